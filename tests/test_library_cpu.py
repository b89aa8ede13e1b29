"""CPU checks of the C ABI library: exports, argument errors, and the host
channel compiler re-executed step by step against the oracle (no GPU)."""

import ctypes
import os
import re

import numpy as np
import pytest

import nbs_inputs as I
from oracle import nbs_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
nbs = pytest.importorskip("paper_1604_07983_gb300.nbs")


@pytest.fixture(scope="module")
def lib():
    try:
        return nbs.lib()
    except ImportError:
        pytest.skip("libnbs.so not built")


def header_functions():
    src = open(os.path.join(ROOT, "include", "nbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(nbs_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    declared = header_functions()
    assert declared == sorted(nbs.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_channel_table(lib):
    names = nbs.channel_names()
    assert len(names) == 52
    assert names[0] == ("p", "n", "p", "n")
    assert len(set(names)) == 52
    for c, ch in enumerate(names):
        _, nl = nbs.channel_info(c)
        assert (nl, 6 - nl) == O.flavour_content(ch)
    # isospin-forbidden Lambda/Sigma0 transitions are not in the table
    assert ("Lambda", "Lambda", "Lambda", "Sigma0") not in names
    assert ("Sigma0", "Sigma0", "Lambda", "Sigma0") not in names


def test_argument_errors_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.nbs_create(ctypes.byref(h), 8, 8, 3) == nbs.NBS_EINVAL
    assert b"flavours" in lib.nbs_last_error(None)
    assert lib.nbs_create(ctypes.byref(h), 5, 8, 2) == nbs.NBS_EINVAL
    assert lib.nbs_create(ctypes.byref(h), 8, 0, 2) == nbs.NBS_EINVAL
    ids = (ctypes.c_int * 1)(99)
    p = ctypes.c_void_p()
    assert lib.nbs_plan_create(ctypes.byref(p), ids, 1) == nbs.NBS_EINVAL
    assert lib.nbs_channel_info(52, None, 0) == nbs.NBS_EINVAL
    assert lib.nbs_set_precision(None, 0) == nbs.NBS_EINVAL


def test_block_types_share_isospin_partners(lib):
    tb = nbs.plan_tables(list(range(52)))
    # p/n, Sigma+/Sigma-, Xi0/Xi-, Lambda, Sigma0: five stored types, 16416 components
    assert len(tb["types"]) == 5
    assert 4 * len(tb["cells"]) == 16416


def test_worked_counts_pn(lib):
    tb = nbs.plan_tables([0])
    terms = tb["terms"]
    assert len(terms) == 9
    assert int(terms[:, 1].sum()) == 586


@pytest.mark.parametrize("L,ids", [(2, list(range(52))), (3, [0, 5, 17, 30, 47, 51])])
def test_compiled_tables_reproduce_oracle(lib, L, ids):
    from plan_emulator import emulate
    names = nbs.channel_names()
    Sl, Ss = I.propagator(61, "l", L, 0), I.propagator(61, "s", L, 0)
    props = {"u": Sl, "d": Sl, "s": Ss}
    F = emulate(ids, Sl, Ss, L)
    for k, c in enumerate(ids):
        Fo = O.correlator(names[c], props, L)
        assert np.linalg.norm(F[k] - Fo) <= 1e-12 * np.linalg.norm(Fo), names[c]
