"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This module only makes inputs: it holds none of the correlator arithmetic.
Every random number comes from one counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): output n of the stream keyed by K is mix64(K + (n+1)*GAMMA),
with GAMMA = 0x9E3779B97F4A7C15 and mix64 the published finaliser.  A value
therefore depends only on (seed, stream, position) and never on the order in
which values are drawn.

Propagator layout (what the C ABI consumes): one timeslice of one flavour is a
complex128 array [V][12][12], site = x + L*(y + L*z), sink index
i = 3*alpha + a (spin alpha, colour a), source index j = 3*alpha' + a'.
"""

from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

FLAVOUR_STREAM = {"l": 1, "u": 1, "d": 2, "s": 3}
_SU3_STREAM = 17


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of the SplitMix64 stream (seed, stream)."""
    with np.errstate(over="ignore"):
        k = _mix64(np.array([seed], dtype=np.uint64))[0]
        k = _mix64(np.array([k ^ np.uint64(stream)], dtype=np.uint64))[0]
    return k


def splitmix64(key: np.uint64, n: np.ndarray) -> np.ndarray:
    """Outputs n (uint64 array of positions) of the stream keyed by `key`."""
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (n.astype(np.uint64) + np.uint64(1)) * _GAMMA
        return _mix64(z)


def uniform01(key: np.uint64, n: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the stream outputs."""
    return (splitmix64(key, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian_c128(key: np.uint64, n: np.ndarray) -> np.ndarray:
    """Complex values with independent N(0,1) real and imaginary parts.

    Box-Muller on the stream positions 2n and 2n+1.
    """
    u1 = uniform01(key, 2 * n)
    u2 = uniform01(key, 2 * n + 1)
    rad = np.sqrt(-2.0 * np.log1p(-u1))
    return rad * np.exp(2j * np.pi * u2)


def propagator(seed: int, flavour: str, L: int, t: int, decay: float = 0.0) -> np.ndarray:
    """One timeslice of a synthetic wall-source propagator, complex128 [V,12,12].

    Entry (site, i, j) of timeslice t is the Gaussian at position
    ((t*V + site)*144 + 12*i + j) of the flavour's stream, times exp(-decay*t).
    """
    V = L * L * L
    key = stream_key(seed, FLAVOUR_STREAM[flavour])
    base = np.uint64(t) * np.uint64(V * 144)
    n = base + np.arange(V * 144, dtype=np.uint64)
    S = gaussian_c128(key, n).reshape(V, 12, 12)
    if decay:
        S *= np.exp(-decay * t)
    return S


def haar_su3(seed: int, L: int, t: int = 0) -> np.ndarray:
    """Haar-random SU(3) matrices, one per site: complex128 [V,3,3].

    QR of a complex Gaussian matrix with the phases of R's diagonal moved into
    Q (Mezzadri, Notices AMS 54 (2007) 592), then divided by a cube root of
    its determinant so that det U = 1.
    """
    V = L * L * L
    key = stream_key(seed, _SU3_STREAM)
    n = np.uint64(t) * np.uint64(V * 9) + np.arange(V * 9, dtype=np.uint64)
    Z = gaussian_c128(key, n).reshape(V, 3, 3) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=1, axis2=2)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    return Q / (det ** (1.0 / 3.0))[:, None, None]


def rotate_sink_colour(S: np.ndarray, U: np.ndarray) -> np.ndarray:
    """S'[x][3*alpha+a][j] = sum_b U[x][a][b] S[x][3*alpha+b][j]."""
    V = S.shape[0]
    Sr = S.reshape(V, 4, 3, 12)
    return np.einsum("xab,xsbj->xsaj", U, Sr).reshape(V, 12, 12)


def rotate_source_colour(S: np.ndarray, U3: np.ndarray) -> np.ndarray:
    """Global source-colour rotation: S'[x][i][3*alpha'+a'] = sum_b S[x][i][3*alpha'+b] U3[b][a']."""
    V = S.shape[0]
    Sr = S.reshape(V, 12, 4, 3)
    return np.einsum("xisb,ba->xisa", Sr, U3).reshape(V, 12, 12)


def translate(S: np.ndarray, L: int, a: tuple[int, int, int]) -> np.ndarray:
    """S'(x) = S(x + a) with periodic boundaries; a = (ax, ay, az)."""
    g = S.reshape(L, L, L, 12, 12)  # [z][y][x]
    g = np.roll(g, shift=(-a[2], -a[1], -a[0]), axis=(0, 1, 2))
    return g.reshape(L * L * L, 12, 12)


def workload_props(seed: int, L: int, T: int, decay: float = 0.0, flavours=("l", "s")):
    """Propagators for timeslices 0..T-1: dict flavour -> complex128 [T,V,12,12]."""
    return {f: np.stack([propagator(seed, f, L, t, decay) for t in range(T)]) for f in flavours}
