"""GB300 implementation of the effective-baryon-block NBS correlator path (arXiv:1604.07983).

The compute path is the CUDA library libnbs.so (C ABI in include/nbs.h); this
package only builds it (build.py) and binds it (nbs.py).
"""

from .nbs import (NBS_BF16X3, NBS_C64, NBS_C128, NBS_FP32, NBS_FP64, NBS_NSPIN, Context, Graph, NBSError, channel_count,  # noqa: F401
                  assemble_full_spin, channel_info, channel_names, full_spin_ids, lib, plan_tables, potential,
                  use_torch_allocator, SlabContext, slab_correlate, slab_layout)
