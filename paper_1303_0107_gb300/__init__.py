"""GB300 (sm_103a) implementation of the lattice Boltzmann shape-optimisation
hot path of Wang, Fan & Luo (arXiv:1303.0107): fused D2Q9 (and D3Q19) BGK stream-collide
with bounce-back and port rules, FP64 pressure-drop / flow-rate reductions,
and the equal-count fluid/solid exchange of the optimality criterion.

The computation lives in the CUDA library built from csrc/ (C ABI in
include/lbm.h, include/lbm3d.h); `lib` and `lib3d` are its ctypes bindings, `inputs` the seeded synthetic
workloads.
"""
from . import inputs  # noqa: F401
from .lib import (F32, BF16_SHIFTED, F16_SHIFTED, OUT_CONST_RHO, OUT_NEUMANN, REINIT_WARM,  # noqa: F401
                  PORTS_REGULARIZED, PORTS_ZOU_HE, COLLIDE_BGK, COLLIDE_REGULARIZED, COLLIDE_SMAGORINSKY,
                  REINIT_COLD, FIELD_RHO, FIELD_UX, FIELD_UY, FIELD_MASK, FIELD_POPS, FIELD_DRHO,
                  Lattice, Batch, Server, LbmError, bytes_per_fluid_update, kernel_launches, load_library,
                  transfer_bytes)
from .lib3d import (Lattice3, FIELD3_DRHO, FIELD3_UX, FIELD3_UY, FIELD3_UZ, FIELD3_MASK,  # noqa: F401
                    FIELD3_POPS)
