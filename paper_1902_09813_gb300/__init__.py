"""GB300-native B-TriRT lattice Boltzmann solver (D2Q9, and D3Q19 in three
dimensions) for nonlinear anisotropic convection-diffusion equations.

The compute path is the CUDA library ``_lib/libbtrt.so`` (sources in ``csrc/``,
C ABI in ``include/btrt.h`` and ``include/btrt3.h``); this package only marshals arguments.  There is
no CPU fallback: importing :class:`Lattice` on a machine without the built
library or a GPU raises.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("Lattice", "Batch", "grid_desc", "coeffs", "workspace_bytes"):
        from . import lattice
        return getattr(lattice, name)
    if name in ("Lattice3", "grid_desc3", "coeffs3"):
        from . import lattice3
        return getattr(lattice3, name)
    raise AttributeError(name)
