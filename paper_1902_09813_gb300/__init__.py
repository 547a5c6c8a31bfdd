"""GB300-native B-TriRT lattice Boltzmann solver (D2Q9) for nonlinear anisotropic
convection-diffusion equations.

The compute path is the CUDA library ``_lib/libbtrt.so`` (sources in ``csrc/``,
C ABI in ``include/btrt.h``); this package only marshals arguments.  There is
no CPU fallback: importing :class:`Lattice` on a machine without the built
library or a GPU raises.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("Lattice", "Batch", "grid_desc", "coeffs", "workspace_bytes"):
        from . import lattice
        return getattr(lattice, name)
    raise AttributeError(name)
