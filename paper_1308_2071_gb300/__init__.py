"""GB300 (sm_103a) implementation of the REV-scale MRT lattice Boltzmann model
for convection heat transfer in porous media (Liu, He, Li, Tao,
arXiv:1308.2071).

The compute path is liblbm (CUDA, include/lbm.h); this package is its thin
Python binding.  Importing the package loads nothing; the first use of the
library raises if liblbm.so has not been built.
"""

__all__ = ["Cavity", "Batch", "make_params", "hot_wall_nusselt", "build"]


def __getattr__(name):
    if name in ("Cavity", "Batch", "make_params"):
        from . import lbm
        return getattr(lbm, name)
    if name == "hot_wall_nusselt":
        from .autograd import hot_wall_nusselt
        return hot_wall_nusselt
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
