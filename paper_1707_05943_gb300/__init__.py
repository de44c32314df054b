"""GB300 (sm_103a) FDTD solver for the 1+1D delay PDE of waveguide QED
(arXiv:1707.05943).  The compute path is libfdtd (include/fdtd.h), built from
csrc/ by build.py; fdtd.py is its Python binding."""
from . import fdtd  # noqa: F401
