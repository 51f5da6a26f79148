"""GB300-native treecode boundary-element Poisson-Boltzmann solver
(Cooper & Barba, arXiv 1506.03745): the C-ABI library libpgb (CUDA, sm_103a)
and its thin Python binding.  The hot path runs only in the CUDA library; if
libpgb.so is missing every call raises."""
from ._lib import *  # noqa: F401,F403
from ._lib import lib, default_params, PgbError  # noqa: F401
