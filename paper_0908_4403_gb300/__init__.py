"""GB300-native hot path of HEGET (arXiv:0908.4403): helicity amplitudes of
u ubar -> n photons, RAMBO phase space and Monte Carlo cross sections behind
the C ABI of include/heget.h.  ``heget`` is the ctypes binding; ``build``
compiles libheget.so for sm_103a."""
from . import heget  # noqa: F401
