"""GB300-native phi-function actions for exponential integrators (Leja and
KIOPS-style Krylov), a CUDA library behind the C-ABI of include/phix.h.

``phix`` is the ctypes binding; ``build`` compiles libphix.so for sm_103a.
"""
