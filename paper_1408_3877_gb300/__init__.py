"""GB300 (sm_103a) LDG diffusion solver: the matrix-free LDG operator of FESTUNG
Part I (arXiv:1408.3877) and its implicit-Euler step, as hand-written CUDA kernels
behind the C ABI of include/festung.h.  ``festung`` is the Python binding."""
