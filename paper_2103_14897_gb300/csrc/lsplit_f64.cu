// double instantiation of the pass and elementwise kernels (see lsplit_kernels.cuh).
#define LS_INST_REAL double
#include "lsplit_kernels.cuh"
