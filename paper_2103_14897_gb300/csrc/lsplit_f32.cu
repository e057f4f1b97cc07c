// float instantiation of the pass and elementwise kernels (see lsplit_kernels.cuh).
#define LS_INST_REAL float
#include "lsplit_kernels.cuh"
