// Persistent batched runner (float and double), a translation unit of its own
// so that it compiles in parallel with the per-precision pass kernels.
#define LS_INST_BATCH
#include "lsplit_kernels.cuh"
