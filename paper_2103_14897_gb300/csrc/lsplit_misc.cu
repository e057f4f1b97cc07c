// Non-templated kernels (reductions, sampler, fills) and host helpers.
#define LS_DEFINE_MISC
#include "lsplit_kernels.cuh"
