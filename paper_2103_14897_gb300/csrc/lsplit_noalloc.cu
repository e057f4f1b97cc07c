// ls_mass_noalloc: the mass sum |phi|^2 of a wave-function array, computed
// without allocating any memory.
//
// Some callers cannot call cudaMalloc: hosts that hand out all device memory
// from their own pool and forbid other allocations, and real-time loops that
// must not pay for or wait on the allocator.  This entry point needs no
// context (ls_create allocates) and uses, as its scratch, a fixed file-scope
// device array instead of memory it would allocate.
//
// The scratch holds one FP64 partial sum per row, kNoAllocMaxRows rows at
// most (512 KB).  It lives in every GPU that loads the library until the
// process exits.  Every call uses the same array and leaves its partial sums
// there; each call overwrites the rows it reads, so nothing needs clearing.
// Calls that overlap on the GPU (different streams, or other threads) race on
// the array and must be ordered by the caller.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "lsplit.h"
#include "lsplit_internal.h"

namespace {

constexpr int64_t kNoAllocMaxRows = 65536;
static __device__ __align__(256) double g_noalloc_rows[kNoAllocMaxRows];

// One warp per row, FP64 accumulation in a fixed order per lane, then a fixed
// shuffle tree: the result does not depend on the launch schedule.
template <typename C>
__global__ void noalloc_row_mass(const C* __restrict__ psi, int64_t rows, int64_t cols, int64_t pitch,
                                 double* rowsum) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows; r += nwarps) {
    double acc = 0.0;
    for (int64_t c = lane; c < cols; c += 32) {
      const C v = psi[r * pitch + c];
      acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) rowsum[r] = acc;
  }
}

__global__ void noalloc_sum_rows(const double* rowsum, int64_t rows, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) acc += rowsum[r];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) out[0] = v;
  }
}

// Device address of the scratch array, looked up once per device with that
// device current (in host code the symbol is only a host-side stand-in).
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    lsk::set_last_error(std::string(std::string("cudaGetDevice: ") + cudaGetErrorString(e)));
    return LS_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    lsk::set_last_error(std::string("device ordinal out of range"));
    return LS_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_rows);
    if (e != cudaSuccess || !p) {
      lsk::set_last_error(std::string(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)));
      return LS_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return LS_OK;
}

}  // namespace

extern "C" int ls_mass_noalloc(const void* psi_dev, int32_t dtype, int64_t rows, int64_t cols, int64_t pitch,
                               double* out_dev, void* stream) {
  lsk::set_last_error("");
  if (!psi_dev || !out_dev) {
    lsk::set_last_error(std::string("psi_dev and out_dev must not be NULL"));
    return LS_ERR_INVALID;
  }
  if (dtype != LS_C64 && dtype != LS_C128) {
    lsk::set_last_error(std::string("dtype must be LS_C64 or LS_C128"));
    return LS_ERR_INVALID;
  }
  if (rows < 1 || cols < 1 || pitch < cols) {
    lsk::set_last_error(std::string("need rows >= 1, cols >= 1 and pitch >= cols"));
    return LS_ERR_INVALID;
  }
  if (rows > kNoAllocMaxRows) {
    lsk::set_last_error(std::string("rows exceeds the fixed scratch of ls_mass_noalloc (65536 rows)"));
    return LS_ERR_INVALID;
  }
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != LS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int threads = 256;
  const int64_t want = (rows * 32 + threads - 1) / threads;
  const unsigned blocks = (unsigned)(want < 4096 ? want : 4096);
  if (dtype == LS_C64)
    noalloc_row_mass<float2><<<blocks, threads, 0, st>>>(static_cast<const float2*>(psi_dev), rows, cols, pitch,
                                                          scratch);
  else
    noalloc_row_mass<double2><<<blocks, threads, 0, st>>>(static_cast<const double2*>(psi_dev), rows, cols, pitch,
                                                           scratch);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    noalloc_sum_rows<<<1, 1024, 0, st>>>(scratch, rows, out_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    lsk::set_last_error(std::string(std::string("kernel launch: ") + cudaGetErrorString(e)));
    return LS_ERR_CUDA;
  }
  return LS_OK;
}
