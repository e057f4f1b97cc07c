// Wave function at real-space points from the plane-wave expansion (Sec. 3):
//   psi(x_j) = sum_{m,n} phi[n][m] exp(i k_mn . x_j),  k_mn = B1 m + B2 n.
// The phase factorises, exp(i k . x) = exp(i m . B1^T x) exp(i n . B2^T x), so
//   T[j][n] = sum_m E1[j][m] phi[n][m],   psi_j = sum_n E2[j][n] T[j][n],
// with E1[j][m] = exp(i m . B1^T x_j), E2[j][n] = exp(i n . B2^T x_j).
// The tables come from exact fixed-point turns (the host gives the components
// of B^T x_j / 2 pi as 64-bit fractions per point; the integer index
// components multiply them modulo 2^64), the contraction over m is a tiled
// complex product (64 x 64 outputs per CTA, 16-wide slabs of m in shared
// memory), the sum over n is one warp per point with FP64 accumulation.
#include "lsplit_kernels.cuh"

namespace lsk {

// E[j][m] = exp(2 pi i (ma fa_j + mb fb_j)), ma = lo_a + m % qa, mb = lo_b + m / qa
// (1D: qa = q and mb = 0), turns modulo 2^64
template <typename Real>
__global__ void density_table_kernel(const uint64_t* __restrict__ f, int64_t nx, int64_t q, int32_t qa,
                                     int32_t lo_a, int32_t lo_b, typename CT<Real>::C* __restrict__ E) {
  const int64_t total = nx * q;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / q, m = idx - j * q;
    const int64_t ma = lo_a + m % qa, mb = lo_b + m / qa;
    const uint64_t t = (uint64_t)ma * f[j] + (uint64_t)mb * f[nx + j];
    E[idx] = phase_of<Real>(t).v;
  }
}

// T[j][n] = sum_m E1[j][m] phi[n][m]; E1: nx x M1 (row j), phi: M2 x M1 (pitch)
template <typename Real>
__global__ void __launch_bounds__(256) density_contract_kernel(const typename CT<Real>::C* __restrict__ E1,
                                                               const typename CT<Real>::C* __restrict__ phi,
                                                               int64_t nx, int64_t M1, int64_t M2, int64_t pitch,
                                                               typename CT<Real>::C* __restrict__ T) {
  using C = typename CT<Real>::C;
  constexpr int TJ = 64, TN = 64, TK = 16;
  __shared__ C sa[TK][TJ + 1], sb[TK][TN + 1];
  const int t = threadIdx.x;
  const int tj = t & 15, tn = t >> 4;      // each thread: rows j0 + tj + 16 a, columns n0 + tn + 16 b
  const int64_t j0 = (int64_t)blockIdx.x * TJ, n0 = (int64_t)blockIdx.y * TN;
  C acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b].x = acc[a][b].y = 0;
  for (int64_t k0 = 0; k0 < M1; k0 += TK) {
    for (int e = t; e < TJ * TK; e += 256) {
      const int r = e / TK, c = e - r * TK;
      const int64_t j = j0 + r, k = k0 + c;
      C v;
      v.x = v.y = 0;
      if (j < nx && k < M1) v = E1[j * M1 + k];
      sa[c][r] = v;
      const int64_t n = n0 + r;
      C w;
      w.x = w.y = 0;
      if (n < M2 && k < M1) w = phi[n * pitch + k];
      sb[c][r] = w;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < TK; ++c) {
      C av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = sa[c][tj + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = sb[c][tn + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc[a][b].x += av[a].x * bv[b].x - av[a].y * bv[b].y;
          acc[a][b].y += av[a].x * bv[b].y + av[a].y * bv[b].x;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t j = j0 + tj + 16 * a, n = n0 + tn + 16 * b;
      if (j < nx && n < M2) T[j * M2 + n] = acc[a][b];
    }
}

// psi_j = sum_n E2[j][n] T[j][n], one warp per point, FP64 accumulation
template <typename Real>
__global__ void density_reduce_kernel(const typename CT<Real>::C* __restrict__ E2,
                                      const typename CT<Real>::C* __restrict__ T, int64_t nx, int64_t M2,
                                      double* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= nx) return;
  double re = 0, im = 0;
  for (int64_t n = lane; n < M2; n += 32) {
    const auto e = E2[j * M2 + n], v = T[j * M2 + n];
    re += (double)e.x * v.x - (double)e.y * v.y;
    im += (double)e.x * v.y + (double)e.y * v.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    out[2 * j] = re;
    out[2 * j + 1] = im;
  }
}

template <typename Real>
cudaError_t launch_density(const DensityArgs& d, cudaStream_t st) {
  using C = typename CT<Real>::C;
  C* E1 = static_cast<C*>(d.e1);
  C* E2 = static_cast<C*>(d.e2);
  C* T = static_cast<C*>(d.t);
  const int64_t n1 = d.nx * d.M1, n2 = d.nx * d.M2;
  density_table_kernel<Real><<<(unsigned)std::min<int64_t>((n1 + 255) / 256, 152 * 16), 256, 0, st>>>(
      d.f1, d.nx, d.M1, d.q1a, d.lo1a, d.lo1b, E1);
  density_table_kernel<Real><<<(unsigned)std::min<int64_t>((n2 + 255) / 256, 152 * 16), 256, 0, st>>>(
      d.f2, d.nx, d.M2, d.q2a, d.lo2a, d.lo2b, E2);
  const dim3 grid((unsigned)((d.nx + 63) / 64), (unsigned)((d.M2 + 63) / 64));
  density_contract_kernel<Real><<<grid, 256, 0, st>>>(E1, static_cast<const C*>(d.psi), d.nx, d.M1, d.M2, d.pitch, T);
  density_reduce_kernel<Real><<<(unsigned)((d.nx + 7) / 8), 256, 0, st>>>(E2, T, d.nx, d.M2, d.out);
  return cudaGetLastError();
}

template cudaError_t launch_density<float>(const DensityArgs&, cudaStream_t);
template cudaError_t launch_density<double>(const DensityArgs&, cudaStream_t);

}  // namespace lsk
