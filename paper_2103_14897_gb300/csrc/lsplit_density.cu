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

// The complex64 contraction on the tensor cores: every real product of
// T = E1 phi^T in split TF32 (x = hi + lo, hi and lo TF32; hi*hi + hi*lo +
// lo*hi accumulated in FP32, the lo*lo term below 2^-22 relative dropped),
// mma.sync m16n8k8.  64 x 64 outputs per CTA of 8 warps (4 along j x 2
// along n, each 16 x 32), 16-wide slabs of m in shared memory as eight planes
// (re/im x hi/lo of E1 and phi) with rows padded to 20 words, so the fragment
// loads (rows g, columns t and t + 4) fall on distinct banks.  Fragment
// layouts of m16n8k8 (g = lane / 4, t = lane % 4): A a0 (g, t), a1 (g + 8, t),
// a2 (g, t + 4), a3 (g + 8, t + 4); B b0 (k = t, n = g), b1 (t + 4, g);
// C c0 (g, 2t), c1 (g, 2t + 1), c2 (g + 8, 2t), c3 (g + 8, 2t + 1).
namespace {
constexpr int kTcR = 20;   // padded row of a plane (words)

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
}  // namespace

__global__ void __launch_bounds__(256) density_contract_tc_kernel(const float2* __restrict__ E1,
                                                                  const float2* __restrict__ phi, int64_t nx,
                                                                  int64_t M1, int64_t M2, int64_t pitch,
                                                                  float2* __restrict__ T) {
  // planes: 0..3 E1 (re hi, re lo, im hi, im lo), 4..7 phi (same), each [64][kTcR]
  __shared__ uint32_t pl[8][64 * kTcR];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wj = warp & 3, wn = warp >> 2;
  const int64_t j0 = (int64_t)blockIdx.x * 64, n0 = (int64_t)blockIdx.y * 64;
  float cr[4][4], ci[4][4];
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int q = 0; q < 4; ++q) cr[b][q] = ci[b][q] = 0.f;
  for (int64_t k0 = 0; k0 < M1; k0 += 16) {
    // stage the slab, split into TF32 hi and lo parts
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + 256 * r;
      const int row = e >> 4, c = e & 15;
      const int64_t k = k0 + c;
      float2 v = make_float2(0.f, 0.f), w = make_float2(0.f, 0.f);
      if (k < M1 && j0 + row < nx) v = E1[(j0 + row) * M1 + k];
      if (k < M1 && n0 + row < M2) w = phi[(n0 + row) * pitch + k];
      const uint32_t vrh = to_tf32(v.x), vih = to_tf32(v.y), wrh = to_tf32(w.x), wih = to_tf32(w.y);
      const int o = row * kTcR + c;
      pl[0][o] = vrh;
      pl[1][o] = to_tf32(v.x - __uint_as_float(vrh));
      pl[2][o] = vih;
      pl[3][o] = to_tf32(v.y - __uint_as_float(vih));
      pl[4][o] = wrh;
      pl[5][o] = to_tf32(w.x - __uint_as_float(wrh));
      pl[6][o] = wih;
      pl[7][o] = to_tf32(w.y - __uint_as_float(wih));
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < 16; ks += 8) {
      // A fragments of this warp's 16 rows: re hi, re lo, im hi, im lo, and -im
      uint32_t a[4][4], na[2][4];
      const int ra = (16 * wj + g) * kTcR + ks + t;
#pragma unroll
      for (int pq = 0; pq < 4; ++pq) {
        a[pq][0] = pl[pq][ra];
        a[pq][1] = pl[pq][ra + 8 * kTcR];
        a[pq][2] = pl[pq][ra + 4];
        a[pq][3] = pl[pq][ra + 8 * kTcR + 4];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        na[0][q] = a[2][q] ^ 0x80000000u;
        na[1][q] = a[3][q] ^ 0x80000000u;
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int rb = (32 * wn + 8 * b + g) * kTcR + ks + t;
        const uint32_t brh0 = pl[4][rb], brh1 = pl[4][rb + 4], brl0 = pl[5][rb], brl1 = pl[5][rb + 4];
        const uint32_t bih0 = pl[6][rb], bih1 = pl[6][rb + 4], bil0 = pl[7][rb], bil1 = pl[7][rb + 4];
        // re += Ar Br - Ai Bi
        mma_tf32(cr[b], a[0], brh0, brh1);
        mma_tf32(cr[b], a[0], brl0, brl1);
        mma_tf32(cr[b], a[1], brh0, brh1);
        mma_tf32(cr[b], na[0], bih0, bih1);
        mma_tf32(cr[b], na[0], bil0, bil1);
        mma_tf32(cr[b], na[1], bih0, bih1);
        // im += Ar Bi + Ai Br
        mma_tf32(ci[b], a[0], bih0, bih1);
        mma_tf32(ci[b], a[0], bil0, bil1);
        mma_tf32(ci[b], a[1], bih0, bih1);
        mma_tf32(ci[b], a[2], brh0, brh1);
        mma_tf32(ci[b], a[2], brl0, brl1);
        mma_tf32(ci[b], a[3], brh0, brh1);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t j = j0 + 16 * wj + g + 8 * (q >> 1), n = n0 + 32 * wn + 8 * b + 2 * t + (q & 1);
      if (j < nx && n < M2) T[j * M2 + n] = make_float2(cr[b][q], ci[b][q]);
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
  if constexpr (sizeof(Real) == 4) {
    if (!d.simt) {
      density_contract_tc_kernel<<<grid, 256, 0, st>>>(E1, static_cast<const C*>(d.psi), d.nx, d.M1, d.M2, d.pitch,
                                                       T);
    } else {
      density_contract_kernel<Real><<<grid, 256, 0, st>>>(E1, static_cast<const C*>(d.psi), d.nx, d.M1, d.M2,
                                                          d.pitch, T);
    }
  } else {
    density_contract_kernel<Real><<<grid, 256, 0, st>>>(E1, static_cast<const C*>(d.psi), d.nx, d.M1, d.M2, d.pitch, T);
  }
  density_reduce_kernel<Real><<<(unsigned)((d.nx + 7) / 8), 256, 0, st>>>(E2, T, d.nx, d.M2, d.out);
  return cudaGetLastError();
}

template cudaError_t launch_density<float>(const DensityArgs&, cudaStream_t);
template cudaError_t launch_density<double>(const DensityArgs&, cudaStream_t);

}  // namespace lsk
