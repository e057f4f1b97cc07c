// Crank-Nicolson layer factors (Sec. 4.2.1, Eq. (tsCN)) for 1D boxes.
//
// A factor of duration s along layer j maps every slice x (fixed index of the
// other layer) to the solution y of
//     (I + i s A/2) y = (I - i s A/2) x,   A = diag(|k|^2/4) + V^j,
// V^j the plane-wave matrix of the layer potential, V[i, i'] = vhat(i - i'),
// banded with half-width hb and truncated at the box ends.  With
// alpha_i = 1 + i (s/2)(|k_i|^2/4 + vhat_0) the off-diagonal part of a row is
// at most rho = (s/2) sum_{h != 0} |vhat_h| / min |alpha_i| < 1/2 (checked on
// the host), so the system is strictly diagonally dominant and the Jacobi
// iteration
//     y <- alpha^{-1} (b - i (s/2) sum_{h != 0} vhat_h y_{i-h}),
//     b = (I - i s A/2) x,  started from alpha^{-1} b,
// contracts by rho per sweep; the host picks the sweep count niter that takes
// rho^niter below the working precision.  A sweep reaches hb indices further,
// so a chunk of TI indices is computed on a tile extending halo = hb (niter + 1)
// indices on each side (the right-hand side needs hb more), and the chunk's
// values after the last sweep equal those of Jacobi on the whole slice.
//
// Tiles: W slices x E = TI + 2 halo indices in shared memory, two buffers.
// Layer 1 (rows): W = 1 and the threads run along the row.  Layer 2 (columns):
// W (a power of two) adjacent columns and the threads run across them, so each
// row segment is one W x 8-byte access.  Each thread keeps the per-element
// terms of its own elements (t + 256 k) in registers.
#include "lsplit_kernels.cuh"

namespace lsk {

// Diagonal Cayley multiplier c = (2 - alpha) / alpha of an element.  For a
// real vhat_0 it has modulus 1 and is returned as a Phase with the deviation
// e = |c|^2 - 1 of its rounded components, so that apply_phase removes the
// bias an element would otherwise meet at every step (the norm drift of a
// plain product); for a complex vhat_0 the factor is not unitary and e = 0.
// Also returns gam = -i (s/2) / alpha.
template <typename Real>
__device__ __forceinline__ Phase<Real> cn_diag(Real z, Real zlo, Real g, Real hs, bool unitary,
                                               typename CT<Real>::C& gam);
template <>
__device__ __forceinline__ Phase<float> cn_diag<float>(float z, float zlo, float g, float hs, bool unitary,
                                                       float2& gam) {
  // alpha = (1 - g) + i z, 2 - alpha = (1 + g) - i z
  Phase<float> p;
  if (unitary) {
    // c = ((1 - z^2) - 2 i z) / (1 + z^2) = exp(-2 i atan z); the low word zlo
    // of z enters as the first-order rotation by -2 zlo / (1 + z^2)
    const float r = __frcp_rn(fmaf(z, z, 1.0f));
    const float cx = fmaf(-z, z, 1.0f) * r, cy = -2.0f * z * r;
    const float dlt = -2.0f * zlo * r;
    gam.x = -hs * z * r;
    gam.y = -hs * r;
    p.v.x = fmaf(-dlt, cy, cx);
    p.v.y = fmaf(dlt, cx, cy);
    const float c2h = __fmul_rn(p.v.x, p.v.x), c2l = fmaf(p.v.x, p.v.x, -c2h);
    const float s2h = __fmul_rn(p.v.y, p.v.y), s2l = fmaf(p.v.y, p.v.y, -s2h);
    p.half_e = 0.5f * __fadd_rn(__fadd_rn(__fadd_rn(c2h, -1.0f), s2h), __fadd_rn(c2l, s2l));
  } else {
    const float ar = 1.0f - g, inv = 1.0f / (ar * ar + z * z);
    const float nr = 1.0f + g, ni = -z;
    p.v.x = (nr * ar + ni * z) * inv;
    p.v.y = (ni * ar - nr * z) * inv;
    p.half_e = 0.0f;
    gam.x = -hs * z * inv;
    gam.y = -hs * ar * inv;
  }
  return p;
}
template <>
__device__ __forceinline__ Phase<double> cn_diag<double>(double z, double zlo, double g, double hs, bool unitary,
                                                         double2& gam) {
  Phase<double> p;
  (void)zlo;
  const double ar = 1.0 - g, inv = 1.0 / (ar * ar + z * z);
  const double nr = 1.0 + g, ni = -z;
  p.v.x = (nr * ar + ni * z) * inv;
  p.v.y = (ni * ar - nr * z) * inv;
  p.half_e = 0.0;
  gam.x = -hs * z * inv;
  gam.y = -hs * ar * inv;
  (void)unitary;
  return p;
}

// z = (s/2)(|k|^2/4 + Re vhat_0) of element (m, n).  Single precision: the
// quadratic form za m^2 + zb m n + zc n^2 + zd with exact integer products
// (|m|, |n| < 2^12) and float-float coefficients, summed with error-free
// transforms into z + zlo (an FP32 k would put ~2e-7 relative error into the
// Cayley angle, the same for an element at every step).  Double: direct.
template <typename Real>
__device__ __forceinline__ void cn_z(const CnArgs& a, int32_t m, int32_t n, Real& z, Real& zlo);
template <>
__device__ __forceinline__ void cn_z<float>(const CnArgs& a, int32_t m, int32_t n, float& z, float& zlo) {
  // 32-bit products and conversions (a 64-bit integer to float conversion
  // runs on the FP64 pipe)
  const float mm = (float)(m * m), mn = (float)(m * n), nn = (float)(n * n);
  const float p1 = __fmul_rn(a.za[0], mm), e1 = fmaf(a.za[0], mm, -p1);
  const float p2 = __fmul_rn(a.zb[0], mn), e2 = fmaf(a.zb[0], mn, -p2);
  const float p3 = __fmul_rn(a.zc[0], nn), e3 = fmaf(a.zc[0], nn, -p3);
  // two-sum chain of the large terms
  float s = p1, err = 0.0f;
  auto add = [&](float b) {
    const float t = __fadd_rn(s, b), bb = __fsub_rn(t, s);
    err = __fadd_rn(err, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(b, bb)));
    s = t;
  };
  add(p2);
  add(p3);
  add(a.zd[0]);
  float small = e1 + e2 + e3 + a.zd[1];
  small = fmaf(a.za[1], mm, small);
  small = fmaf(a.zb[1], mn, small);
  small = fmaf(a.zc[1], nn, small);
  const float lo = __fadd_rn(err, small);
  z = __fadd_rn(s, lo);
  zlo = __fsub_rn(lo, __fsub_rn(z, s));
}
template <>
__device__ __forceinline__ void cn_z<double>(const CnArgs& a, int32_t m, int32_t n, double& z, double& zlo) {
  const double kk = a.b_own * (double)m + a.b_oth * (double)n;
  z = a.half_s * (0.25 * kk * kk + a.v_re[kCnMaxBand]);
  zlo = 0.0;
}

// Per element: y = c x + gam (sx + sum_{h != 0} vhat_h y_{i-h}), with
// gam = -i (s/2) / alpha and sx = sum_{h != 0} vhat_h x_{i-h}; the first
// iterate takes y = 0 inside the sum (that is alpha^{-1} b).  The tile buffers
// carry HB * hstep zero entries before and after, so neighbour reads need no
// bounds checks (beyond the box and beyond the tile both read zero).
template <typename Real, bool STRIDED, int HB>
__global__ void __launch_bounds__(256) cn_pass_kernel(const CnArgs a) {
  using C = typename CT<Real>::C;
  constexpr int KE = kCnPerThread;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ C s_v[2 * kCnMaxBand + 1];
  const int W = a.W, lw = STRIDED ? 31 - __clz(W) : 0;
  const int E = a.TI + 2 * a.halo, span = W * E;
  const int hstep = STRIDED ? W : 1;
  const int pad = HB * hstep;
  const int t = threadIdx.x;
  if (t < 2 * kCnMaxBand + 1) {
    s_v[t].x = (Real)a.v_re[t];
    s_v[t].y = (Real)a.v_im[t];
  }
  C* cur = reinterpret_cast<C*>(smraw) + pad;
  C* nxt = cur + span + 2 * pad;
  for (int e = t; e < pad; e += 256) {
    C z;
    z.x = z.y = 0;
    cur[-1 - e] = z;
    cur[span + e] = z;
    nxt[-1 - e] = z;
    nxt[span + e] = z;
  }
  // 32-bit index arithmetic (a 64-bit division runs on the FP64 pipe)
  const unsigned nch = (unsigned)a.nchunks;
  const unsigned grp = blockIdx.x / nch, ch = blockIdx.x - grp * nch;
  const int64_t s0 = (int64_t)grp * W;
  const int i0 = (int)(ch * (unsigned)a.TI) - a.halo;
  C* psi = reinterpret_cast<C*>(a.psi);
  Real hs;
  if constexpr (sizeof(Real) == 4) hs = a.half_s_f;
  else hs = a.half_s;
  const bool unitary = a.unitary != 0;

  C xk[KE];
#pragma unroll
  for (int k = 0; k < KE; ++k) {
    const int e = t + 256 * k;
    xk[k].x = xk[k].y = 0;
    if (e >= span) continue;
    const int w = STRIDED ? (e & (W - 1)) : 0, j = STRIDED ? (e >> lw) : e;
    const int i = i0 + j;
    const int64_t s = s0 + w;
    if (s < a.nslices && i >= 0 && i < a.q) xk[k] = psi[s * a.slice_stride + (int64_t)i * a.ea];
    nxt[e] = xk[k];
  }
  __syncthreads();
  C px[KE], gam[KE], sx[KE];
  const C v0 = s_v[kCnMaxBand];
#pragma unroll
  for (int k = 0; k < KE; ++k) {
    const int e = t + 256 * k;
    px[k].x = px[k].y = 0;
    gam[k].x = gam[k].y = 0;
    sx[k].x = sx[k].y = 0;
    if (e >= span) continue;
    const int w = STRIDED ? (e & (W - 1)) : 0, j = STRIDED ? (e >> lw) : e;
    const int i = i0 + j;
    const int64_t s = s0 + w;
    C y;
    y.x = y.y = 0;
    if (s < a.nslices && i >= 0 && i < a.q) {
      Real z, zlo;
      cn_z<Real>(a, a.lo + i, a.olo + (int32_t)s, z, zlo);
      const Real g = hs * v0.y;
      px[k] = apply_phase<Real>(xk[k], cn_diag<Real>(z, zlo, g, hs, unitary, gam[k]));
      C acc;
      acc.x = acc.y = 0;
#pragma unroll
      for (int h = 1; h <= HB; ++h) {
        if (h > a.hb) break;
        const C vl = s_v[kCnMaxBand + h], vr = s_v[kCnMaxBand - h];
        const C xl = nxt[e - h * hstep], xr = nxt[e + h * hstep];
        acc.x += vl.x * xl.x - vl.y * xl.y + vr.x * xr.x - vr.y * xr.y;
        acc.y += vl.x * xl.y + vl.y * xl.x + vr.x * xr.y + vr.y * xr.x;
      }
      sx[k] = acc;
      y = px[k];
      y.x += gam[k].x * acc.x - gam[k].y * acc.y;
      y.y += gam[k].x * acc.y + gam[k].y * acc.x;
    }
    cur[e] = y;
  }
  __syncthreads();
  for (int it = 0; it < a.niter; ++it) {
#pragma unroll
    for (int k = 0; k < KE; ++k) {
      const int e = t + 256 * k;
      if (e >= span) continue;
      C acc = sx[k];
#pragma unroll
      for (int h = 1; h <= HB; ++h) {
        if (h > a.hb) break;
        const C vl = s_v[kCnMaxBand + h], vr = s_v[kCnMaxBand - h];
        const C yl = cur[e - h * hstep], yr = cur[e + h * hstep];
        acc.x += vl.x * yl.x - vl.y * yl.y + vr.x * yr.x - vr.y * yr.y;
        acc.y += vl.x * yl.y + vl.y * yl.x + vr.x * yr.y + vr.y * yr.x;
      }
      C y = px[k];
      y.x += gam[k].x * acc.x - gam[k].y * acc.y;
      y.y += gam[k].x * acc.y + gam[k].y * acc.x;
      nxt[e] = y;
    }
    __syncthreads();
    C* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
#pragma unroll
  for (int k = 0; k < KE; ++k) {
    const int e = t + 256 * k;
    if (e >= span) continue;
    const int w = STRIDED ? (e & (W - 1)) : 0, j = STRIDED ? (e >> lw) : e;
    if (j < a.halo || j >= a.halo + a.TI) continue;
    const int i = i0 + j;
    const int64_t s = s0 + w;
    if (s < a.nslices && i < a.q) psi[s * a.slice_stride + (int64_t)i * a.ea] = cur[e];
  }
}

// ---------------------------------------------------------------- semi-implicit step
// One CTA: a column tile of 256 consecutive m by kSiRows consecutive rows n;
// thread t owns column m0 + t.  Neighbours come through the read-only cache
// (the step is out of place).  Row / column weights of the random batch form
// are looked up once per CTA by binary search in the sorted sample lists.
constexpr int kSiRows = 4;

__device__ __forceinline__ bool si_member(const int32_t* list, int32_t n, int32_t v) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int32_t x = __ldg(list + mid);
    if (x == v) return true;
    if (x < v) lo = mid + 1;
    else hi = mid - 1;
  }
  return false;
}

template <typename Real>
__global__ void __launch_bounds__(256) si_kernel(const SiArgs a) {
  using C = typename CT<Real>::C;
  __shared__ C s_v1[2 * kCnMaxBand + 1], s_v2[2 * kCnMaxBand + 1];
  __shared__ Real s_wr[kSiRows];
  const int t = threadIdx.x;
  if (t < 2 * kCnMaxBand + 1) {
    s_v1[t].x = (Real)a.v1_re[t];
    s_v1[t].y = (Real)a.v1_im[t];
    s_v2[t].x = (Real)a.v2_re[t];
    s_v2[t].y = (Real)a.v2_im[t];
  }
  const int64_t m = (int64_t)blockIdx.x * 256 + t;
  const int64_t n0 = (int64_t)blockIdx.y * kSiRows;
  if (t < kSiRows) {
    Real w = 1;
    if (a.rows) w = (n0 + t < a.M2 && si_member(a.rows, a.nrows, (int32_t)(n0 + t))) ? (Real)a.w_row : (Real)0;
    s_wr[t] = w;
  }
  __syncthreads();
  if (m >= a.M1) return;
  Real wc = 1;
  if (a.cols) wc = si_member(a.cols, a.ncols, (int32_t)m) ? (Real)a.w_col : (Real)0;
  const C* src = reinterpret_cast<const C*>(a.src);
  C* dst = reinterpret_cast<C*>(a.dst);
  Real tau;
  if constexpr (sizeof(Real) == 4) tau = a.tau_f;
  else tau = a.tau;
  const int32_t mi = a.lo1 + (int32_t)m;
  for (int r = 0; r < kSiRows; ++r) {
    const int64_t n = n0 + r;
    if (n >= a.M2) break;
    const C* row = src + n * a.pitch;
    // s1 = sum_h vhat1_h x[n][m - h], s2 = sum_h vhat2_h x[n - h][m]
    C s1, s2;
    s1.x = s1.y = 0;
    s2.x = s2.y = 0;
    for (int h = -a.hb1; h <= a.hb1; ++h) {
      const int64_t mm = m - h;
      if (mm < 0 || mm >= a.M1) continue;
      const C x = __ldg(row + mm), v = s_v1[h + kCnMaxBand];
      s1.x += v.x * x.x - v.y * x.y;
      s1.y += v.x * x.y + v.y * x.x;
    }
    for (int h = -a.hb2; h <= a.hb2; ++h) {
      const int64_t nn = n - h;
      if (nn < 0 || nn >= a.M2) continue;
      const C x = __ldg(src + nn * a.pitch + m), v = s_v2[h + kCnMaxBand];
      s2.x += v.x * x.x - v.y * x.y;
      s2.y += v.x * x.y + v.y * x.x;
    }
    const Real wr = s_wr[r];
    C acc;
    acc.x = wr * s1.x + wc * s2.x;
    acc.y = wr * s1.y + wc * s2.y;
    const C x = __ldg(row + m);
    // num = x - i tau acc
    C num;
    num.x = x.x + tau * acc.y;
    num.y = x.y - tau * acc.x;
    // z = tau |k|^2 / 2; dst = num (1 - i z) / (1 + z^2)
    Real z, zlo;
    if constexpr (sizeof(Real) == 4) {
      CnArgs q;
      q.za[0] = a.za[0]; q.za[1] = a.za[1];
      q.zb[0] = a.zb[0]; q.zb[1] = a.zb[1];
      q.zc[0] = a.zc[0]; q.zc[1] = a.zc[1];
      q.zd[0] = 0.0f; q.zd[1] = 0.0f;
      cn_z<float>(q, mi, a.lo2 + (int32_t)n, z, zlo);
    } else {
      const double md = (double)mi, nd = (double)(a.lo2 + n);
      z = a.zad * md * md + a.zbd * md * nd + a.zcd * nd * nd;
      zlo = 0;
    }
    (void)zlo;
    const Real rr = (Real)1 / ((Real)1 + z * z);
    C y;
    y.x = (num.x + z * num.y) * rr;
    y.y = (num.y - z * num.x) * rr;
    dst[n * a.pitch + m] = y;
  }
}

template <typename Real> cudaError_t launch_si(const SiArgs& a, cudaStream_t st) {
  if (a.hb1 > kCnMaxBand || a.hb2 > kCnMaxBand) return cudaErrorInvalidValue;
  if (a.M1 <= 0 || a.M2 <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((a.M1 + 255) / 256), (unsigned)((a.M2 + kSiRows - 1) / kSiRows));
  si_kernel<Real><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_si<float>(const SiArgs&, cudaStream_t);
template cudaError_t launch_si<double>(const SiArgs&, cudaStream_t);

size_t cn_smem_bytes(const CnArgs& a, size_t elem_bytes) {
  // two tile buffers, each with kCnMaxBand * W zero entries on both sides
  return 2 * ((size_t)a.W * (size_t)(a.TI + 2 * a.halo) + 2 * (size_t)kCnMaxBand * a.W) * elem_bytes;
}

template <typename Real> cudaError_t launch_cn(const CnArgs& a, cudaStream_t st) {
  using C = typename CT<Real>::C;
  if (a.W < 1 || a.TI < 1 || a.W * (a.TI + 2 * a.halo) > 256 * kCnPerThread || a.hb > kCnMaxBand ||
      (a.W & (a.W - 1)) != 0 || (!a.strided && a.W != 1))
    return cudaErrorInvalidValue;
  const int64_t groups = (a.nslices + a.W - 1) / a.W;
  const int64_t blocks = groups * a.nchunks;
  if (blocks <= 0) return cudaSuccess;
  const size_t smem = cn_smem_bytes(a, sizeof(C));
  const bool one = a.hb <= 1;
  if (a.strided) {
    if (one) cn_pass_kernel<Real, true, 1><<<(unsigned)blocks, 256, smem, st>>>(a);
    else cn_pass_kernel<Real, true, kCnMaxBand><<<(unsigned)blocks, 256, smem, st>>>(a);
  } else {
    if (one) cn_pass_kernel<Real, false, 1><<<(unsigned)blocks, 256, smem, st>>>(a);
    else cn_pass_kernel<Real, false, kCnMaxBand><<<(unsigned)blocks, 256, smem, st>>>(a);
  }
  return cudaGetLastError();
}

template <typename Real> cudaError_t cn_prepare(size_t max_smem) {
  cudaError_t e = allow_smem(cn_pass_kernel<Real, true, 1>, max_smem);
  if (e == cudaSuccess) e = allow_smem(cn_pass_kernel<Real, true, kCnMaxBand>, max_smem);
  if (e == cudaSuccess) e = allow_smem(cn_pass_kernel<Real, false, 1>, max_smem);
  if (e == cudaSuccess) e = allow_smem(cn_pass_kernel<Real, false, kCnMaxBand>, max_smem);
  return e;
}

template cudaError_t launch_cn<float>(const CnArgs&, cudaStream_t);
template cudaError_t launch_cn<double>(const CnArgs&, cudaStream_t);
template cudaError_t cn_prepare<float>(size_t);
template cudaError_t cn_prepare<double>(size_t);

}  // namespace lsk
