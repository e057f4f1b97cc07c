// CUDA kernels of the layer-split stepper (sm_103a).
//
// One launch of pass_kernel applies one layer factor of the splitting to the
// whole lifted array (Algorithm 3 steps 1-5 for layer j, with the kinetic
// factors on either side fused in):
//
//   for every slice (fixed index of the other layer):
//     x_i    <- psi_i * exp(-i u_pre s_K |k|^2/2)          kinetic pre-phase
//     y_p    <- sum_i x_i exp(+2 pi i i p / q)             to layer j's grid
//     y_p    <- y_p * exp(-i s v_j(x_p)) / q               potential phase
//     x_k    <- sum_p y_p exp(-2 pi i p k / q)             back to coefficients
//     psi_k  <- x_k * exp(-i u_post s_K |k|^2/2)           kinetic post-phase
//
// The whole slice (or a tile of W slices) lives in shared memory, so a pass is
// one read and one write of the array.  Transforms are radix-8/4/2 Stockham
// FFTs in shared memory; slice lengths that are not powers of two use
// Bluestein's chirp-z identity with a power-of-two convolution of length
// np >= 2q - 2 (the chirp is even, so index q-1 and np-(q-1) may coincide).
// Between the inverse and the forward Bluestein transform the chirps cancel.
//
// Kinetic phases are exact: the phase of |k|^2/2 in turns is a quadratic form
// in the integer indices with coefficients held as 64-bit fixed-point
// fractions (2^-64 turns), so reduction modulo one turn is integer
// wrap-around; only the final sub-quadrant angle goes through sincospi.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lsplit_internal.h"

namespace lsk {

template <typename Real> struct CT;
template <> struct CT<float> { using C = float2; };
template <> struct CT<double> { using C = double2; };

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C> __device__ __forceinline__ C cmulconj(C a, C b) {  // a * conj(b)
  C r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C czero() { C r; r.x = 0; r.y = 0; return r; }

// Shared-memory padding: one spare element after every 16 breaks the
// power-of-two strides of the first Stockham stages across banks.
__device__ __forceinline__ int phys(int i) { return i + (i >> 4); }

// exp(2 pi i t / 2^64) for a fixed-point angle t.  The nearest quadrant is
// removed exactly with integer arithmetic; the remainder (|angle| <= pi/4)
// goes to sincospi.
template <typename Real> __device__ __forceinline__ typename CT<Real>::C phase_of(uint64_t t);
template <> __device__ __forceinline__ float2 phase_of<float>(uint64_t t) {
  const uint64_t q = (t + (1ull << 61)) >> 62;
  const int64_t r = (int64_t)(t - (q << 62));
  const float x = (float)(int)(r >> 32) * 0x1p-31f;  // units of pi
  float s, c;
  sincospif(x, &s, &c);
  switch (q & 3) {
    case 0: return make_float2(c, s);
    case 1: return make_float2(-s, c);
    case 2: return make_float2(-c, -s);
    default: return make_float2(s, -c);
  }
}
template <> __device__ __forceinline__ double2 phase_of<double>(uint64_t t) {
  const uint64_t q = (t + (1ull << 61)) >> 62;
  const int64_t r = (int64_t)(t - (q << 62));
  const double x = (double)r * 0x1p-63;
  double s, c;
  sincospi(x, &s, &c);
  switch (q & 3) {
    case 0: return make_double2(c, s);
    case 1: return make_double2(-s, c);
    case 2: return make_double2(-c, -s);
    default: return make_double2(s, -c);
  }
}

// ---------------------------------------------------------------- radix DFTs
// exp(-2 pi i k / 8) components for k = 0..7 (cos, sin of multiples of pi/4).
#define LS_R2 0.70710678118654752440
template <typename C, bool INV> __device__ __forceinline__ C rot8(C v, int k) {
  // multiply by exp(-+ 2 pi i k / 8) (minus for forward, plus for INV)
  typedef decltype(v.x) R;
  const R h = (R)LS_R2;
  C r;
  switch (k & 7) {
    case 0: return v;
    case 1: r.x = h * (v.x + (INV ? -v.y : v.y)); r.y = h * (v.y + (INV ? v.x : -v.x)); return r;
    case 2: r.x = INV ? -v.y : v.y; r.y = INV ? v.x : -v.x; return r;
    case 3: r.x = h * (-v.x + (INV ? -v.y : v.y)); r.y = h * (-v.y + (INV ? v.x : -v.x)); return r;
    default: return v;  // unused
  }
}

template <typename C, bool INV> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}
template <typename C, bool INV> __device__ __forceinline__ void dft4(C* v) {
  // natural order in and out
  C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
  C b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
  b1 = rot8<C, INV>(b1, 2);
  v[0] = cadd(a0, b0);
  v[2] = csub(a0, b0);
  v[1] = cadd(a1, b1);
  v[3] = csub(a1, b1);
}
template <typename C, bool INV> __device__ __forceinline__ void dft8(C* v) {
  C e[4] = {v[0], v[2], v[4], v[6]};
  C o[4] = {v[1], v[3], v[5], v[7]};
  dft4<C, INV>(e);
  dft4<C, INV>(o);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    C t = rot8<C, INV>(o[k], k);
    v[k] = cadd(e[k], t);
    v[k + 4] = csub(e[k], t);
  }
}
template <int R, typename C, bool INV> __device__ __forceinline__ void dftR(C* v) {
  if constexpr (R == 2) dft2<C, INV>(v[0], v[1]);
  else if constexpr (R == 4) dft4<C, INV>(v);
  else dft8<C, INV>(v);
}

// ---------------------------------------------------------------- Stockham FFT
// Batched in-place FFT of length n over W slices in shared memory.  Slice w's
// buffer starts at w * sb; transform t of a slice has elements at logical
// offsets t * bs + e * es (e = 0..n-1), physical index phys(logical).
// JFAST: consecutive threads take consecutive butterflies of one transform
// (es == 1); otherwise consecutive threads take consecutive transforms.
struct FftGeo {
  int W, sb, n, nbatch, es, bs;
};

template <typename Real, int R, bool INV, bool JFAST, int BPT>
__device__ __forceinline__ void fft_stage(typename CT<Real>::C* sm, const FftGeo& f, int ns,
                                          const typename CT<Real>::C* __restrict__ tw) {
  using C = typename CT<Real>::C;
  const int nR = f.n / R;
  const int total = f.W * f.nbatch * nR;
  const int tstride = f.n / (ns * R);
  C v[BPT][R];
  int dst[BPT];
#pragma unroll
  for (int u = 0; u < BPT; ++u) {
    const int b = threadIdx.x + u * blockDim.x;
    dst[u] = -1;
    if (b < total) {
      int j, t, w;
      if (JFAST) {
        j = b % nR;
        const int rest = b / nR;
        t = rest % f.nbatch;
        w = rest / f.nbatch;
      } else {
        t = b % f.nbatch;
        const int rest = b / f.nbatch;
        j = rest % nR;
        w = rest / nR;
      }
      const int base = w * f.sb;
      const int off = t * f.bs;
      const int k = j & (ns - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) v[u][r] = sm[base + phys(off + (j + r * nR) * f.es)];
      if (ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w0 = tw[r * k * tstride];
          v[u][r] = INV ? cmulconj(v[u][r], w0) : cmul(v[u][r], w0);
        }
      }
      dftR<R, C, INV>(v[u]);
      dst[u] = b;  // the store position is recomputed from b after the barrier
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < BPT; ++u) {
    const int b = dst[u];
    if (b >= 0) {
      int j, t, w;
      if (JFAST) {
        j = b % nR;
        const int rest = b / nR;
        t = rest % f.nbatch;
        w = rest / f.nbatch;
      } else {
        t = b % f.nbatch;
        const int rest = b / f.nbatch;
        j = rest % nR;
        w = rest / nR;
      }
      const int base = w * f.sb;
      const int off = t * f.bs;
      const int k = j & (ns - 1);
      const int i0 = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) sm[base + phys(off + (i0 + r * ns) * f.es)] = v[u][r];
    }
  }
  __syncthreads();
}

// Stage plan: 3 bits per stage, ending in 2+2 or 1 bit (radix >= 4 unless n = 2).
__host__ __device__ __forceinline__ int stage_bits(int rem) {
  if (rem == 4 || rem == 2) return 2;
  if (rem == 1) return 1;
  return 3;
}

template <typename Real, bool INV, bool JFAST, int BPT>
__device__ void fft_all(typename CT<Real>::C* sm, const FftGeo& f, const typename CT<Real>::C* tw) {
  int rem = 31 - __clz(f.n);
  int ns = 1;
  while (rem > 0) {
    const int bits = stage_bits(rem);
    // radix-8 stages have half the butterflies of a radix-4 stage: BPT/2 suffices
    if (bits == 3) fft_stage<Real, 8, INV, JFAST, (BPT > 1 ? BPT / 2 : 1)>(sm, f, ns, tw);
    else if (bits == 2) fft_stage<Real, 4, INV, JFAST, BPT>(sm, f, ns, tw);
    else fft_stage<Real, 2, INV, JFAST, BPT * 2>(sm, f, ns, tw);
    ns <<= bits;
    rem -= bits;
  }
}

// ---------------------------------------------------------------- pass kernel
// Threads per CTA bound: register arrays hold 8 * BPT reals per thread.
template <typename Real, int BPT> struct PassTraits {
  static constexpr int kMaxNT = (sizeof(Real) == 4 ? 2048 : 1024) / BPT;
};

__device__ __forceinline__ uint64_t quad_turns(const LayerGeom& g, int64_t mua, int64_t mub,
                                               uint64_t la, uint64_t lb, uint64_t c0) {
  const uint64_t a = (uint64_t)mua, b = (uint64_t)mub;
  return g.A_aa * (a * a) + g.A_ab * (a * b) + g.A_bb * (b * b) + la * a + lb * b + c0;
}

template <typename Real, bool INV, int BPT>
__device__ __forceinline__ void transform(typename CT<Real>::C* sm, const LayerGeom& g, int W,
                                          bool bluestein_half_fwd) {
  using C = typename CT<Real>::C;
  (void)bluestein_half_fwd;
  if (g.d == 1) {
    FftGeo f{W, g.sb, g.np, 1, 1, 0};
    fft_all<Real, INV, true, BPT>(sm, f, (const C*)g.tw);
  } else {
    FftGeo fa{W, g.sb, g.qa, g.qb, 1, g.qa};
    fft_all<Real, INV, true, BPT>(sm, fa, (const C*)g.tw);
    FftGeo fb{W, g.sb, g.qb, g.qa, g.qa, 1};
    fft_all<Real, INV, false, BPT>(sm, fb, (const C*)g.twb);
  }
}

// Bluestein convolution on every slice: x <- IFFT(FFT(x) * tab) (tab has the 1/np).
template <typename Real, int BPT>
__device__ __forceinline__ void bluestein_conv(typename CT<Real>::C* sm, const LayerGeom& g, int W,
                                               const typename CT<Real>::C* __restrict__ tab) {
  using C = typename CT<Real>::C;
  FftGeo f{W, g.sb, g.np, 1, 1, 0};
  fft_all<Real, false, true, BPT>(sm, f, (const C*)g.tw);
  for (int e = threadIdx.x; e < W * g.np; e += blockDim.x) {
    const int w = e / g.np, k = e - w * g.np;
    const int pi = w * g.sb + phys(k);
    sm[pi] = cmul(sm[pi], tab[k]);
  }
  __syncthreads();
  fft_all<Real, true, true, BPT>(sm, f, (const C*)g.tw);
}

template <typename Real, int BPT>
__global__ void __launch_bounds__(PassTraits<Real, BPT>::kMaxNT)
pass_kernel(const PassArgs a) {
  using C = typename CT<Real>::C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const LayerGeom& g = a.g;
  const int W = a.W;
  C* sml = sm + (size_t)W * g.sb;  // adjoint: lambda tile
  __shared__ int64_t s_slice[kMaxTileSlices];
  __shared__ uint64_t s_la[kMaxTileSlices], s_lb[kMaxTileSlices], s_c0[kMaxTileSlices];
  __shared__ int32_t s_touch[kMaxTileSlices];
  __shared__ double s_red[32];

  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  const bool adj = (a.mode == MODE_ADJOINT);
  const bool lazy = (a.mode == MODE_LAZY);
  const bool kin_only = (a.mode == MODE_KIN);
  const bool measure = (a.mode == MODE_MEASURE);

  if (tid < W) {
    int64_t s = -1;
    if (a.list) {
      const int64_t li = (int64_t)blockIdx.x * W + tid;
      if (li < a.nlist) s = a.list[li];
    } else {
      s = (int64_t)blockIdx.x * W + tid;
      if (s >= g.nslices) s = -1;
    }
    s_slice[tid] = s;
    uint64_t la = 0, lb = 0, c0 = 0;
    int32_t touch = 0;
    if (s >= 0) {
      const int64_t nua = s % g.oqa + g.olo_a;
      const int64_t nub = s / g.oqa + g.olo_b;
      const uint64_t ua = (uint64_t)nua, ub = (uint64_t)nub;
      la = g.X_aa * ua + g.X_ab * ub;
      lb = g.X_ba * ua + g.X_bb * ub;
      c0 = g.C_aa * (ua * ua) + g.C_ab * (ua * ub) + g.C_bb * (ub * ub);
      if (lazy || kin_only) touch = a.touch_own[s];
    }
    s_la[tid] = la;
    s_lb[tid] = lb;
    s_c0[tid] = c0;
    s_touch[tid] = touch;
  }
  __syncthreads();

  C* psi = reinterpret_cast<C*>(a.psi);
  C* lam = reinterpret_cast<C*>(a.lam);
  const int M = g.M;
  const int q = g.qa;  // 1D slice length (chirp index range)

  // ---- load + kinetic pre-phase (+ Bluestein pre-chirp)
  for (int e = tid; e < W * M; e += NT) {
    int w, i;
    if (a.strided) { w = e % W; i = e / W; } else { w = e / M; i = e - w * M; }
    const int64_t s = s_slice[w];
    C x = czero<C>(), xl = czero<C>();
    if (s >= 0) {
      const int ia = i % g.qa, ib = i / g.qa;
      const int64_t off = s * g.slice_stride + ia * g.ea + ib * g.eb;
      x = psi[off];
      if (adj) xl = lam[off];
      if (!measure) {
        const uint64_t qd = quad_turns(g, g.lo_a + ia, g.lo_b + ib, s_la[w], s_lb[w], s_c0[w]);
        int64_t units = a.units_pre;
        if (lazy || kin_only) {
          const int32_t t2 = a.touch_other[i];
          units = (int64_t)a.now - (int64_t)(s_touch[w] > t2 ? s_touch[w] : t2);
        }
        uint64_t t = (uint64_t)0 - (uint64_t)units * qd;
        if (g.bluestein && !kin_only) t += (uint64_t)(((int64_t)i * i) % g.two_q) * g.chirp_unit;
        const C ph = phase_of<Real>(t);
        x = cmul(x, ph);
        if (adj) xl = cmul(xl, ph);
      } else if (g.bluestein) {
        const C ph = phase_of<Real>((uint64_t)(((int64_t)i * i) % g.two_q) * g.chirp_unit);
        x = cmul(x, ph);
      }
    }
    if (kin_only) {
      if (s >= 0) {
        const int ia = i % g.qa, ib = i / g.qa;
        psi[s * g.slice_stride + ia * g.ea + ib * g.eb] = x;
      }
      continue;
    }
    sm[w * g.sb + phys(i)] = x;
    if (adj) sml[w * g.sb + phys(i)] = xl;
  }
  if (kin_only) return;
  if (g.bluestein) {
    const int pad = g.np - q;
    for (int e = tid; e < W * pad; e += NT) {
      const int w = e / pad, i = q + (e - w * pad);
      sm[w * g.sb + phys(i)] = czero<C>();
      if (adj) sml[w * g.sb + phys(i)] = czero<C>();
    }
  }
  __syncthreads();

  // ---- to layer j's real-space grid (unnormalised inverse transform)
  if (g.bluestein) {
    bluestein_conv<Real, BPT>(sm, g, W, (const C*)g.bm);
    if (adj) bluestein_conv<Real, BPT>(sml, g, W, (const C*)g.bm);
  } else {
    transform<Real, true, BPT>(sm, g, W, false);
    if (adj) transform<Real, true, BPT>(sml, g, W, false);
  }

  // ---- pointwise potential factor (or measurement / gradient)
  if (measure) {
    double acc = 0.0;
    for (int e = tid; e < W * M; e += NT) {
      const int w = e / M, p = e - w * M;
      if (s_slice[w] < 0) continue;
      const C y = sm[w * g.sb + phys(p)];
      acc += g.vgrid[p] * ((double)y.x * y.x + (double)y.y * y.y);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = acc;
    __syncthreads();
    if (tid < 32) {
      double v = tid < (NT + 31) / 32 ? s_red[tid] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (tid == 0) a.partials[blockIdx.x] = v / (double)M;
    }
    return;
  }
  {
    const C* T = reinterpret_cast<const C*>(a.T);
    const int span = g.bluestein ? g.np : M;
    for (int e = tid; e < W * span; e += NT) {
      const int w = e / span, p = e - w * span;
      const int pi = w * g.sb + phys(p);
      if (p >= M) {
        sm[pi] = czero<C>();
        if (adj) sml[pi] = czero<C>();
        continue;
      }
      const C tp = T[p];
      if (adj) {
        if (s_slice[w] >= 0) {
          const C yp = sm[pi], yl = sml[pi];
          // dL/dv_p += 2 s Im(conj(mu_p) psi_p), mu, psi unitary transforms (1/M)
          const double im = (double)yl.x * yp.y - (double)yl.y * yp.x;
          atomicAdd(&a.grad[p], 2.0 * a.sdur * im / (double)M);
        }
        sml[pi] = cmul(sml[pi], tp);
      }
      sm[pi] = cmul(sm[pi], tp);
    }
    __syncthreads();
  }

  // ---- back to coefficients (forward transform; 1/M is folded into T)
  if (g.bluestein) {
    bluestein_conv<Real, BPT>(sm, g, W, (const C*)g.bp);
    if (adj) bluestein_conv<Real, BPT>(sml, g, W, (const C*)g.bp);
  } else {
    transform<Real, false, BPT>(sm, g, W, false);
    if (adj) transform<Real, false, BPT>(sml, g, W, false);
  }

  // ---- store + kinetic post-phase (+ Bluestein post-chirp)
  for (int e = tid; e < W * M; e += NT) {
    int w, i;
    if (a.strided) { w = e % W; i = e / W; } else { w = e / M; i = e - w * M; }
    const int64_t s = s_slice[w];
    if (s < 0) continue;
    const int ia = i % g.qa, ib = i / g.qa;
    const int64_t off = s * g.slice_stride + ia * g.ea + ib * g.eb;
    uint64_t t = 0;
    if (!lazy && a.units_post != 0) {
      const uint64_t qd = quad_turns(g, g.lo_a + ia, g.lo_b + ib, s_la[w], s_lb[w], s_c0[w]);
      t = (uint64_t)0 - (uint64_t)a.units_post * qd;
    }
    if (g.bluestein) t -= (uint64_t)(((int64_t)i * i) % g.two_q) * g.chirp_unit;
    C x = sm[w * g.sb + phys(i)];
    if (t != 0) {
      const C ph = phase_of<Real>(t);
      x = cmul(x, ph);
      if (adj) lam[off] = cmul(sml[w * g.sb + phys(i)], ph);
    } else if (adj) {
      lam[off] = sml[w * g.sb + phys(i)];
    }
    psi[off] = x;
  }
  if (lazy && tid < W && s_slice[tid] >= 0) a.touch_own[s_slice[tid]] = a.now;
}

int pass_threads(const LayerGeom& g, int W, int bpt) {
  // Largest butterfly count over all stages of all transforms of a pass.
  auto worst = [&](int n, int nbatch) {
    int rem = 0;
    while ((1 << rem) < n) ++rem;
    int most = 0;
    while (rem > 0) {
      const int bits = stage_bits(rem);
      const int R = 1 << bits;
      const int per = (bits == 3) ? (bpt > 1 ? bpt / 2 : 1) : (bits == 2 ? bpt : bpt * 2);
      const int need = (W * nbatch * (n / R) + per - 1) / per;
      if (need > most) most = need;
      rem -= bits;
    }
    return most;
  };
  int nt = (g.d == 1) ? worst(g.np, 1) : (worst(g.qa, g.qb) > worst(g.qb, g.qa) ? worst(g.qa, g.qb) : worst(g.qb, g.qa));
  if (nt < 64) nt = 64;
  nt = (nt + 31) / 32 * 32;
  return nt;
}

template <typename Real> size_t pass_smem_bytes(const LayerGeom& g, int W, int mode) {
  using C = typename CT<Real>::C;
  return (size_t)W * g.sb * sizeof(C) * (mode == MODE_ADJOINT ? 2 : 1);
}

template <typename Real> cudaError_t pass_prepare(size_t max_smem) {
  cudaError_t e = cudaFuncSetAttribute(pass_kernel<Real, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(pass_kernel<Real, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
}

template <typename Real> cudaError_t launch_pass(const PassArgs& a, int bpt, int nthreads, int64_t ntiles,
                                                 cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  const size_t smem = pass_smem_bytes<Real>(a.g, a.W, a.mode);
  if (bpt == 4) pass_kernel<Real, 4><<<(unsigned)ntiles, nthreads, smem, st>>>(a);
  else pass_kernel<Real, 2><<<(unsigned)ntiles, nthreads, smem, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- elementwise kernels
struct Idx {
  int64_t n, m;
};

__device__ __forceinline__ void decode_mn(const ElemArgs& e, int64_t row, int64_t col, double* mv,
                                          double* nv) {
  mv[0] = (double)(col % e.q1a + e.lo1a);
  mv[1] = (double)(col / e.q1a + e.lo1b);
  nv[0] = (double)(row % e.q2a + e.lo2a);
  nv[1] = (double)(row / e.q2a + e.lo2b);
}

// k = B1 m + B2 n with the operation order of the index-set predicate,
// without contraction (explicit round-to-nearest intrinsics).
__device__ __forceinline__ void kvec(const ElemArgs& e, const double* mv, const double* nv, double* k) {
  for (int i = 0; i < e.d; ++i) {
    double acc = __dmul_rn(e.B1[i * e.d + 0], mv[0]);
    for (int j = 1; j < e.d; ++j) acc = __dadd_rn(acc, __dmul_rn(e.B1[i * e.d + j], mv[j]));
    for (int j = 0; j < e.d; ++j) acc = __dadd_rn(acc, __dmul_rn(e.B2[i * e.d + j], nv[j]));
    k[i] = acc;
  }
}
__device__ __forceinline__ double half_k2(const ElemArgs& e, const double* k) {
  double acc = __dmul_rn(k[0], k[0]);
  for (int i = 1; i < e.d; ++i) acc = __dadd_rn(acc, __dmul_rn(k[i], k[i]));
  return __dmul_rn(0.5, acc);
}

template <typename Real>
__global__ void gaussian_kernel(const ElemArgs e, typename CT<Real>::C* psi, double x00, double x01,
                                double w, double k00, double k01, double* partials) {
  using C = typename CT<Real>::C;
  double acc = 0.0;
  const int64_t total = e.M1 * e.M2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / e.M1, col = idx - row * e.M1;
    double mv[2], nv[2], k[2] = {0, 0};
    decode_mn(e, row, col, mv, nv);
    kvec(e, mv, nv, k);
    const bool in = half_k2(e, k) <= e.ecut;
    double re = 0, im = 0;
    if (in) {
      const double d0 = k[0] - k00, d1 = (e.d > 1) ? k[1] - k01 : 0.0;
      const double amp = exp(-0.5 * w * w * (d0 * d0 + d1 * d1));
      const double kx = k[0] * x00 + ((e.d > 1) ? k[1] * x01 : 0.0);
      double s, c;
      sincos(kx, &s, &c);
      re = amp * c;
      im = -amp * s;
      acc += re * re + im * im;
    }
    C v;
    v.x = (Real)re;
    v.y = (Real)im;
    psi[row * e.pitch + col] = v;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) partials[blockIdx.x * kObsQ] = v;
  }
}

template <typename Real>
__global__ void scale_kernel(const ElemArgs e, typename CT<Real>::C* psi, const double* sumsq) {
  const double f = 1.0 / sqrt(sumsq[0]);
  const int64_t total = e.M1 * e.M2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / e.M1, col = idx - row * e.M1;
    auto v = psi[row * e.pitch + col];
    v.x = (Real)(v.x * f);
    v.y = (Real)(v.y * f);
    psi[row * e.pitch + col] = v;
  }
}

template <typename Real>
__global__ void elem_obs_kernel(const ElemArgs e, const typename CT<Real>::C* psi,
                                const typename CT<Real>::C* chi, double* partials) {
  double acc[kObsQ];
#pragma unroll
  for (int i = 0; i < kObsQ; ++i) acc[i] = 0.0;
  const int64_t total = e.M1 * e.M2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / e.M1, col = idx - row * e.M1;
    const auto v = psi[row * e.pitch + col];
    const double re = v.x, im = v.y;
    const double a2 = re * re + im * im;
    double mv[2], nv[2], k[2] = {0, 0};
    decode_mn(e, row, col, mv, nv);
    kvec(e, mv, nv, k);
    acc[0] += a2;
    acc[1] += half_k2(e, k) * a2;
    acc[2] += k[0] * a2;
    acc[3] += k[1] * a2;
    if (chi) {
      const auto c = chi[row * e.pitch + col];
      acc[4] += (double)c.x * re + (double)c.y * im;
      acc[5] += (double)c.x * im - (double)c.y * re;
    }
  }
  __shared__ double red[32][kObsQ];
#pragma unroll
  for (int q = 0; q < kObsQ; ++q) {
    double x = acc[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < kObsQ) {
    double x = 0.0;
    for (int wv = 0; wv < (int)(blockDim.x + 31) / 32; ++wv) x += red[wv][threadIdx.x];
    partials[blockIdx.x * kObsQ + threadIdx.x] = x;
  }
}

// Sum partials[nparts][nq] over parts in a fixed order (deterministic).
__global__ void reduce_kernel(const double* partials, int nparts, int nq, double* out) {
  __shared__ double red[32];
  for (int q = 0; q < nq; ++q) {
    double x = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) x += partials[(int64_t)i * nq + q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (threadIdx.x == 0) out[q] = v;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- stochastic sampler
// SplitMix64 (Steele, Lea & Flood 2014) driving a partial Fisher-Yates shuffle;
// one block per sub-step g = g0 + blockIdx.x, output sorted ascending.
__device__ __forceinline__ uint64_t splitmix64_next(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void sampler_kernel(SamplerArgs sa, const uint64_t* seed_g0, int32_t* out) {
  extern __shared__ int32_t perm[];  // Smax ints, then Smax flag bytes
  const int64_t rel = blockIdx.x;
  const int layer = sa.pattern[rel % sa.npf];
  const int S = layer == 1 ? sa.S1 : sa.S2;
  const int p = layer == 1 ? sa.p1 : sa.p2;
  unsigned char* flag = reinterpret_cast<unsigned char*>(perm + sa.Smax);
  const uint64_t seed = seed_g0 ? seed_g0[0] : sa.seed;
  const uint64_t g = (seed_g0 ? seed_g0[1] : sa.g0) + (uint64_t)rel;
  for (int i = threadIdx.x; i < S; i += blockDim.x) {
    perm[i] = i;
    flag[i] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t state = seed ^ (g * 0xD1B54A32D192ED03ull);
    for (int i = 0; i < p; ++i) {
      const uint64_t r = splitmix64_next(state);
      const int j = i + (int)(r % (uint64_t)(S - i));
      const int t = perm[i];
      perm[i] = perm[j];
      perm[j] = t;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += blockDim.x) flag[perm[i]] = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t* o = out + rel * sa.pmax;
    int c = 0;
    for (int i = 0; i < S; ++i)
      if (flag[i]) o[c++] = i;
  }
}

__global__ void zero_i32_kernel(int32_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0;
}
__global__ void zero_f64_kernel(double* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0.0;
}

template <typename Real>
cudaError_t launch_gaussian(const ElemArgs& e, void* psi, const double* x0, double w, const double* k0,
                            double* partials, int nblocks, cudaStream_t st) {
  gaussian_kernel<Real><<<nblocks, 256, 0, st>>>(e, reinterpret_cast<typename CT<Real>::C*>(psi), x0[0],
                                                 e.d > 1 ? x0[1] : 0.0, w, k0[0], e.d > 1 ? k0[1] : 0.0,
                                                 partials);
  return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_scale(const ElemArgs& e, void* psi, const double* sumsq, cudaStream_t st) {
  scale_kernel<Real><<<kReduceBlocks, 256, 0, st>>>(e, reinterpret_cast<typename CT<Real>::C*>(psi), sumsq);
  return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_elem_obs(const ElemArgs& e, const void* psi, const void* chi, double* partials, int nblocks,
                            cudaStream_t st) {
  using C = typename CT<Real>::C;
  elem_obs_kernel<Real><<<nblocks, 256, 0, st>>>(e, reinterpret_cast<const C*>(psi),
                                                 reinterpret_cast<const C*>(chi), partials);
  return cudaGetLastError();
}
cudaError_t launch_reduce(const double* partials, int nparts, int nq, double* out, cudaStream_t st) {
  reduce_kernel<<<1, 1024, 0, st>>>(partials, nparts, nq, out);
  return cudaGetLastError();
}
cudaError_t launch_sampler(const SamplerArgs& sa, const uint64_t* seed_g0_dev, int32_t count, int32_t* out,
                           cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = (size_t)sa.Smax * 5;
  sampler_kernel<<<count, 256, smem, st>>>(sa, seed_g0_dev, out);
  return cudaGetLastError();
}
cudaError_t sampler_prepare(size_t smem) {
  return cudaFuncSetAttribute(sampler_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
cudaError_t launch_zero_i32(int32_t* p, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  zero_i32_kernel<<<256, 256, 0, st>>>(p, n);
  return cudaGetLastError();
}
cudaError_t launch_zero_f64(double* p, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  zero_f64_kernel<<<256, 256, 0, st>>>(p, n);
  return cudaGetLastError();
}

#define LS_INST(R)                                                                                        \
  template cudaError_t launch_pass<R>(const PassArgs&, int, int, int64_t, cudaStream_t);                 \
  template size_t pass_smem_bytes<R>(const LayerGeom&, int, int);                                        \
  template cudaError_t pass_prepare<R>(size_t);                                                          \
  template cudaError_t launch_gaussian<R>(const ElemArgs&, void*, const double*, double, const double*, \
                                          double*, int, cudaStream_t);                                   \
  template cudaError_t launch_scale<R>(const ElemArgs&, void*, const double*, cudaStream_t);             \
  template cudaError_t launch_elem_obs<R>(const ElemArgs&, const void*, const void*, double*, int,      \
                                          cudaStream_t);
LS_INST(float)
LS_INST(double)

}  // namespace lsk

namespace lsk {
template <typename Real> int pass_max_threads(int bpt) {
  return bpt == 4 ? PassTraits<Real, 4>::kMaxNT : PassTraits<Real, 2>::kMaxNT;
}
template int pass_max_threads<float>(int);
template int pass_max_threads<double>(int);
}  // namespace lsk
