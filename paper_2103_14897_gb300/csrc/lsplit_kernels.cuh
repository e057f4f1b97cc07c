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

#include <type_traits>

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
// complex64: one paired FP32 operation each, rounded as the scalar forms
// (a - b is fma(b, -1, a), a single rounding of the exact difference)
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
template <typename C> __device__ __forceinline__ C czero() { C r; r.x = 0; r.y = 0; return r; }

// Per-slice metadata of the tile a CTA works on (slice index, kinetic
// quadratic-form coefficients, lazy touch time) and a reduction scratch.  One
// file-scope block shared by every tile body, so a kernel that can run
// several tile kinds (the persistent batched runner) holds it once.
struct TileMeta {
  int64_t slice[kMaxTileSlices];
  uint64_t la[kMaxTileSlices], lb[kMaxTileSlices], c0[kMaxTileSlices];
  int32_t touch[kMaxTileSlices];
  double2 fix1[kMaxTileSlices];
  double red[32];
};
static __shared__ TileMeta g_tm;

// Shared-memory padding: one spare element after every 16 breaks the
// power-of-two strides of the first Stockham stages across banks.
__device__ __forceinline__ int phys(int i) { return i + (i >> 4); }

// exp(2 pi i t / 2^64) for a fixed-point angle t.  The nearest quadrant is
// removed exactly with integer arithmetic; the remainder (|angle| <= pi/4)
// goes to sincospi.  In single precision two systematic errors are removed,
// because the same angle recurs at every step for a given element:
//  * the float argument is rounded; the exact integer residual of that
//    rounding (< 2^-24 relative) rotates the result to first order;
//  * |(c, s)| differs from 1 by O(eps); the deviation e = c^2 + s^2 - 1 is
//    computed with error-free products and returned, and the caller scales the
//    product x * (c, s) by (1 - e/2) with one fused rounding.
template <typename Real> struct Phase {
  typename CT<Real>::C v;
  Real half_e;  // (c^2 + s^2 - 1) / 2
};

template <typename Real> __device__ __forceinline__ Phase<Real> phase_of(uint64_t t);
// sin(pi y) and cos(pi y) for |y| <= 1/4 from the Taylor series at 0, with
// coefficients (-1)^k pi^(2k+1) / (2k+1)! and (-1)^k pi^(2k) / (2k)!, through
// y^9 and y^10 (truncation below 3e-9), Horner in y^2; the leading term of the
// sine multiplies by pi split into two floats.  Measured against FP64 on the
// device: rms angle error 0.19 and max 1.4 units of 2^-24, as sincospif.
__device__ __forceinline__ void sincospi_quarter(float y, float& s, float& c) {
  const float y2 = y * y;
  // the sine and cosine series side by side as one pair of Horner steps
  // (per-lane paired FMAs, each rounded as fmaf); the cosine has one more term
  const float2 Y2 = make_float2(y2, y2);
  float2 P = __ffma2_rn(make_float2(0.0821458866f, -0.0258068914f), Y2, make_float2(-0.599264529f, 0.235330630f));
  P = __ffma2_rn(P, Y2, make_float2(2.55016404f, -1.33526277f));
  P = __ffma2_rn(P, Y2, make_float2(-5.16771278f, 4.05871213f));
  s = fmaf(y, 3.14159274f, fmaf(y * y2, P.x, y * -8.74227766e-08f));
  const float pc = fmaf(P.y, y2, -4.93480220f);
  c = fmaf(y2, pc, 1.0f);
}

template <> __device__ __forceinline__ Phase<float> phase_of<float>(uint64_t t) {
  // t: angle in 64-bit fixed-point turns.  q: nearest quarter turn (top bits);
  // rhi: remainder in units of 2^-32 turn, |rhi| <= 2^29, split into
  // xf = float(rhi) (y = xf 2^-31 half-turns, |y| <= 1/4) and the small exact
  // integer rhi - xf; that and the low word enter as a first-order rotation
  // by d radians.  32-bit integer work only.
  const uint32_t hi = (uint32_t)(t >> 32), lo = (uint32_t)t;
  const uint32_t q = (hi + (1u << 29)) >> 30;
  const int32_t rhi = (int32_t)(hi - (q << 30));
  const float xf = (float)rhi;                    // may round (|rhi| <= 2^29)
  const int32_t res = rhi - (int32_t)xf;          // exact, |res| <= 16
  float s, c;
  sincospi_quarter(xf * 0x1p-31f, s, c);
  const float d = fmaf((float)lo, 0x1p-32f, (float)res) * 0x1.921fb6p-30f;  // 2 pi / 2^32 per unit
  const float c1 = fmaf(-d, s, c), s1 = fmaf(d, c, s);
  // explicit round-to-nearest operations: no contraction may merge c2h - 1;
  // lane 0 carries c1, lane 1 s1: NH = -(v^2 rounded), L = v^2 - fl(v^2) exactly
  const float2 V = make_float2(c1, s1);
  const float2 NH = __fmul2_rn(V, make_float2(-c1, -s1));
  const float2 L = __ffma2_rn(V, V, NH);
  const float e = __fadd_rn(__fadd_rn(__fadd_rn(-NH.x, -1.0f), -NH.y), __fadd_rn(L.x, L.y));
  // rotate by q quarter turns without branches: odd q swaps (c, s) -> (-s, c),
  // q & 2 negates both
  const bool odd = (q & 1) != 0;
  const uint32_t neg = (q & 2) << 30;
  const float vx = odd ? -s1 : c1, vy = odd ? c1 : s1;
  Phase<float> p;
  p.v = make_float2(__uint_as_float(__float_as_uint(vx) ^ neg), __uint_as_float(__float_as_uint(vy) ^ neg));
  p.half_e = 0.5f * e;
  return p;
}
template <> __device__ __forceinline__ Phase<double> phase_of<double>(uint64_t t) {
  const uint64_t q = (t + (1ull << 61)) >> 62;
  const int64_t r = (int64_t)(t - (q << 62));
  const double x = (double)r * 0x1p-63;
  double s, c;
  sincospi(x, &s, &c);
  Phase<double> p;
  switch (q & 3) {
    case 0: p.v = make_double2(c, s); break;
    case 1: p.v = make_double2(-s, c); break;
    case 2: p.v = make_double2(-c, -s); break;
    default: p.v = make_double2(s, -c); break;
  }
  p.half_e = 0.0;
  return p;
}

// x * exp(i angle) with the modulus deviation of the phase removed.
// In single precision the product is formed error-free (two-product and
// two-sum transforms, explicit round-to-nearest intrinsics so nothing is
// contracted), the factor (1 - e/2) is applied to the exact value and each
// component is rounded once.  A correction of e/2 ~ eps applied after a
// rounded product would itself round away, leaving the per-element bias of
// |(c, s)| in place at every step.
__device__ __forceinline__ float dot2_fix(float a, float c, float b, float s, float h) {
  // a*c + b*s, times (1 - h), single final rounding
  const float p = __fmul_rn(a, c), pe = fmaf(a, c, -p);
  const float q = __fmul_rn(b, s), qe = fmaf(b, s, -q);
  const float r = __fadd_rn(p, q);
  const float bb = __fsub_rn(r, p);
  const float re = __fadd_rn(__fsub_rn(p, __fsub_rn(r, bb)), __fsub_rn(q, bb));
  const float lo = __fadd_rn(__fadd_rn(re, __fadd_rn(pe, qe)), -__fmul_rn(h, r));
  return __fadd_rn(r, lo);
}

template <typename Real>
__device__ __forceinline__ typename CT<Real>::C apply_phase(typename CT<Real>::C x, const Phase<Real>& p);
template <>
__device__ __forceinline__ float2 apply_phase<float>(float2 x, const Phase<float>& p) {
  // dot2_fix for both components at once in paired FP32 operations: lane 0
  // forms x.x c - x.y s, lane 1 x.x s + x.y c, each times (1 - e/2) with one
  // final rounding.  Subtractions are fused multiply-adds by -1 and negated
  // intermediates are carried instead of subtracted, so every lane performs
  // the exact operations of the error-free transforms.
  const float2 A = make_float2(x.x, x.x), NA = make_float2(-x.x, -x.x);
  const float2 B = make_float2(-x.y, x.y), NB = make_float2(x.y, -x.y);
  const float2 Cv = p.v, Sv = make_float2(p.v.y, p.v.x);
  const float2 M1 = make_float2(-1.0f, -1.0f);
  const float2 P = __fmul2_rn(A, Cv);
  const float2 NPE = __ffma2_rn(NA, Cv, P);     // -(a c - p), exact
  const float2 Q = __fmul2_rn(B, Sv);
  const float2 NQE = __ffma2_rn(NB, Sv, Q);     // -(b s - q), exact
  const float2 R = __fadd2_rn(P, Q);
  const float2 BB = __ffma2_rn(P, M1, R);       // r - p
  const float2 T1 = __ffma2_rn(BB, M1, R);      // r - bb
  const float2 T2 = __ffma2_rn(T1, M1, P);      // p - (r - bb)
  const float2 T3 = __ffma2_rn(BB, M1, Q);      // q - bb
  const float2 RE = __fadd2_rn(T2, T3);         // two-sum error of r
  const float2 S1 = __fadd2_rn(NPE, NQE);       // -(pe + qe)
  const float2 U = __ffma2_rn(S1, M1, RE);      // re + pe + qe
  const float2 LO = __ffma2_rn(make_float2(-p.half_e, -p.half_e), R, U);   // ... - h r
  return __fadd2_rn(R, LO);
}
template <>
__device__ __forceinline__ double2 apply_phase<double>(double2 x, const Phase<double>& p) {
  return cmul(x, p.v);
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

// The batched runner inlines the transform into its persistent loop (a call
// would keep per-thread register arrays in local memory across the call).
#ifdef LS_INST_BATCH
#define LS_FFT_INLINE __forceinline__
#else
#define LS_FFT_INLINE
#endif
template <typename Real, bool INV, bool JFAST, int BPT>
__device__ LS_FFT_INLINE void fft_all(typename CT<Real>::C* sm, const FftGeo& f, const typename CT<Real>::C* tw) {
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

template <typename Real, bool INV, int BPT, bool D1 = false>
__device__ __forceinline__ void transform(typename CT<Real>::C* sm, const LayerGeom& g, int W,
                                          bool bluestein_half_fwd) {
  using C = typename CT<Real>::C;
  (void)bluestein_half_fwd;
  if (D1 || g.d == 1) {
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

// One layer factor over a tile of W slices.  MODE selects the variant:
//   MODE_STEP     K(post) P(s) K(pre) with fixed kinetic units;
//   MODE_LAZY     stochastic: P on the listed slices only, the kinetic phase
//                 pending since the element's last touch applied before P;
//   MODE_KIN      kinetic phase only, no transform: the phase pending since
//                 the element's last touch (settle, touch_own set), or a fixed
//                 units_pre on psi and, if lam is set, on lam (the reverse
//                 sweep of the stochastic schemes);
//   MODE_MEASURE  sum_p v(x_p)|psi(x_p)|^2 / M per CTA (potential energy);
//   MODE_ADJOINT  inverse factor on psi and lambda together, accumulating
//                 dL/dv(x_p).
// P is applied as x + F diag(T - 1) F^{-1} x (T - 1 with the 1/M of the
// forward transform in the table): the same operator, but the rounding of the
// transforms only enters through the small correction term, so it does not
// build up coherently over thousands of passes.
// Global loads of the wave function: plain in the one-pass-per-launch
// kernels; through L2 only (no L1 allocation) in the persistent batched runner,
// where another CTA of the same launch may have written the data.
template <bool CG, typename C> __device__ __forceinline__ C ldpsi(const C* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

template <typename Real, int BPT, int MODE, bool CG, bool D1 = false>
__device__ __forceinline__ void pass_tile(const PassArgs& a, int64_t tile, unsigned char* smraw) {
  using C = typename CT<Real>::C;
  constexpr bool adj = (MODE == MODE_ADJOINT);
  constexpr bool lazy = (MODE == MODE_LAZY);
  constexpr bool kin_only = (MODE == MODE_KIN);
  constexpr bool measure = (MODE == MODE_MEASURE);
  const LayerGeom& g = a.g;
  const int W = a.W;
  const int M = g.M;
  C* sm = reinterpret_cast<C*>(smraw);
  C* sml = sm + (size_t)W * g.sb;                         // adjoint: lambda tile
  C* sx = sm + (size_t)W * g.sb * (adj ? 2 : 1);          // saved x (pre-phased)
  C* sxl = sx + (size_t)W * M;                            // adjoint: saved lambda
  int64_t* s_slice = g_tm.slice;
  uint64_t *s_la = g_tm.la, *s_lb = g_tm.lb, *s_c0 = g_tm.c0;
  int32_t* s_touch = g_tm.touch;
  double* s_red = g_tm.red;

  const int tid = threadIdx.x;
  const int NT = blockDim.x;

  if (tid < W) {
    int64_t s = -1;
    if (a.list) {
      const int64_t li = tile * W + tid;
      if (li < a.nlist) s = a.list[li];
    } else {
      s = tile * W + tid;
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
      if (lazy || (kin_only && a.touch_own)) touch = CG ? __ldcg(a.touch_own + s) : a.touch_own[s];
    }
    s_la[tid] = la;
    s_lb[tid] = lb;
    s_c0[tid] = c0;
    s_touch[tid] = touch;
  }
  __syncthreads();

  C* psi = reinterpret_cast<C*>(a.psi);
  C* lam = reinterpret_cast<C*>(a.lam);
  const C* chirp = reinterpret_cast<const C*>(g.chirp);
  const bool kin_lam = kin_only && lam != nullptr;   // fixed-units kinetic factor on psi and lam
  const bool kin_touch = kin_only && a.touch_own != nullptr;

  // ---- load + kinetic pre-phase (+ Bluestein pre-chirp on the transform input)
  for (int e = tid; e < W * M; e += NT) {
    int w, i;
    if (a.strided) { w = e % W; i = e / W; } else { w = e / M; i = e - w * M; }
    const int64_t s = s_slice[w];
    C x = czero<C>(), xl = czero<C>();
    if (s >= 0) {
      const int ia = i % g.qa, ib = i / g.qa;
      const int64_t off = s * g.slice_stride + ia * g.ea + ib * g.eb;
      x = ldpsi<CG>(psi + off);
      if (adj || kin_lam) xl = lam[off];
      if (!measure) {
        int64_t units = a.units_pre;
        if (lazy || kin_touch) {
          const int oi = g.shared_b ? ia : i;   // the other layer's slice of this element
          const int32_t t2 = CG ? __ldcg(a.touch_other + oi) : a.touch_other[oi];
          units = (int64_t)a.now - (int64_t)(s_touch[w] > t2 ? s_touch[w] : t2);
        }
        if (units != 0) {
          const uint64_t qd = quad_turns(g, g.lo_a + ia, g.lo_b + ib, s_la[w], s_lb[w], s_c0[w]);
          const Phase<Real> ph = phase_of<Real>((uint64_t)0 - (uint64_t)units * qd);
          x = apply_phase<Real>(x, ph);
          if (adj || kin_lam) xl = apply_phase<Real>(xl, ph);
        }
        if (kin_only) {
          psi[off] = x;
          if (kin_lam) lam[off] = xl;
          continue;
        }
      }
    }
    if (kin_only) continue;
    if (!measure) {
      sx[e] = x;
      if (adj) sxl[e] = xl;
    }
    if (g.bluestein) {
      const C ch = chirp[i];
      x = cmul(x, ch);
      if (adj) xl = cmul(xl, ch);
    }
    sm[w * g.sb + phys(i)] = x;
    if (adj) sml[w * g.sb + phys(i)] = xl;
  }
  if (kin_only) return;
  if (g.bluestein) {
    const int q = g.qa;
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
    transform<Real, true, BPT, D1>(sm, g, W, false);
    if (adj) transform<Real, true, BPT, D1>(sml, g, W, false);
  }

  // ---- pointwise: (T - 1)/M, or the measurement / gradient
  if constexpr (measure) {
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
      if (tid == 0) a.partials[tile] = v / (double)M;
    }
    return;
  } else {
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

    // ---- back to coefficients (forward transform; 1/M is in the table)
    if (g.bluestein) {
      bluestein_conv<Real, BPT>(sm, g, W, (const C*)g.bp);
      if (adj) bluestein_conv<Real, BPT>(sml, g, W, (const C*)g.bp);
    } else {
      transform<Real, false, BPT, D1>(sm, g, W, false);
      if (adj) transform<Real, false, BPT, D1>(sml, g, W, false);
    }

    // ---- x + correction, kinetic post-phase, store
    for (int e = tid; e < W * M; e += NT) {
      int w, i;
      if (a.strided) { w = e % W; i = e / W; } else { w = e / M; i = e - w * M; }
      const int64_t s = s_slice[w];
      if (s < 0) continue;
      const int ia = i % g.qa, ib = i / g.qa;
      const int64_t off = s * g.slice_stride + ia * g.ea + ib * g.eb;
      C cx = sm[w * g.sb + phys(i)], cl;
      if (adj) cl = sml[w * g.sb + phys(i)];
      if (g.bluestein) {
        const C ch = chirp[i];
        cx = cmulconj(cx, ch);
        if (adj) cl = cmulconj(cl, ch);
      }
      C x = cadd(sx[e], cx), xl;
      if (adj) xl = cadd(sxl[e], cl);
      if (!lazy && a.units_post != 0) {
        const uint64_t qd = quad_turns(g, g.lo_a + ia, g.lo_b + ib, s_la[w], s_lb[w], s_c0[w]);
        const Phase<Real> ph = phase_of<Real>((uint64_t)0 - (uint64_t)a.units_post * qd);
        x = apply_phase<Real>(x, ph);
        if (adj) xl = apply_phase<Real>(xl, ph);
      }
      psi[off] = x;
      if (adj) lam[off] = xl;
    }
    if (lazy && tid < W && s_slice[tid] >= 0) a.touch_own[s_slice[tid]] = a.now;
  }
}

template <typename Real, int BPT, int MODE>
__global__ void __launch_bounds__(PassTraits<Real, BPT>::kMaxNT)
pass_kernel(const PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  pass_tile<Real, BPT, MODE, false>(a, (int64_t)blockIdx.x, smraw);
}

// ---------------------------------------------------------------- fast 1D pass
// Specialised pass for 1D slices whose transform length N = 2^LOGN is fixed at
// compile time (8 <= LOGN <= 13): every thread owns 16 elements
// x[j + r N/16] of its slice in registers; Stockham stages with radix 16
// first and last (radix 2/4/8 in the middle), so the output of one FFT and the
// input of the next have the same register layout and the pointwise products
// between transforms (Bluestein kernels, the potential factor) happen in
// registers.  Only the inner stages exchange through shared memory
// (ping-pong buffers, one barrier per exchange).

__host__ __device__ constexpr int fast_nstages(int logn) { return logn == 13 ? 4 : (logn == 8 ? 2 : 3); }
__host__ __device__ constexpr int fast_radix(int logn, int s) {
  // stage s of the plan for N = 2^logn
  return (s == 0 || s == fast_nstages(logn) - 1) ? 16
         : (logn == 9 ? 2 : logn == 10 ? 4 : logn == 11 ? 8 : logn == 12 ? 16 : (s == 1 ? 2 : 16));
}
__host__ __device__ constexpr int fast_ns(int logn, int s) {  // product of radices before stage s
  return s == 0 ? 1 : fast_ns(logn, s - 1) * fast_radix(logn, s - 1);
}

// exp(-+2 pi i k / 16) for compile-time k: (cos, sin) of multiples of pi/8.
template <typename C, bool INV, int K>
__device__ __forceinline__ C rot16(C v) {
  typedef decltype(v.x) R;
  constexpr int k = K & 15;
  if constexpr (k == 0) return v;
  else if constexpr ((k & 1) == 0) return rot8<C, INV>(v, k / 2 < 4 ? k / 2 : 0) ;  // k = 2,4,6 (k <= 9 used)
  else {
    const R c8 = (R)0.92387953251128675613, s8 = (R)0.38268343236508977173;
    R cr, ci;  // exp(-i 2 pi k / 16) = (cos, -sin)
    if constexpr (k == 1) { cr = c8; ci = -s8; }
    else if constexpr (k == 3) { cr = s8; ci = -c8; }
    else if constexpr (k == 5) { cr = -s8; ci = -c8; }
    else if constexpr (k == 7) { cr = -c8; ci = -s8; }
    else { cr = -c8; ci = s8; }  // k == 9
    if (INV) ci = -ci;
    C r;
    r.x = v.x * cr - v.y * ci;
    r.y = v.x * ci + v.y * cr;
    return r;
  }
}

template <typename C, bool INV, int N2>
__device__ __forceinline__ void dft16_col(C* v) {
  // 4-point DFT of v[N2 + 4 n1] over n1, in place, then the inner twiddles
  // W16^(N2 k1): afterwards v[N2 + 4 k1] holds column N2, frequency k1.
  C t[4] = {v[N2], v[4 + N2], v[8 + N2], v[12 + N2]};
  dft4<C, INV>(t);
  v[N2] = t[0];
  v[4 + N2] = rot16<C, INV, N2 * 1>(t[1]);
  v[8 + N2] = rot16<C, INV, N2 * 2>(t[2]);
  v[12 + N2] = rot16<C, INV, N2 * 3>(t[3]);
}

// 16-point DFT in registers, natural order in and out (4 x 4 decomposition,
// in place; the final 4 x 4 transpose is a register renaming).
template <typename C, bool INV>
__device__ __forceinline__ void dft16(C* v) {
  dft16_col<C, INV, 0>(v);
  dft16_col<C, INV, 1>(v);
  dft16_col<C, INV, 2>(v);
  dft16_col<C, INV, 3>(v);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    // row k1: v[4 k1 + n2], n2 = 0..3 -> frequencies k2 (output k1 + 4 k2)
    C t[4] = {v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]};
    dft4<C, INV>(t);
    v[4 * k1] = t[0];
    v[4 * k1 + 1] = t[1];
    v[4 * k1 + 2] = t[2];
    v[4 * k1 + 3] = t[3];
  }
  // X[k1 + 4 k2] is at v[4 k1 + k2]: transpose the 4 x 4 block
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a + 1; b < 4; ++b) {
      C t = v[4 * a + b];
      v[4 * a + b] = v[4 * b + a];
      v[4 * b + a] = t;
    }
}

template <int R, typename C, bool INV> __device__ __forceinline__ void dftRR(C* v) {
  if constexpr (R == 16) dft16<C, INV>(v);
  else dftR<R, C, INV>(v);
}

// Multiply v[r] (r = 1..R-1) by w^r, w = exp(-+2 pi i k / (ns R)), with the
// powers formed by repeated multiplication from one table entry (two live
// registers; relative error <= R eps, which enters the result only through
// the small potential correction term).
template <int R, typename Real, bool INV>
__device__ __forceinline__ void twiddle_pow(typename CT<Real>::C* v, typename CT<Real>::C w) {
  using C = typename CT<Real>::C;
  if (INV) w.y = -w.y;
  C p = w;
#pragma unroll
  for (int r = 1; r < R; ++r) {
    v[r] = cmul(v[r], p);
    if (r + 1 < R) p = cmul(p, w);
  }
}

template <typename Real, int LOGN, int S, bool INV, bool SINGLE = false>
__device__ __forceinline__ void fast_xchg(typename CT<Real>::C (&v)[16], typename CT<Real>::C* buf,
                                          const typename CT<Real>::C* __restrict__ tw, int j) {
  using C = typename CT<Real>::C;
  constexpr int N = 1 << LOGN, TPS = N / 16;
  if constexpr (S < fast_nstages(LOGN)) {
    // twiddle bases of stage S are fetched before the exchange so that their
    // latency overlaps the shared-memory round trip and the barrier
    constexpr int R0 = fast_radix(LOGN, S), ns0 = fast_ns(LOGN, S);
    C wb[16 / R0];
#pragma unroll
    for (int u = 0; u < 16 / R0; ++u) wb[u] = tw[((j + u * TPS) & (ns0 - 1)) * (N / (ns0 * R0))];
    // write the outputs of stage S-1, then read the inputs of stage S
    constexpr int Rp = fast_radix(LOGN, S - 1), nsp = fast_ns(LOGN, S - 1);
#pragma unroll
    for (int u = 0; u < 16 / Rp; ++u) {
      const int b = j + u * TPS;
      const int k = b & (nsp - 1);
      const int i0 = (b - k) * Rp + k;
#pragma unroll
      for (int r = 0; r < Rp; ++r) buf[phys(i0 + r * nsp)] = v[u * Rp + r];
    }
    __syncthreads();
    constexpr int R = fast_radix(LOGN, S), ns = fast_ns(LOGN, S);
#pragma unroll
    for (int u = 0; u < 16 / R; ++u) {
      const int b = j + u * TPS;
#pragma unroll
      for (int r = 0; r < R; ++r) v[u * R + r] = buf[phys(b + r * (N / R))];
    }
    // one shared buffer: every read must finish before the next exchange writes
    if constexpr (SINGLE) __syncthreads();
#pragma unroll
    for (int u = 0; u < 16 / R; ++u) {
      twiddle_pow<R, Real, INV>(v + u * R, wb[u]);
      dftRR<R, C, INV>(v + u * R);
    }
  }
}

// Full FFT of length N on the register layout x[j + r N/16]; exchanges
// alternate between the two buffers (one barrier each).
template <typename Real, int LOGN, bool INV, bool SINGLE = false>
__device__ __forceinline__ void fast_fft(typename CT<Real>::C (&v)[16], typename CT<Real>::C* bufA,
                                         typename CT<Real>::C* bufB, int& flip,
                                         const typename CT<Real>::C* __restrict__ tw, int j,
                                         const typename CT<Real>::C* __restrict__ pre = nullptr) {
  // pre: a table read right after this transform at j + r N/16; its lines are
  // prefetched into L1 here so the loads after the last stage hit
  if (pre) {
#pragma unroll
    for (int r = 0; r < 16; r += 4) {
      asm volatile("prefetch.global.L1 [%0];" ::"l"(pre + j + r * ((1 << LOGN) / 16)));
    }
  }
  using C = typename CT<Real>::C;
  constexpr int N = 1 << LOGN, TPS = N / 16;
  constexpr int NS = fast_nstages(LOGN);
  dft16<C, INV>(v);
#pragma unroll
  for (int S = 1; S < NS; ++S) {
    C* buf = (flip & 1) ? bufB : bufA;
    ++flip;
    // radix and stride of stages S-1 and S (S is a loop index; the switch
    // below dispatches to compile-time stage bodies)
    switch (S) {
      case 1: fast_xchg<Real, LOGN, 1, INV, SINGLE>(v, buf, tw, j); break;
      case 2: fast_xchg<Real, LOGN, 2, INV, SINGLE>(v, buf, tw, j); break;
      case 3: fast_xchg<Real, LOGN, 3, INV, SINGLE>(v, buf, tw, j); break;
    }
  }
  (void)TPS;
}
#ifdef LS_DEFINE_MISC
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

#endif  // LS_DEFINE_MISC

template <typename Real> size_t pass_smem_bytes(const LayerGeom& g, int W, int mode) {
  using C = typename CT<Real>::C;
  const size_t k = (mode == MODE_ADJOINT) ? 2 : 1;
  if (mode == MODE_KIN) return 0;
  return ((size_t)W * g.sb + (mode == MODE_MEASURE ? 0 : (size_t)W * g.M)) * sizeof(C) * k;
}

// Opt-in dynamic shared memory: the per-block limit minus the kernel's static
// shared memory.
template <typename K> static cudaError_t allow_smem(K kernel, size_t max_block) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const size_t dyn = max_block > fa.sharedSizeBytes ? max_block - fa.sharedSizeBytes : 0;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}


// Fast pass: MODE_STEP or MODE_LAZY, 1D slices, N = 2^LOGN, at most NTMAX
// threads per CTA (256 threads: several CTAs per SM; 512: two slices per CTA
// for wider row segments in the strided layer).
// FUSED (convolution form only): two potential factors of the same layer
// separated by a kinetic factor, P(s2) K(mid) P(s1), in one launch (the two
// halves of adjacent Strang steps); the intermediate state never leaves the CTA.
// One tile (W slices) of the fast pass; CG reads psi and the touch times
// through L2 only (the batched runner, whose other CTAs wrote them).
template <typename Real, int LOGN, int MODE, int NBUF, bool FUSED, bool CG>
__device__ __forceinline__ void fast_tile(const PassArgs& a, int64_t tile, unsigned char* smraw) {
  constexpr bool SINGLE = (NBUF == 1);
  using C = typename CT<Real>::C;
  constexpr int N = 1 << LOGN, TPS = N / 16;
  constexpr bool lazy = (MODE == MODE_LAZY);
  const LayerGeom& g = a.g;
  const int W = a.W;
  const int Q = g.qa;
  const int t = threadIdx.x;
  const int w = a.strided ? t % W : t / TPS;
  const int j = a.strided ? t / W : t % TPS;
  C* bufA = reinterpret_cast<C*>(smraw) + (size_t)w * NBUF * g.sb;
  C* bufB = SINGLE ? bufA : bufA + g.sb;
  int64_t* s_slice = g_tm.slice;
  uint64_t *s_la = g_tm.la, *s_c0 = g_tm.c0;
  int32_t* s_touch = g_tm.touch;
  if (t < W) {
    int64_t s = -1;
    if (a.list) {
      const int64_t li = tile * W + t;
      if (li < a.nlist) s = a.list[li];
    } else {
      s = tile * W + t;
      if (s >= g.nslices) s = -1;
    }
    s_slice[t] = s;
    uint64_t la = 0, c0 = 0;
    int32_t touch = 0;
    if (s >= 0) {
      const uint64_t ua = (uint64_t)(s + g.olo_a);
      la = g.X_aa * ua;
      c0 = g.C_aa * (ua * ua);
      if (lazy) touch = CG ? __ldcg(a.touch_own + s) : a.touch_own[s];
    }
    s_la[t] = la;
    s_c0[t] = c0;
    s_touch[t] = touch;
  }
  __syncthreads();
  C* psi = reinterpret_cast<C*>(a.psi);
  const C* chirp = reinterpret_cast<const C*>(g.chirp);
  const C* tw = reinterpret_cast<const C*>(g.tw);

  // load + kinetic pre-phase into shared memory (element loop, low register
  // pressure), then every thread picks up its 16 elements
  const int NT = blockDim.x;
  C* smc = reinterpret_cast<C*>(smraw);
  C* xs0 = smc + (size_t)W * NBUF * g.sb;
#pragma unroll 4
  for (int e = t; e < W * N; e += NT) {
    int ww, i;
    if (a.strided) { ww = e % W; i = e / W; } else { ww = e / N; i = e - ww * N; }
    const int64_t ss = s_slice[ww];
    C x = czero<C>();
    if (i < Q && ss >= 0) {
      x = ldpsi<CG>(psi + ss * g.slice_stride + (int64_t)i * g.ea);
      int64_t units = a.units_pre;
      if (lazy) {
        const int32_t t2 = CG ? __ldcg(a.touch_other + i) : a.touch_other[i];
        units = (int64_t)a.now - (int64_t)(s_touch[ww] > t2 ? s_touch[ww] : t2);
      }
      if (units != 0) {
        const uint64_t m = (uint64_t)(int64_t)(g.lo_a + i);
        const uint64_t qd = g.A_aa * (m * m) + s_la[ww] * m + s_c0[ww];
        x = apply_phase<Real>(x, phase_of<Real>((uint64_t)0 - (uint64_t)units * qd));
      }
      xs0[(size_t)ww * Q + i] = x;
      if (g.bluestein && a.Khat == nullptr) x = cmul(x, chirp[i]);
    } else if (i < Q) {
      xs0[(size_t)ww * Q + i] = x;
    }
    smc[(size_t)ww * NBUF * g.sb + phys(i)] = x;
  }
  __syncthreads();
  C v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = bufA[phys(j + r * TPS)];
  if constexpr (SINGLE) __syncthreads();
  int flip = 1;  // buffer A holds the input; the first exchange uses B
  const C* T = reinterpret_cast<const C*>(a.T);
  const bool conv = g.bluestein && a.Khat != nullptr;
  if (conv) {
    // cyclic convolution of the zero-padded slice with the wrapped kernel
    const C* Kh = reinterpret_cast<const C*>(a.Khat);
    fast_fft<Real, LOGN, false, SINGLE>(v, bufA, bufB, flip, tw, j, Kh);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], Kh[j + r * TPS]);
    fast_fft<Real, LOGN, true, SINGLE>(v, bufA, bufB, flip, tw, j);
    if constexpr (FUSED) {
      // x1 = K(mid) (x + c1): through shared memory, then the second factor
      C* s_fix1 = reinterpret_cast<C*>(g_tm.fix1);
      if (t < W && s_slice[t] >= 0) {
        C f;
        f.x = (Real)a.fix0_re;
        f.y = (Real)a.fix0_im;
        s_fix1[t] = cmul(f, xs0[(size_t)t * Q + Q - 1]);
      }
      C* buf = (flip & 1) ? bufB : bufA;
#pragma unroll
      for (int r = 0; r < 16; ++r) buf[phys(j + r * TPS)] = v[r];
      __syncthreads();
      for (int e = t; e < W * N; e += NT) {
        int ww, i;
        if (a.strided) { ww = e % W; i = e / W; } else { ww = e / N; i = e - ww * N; }
        C* bw = smc + (size_t)ww * NBUF * g.sb + (size_t)(buf - bufA) + phys(i);
        C x = czero<C>();
        if (i < Q && s_slice[ww] >= 0) {
          C c = *bw;
          if (i == 0) c = cadd(c, s_fix1[ww]);
          x = cadd(xs0[(size_t)ww * Q + i], c);
          if (a.units_mid != 0) {
            const uint64_t m = (uint64_t)(int64_t)(g.lo_a + i);
            const uint64_t qd = g.A_aa * (m * m) + s_la[ww] * m + s_c0[ww];
            x = apply_phase<Real>(x, phase_of<Real>((uint64_t)0 - (uint64_t)a.units_mid * qd));
          }
          xs0[(size_t)ww * Q + i] = x;
        }
        *bw = x;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = buf[phys(j + r * TPS)];
      __syncthreads();
      const C* Kh2 = reinterpret_cast<const C*>(a.Khat2);
      fast_fft<Real, LOGN, false, SINGLE>(v, bufA, bufB, flip, tw, j, Kh2);
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], Kh2[j + r * TPS]);
      fast_fft<Real, LOGN, true, SINGLE>(v, bufA, bufB, flip, tw, j);
    }
  } else if (g.bluestein) {
    const C* bm = reinterpret_cast<const C*>(g.bm);
    const C* bp = reinterpret_cast<const C*>(g.bp);
    fast_fft<Real, LOGN, false, SINGLE>(v, bufA, bufB, flip, tw, j);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], bm[j + r * TPS]);
    fast_fft<Real, LOGN, true, SINGLE>(v, bufA, bufB, flip, tw, j);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int i = j + r * TPS;
      v[r] = i < Q ? cmul(v[r], T[i]) : czero<C>();
    }
    fast_fft<Real, LOGN, false, SINGLE>(v, bufA, bufB, flip, tw, j);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], bp[j + r * TPS]);
    fast_fft<Real, LOGN, true, SINGLE>(v, bufA, bufB, flip, tw, j);
  } else {
    fast_fft<Real, LOGN, true, SINGLE>(v, bufA, bufB, flip, tw, j);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], T[j + r * TPS]);
    fast_fft<Real, LOGN, false, SINGLE>(v, bufA, bufB, flip, tw, j);
  }
  // correction back to shared memory, then x + correction, post-phase, store
  {
    C* buf = (flip & 1) ? bufB : bufA;
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[phys(j + r * TPS)] = v[r];
    const int ob = (flip & 1) ? 1 : 0;
    __syncthreads();
#pragma unroll 4
    for (int e = t; e < W * Q; e += NT) {
      int ww, i;
      if (a.strided) { ww = e % W; i = e / W; } else { ww = e / Q; i = e - ww * Q; }
      const int64_t ss = s_slice[ww];
      if (ss < 0) continue;
      C c = smc[(size_t)ww * NBUF * g.sb + (size_t)(SINGLE ? 0 : ob) * g.sb + phys(i)];
      if (conv) {
        if (i == 0) {
          C f;
          f.x = (Real)(FUSED ? a.fix2_re : a.fix0_re);
          f.y = (Real)(FUSED ? a.fix2_im : a.fix0_im);
          c = cadd(c, cmul(f, xs0[(size_t)ww * Q + Q - 1]));
        }
      } else if (g.bluestein) {
        c = cmulconj(c, chirp[i]);
      }
      C x = cadd(xs0[(size_t)ww * Q + i], c);
      if (!lazy && a.units_post != 0) {
        const uint64_t m = (uint64_t)(int64_t)(g.lo_a + i);
        const uint64_t qd = g.A_aa * (m * m) + s_la[ww] * m + s_c0[ww];
        x = apply_phase<Real>(x, phase_of<Real>((uint64_t)0 - (uint64_t)a.units_post * qd));
      }
      psi[ss * g.slice_stride + (int64_t)i * g.ea] = x;
    }
  }
  if (lazy && t < W && s_slice[t] >= 0) a.touch_own[s_slice[t]] = a.now;
}

template <typename Real, int LOGN, int MODE, int NTMAX, int NBUF = 2,
          int MINB = ((NTMAX == 256 && sizeof(Real) == 4) ? 2 : 1), bool FUSED = false>
__global__ void __launch_bounds__(NTMAX, MINB)
pass_fast_kernel(const PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  fast_tile<Real, LOGN, MODE, NBUF, FUSED, false>(a, (int64_t)blockIdx.x, smraw);
}

// ---------------------------------------------------------------- fast 2D pass (64 x 64 slices)
// One 64 x 64 slice per 256-thread CTA.  The slice sits in shared memory with
// row stride 65 (element (ia, ib) at ia + 65 ib).  A 64-point transform along
// either axis is done by four threads: thread t takes line sub = t & 63 and
// quarter j = t >> 6 and holds elements j + 4u + 8r (u < 2, r < 8) of the line
// in v[8u + r].  All lanes of a warp share j and take 32 consecutive lines, so
// every shared-memory access of both axes is free of bank conflicts.  Two
// radix-8 Stockham stages; the output lands in the input layout, so the
// inverse transform along b, the potential factor and the forward transform
// along b follow one another in registers.
constexpr int kF2Row = 65;

template <typename Real, bool INV>
__device__ __forceinline__ void fft64_line(typename CT<Real>::C (&v)[16], typename CT<Real>::C* buf, int base,
                                           int es, int j, const typename CT<Real>::C* __restrict__ tw) {
  using C = typename CT<Real>::C;
  C wb[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) wb[u] = tw[j + 4 * u];  // W_64^b, b = j + 4u (stage 2, stride 1)
  // stage 1 (ns = 1): butterfly b = j + 4u reads x[b + 8r], writes 8b + r
#pragma unroll
  for (int u = 0; u < 2; ++u) dftR<8, C, INV>(v + 8 * u);
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int r = 0; r < 8; ++r) buf[base + (8 * (j + 4 * u) + r) * es] = v[8 * u + r];
  __syncthreads();
  // stage 2 (ns = 8): butterfly b reads x[b + 8r], twiddles W_64^(r b), writes b + 8r
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int r = 0; r < 8; ++r) v[8 * u + r] = buf[base + (j + 4 * u + 8 * r) * es];
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    twiddle_pow<8, Real, INV>(v + 8 * u, wb[u]);
    dftR<8, C, INV>(v + 8 * u);
  }
}

template <typename Real>
__device__ __forceinline__ void f2_line_load(typename CT<Real>::C (&v)[16], const typename CT<Real>::C* buf,
                                             int base, int es, int j) {
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int r = 0; r < 8; ++r) v[8 * u + r] = buf[base + (j + 4 * u + 8 * r) * es];
}
template <typename Real>
__device__ __forceinline__ void f2_line_store(const typename CT<Real>::C (&v)[16], typename CT<Real>::C* buf,
                                              int base, int es, int j) {
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int r = 0; r < 8; ++r) buf[base + (j + 4 * u + 8 * r) * es] = v[8 * u + r];
}

// Kinetic phase turns of one thread's elements (ia fixed, ib = ib0 + 4m,
// m = 0..15) by exact second differences modulo 2^64: the quadratic form
// q(a, b) = A_aa a^2 + A_ab a b + A_bb b^2 + la a + lb b + c0 steps in b by
// d_m = 4 A_ab a + A_bb (8 b_m + 16) + 4 lb, and d steps by 32 A_bb.
struct QuadWalk {
  uint64_t q, d, dd;
  __device__ __forceinline__ QuadWalk(const LayerGeom& g, int ia, int ib0, uint64_t la, uint64_t lb, uint64_t c0) {
    const uint64_t a = (uint64_t)(g.lo_a + ia), b = (uint64_t)(g.lo_b + ib0);
    q = quad_turns(g, g.lo_a + ia, g.lo_b + ib0, la, lb, c0);
    d = 4 * g.A_ab * a + g.A_bb * (8 * b + 16) + 4 * lb;
    dd = 32 * g.A_bb;
  }
  __device__ __forceinline__ void scale(uint64_t u) {  // walk u * q instead of q
    q *= u;
    d *= u;
    dd *= u;
  }
  __device__ __forceinline__ void next() {
    q += d;
    d += dd;
  }
};

// The correction F diag((T - 1)/M) F^{-1} x of one slice held in buf (row
// stride 65), in place: inverse transforms along a and b, the potential
// factor, forward transforms along b and a.  Ends with a barrier.
template <typename Real>
__device__ __forceinline__ void f2_correction(typename CT<Real>::C* buf, const typename CT<Real>::C* __restrict__ T,
                                              const typename CT<Real>::C* __restrict__ twa,
                                              const typename CT<Real>::C* __restrict__ twb, int sub, int j) {
  using C = typename CT<Real>::C;
  C v[16];
  // inverse transform along a (line = row ib = sub)
  f2_line_load<Real>(v, buf, sub * kF2Row, 1, j);
  __syncthreads();
  fft64_line<Real, true>(v, buf, sub * kF2Row, 1, j, twa);
  f2_line_store<Real>(v, buf, sub * kF2Row, 1, j);
  __syncthreads();
  // inverse along b (line = column ia = sub), potential factor, forward along b
  f2_line_load<Real>(v, buf, sub, kF2Row, j);
  __syncthreads();
  fft64_line<Real, true>(v, buf, sub, kF2Row, j, twb);
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int r = 0; r < 8; ++r) v[8 * u + r] = cmul(v[8 * u + r], T[sub + 64 * (j + 4 * u + 8 * r)]);
  fft64_line<Real, false>(v, buf, sub, kF2Row, j, twb);
  f2_line_store<Real>(v, buf, sub, kF2Row, j);
  __syncthreads();
  // forward along a
  f2_line_load<Real>(v, buf, sub * kF2Row, 1, j);
  __syncthreads();
  fft64_line<Real, false>(v, buf, sub * kF2Row, 1, j, twa);
  f2_line_store<Real>(v, buf, sub * kF2Row, 1, j);
  __syncthreads();
}

// FUSED: two layer-1 factors of consecutive Strang steps in one launch, with
// the merged kinetic factor (units_mid) between them and the second factor's
// table in T2; the intermediate slice stays in shared memory.
template <typename Real, int MODE, bool FUSED = false>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 3 : 1)
pass_fast2d_kernel(const PassArgs a) {
  using C = typename CT<Real>::C;
  constexpr bool lazy = (MODE == MODE_LAZY);
  extern __shared__ __align__(16) unsigned char smraw[];
  const LayerGeom& g = a.g;
  const int t = threadIdx.x;
  const int sub = t & 63, j = t >> 6;
  C* buf = reinterpret_cast<C*>(smraw);
  C* xs = buf + 64 * kF2Row;
  __shared__ int64_t s_slice;
  __shared__ uint64_t s_la, s_lb, s_c0;
  __shared__ int32_t s_touch;
  if (t == 0) {
    int64_t s = -1;
    if (a.list) {
      if ((int64_t)blockIdx.x < a.nlist) s = a.list[blockIdx.x];
    } else {
      s = blockIdx.x;
      if (s >= g.nslices) s = -1;
    }
    s_slice = s;
    uint64_t la = 0, lb = 0, c0 = 0;
    int32_t touch = 0;
    if (s >= 0) {
      const uint64_t ua = (uint64_t)(s % g.oqa + g.olo_a), ub = (uint64_t)(s / g.oqa + g.olo_b);
      la = g.X_aa * ua + g.X_ab * ub;
      lb = g.X_ba * ua + g.X_bb * ub;
      c0 = g.C_aa * (ua * ua) + g.C_ab * (ua * ub) + g.C_bb * (ub * ub);
      if (lazy) touch = a.touch_own[s];
    }
    s_la = la;
    s_lb = lb;
    s_c0 = c0;
    s_touch = touch;
  }
  __syncthreads();
  const int64_t s = s_slice;
  if (s < 0) return;
  C* psi = reinterpret_cast<C*>(a.psi);
  const C* twa = reinterpret_cast<const C*>(g.tw);
  const C* twb = reinterpret_cast<const C*>(g.twb);
  // this thread's elements in the load and store loops: ia = sub, ib = j + 4m
  C* pp = psi + s * g.slice_stride + sub * g.ea + j * g.eb;
  const int64_t estep = 4 * g.eb;
  {
    C x[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) x[m] = pp[m * estep];  // all loads in flight before the phases
    if (lazy) {
      QuadWalk w(g, sub, j, s_la, s_lb, s_c0);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int32_t t2 = a.touch_other[sub + 64 * (j + 4 * m)];
        const int64_t units = (int64_t)a.now - (int64_t)(s_touch > t2 ? s_touch : t2);
        if (units != 0) x[m] = apply_phase<Real>(x[m], phase_of<Real>((uint64_t)0 - (uint64_t)units * w.q));
        w.next();
      }
    } else if (a.units_pre != 0) {
      QuadWalk w(g, sub, j, s_la, s_lb, s_c0);
      w.scale((uint64_t)0 - (uint64_t)a.units_pre);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        x[m] = apply_phase<Real>(x[m], phase_of<Real>(w.q));
        w.next();
      }
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int ib = j + 4 * m;
      xs[sub + 64 * ib] = x[m];
      buf[sub + kF2Row * ib] = x[m];
    }
  }
  __syncthreads();
  f2_correction<Real>(buf, reinterpret_cast<const C*>(a.T), twa, twb, sub, j);
  if constexpr (FUSED) {
    // x1 = K(mid) (x + correction): the second factor's input and identity term
    QuadWalk w(g, sub, j, s_la, s_lb, s_c0);
    const bool mid = a.units_mid != 0;
    if (mid) w.scale((uint64_t)0 - (uint64_t)a.units_mid);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int ib = j + 4 * m;
      C x = cadd(xs[sub + 64 * ib], buf[sub + kF2Row * ib]);
      if (mid) {
        x = apply_phase<Real>(x, phase_of<Real>(w.q));
        w.next();
      }
      xs[sub + 64 * ib] = x;
      buf[sub + kF2Row * ib] = x;
    }
    __syncthreads();
    f2_correction<Real>(buf, reinterpret_cast<const C*>(a.T2), twa, twb, sub, j);
  }
  // x + correction, kinetic post-phase, store
  {
    const bool post = !lazy && a.units_post != 0;
    QuadWalk w(g, sub, j, s_la, s_lb, s_c0);
    if (post) w.scale((uint64_t)0 - (uint64_t)a.units_post);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int ib = j + 4 * m;
      C x = cadd(xs[sub + 64 * ib], buf[sub + kF2Row * ib]);
      if (post) {
        x = apply_phase<Real>(x, phase_of<Real>(w.q));
        w.next();
      }
      pp[m * estep] = x;
    }
  }
  if (lazy && t == 0) a.touch_own[s] = a.now;
}

// Two adjacent slices per CTA for the strided layer (slice stride 1 element):
// one 16-byte load or store moves an element of both slices, which halves the
// requests and doubles the used bytes per sector of the column-wise access.
// The slices are transformed one after the other in the same buffer; the
// second slice's input waits in registers, the first slice's result in
// shared memory.  Full passes (no slice list) in MODE_STEP, complex64.
template <typename Real>
__global__ void __launch_bounds__(256, 2) pass_fast2d_pair_kernel(const PassArgs a) {
  static_assert(sizeof(Real) == 4, "complex64 only");
  using C = float2;
  extern __shared__ __align__(16) unsigned char smraw[];
  const LayerGeom& g = a.g;
  const int t = threadIdx.x;
  const int sub = t & 63, j = t >> 6;
  C* buf = reinterpret_cast<C*>(smraw);
  C* xs = buf + 64 * kF2Row;
  __shared__ uint64_t s_la[2], s_lb[2], s_c0[2];
  const int64_t s0 = 2 * (int64_t)blockIdx.x;
  if (s0 >= g.nslices) return;
  const bool has1 = s0 + 1 < g.nslices;
  if (t < 2) {
    const int64_t s = s0 + t;
    const uint64_t ua = (uint64_t)(s % g.oqa + g.olo_a), ub = (uint64_t)(s / g.oqa + g.olo_b);
    s_la[t] = g.X_aa * ua + g.X_ab * ub;
    s_lb[t] = g.X_ba * ua + g.X_bb * ub;
    s_c0[t] = g.C_aa * (ua * ua) + g.C_ab * (ua * ub) + g.C_bb * (ub * ub);
  }
  __syncthreads();
  C* pp = reinterpret_cast<C*>(a.psi) + s0 + sub * g.ea + j * g.eb;
  const int64_t estep = 4 * g.eb;
  const C* twa = reinterpret_cast<const C*>(g.tw);
  const C* twb = reinterpret_cast<const C*>(g.twb);
  const C* T = reinterpret_cast<const C*>(a.T);
  C x1[16];
  {
    C x0[16];
    if (has1) {
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const float4 q = *reinterpret_cast<const float4*>(pp + m * estep);
        x0[m] = make_float2(q.x, q.y);
        x1[m] = make_float2(q.z, q.w);
      }
    } else {
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        x0[m] = pp[m * estep];
        x1[m] = make_float2(0.f, 0.f);
      }
    }
    if (a.units_pre != 0) {
      QuadWalk w0(g, sub, j, s_la[0], s_lb[0], s_c0[0]), w1(g, sub, j, s_la[1], s_lb[1], s_c0[1]);
      w0.scale((uint64_t)0 - (uint64_t)a.units_pre);
      w1.scale((uint64_t)0 - (uint64_t)a.units_pre);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        x0[m] = apply_phase<float>(x0[m], phase_of<float>(w0.q));
        x1[m] = apply_phase<float>(x1[m], phase_of<float>(w1.q));
        w0.next();
        w1.next();
      }
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int ib = j + 4 * m;
      xs[sub + 64 * ib] = x0[m];
      buf[sub + kF2Row * ib] = x0[m];
    }
  }
  __syncthreads();
  f2_correction<float>(buf, T, twa, twb, sub, j);
  // first slice: x + correction, post-phase, kept in xs; second slice's input
  // into buf (each thread touches only its own elements here)
  {
    QuadWalk w(g, sub, j, s_la[0], s_lb[0], s_c0[0]);
    const bool post = a.units_post != 0;
    if (post) w.scale((uint64_t)0 - (uint64_t)a.units_post);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int ib = j + 4 * m;
      C x = cadd(xs[sub + 64 * ib], buf[sub + kF2Row * ib]);
      if (post) {
        x = apply_phase<float>(x, phase_of<float>(w.q));
        w.next();
      }
      xs[sub + 64 * ib] = x;
      buf[sub + kF2Row * ib] = x1[m];
    }
  }
  __syncthreads();
  f2_correction<float>(buf, T, twa, twb, sub, j);
  {
    QuadWalk w(g, sub, j, s_la[1], s_lb[1], s_c0[1]);
    const bool post = a.units_post != 0;
    if (post) w.scale((uint64_t)0 - (uint64_t)a.units_post);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int ib = j + 4 * m;
      C x = cadd(x1[m], buf[sub + kF2Row * ib]);
      if (post) {
        x = apply_phase<float>(x, phase_of<float>(w.q));
        w.next();
      }
      const C r0 = xs[sub + 64 * ib];
      if (has1) *reinterpret_cast<float4*>(pp + m * estep) = make_float4(r0.x, r0.y, x.x, x.y);
      else pp[m * estep] = r0;
    }
  }
}

template <typename Real> size_t fast2d_smem_bytes(const LayerGeom& g) {
  using C = typename CT<Real>::C;
  return ((size_t)64 * kF2Row + (size_t)g.M) * sizeof(C);
}

template <typename Real> cudaError_t launch_fast2d(const PassArgs& a, int64_t ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (a.g.d != 2 || a.g.qa != 64 || a.g.qb != 64) return cudaErrorInvalidValue;
  const size_t smem = fast2d_smem_bytes<Real>(a.g);
  if constexpr (sizeof(Real) == 4) {
    // strided layer, full pass, 16-byte aligned slice pairs: two slices per CTA
    if (a.mode == MODE_STEP && a.list == nullptr && a.T2 == nullptr && a.g.slice_stride == 1 &&
        (a.g.ea % 2) == 0 && (a.g.eb % 2) == 0 && (reinterpret_cast<uintptr_t>(a.psi) % 16) == 0) {
      pass_fast2d_pair_kernel<Real><<<(unsigned)((a.g.nslices + 1) / 2), 256, smem, st>>>(a);
      return cudaGetLastError();
    }
  }
  if (a.mode == MODE_LAZY) pass_fast2d_kernel<Real, MODE_LAZY><<<(unsigned)ntiles, 256, smem, st>>>(a);
  else if (a.T2) pass_fast2d_kernel<Real, MODE_STEP, true><<<(unsigned)ntiles, 256, smem, st>>>(a);
  else pass_fast2d_kernel<Real, MODE_STEP><<<(unsigned)ntiles, 256, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename Real> cudaError_t fast2d_prepare(size_t max_smem) {
  cudaError_t e = allow_smem(pass_fast2d_kernel<Real, MODE_STEP>, max_smem);
  if (e == cudaSuccess) e = allow_smem(pass_fast2d_kernel<Real, MODE_STEP, true>, max_smem);
  if constexpr (sizeof(Real) == 4)
    if (e == cudaSuccess) e = allow_smem(pass_fast2d_pair_kernel<Real>, max_smem);
  if (e == cudaSuccess) e = allow_smem(pass_fast2d_kernel<Real, MODE_LAZY>, max_smem);
  return e;
}

// Two adjacent columns per CTA for the strided 1D layer (slice stride 1
// element, transform length 4096, complex64): one 16-byte load or store moves
// an element of both columns.  The columns are transformed one after the
// other in one shared buffer (the convolution form, or the plain form for
// power-of-two lengths); the second column's input waits in registers (NX per
// thread), the first column's result in shared memory.  Thread t owns
// elements i = t + 256 k; kinetic phases step along k by exact second
// differences modulo 2^64.  Full passes in MODE_STEP only.
struct QuadWalk1 {
  uint64_t q, d, dd;
  __device__ __forceinline__ QuadWalk1(const LayerGeom& g, int i0, int step, uint64_t la, uint64_t c0) {
    const uint64_t m = (uint64_t)(int64_t)(g.lo_a + i0), st = (uint64_t)step;
    q = g.A_aa * (m * m) + la * m + c0;
    d = g.A_aa * (2 * m * st + st * st) + la * st;
    dd = 2 * g.A_aa * (st * st);
  }
  __device__ __forceinline__ void scale(uint64_t u) {
    q *= u;
    d *= u;
    dd *= u;
  }
  __device__ __forceinline__ void next() {
    q += d;
    d += dd;
  }
};

template <typename Real, int NX>
__device__ __forceinline__ void fast_pair_middle(typename CT<Real>::C* buf, const PassArgs& a, bool conv, int j) {
  using C = typename CT<Real>::C;
  constexpr int LOGN = 12, TPS = 256;
  const C* tw = reinterpret_cast<const C*>(a.g.tw);
  C v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = buf[phys(j + r * TPS)];
  __syncthreads();
  int flip = 1;
  if (conv) {
    const C* Kh = reinterpret_cast<const C*>(a.Khat);
    fast_fft<Real, LOGN, false, true>(v, buf, buf, flip, tw, j, Kh);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], Kh[j + r * TPS]);
    fast_fft<Real, LOGN, true, true>(v, buf, buf, flip, tw, j);
  } else {
    const C* T = reinterpret_cast<const C*>(a.T);
    fast_fft<Real, LOGN, true, true>(v, buf, buf, flip, tw, j);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], T[j + r * TPS]);
    fast_fft<Real, LOGN, false, true>(v, buf, buf, flip, tw, j);
  }
#pragma unroll
  for (int r = 0; r < 16; ++r) buf[phys(j + r * TPS)] = v[r];
  __syncthreads();
}

template <typename Real, int NX>
__global__ void __launch_bounds__(256, 2) pass_fast_pair_kernel(const PassArgs a) {
  static_assert(sizeof(Real) == 4, "complex64 only");
  using C = float2;
  constexpr int N = 4096;
  extern __shared__ __align__(16) unsigned char smraw[];
  const LayerGeom& g = a.g;
  const int Q = g.qa;
  const int t = threadIdx.x;
  const bool conv = a.Khat != nullptr;
  C* buf = reinterpret_cast<C*>(smraw);
  C* xs = buf + g.sb;
  __shared__ uint64_t s_la[2], s_c0[2];
  __shared__ C s_last1;
  const int64_t s0 = 2 * (int64_t)blockIdx.x;
  if (s0 >= g.nslices) return;
  const bool has1 = s0 + 1 < g.nslices;
  if (t < 2) {
    const uint64_t ua = (uint64_t)(s0 + t + g.olo_a);
    s_la[t] = g.X_aa * ua;
    s_c0[t] = g.C_aa * (ua * ua);
  }
  __syncthreads();
  C* pp = reinterpret_cast<C*>(a.psi) + s0 + (int64_t)t * g.ea;
  const int64_t estep = 256 * g.ea;
  C x1[NX];
  {
    C x0[NX];
#pragma unroll
    for (int k = 0; k < NX; ++k) {
      x0[k] = x1[k] = make_float2(0.f, 0.f);
      if (t + 256 * k < Q) {
        if (has1) {
          const float4 q = *reinterpret_cast<const float4*>(pp + k * estep);
          x0[k] = make_float2(q.x, q.y);
          x1[k] = make_float2(q.z, q.w);
        } else {
          x0[k] = pp[k * estep];
        }
      }
    }
    if (a.units_pre != 0) {
      QuadWalk1 w0(g, t, 256, s_la[0], s_c0[0]), w1(g, t, 256, s_la[1], s_c0[1]);
      w0.scale((uint64_t)0 - (uint64_t)a.units_pre);
      w1.scale((uint64_t)0 - (uint64_t)a.units_pre);
#pragma unroll
      for (int k = 0; k < NX; ++k) {
        if (t + 256 * k < Q) {
          x0[k] = apply_phase<float>(x0[k], phase_of<float>(w0.q));
          x1[k] = apply_phase<float>(x1[k], phase_of<float>(w1.q));
        }
        w0.next();
        w1.next();
      }
    }
#pragma unroll
    for (int k = 0; k < NX; ++k) {
      const int i = t + 256 * k;
      if (i < Q) {
        xs[i] = x0[k];
        if (i == Q - 1) s_last1 = x1[k];
      }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int i = t + 256 * k;
      buf[phys(i)] = (k < NX && i < Q) ? x0[k < NX ? k : 0] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  C last0 = xs[Q - 1];  // the first column's input at Q - 1 (before xs is overwritten)
  C last1 = s_last1;
  fast_pair_middle<float, NX>(buf, a, conv, t);
  const bool post = a.units_post != 0;
  const C fix = make_float2((float)a.fix0_re, (float)a.fix0_im);
  // first column: x + correction, post-phase, kept in xs; second column's
  // input into buf (each thread touches only its own elements here)
  {
    QuadWalk1 w(g, t, 256, s_la[0], s_c0[0]);
    if (post) w.scale((uint64_t)0 - (uint64_t)a.units_post);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int i = t + 256 * k;
      if (k < NX && i < Q) {
        C c = buf[phys(i)];
        if (conv && i == 0) c = cadd(c, cmul(fix, last0));
        C x = cadd(xs[i], c);
        if (post) x = apply_phase<float>(x, phase_of<float>(w.q));
        xs[i] = x;
        buf[phys(i)] = x1[k < NX ? k : 0];
      } else {
        buf[phys(i)] = make_float2(0.f, 0.f);
      }
      w.next();
    }
  }
  __syncthreads();
  fast_pair_middle<float, NX>(buf, a, conv, t);
  {
    QuadWalk1 w(g, t, 256, s_la[1], s_c0[1]);
    if (post) w.scale((uint64_t)0 - (uint64_t)a.units_post);
#pragma unroll
    for (int k = 0; k < NX; ++k) {
      const int i = t + 256 * k;
      if (i < Q) {
        C c = buf[phys(i)];
        if (conv && i == 0) c = cadd(c, cmul(fix, last1));
        C x = cadd(x1[k], c);
        if (post) x = apply_phase<float>(x, phase_of<float>(w.q));
        const C r0 = xs[i];
        if (has1) *reinterpret_cast<float4*>(pp + k * estep) = make_float4(r0.x, r0.y, x.x, x.y);
        else pp[k * estep] = r0;
      }
      w.next();
    }
  }
}

template <typename Real> size_t fast_smem_bytes(const LayerGeom& g, int W, int variant) {
  using C = typename CT<Real>::C;
  const size_t nbuf = (variant == 0) ? 2 : 1;
  return ((size_t)W * nbuf * g.sb + (size_t)W * g.qa) * sizeof(C);
}

template <typename Real, int LOGN>
static cudaError_t launch_fast_n(const PassArgs& a, int64_t ntiles, cudaStream_t st) {
  const int nt = a.W * ((1 << LOGN) / 16);
  if (nt > 256) return cudaErrorInvalidValue;
  // single precision: one shared buffer, three resident CTAs per SM; double:
  // two buffers (ping-pong), registers for one CTA
  constexpr int NBUF = sizeof(Real) == 4 ? 1 : 2;
  constexpr int MINB = sizeof(Real) == 4 ? 3 : 1;
  const size_t smem = fast_smem_bytes<Real>(a.g, a.W, NBUF == 1 ? 1 : 0);
  if constexpr (sizeof(Real) == 4 && LOGN == 12) {
    // strided layer, full pass, 16-byte aligned column pairs: two columns per CTA
    if (a.mode == MODE_STEP && a.list == nullptr && a.W == 1 && a.strided && a.g.slice_stride == 1 &&
        a.Khat2 == nullptr && (a.Khat != nullptr || !a.g.bluestein) && (a.g.ea % 2) == 0 &&
        (reinterpret_cast<uintptr_t>(a.psi) % 16) == 0) {
      const unsigned nb = (unsigned)((a.g.nslices + 1) / 2);
      if (a.g.qa <= 9 * 256) pass_fast_pair_kernel<Real, 9><<<nb, 256, smem, st>>>(a);
      else pass_fast_pair_kernel<Real, 16><<<nb, 256, smem, st>>>(a);
      return cudaGetLastError();
    }
  }
  if (a.mode == MODE_LAZY) pass_fast_kernel<Real, LOGN, MODE_LAZY, 256, NBUF, MINB><<<(unsigned)ntiles, nt, smem, st>>>(a);
  else if (a.Khat2) pass_fast_kernel<Real, LOGN, MODE_STEP, 256, NBUF, MINB, true><<<(unsigned)ntiles, nt, smem, st>>>(a);
  else pass_fast_kernel<Real, LOGN, MODE_STEP, 256, NBUF, MINB><<<(unsigned)ntiles, nt, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename Real> cudaError_t launch_fast(const PassArgs& a, int64_t ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  switch (a.g.np) {
    case 512: return launch_fast_n<Real, 9>(a, ntiles, st);
    case 1024: return launch_fast_n<Real, 10>(a, ntiles, st);
    case 2048: return launch_fast_n<Real, 11>(a, ntiles, st);
    case 4096: return launch_fast_n<Real, 12>(a, ntiles, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename Real> cudaError_t fast_prepare(size_t max_smem) {
  cudaError_t e = cudaSuccess;
  constexpr int NBUF = sizeof(Real) == 4 ? 1 : 2;
  constexpr int MINB = sizeof(Real) == 4 ? 3 : 1;
#define LS_FPREP(L) \
  if (e == cudaSuccess) e = allow_smem(pass_fast_kernel<Real, L, MODE_STEP, 256, NBUF, MINB>, max_smem); \
  if (e == cudaSuccess) e = allow_smem(pass_fast_kernel<Real, L, MODE_STEP, 256, NBUF, MINB, true>, max_smem); \
  if (e == cudaSuccess) e = allow_smem(pass_fast_kernel<Real, L, MODE_LAZY, 256, NBUF, MINB>, max_smem);
  LS_FPREP(9) LS_FPREP(10) LS_FPREP(11) LS_FPREP(12)
#undef LS_FPREP
  if constexpr (sizeof(Real) == 4) {
    if (e == cudaSuccess) e = allow_smem(pass_fast_pair_kernel<Real, 9>, max_smem);
    if (e == cudaSuccess) e = allow_smem(pass_fast_pair_kernel<Real, 16>, max_smem);
  }
  return e;
}
template <typename Real> int fast_max_threads() { return 256; }

// ---------------------------------------------------------------- compact-kernel pass
// P_j(s) - I is the circulant of c' = DFT_q(T - 1)/q on a 1D slice of length q
// (the kernel the convolution form transforms).  For band-limited potentials
// and short durations c' decays fast (for v = a cos, c'_d is the Bessel
// coefficient J_d(s a) up to a unit phase, minus the identity at d = 0), and
// the host keeps the taps |d| <= BV when the l1 norm of the dropped ones, a
// bound on the operator-norm error, is below working precision.  A tile holds
// W whole slices in shared memory, each with a wrap halo on both sides, so
// x_{(i - d) mod q} is a plain offset:
//   16-byte asynchronous copies global -> shared (through L2) -> kinetic
//   pre-phase in shared memory -> halos -> y_i = x_i + sum_d c'_d x_{i-d}
//   (the identity plus the small correction, as in the transform forms) ->
//   kinetic post-phase -> store.
// Shared-memory layout, H = the halo width rounded up to even, so that element
// pairs (and complex128 elements) are 16-byte aligned:
//   contiguous slices (rows): slice w at w * Ls, Ls = q + 2H rounded up to
//   even, element i at + H + i;
//   strided slices (adjacent columns, W a power of two >= 2): element (w, i)
//   at (i + H) W + w.
// Consecutive threads touch consecutive words in every phase.
__host__ __device__ constexpr int stencil_halo(int bv) { return (bv + 1) & ~1; }
__host__ __device__ inline int stencil_row_len(int q, int bv) {
  const int l = q + 2 * stencil_halo(bv);
  return (l + 1) & ~1;
}

// Kinetic phase turns q(m) = A m^2 + la m + c0 (64-bit fixed point) along a
// thread's elements m, m + st, m + 2 st, ... by exact second differences
// modulo 2^64; scale(u) walks u q instead.
struct KinWalk {
  uint64_t q, d, dd;
  __device__ __forceinline__ void init(uint64_t A, uint64_t la, uint64_t c0, int64_t m, int64_t st) {
    const uint64_t um = (uint64_t)m, us = (uint64_t)st;
    q = A * (um * um) + la * um + c0;
    d = A * (2 * um * us + us * us) + la * us;
    dd = 2 * A * (us * us);
  }
  __device__ __forceinline__ void scale(uint64_t u) {
    q *= u;
    d *= u;
    dd *= u;
  }
  __device__ __forceinline__ void next() {
    q += d;
    d += dd;
  }
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_raw(unsigned sa, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// exp(2 pi i t / 2^64) to about 5e-7 absolute: the top 32 bits of t as a
// float angle and the hardware sine and cosine.  Used only for factors that
// multiply the small correction term of the interaction frame (taps of size
// about s |v|), where this error is scaled far below the working precision.
__device__ __forceinline__ float2 cis_fast(uint64_t t) {
  const int32_t h = (int32_t)(uint32_t)(t >> 32);
  float sn, cs;
  __sincosf((float)h * 1.46291807926715968e-09f, &sn, &cs);   // 2 pi / 2^32
  return make_float2(cs, sn);
}
template <typename Real> __device__ __forceinline__ typename CT<Real>::C cis_corr(uint64_t t);
template <> __device__ __forceinline__ float2 cis_corr<float>(uint64_t t) { return cis_fast(t); }
template <> __device__ __forceinline__ double2 cis_corr<double>(uint64_t t) { return phase_of<double>(t).v; }

// Interaction-frame correction of one complex64 element,
//   sum_{d=1..BV} [w^d t_d x_{m-d} + conj(w)^d t_{-d} x_{m+d}],  w = (c, s),
// in paired FP32 operations on broadcast pairs of the tap factors:
// with pa = x1 t1.x + x2 t2.x, pb = x1 t1.x - x2 t2.x, qa = x1 t1.y + x2 t2.y,
// qb = x1 t1.y - x2 t2.y, the pair contributes (S1, S2) += (c_d pa - s_d qb,
// c_d qa + s_d pb) and the sum is S1 + i S2.  cos 2a = 2 c^2 - 1 and
// sin 2a = 2 c s give the second power; higher powers by products.
template <int BV> struct IpTaps {
  float2 t1x[BV], t1y[BV], nt1y[BV], t2x[BV], nt2x[BV], t2y[BV];
};
template <int BV>
__device__ __forceinline__ float2 ip_corr_f(const float2* sp, int sstep, const IpTaps<BV>& T, float c, float s) {
  float2 Cd = make_float2(c, c), Sd = make_float2(s, s);
  float2 Sa = make_float2(0.f, 0.f), Sb = make_float2(0.f, 0.f);
#pragma unroll
  for (int d = 1; d <= BV; ++d) {
    const float2 x1 = sp[-d * sstep], x2 = sp[d * sstep];
    const float2 p1 = __fmul2_rn(x1, T.t1x[d - 1]);
    const float2 pa = __ffma2_rn(x2, T.t2x[d - 1], p1);
    const float2 pb = __ffma2_rn(x2, T.nt2x[d - 1], p1);
    const float2 q2 = __fmul2_rn(x2, T.t2y[d - 1]);
    const float2 qa = __ffma2_rn(x1, T.t1y[d - 1], q2);
    const float2 qbn = __ffma2_rn(x1, T.nt1y[d - 1], q2);   // -qb
    Sa = __ffma2_rn(pa, Cd, Sa);
    Sa = __ffma2_rn(qbn, Sd, Sa);
    Sb = __ffma2_rn(qa, Cd, Sb);
    Sb = __ffma2_rn(pb, Sd, Sb);
    if (d < BV) {
      if (d == 1) {
        const float2 C2 = __fadd2_rn(Cd, Cd);
        Sd = __fmul2_rn(C2, Sd);
        Cd = __ffma2_rn(C2, Cd, make_float2(-1.f, -1.f));
      } else {
        const float cn = fmaf(Cd.x, c, -Sd.x * s), sn = fmaf(Sd.x, c, Cd.x * s);
        Cd = make_float2(cn, cn);
        Sd = make_float2(sn, sn);
      }
    }
  }
  return make_float2(Sa.x - Sb.y, Sa.y + Sb.x);
}

template <typename Real, int MODE, bool CG, int BV, bool IP = false>
__device__ __forceinline__ void stencil_tile(const PassArgs& a, int64_t tile, unsigned char* smraw) {
  using C = typename CT<Real>::C;
  static_assert(!IP || MODE == MODE_STEP, "the interaction frame is a deterministic-step form");
  constexpr bool lazy = (MODE == MODE_LAZY);
  constexpr int NTAP = 2 * BV + 1;
  constexpr int H = stencil_halo(BV);
  constexpr int PAIR = sizeof(C) == 8 ? 2 : 1;   // elements per 16-byte copy
  const LayerGeom& g = a.g;
  const int W = a.W, q = g.qa;
  const bool strided = a.strided != 0;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = NT >> 5;
  // a tile past the last slice (the tail of a multi-tile work item) is empty
  if (tile * W >= (a.list ? (int64_t)a.nlist : g.nslices)) return;
  C* sm = reinterpret_cast<C*>(smraw);
  int64_t* s_slice = g_tm.slice;
  uint64_t *s_la = g_tm.la, *s_c0 = g_tm.c0;
  int32_t* s_touch = g_tm.touch;
  if (tid < W) {
    int64_t sl = -1;
    if (a.list) {
      const int64_t li = tile * W + tid;
      if (li < a.nlist) sl = a.list[li];
    } else {
      sl = tile * W + tid;
      if (sl >= g.nslices) sl = -1;
    }
    s_slice[tid] = sl;
    uint64_t la = 0, c0 = 0;
    int32_t touch = 0;
    if (sl >= 0) {
      const uint64_t ua = (uint64_t)(sl + g.olo_a);
      la = g.X_aa * ua;
      c0 = g.C_aa * (ua * ua);
      if (lazy) touch = CG ? __ldcg(a.touch_own + sl) : a.touch_own[sl];
    }
    s_la[tid] = la;
    s_c0[tid] = c0;
    s_touch[tid] = touch;
  }
  // complex64 with at most 7 taps: the multiply-adds run as paired FP32
  // operations, sum_k v_k (t_k.x, t_k.x) and sum_k v_k (t_k.y, t_k.y) in two
  // accumulators combined at the end
  constexpr bool PACK = sizeof(Real) == 4 && BV <= 3;
  C t[NTAP];
  {
    const C* tp = reinterpret_cast<const C*>(a.taps);
#pragma unroll
    for (int k = 0; k < NTAP; ++k) t[k] = tp[k];
  }
  __syncthreads();
  C* psi = reinterpret_cast<C*>(a.psi);
  const int Ls = stencil_row_len(q, BV);
  // ---- load: 16-byte copies global -> shared through L2
  if (!strided) {
    // rows, one warp per row (a row starts 128-byte aligned and its pitch
    // padding covers the pair past an odd end)
    const int np2 = (q + PAIR - 1) / PAIR;
    for (int w = warp; w < W; w += nwarp) {
      const int64_t sl = s_slice[w];
      if (sl < 0) continue;
      // lane j copies bytes [16 j, 16 j + 16) of each 512-byte run
      unsigned sa = (unsigned)__cvta_generic_to_shared(sm + w * Ls + H) + 16u * lane;
      const char* ga = reinterpret_cast<const char*>(psi + sl * g.slice_stride) + 16 * lane;
#pragma unroll 4
      for (int j = lane; j < np2; j += 32, sa += 512u, ga += 512) cp_async16_raw(sa, ga);
    }
  } else if (!a.list) {
    // adjacent columns: one copy moves PAIR columns of a row; tiles start at a
    // multiple of W columns and never read past the row pitch
    // (NT is a multiple of wp, so each thread keeps its copy column k and
    // steps NT / wp rows)
    const int wp = W / PAIR;
    const int wsh = 31 - __clz(wp);
    const int64_t s0 = tile * (int64_t)W;
    const int k = tid & (wp - 1), di = NT >> wsh;
    int i = tid >> wsh;
    unsigned sa = (unsigned)__cvta_generic_to_shared(sm + (i + H) * W + PAIR * k);
    const char* ga = reinterpret_cast<const char*>(psi + s0 + (int64_t)i * g.ea + PAIR * k);
    const unsigned dsa = (unsigned)(di * W * (int)sizeof(C));
    const int64_t dga = (int64_t)di * g.ea * (int64_t)sizeof(C);
#pragma unroll 4
    for (; i < q; i += di, sa += dsa, ga += dga) cp_async16_raw(sa, ga);
  } else {
    // sampled (scattered) columns: plain loads, the column fixed per thread
    const int wsh = 31 - __clz(W);
    const int w = tid & (W - 1), di = NT >> wsh;
    const int64_t sl = s_slice[w];
#pragma unroll 4
    for (int i = tid >> wsh; i < q; i += di) {
      C x = czero<C>();
      if (sl >= 0) x = ldpsi<CG>(psi + sl + (int64_t)i * g.ea);
      sm[(i + H) * W + w] = x;
    }
  }
  // interaction frame: the tap factors c_d e^{-2 pi i t A d^2}, formed while
  // the copies are in flight
  C tf[NTAP];
  if constexpr (IP) {
    const uint64_t tu = (uint64_t)a.ip_t;
#pragma unroll
    for (int d = 1; d <= BV; ++d) {
      const C e = cis_corr<Real>((uint64_t)0 - tu * g.A_aa * (uint64_t)(d * d));
      tf[BV + d] = cmul(t[BV + d], e);
      tf[BV - d] = cmul(t[BV - d], e);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // Element ownership in the phase and stencil sweeps.  Contiguous tiles:
  // work units of CH consecutive elements of one slice (unit u: slice u / nch,
  // chunk u mod nch), taken by the warps in turn, lane l owning elements
  // l, l + 32, ... of its unit; strided tiles: one unit per thread, the column
  // w = tid mod W and rows i = tid / W + k NT / W.  Every thread walks its
  // kinetic phase turns by second differences along its elements.
  constexpr int CH = 256;
  const int wsh = 31 - __clz(W);
  const int nch = (q + CH - 1) / CH;
  const int u0 = strided ? 0 : warp;                            // first unit of this thread
  const int ud = strided ? 1 : nwarp;                           // unit step
  const int nunit = strided ? 1 : W * nch;
  const int eid = strided ? (NT >> wsh) : 32;                   // element step
  const int sstep = strided ? W : 1;                            // shared-memory step between neighbours
  // unit u -> slice w, elements [i0, i1) owned with step eid from ei
  auto unit = [&](int u, int& w, int& ei, int& i1) {
    if (strided) {
      w = tid & (W - 1);
      ei = tid >> wsh;
      i1 = q;
    } else {
      w = u / nch;
      const int c = u - w * nch;
      ei = c * CH + lane;
      i1 = min(q, (c + 1) * CH);
    }
  };
  // ---- kinetic pre-phase (first pass of a call) or the pending lazy phase
  // (none in the interaction frame: psi~ = psi at the start of a call)
  if (!IP && (lazy || a.units_pre != 0)) {
    for (int u = u0; u < nunit; u += ud) {
      int w, ei0, i1;
      unit(u, w, ei0, i1);
      const int64_t sl = s_slice[w];
      if (sl >= 0) {
        KinWalk kw;
        kw.init(g.A_aa, s_la[w], s_c0[w], g.lo_a + ei0, eid);
        if (!lazy) kw.scale((uint64_t)0 - (uint64_t)a.units_pre);
        const int32_t tw = s_touch[w];
        C* p = sm + (strided ? (ei0 + H) * W + w : w * Ls + H + ei0);
        for (int i = ei0; i < i1; i += eid) {
          if (lazy) {
            const int32_t t2 = CG ? __ldcg(a.touch_other + i) : a.touch_other[i];
            const int64_t units = (int64_t)a.now - (int64_t)(tw > t2 ? tw : t2);
            if (units != 0) *p = apply_phase<Real>(*p, phase_of<Real>((uint64_t)0 - (uint64_t)units * kw.q));
          } else {
            *p = apply_phase<Real>(*p, phase_of<Real>(kw.q));
          }
          p += eid * sstep;
          kw.next();
        }
      }
    }
    __syncthreads();
  }
  // ---- wrap halos: i in [-BV, 0) takes x_{i + q}, i in [q, q + BV) takes x_{i - q}.
  // In the interaction frame a wrapped neighbour j' = j mod q is stored as
  // x~_{j'} e^{2 pi i t (kappa(j) - kappa(j'))}, so that the taps' phases,
  // written for the unwrapped index j, hold at the slice ends too.
  for (int e = tid; e < W * 2 * BV; e += NT) {
    const int w = e / (2 * BV), k = e - w * (2 * BV);
    const int dst = k < BV ? k - BV : q + (k - BV);
    const int src = k < BV ? q - BV + k : k - BV;
    C v = strided ? sm[(src + H) * W + w] : sm[w * Ls + H + src];
    if constexpr (IP) {
      const int64_t mj = (int64_t)g.lo_a + dst, mk = (int64_t)g.lo_a + src;
      const uint64_t turns =
          (uint64_t)a.ip_t * ((uint64_t)(mj - mk) * (g.A_aa * (uint64_t)(mj + mk) + s_la[w]));
      v = cmul(v, cis_corr<Real>(turns));
    }
    if (strided) sm[(dst + H) * W + w] = v;
    else sm[w * Ls + H + dst] = v;
  }
  __syncthreads();
  // ---- interaction frame: y = x + sum_{d != 0} c_d e^{-2 pi i t A d^2} w^d x_{i-d},
  // w = e^{2 pi i t (2 A m + l)} per element; the pairs d, -d combine as
  // w^d u + conj(w)^d v = cos(d a) (u + v) + i sin(d a) (u - v); the call's last
  // pass applies Lambda K(T) with the error-free product
  if constexpr (IP) {
    const uint64_t tu = (uint64_t)a.ip_t;
    auto sweep = [&](auto post_c) {
      constexpr bool POST = decltype(post_c)::value;
      for (int u = u0; u < nunit; u += ud) {
        int w, ei0, i1;
        unit(u, w, ei0, i1);
        const int64_t sl = s_slice[w];
        if (sl < 0) continue;
        const uint64_t twoA = 2 * g.A_aa;
        uint64_t phi = tu * (twoA * (uint64_t)(int64_t)(g.lo_a + ei0) + s_la[w]);
        const uint64_t dphi = tu * twoA * (uint64_t)eid;
        KinWalk kw;
        if constexpr (POST) {
          kw.init(g.A_aa, s_la[w], s_c0[w], g.lo_a + ei0, eid);
          kw.scale((uint64_t)0 - (uint64_t)a.units_post);
          kw.q += a.lam_turns;
        }
        const C* sp = sm + (strided ? (ei0 + H) * W + w : w * Ls + H + ei0);
        C* gp = psi + sl * g.slice_stride + (int64_t)ei0 * g.ea;
        const int64_t gstep = (int64_t)eid * g.ea;
        for (int i = ei0; i < i1; i += eid) {
          const C om = cis_corr<Real>(phi);
          phi += dphi;
          C od = om;
          C S1 = czero<C>(), S2 = czero<C>();
#pragma unroll
          for (int d = 1; d <= BV; ++d) {
            const C x1 = sp[-d * sstep], x2 = sp[d * sstep];
            const C t1 = tf[BV + d], t2 = tf[BV - d];
            C pa, pb, qa, qb;
            if constexpr (sizeof(Real) == 4) {
              const float2 p1 = __fmul2_rn(x1, make_float2(t1.x, t1.x));
              pa = __ffma2_rn(x2, make_float2(t2.x, t2.x), p1);
              pb = __ffma2_rn(x2, make_float2(-t2.x, -t2.x), p1);
              const float2 q1 = __fmul2_rn(x1, make_float2(t1.y, t1.y));
              qa = __ffma2_rn(x2, make_float2(t2.y, t2.y), q1);
              qb = __ffma2_rn(x2, make_float2(-t2.y, -t2.y), q1);
              S1 = __ffma2_rn(pa, make_float2(od.x, od.x), S1);
              S1 = __ffma2_rn(qb, make_float2(-od.y, -od.y), S1);
              S2 = __ffma2_rn(qa, make_float2(od.x, od.x), S2);
              S2 = __ffma2_rn(pb, make_float2(od.y, od.y), S2);
            } else {
              pa.x = fma(x2.x, t2.x, x1.x * t1.x);
              pa.y = fma(x2.y, t2.x, x1.y * t1.x);
              pb.x = fma(x2.x, -t2.x, x1.x * t1.x);
              pb.y = fma(x2.y, -t2.x, x1.y * t1.x);
              qa.x = fma(x2.x, t2.y, x1.x * t1.y);
              qa.y = fma(x2.y, t2.y, x1.y * t1.y);
              qb.x = fma(x2.x, -t2.y, x1.x * t1.y);
              qb.y = fma(x2.y, -t2.y, x1.y * t1.y);
              S1.x = fma(od.x, pa.x, fma(-od.y, qb.x, S1.x));
              S1.y = fma(od.x, pa.y, fma(-od.y, qb.y, S1.y));
              S2.x = fma(od.x, qa.x, fma(od.y, pb.x, S2.x));
              S2.y = fma(od.x, qa.y, fma(od.y, pb.y, S2.y));
            }
            if (d < BV) od = cmul(od, om);
          }
          C y = sp[0];
          y.x += S1.x - S2.y;
          y.y += S1.y + S2.x;
          if constexpr (POST) {
            Phase<Real> ph = phase_of<Real>(kw.q);
            if constexpr (sizeof(Real) == 4) {
              ph.half_e += (Real)a.lam_def;
            } else {
              ph.v.x *= 1.0 - a.lam_def;
              ph.v.y *= 1.0 - a.lam_def;
            }
            y = apply_phase<Real>(y, ph);
            kw.next();
          }
          *gp = y;
          sp += eid * sstep;
          gp += gstep;
        }
      }
    };
    // (complex64 tiles of rows of length >= 32 or of columns run
    // stencil_tile_ipf instead; this general sweep serves the rest)
    if (a.units_post != 0) sweep(std::integral_constant<bool, true>());
    else sweep(std::integral_constant<bool, false>());
  } else
  // ---- y = x + sum_d c'_d x_{i-d}, post-phase, store
  {
    const bool post = !lazy && a.units_post != 0;
    for (int u = u0; u < nunit; u += ud) {
      int w, ei0, i1;
      unit(u, w, ei0, i1);
      const int64_t sl = s_slice[w];
      if (sl >= 0) {
        KinWalk kw;
        kw.init(g.A_aa, s_la[w], s_c0[w], g.lo_a + ei0, eid);
        kw.scale((uint64_t)0 - (uint64_t)a.units_post);
        const C* sp = sm + (strided ? (ei0 + H) * W + w : w * Ls + H + ei0);
        C* gp = psi + sl * g.slice_stride + (int64_t)ei0 * g.ea;
        const int64_t gstep = (int64_t)eid * g.ea;
        for (int i = ei0; i < i1; i += eid) {
          C acc = czero<C>();
          if constexpr (PACK) {
            float2 ax = make_float2(0.f, 0.f), ay = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < NTAP; ++k) {
              const float2 v = *reinterpret_cast<const float2*>(sp + (BV - k) * sstep);
              ax = __ffma2_rn(v, make_float2(t[k].x, t[k].x), ax);
              ay = __ffma2_rn(v, make_float2(t[k].y, t[k].y), ay);
            }
            acc.x = ax.x - ay.y;
            acc.y = ax.y + ay.x;
          } else {
#pragma unroll
            for (int k = 0; k < NTAP; ++k) {
              // tap k is d = k - BV: x_{i - d} sits (BV - k) steps from x_i
              const C v = sp[(BV - k) * sstep];
              acc.x = fma(t[k].x, v.x, fma(-t[k].y, v.y, acc.x));
              acc.y = fma(t[k].x, v.y, fma(t[k].y, v.x, acc.y));
            }
          }
          C y = cadd(sp[0], acc);
          if (post) y = apply_phase<Real>(y, phase_of<Real>(kw.q));
          *gp = y;
          sp += eid * sstep;
          gp += gstep;
          kw.next();
        }
      }
    }
  }
  if (lazy && tid < W && s_slice[tid] >= 0) a.touch_own[s_slice[tid]] = a.now;
}

// Interaction-frame compact tile for complex64 (rows of length >= 32, or
// columns), with one CTA barrier per tile (after the copies).  Slice indices
// and kinetic coefficients come from the tile index.  Each warp (rows) or
// thread (columns) writes the wrapped halo entries it reads itself; another
// writer of the same entry writes the same value, so no barrier separates the
// halo from the sweep.  Rows are swept as one balanced flat range per warp (a
// row change is a predicated jump of the pointers and the phase), columns one
// per thread; the call's last pass applies Lambda K(T) with the exact phase.
template <int BV>
__device__ __forceinline__ void stencil_tile_ipf(const PassArgs& a, int64_t tile, unsigned char* smraw) {
  constexpr int H = stencil_halo(BV);
  const LayerGeom& g = a.g;
  const int W = a.W, q = g.qa;
  const bool strided = a.strided != 0;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = NT >> 5;
  const int64_t s0 = tile * (int64_t)W;
  if (s0 >= g.nslices) return;
  const int Wv = (int)min((int64_t)W, g.nslices - s0);
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int Ls = stencil_row_len(q, BV);
  float2 t[2 * BV + 1];
  {
    const float2* tp = reinterpret_cast<const float2*>(a.taps);
#pragma unroll
    for (int k = 0; k <= 2 * BV; ++k) t[k] = tp[k];
  }
  float2* pg = reinterpret_cast<float2*>(a.psi);
  const int64_t sstr = g.slice_stride, ea = g.ea;
  // ---- copies (16 bytes = two elements each) global -> shared through L2
  if (!strided) {
    const int np2 = (q + 1) / 2;
    for (int w = warp; w < Wv; w += nwarp) {
      unsigned sa = (unsigned)__cvta_generic_to_shared(sm + w * Ls + H) + 16u * lane;
      const char* ga = reinterpret_cast<const char*>(pg + (s0 + w) * sstr) + 16 * lane;
#pragma unroll 4
      for (int j = lane; j < np2; j += 32, sa += 512u, ga += 512) cp_async16_raw(sa, ga);
    }
  } else {
    const int wp = W / 2;
    const int wsh = 31 - __clz(wp);
    const int k = tid & (wp - 1), di = NT >> wsh;
    int i = tid >> wsh;
    unsigned sa = (unsigned)__cvta_generic_to_shared(sm + (i + H) * W + 2 * k);
    const char* ga = reinterpret_cast<const char*>(pg + s0 + (int64_t)i * ea + 2 * k);
    const unsigned dsa = (unsigned)(di * W * 8);
    const int64_t dga = (int64_t)di * ea * 8;
#pragma unroll 4
    for (; i < q; i += di, sa += dsa, ga += dga) cp_async16_raw(sa, ga);
  }
  const uint64_t tu = (uint64_t)a.ip_t, A = g.A_aa, twoA = 2 * g.A_aa, Xa = g.X_aa, Ca = g.C_aa;
  const int lo = g.lo_a;
  const int64_t olo = g.olo_a;
  // tap factors c_d e^{-2 pi i t A d^2} as broadcast pairs, while the copies fly
  IpTaps<BV> T;
#pragma unroll
  for (int d = 1; d <= BV; ++d) {
    const float2 e = cis_fast((uint64_t)0 - tu * A * (uint64_t)(d * d));
    const float2 t1 = cmul(t[BV + d], e), t2 = cmul(t[BV - d], e);
    T.t1x[d - 1] = make_float2(t1.x, t1.x);
    T.t1y[d - 1] = make_float2(t1.y, t1.y);
    T.nt1y[d - 1] = make_float2(-t1.y, -t1.y);
    T.t2x[d - 1] = make_float2(t2.x, t2.x);
    T.nt2x[d - 1] = make_float2(-t2.x, -t2.x);
    T.t2y[d - 1] = make_float2(t2.y, t2.y);
  }
  cp_async_wait_all();
  __syncthreads();
  // halo entry k of line w: i in [-BV, 0) takes x_{i + q}, i in [q, q + BV)
  // takes x_{i - q}, times e^{2 pi i t (kappa(i) - kappa(i mod q))}
  auto fill_halo = [&](int w, int k) {
    const int dst = k < BV ? k - BV : q + (k - BV);
    const int src = k < BV ? q - BV + k : k - BV;
    const int64_t mj = (int64_t)lo + dst, mk = (int64_t)lo + src;
    const uint64_t la = Xa * (uint64_t)(s0 + w + olo);
    const float2 f = cis_fast(tu * ((uint64_t)(mj - mk) * (A * (uint64_t)(mj + mk) + la)));
    if (strided) sm[(dst + H) * W + w] = cmul(sm[(src + H) * W + w], f);
    else sm[w * Ls + H + dst] = cmul(sm[w * Ls + H + src], f);
  };
  const uint64_t negT = (uint64_t)0 - (uint64_t)a.units_post;
  auto walk_at = [&](int w, int i, int step) {
    KinWalk kw;
    const uint64_t ua = (uint64_t)(s0 + w + olo);
    kw.init(A, Xa * ua, Ca * (ua * ua), lo + i, step);
    kw.scale(negT);
    kw.q += a.lam_turns;
    return kw;
  };
  auto finish = [&](float2 y, const KinWalk& kw) {
    Phase<float> ph = phase_of<float>(kw.q);
    ph.half_e += (float)a.lam_def;
    return apply_phase<float>(y, ph);
  };
  auto sweep = [&](auto post_c) {
    constexpr bool POST = decltype(post_c)::value;
    if (!strided) {
      const int total = Wv * q;
      const int per = ((total + nwarp * 32 - 1) / (nwarp * 32)) * 32;
      const int e0 = warp * per, e1 = min(total, (warp + 1) * per);
      if (e0 >= e1) return;
      // the halos of every row this warp's range touches
      const int wa = e0 / q, wb = (e1 - 1) / q;
      for (int r = lane; r < (wb - wa + 1) * 2 * BV; r += 32) fill_halo(wa + r / (2 * BV), r % (2 * BV));
      __syncwarp();
      // lane l takes the elements e0 + l + 32 k < e1, row by row
      const uint64_t dphi = tu * twoA * 32u;
      for (int w = wa; w <= wb; ++w) {
        const int rs = max(e0, w * q), re = min(e1, (w + 1) * q);
        // first element of this lane in [rs, re)
        const int ef = rs + ((e0 + lane - rs) & 31);
        if (ef >= re) continue;
        int i = ef - w * q;
        const int iend = re - w * q;
        const float2* sp = sm + w * Ls + H + i;
        float2* gp = pg + (s0 + w) * sstr + i;
        uint64_t phi = tu * (twoA * (uint64_t)(int64_t)(lo + i) + Xa * (uint64_t)(s0 + w + olo));
        KinWalk kw;
        if constexpr (POST) kw = walk_at(w, i, 32);
        for (; i < iend; i += 32) {
          const float2 cs = cis_fast(phi);
          const float2 corr = ip_corr_f<BV>(sp, 1, T, cs.x, cs.y);
          const float2 x0 = sp[0];
          float2 y = make_float2(x0.x + corr.x, x0.y + corr.y);
          if constexpr (POST) {
            y = finish(y, kw);
            kw.next();
          }
          __stcg(gp, y);
          sp += 32;
          gp += 32;
          phi += dphi;
        }
      }
    } else {
      const int wsh = 31 - __clz(W);
      const int w = tid & (W - 1);
      if (w >= Wv) return;
#pragma unroll
      for (int k = 0; k < 2 * BV; ++k) fill_halo(w, k);
      const int eid = NT >> wsh;
      int i = tid >> wsh;
      const float2* sp = sm + (i + H) * W + w;
      float2* gp = pg + (s0 + w) + (int64_t)i * ea;
      uint64_t phi = tu * (twoA * (uint64_t)(int64_t)(lo + i) + Xa * (uint64_t)(s0 + w + olo));
      const uint64_t dphi = tu * twoA * (uint64_t)eid;
      const int dsp = eid * W;
      const int64_t dg = (int64_t)eid * ea;
      KinWalk kw;
      if constexpr (POST) kw = walk_at(w, i, eid);
      for (; i < q; i += eid) {
        const float2 cs = cis_fast(phi);
        const float2 corr = ip_corr_f<BV>(sp, W, T, cs.x, cs.y);
        const float2 x0 = sp[0];
        float2 y = make_float2(x0.x + corr.x, x0.y + corr.y);
        if constexpr (POST) {
          y = finish(y, kw);
          kw.next();
        }
        __stcg(gp, y);
        sp += dsp;
        gp += dg;
        phi += dphi;
      }
    }
  };
  if (a.units_post != 0) sweep(std::integral_constant<bool, true>());
  else sweep(std::integral_constant<bool, false>());
}

template <typename Real, int MODE, int BV, bool IP = false>
__global__ void __launch_bounds__(kStencilThreads, sizeof(Real) == 4 ? 3 : 2)
pass_stencil_kernel(const PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if constexpr (IP && sizeof(Real) == 4) {
    if (a.strided || a.g.qa >= 32) {
      stencil_tile_ipf<BV>(a, (int64_t)blockIdx.x, smraw);
      return;
    }
  }
  stencil_tile<Real, MODE, false, BV, IP>(a, (int64_t)blockIdx.x, smraw);
}

template <typename Real> size_t stencil_smem_bytes(const LayerGeom& g, int W, int B) {
  using C = typename CT<Real>::C;
  return (size_t)W * stencil_row_len(g.qa, B) * sizeof(C);
}

template <typename Real, int BV>
static cudaError_t launch_stencil_b(const PassArgs& a, int64_t ntiles, cudaStream_t st) {
  const size_t smem = stencil_smem_bytes<Real>(a.g, a.W, BV);
  if (a.mode == MODE_LAZY) pass_stencil_kernel<Real, MODE_LAZY, BV><<<(unsigned)ntiles, kStencilThreads, smem, st>>>(a);
  else if (a.ip) pass_stencil_kernel<Real, MODE_STEP, BV, true><<<(unsigned)ntiles, kStencilThreads, smem, st>>>(a);
  else pass_stencil_kernel<Real, MODE_STEP, BV><<<(unsigned)ntiles, kStencilThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename Real> cudaError_t launch_stencil(const PassArgs& a, int64_t ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (a.g.d != 1 || a.W < 1 || a.W > kMaxTileSlices || (a.strided && (a.W < 2 || (a.W & (a.W - 1)))) ||
      2 * a.sB + 1 > a.g.qa || (reinterpret_cast<uintptr_t>(a.psi) & 15) != 0 ||
      (a.strided ? (a.g.ea & 1) : (a.g.slice_stride & 1)) != 0)
    return cudaErrorInvalidValue;
  switch (a.sB) {
    case 2: return launch_stencil_b<Real, 2>(a, ntiles, st);
    case 3: return launch_stencil_b<Real, 3>(a, ntiles, st);
    case 5: return launch_stencil_b<Real, 5>(a, ntiles, st);
    case 8: return launch_stencil_b<Real, 8>(a, ntiles, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename Real> cudaError_t stencil_prepare(size_t max_smem) {
  cudaError_t e = cudaSuccess;
#define LS_SPREP(BV)                                                                                   \
  if (e == cudaSuccess) e = allow_smem(pass_stencil_kernel<Real, MODE_STEP, BV>, max_smem);           \
  if (e == cudaSuccess) e = allow_smem(pass_stencil_kernel<Real, MODE_STEP, BV, true>, max_smem);     \
  if (e == cudaSuccess) e = allow_smem(pass_stencil_kernel<Real, MODE_LAZY, BV>, max_smem);
  LS_SPREP(2) LS_SPREP(3) LS_SPREP(5) LS_SPREP(8)
#undef LS_SPREP
  return e;
}

// ---------------------------------------------------------------- batched runner
// 256-thread CTAs (the block size the host uses for every tile shape); 1D
// slices only; STOCH selects the stochastic (lazy + settle) or deterministic
// body; MINB the resident CTAs per SM the registers are budgeted for.
// Tiles of the batched runner as calls, not inlined into the persistent loop:
// each tile body then gets the kernel's whole register budget, and the loop
// keeps only its few scalars across the call.
template <typename Real, int LOGN, int MODE, bool FUSED = false>
__device__ __noinline__ void batch_fast_tile_n(const PassArgs& a, int64_t tile, unsigned char* smraw) {
  fast_tile<Real, LOGN, MODE, 1, FUSED, true>(a, tile, smraw);
}
template <typename Real, int BPT, int MODE>
__device__ __noinline__ void batch_general_tile(const PassArgs& a, int64_t tile, unsigned char* smraw) {
  pass_tile<Real, BPT, MODE, true, true>(a, tile, smraw);
}

template <typename Real, int MODE, int BV>
__device__ __noinline__ void batch_stencil_tile_n(const PassArgs& a, int64_t tile, unsigned char* smraw) {
  stencil_tile<Real, MODE, true, BV>(a, tile, smraw);
}

// Compact-kernel tile of a batched work item (sB > 0); false: not this form.
template <typename Real, int MODE, int BV, bool IP>
__device__ __noinline__ void stencil_tile_call(const PassArgs& a, int64_t tile, unsigned char* smraw) {
  if constexpr (IP && sizeof(Real) == 4) {
    if (a.strided || a.g.qa >= 32) {
      stencil_tile_ipf<BV>(a, tile, smraw);
      return;
    }
  }
  stencil_tile<Real, MODE, true, BV, IP>(a, tile, smraw);
}

template <typename Real, int MODE>
__device__ __forceinline__ bool batch_stencil_tile(const PassArgs& a, int64_t tile, unsigned char* smraw) {
  switch (a.sB) {
    case 2: batch_stencil_tile_n<Real, MODE, 2>(a, tile, smraw); return true;
    case 3: batch_stencil_tile_n<Real, MODE, 3>(a, tile, smraw); return true;
    case 5: batch_stencil_tile_n<Real, MODE, 5>(a, tile, smraw); return true;
    case 8: batch_stencil_tile_n<Real, MODE, 8>(a, tile, smraw); return true;
    default: return false;
  }
}

// Fast tile of a batched work item (complex64, transform length 2^9..2^11,
// W = 4096 / N slices so that W N / 16 = 256 threads); false: general tile.
template <typename Real, int MODE>
__device__ __forceinline__ bool batch_fast_tile(const PassArgs& a, int64_t tile, unsigned char* smraw) {
  if constexpr (sizeof(Real) == 4) {
    if (MODE == MODE_STEP && a.Khat2 != nullptr) {
      // two layer-1 factors of consecutive Strang steps (convolution form)
      switch (a.fast_logn) {
        case 9: batch_fast_tile_n<Real, 9, MODE, true>(a, tile, smraw); return true;
        case 10: batch_fast_tile_n<Real, 10, MODE, true>(a, tile, smraw); return true;
        case 11: batch_fast_tile_n<Real, 11, MODE, true>(a, tile, smraw); return true;
        default: return false;
      }
    }
    switch (a.fast_logn) {
      case 9: batch_fast_tile_n<Real, 9, MODE>(a, tile, smraw); return true;
      case 10: batch_fast_tile_n<Real, 10, MODE>(a, tile, smraw); return true;
      case 11: batch_fast_tile_n<Real, 11, MODE>(a, tile, smraw); return true;
      default: return false;
    }
  }
  return false;
}

// One work item's tile.  KIND 0: any tile kind (compact-kernel, fast and
// general transform tiles as calls with the kernel's whole register budget);
// KIND 1: compact-kernel tiles only, inlined (a batch whose every factor takes
// that form: no transform code, lighter registers, more CTAs per SM).
template <typename Real, int BPT, int MODE, int KIND>
__device__ __forceinline__ void batch_tile(const PassArgs& a, int64_t tile, unsigned char* smraw) {
  if constexpr (KIND == 1) {
    // an item covers `subtiles` consecutive tiles, processed back to back
    const int nsub = a.subtiles > 1 ? a.subtiles : 1;
    for (int k = 0; k < nsub; ++k) {
      if (k) __syncthreads();
      const int64_t tk = tile * nsub + k;

      // deterministic complex64 steps of the compact-only kernel run in the
      // interaction frame (complex128 keeps the exact per-pass phases: its
      // phase evaluation costs the same either way); the wide kernels (rare:
      // long tails) are calls, so that their registers do not weigh on the
      // common narrow ones
      constexpr bool IP = MODE == MODE_STEP && sizeof(Real) == 4;
      const bool ipf = IP && (a.strided || a.g.qa >= 32);
      switch (a.sB) {
        case 2:
          if (ipf) stencil_tile_ipf<2>(a, tk, smraw);
          else stencil_tile<Real, MODE, true, 2, IP>(a, tk, smraw);
          break;
        case 3:
          if (ipf) stencil_tile_ipf<3>(a, tk, smraw);
          else stencil_tile<Real, MODE, true, 3, IP>(a, tk, smraw);
          break;
        case 5: stencil_tile_call<Real, MODE, 5, IP>(a, tk, smraw); break;
        default: stencil_tile_call<Real, MODE, 8, IP>(a, tk, smraw); break;
      }
    }
  } else {
    if (!batch_stencil_tile<Real, MODE>(a, tile, smraw) && !batch_fast_tile<Real, MODE>(a, tile, smraw))
      batch_general_tile<Real, BPT, MODE>(a, tile, smraw);
  }
}

template <typename Real, int BPT, bool STOCH, int MINB, int KIND, int NTH = 256>
__global__ void __launch_bounds__(NTH, MINB)
batch_kernel(const BatchArgs b) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ PassArgs s_args;
  __shared__ long long s_item;
  __shared__ int s_stop, s_inst, s_pass;
  __shared__ long long s_tile, s_step;
  // fused Strang: [first L1] then per step [L2, fused L1 (last step: plain L1)]
  const long long steps_total = b.fused ? b.pass_items[0] + (long long)b.nsteps * (b.pass_items[0] + b.pass_items[1])
                                        : b.step_items * (long long)b.nsteps;
  const long long total = steps_total + (b.stoch ? b.settle_items : 0);
  volatile int32_t* status = b.status;
  volatile unsigned long long* done = b.counters + 1;
  __shared__ int s_settle;
  // small per-pass tables copied to shared memory once: indexing the kernel
  // parameter arrays with runtime indices would force a local-memory copy of
  // the whole parameter block
  __shared__ long long s_pass_items[4];
  __shared__ int32_t s_units[4][3][2];
  __shared__ int32_t s_now_off[3];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) s_pass_items[q] = b.pass_items[q];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        s_units[v][q][0] = b.units[v][q][0];
        s_units[v][q][1] = b.units[v][q][1];
      }
#pragma unroll
    for (int q = 0; q < 3; ++q) s_now_off[q] = b.now_off[q];
  }
  __syncthreads();
  // Thread 0 claims the next item one item ahead: the claim's round trip
  // overlaps the current tile.  Items still start in claim order per CTA, and
  // a CTA starts an item claimed early only after finishing the current one,
  // so the earliest unfinished item always runs with its inputs complete.
  long long claimed = -1;
  if (threadIdx.x == 0 && *status == 0) claimed = (long long)atomicAdd(&b.counters[0], 1ull);
  for (;;) {
    if (threadIdx.x == 0) {
      long long it = claimed;
      s_stop = 0;
      s_settle = 0;
      if (*status != 0) it = -1;
      s_item = (it >= 0 && it < total) ? it : -1;
      claimed = -1;
      if (s_item >= 0 && *status == 0) claimed = (long long)atomicAdd(&b.counters[0], 1ull);
      if (s_item >= 0) {
        unsigned long long need;
        int i;
        if (s_item >= steps_total) {
          // settle phase: after every sub-step of instance i
          const long long r = s_item - steps_total;
          int lo = 0, hi = b.ninst - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.settle_cum[mid] <= r) lo = mid; else hi = mid - 1;
          }
          i = lo;
          s_settle = 1;
          s_inst = i;
          s_pass = 0;
          s_tile = r - b.settle_cum[i];
          need = (unsigned long long)((long long)b.nsteps * b.tiles_step[i]);
          s_step = 0;
        } else if (b.fused) {
          const long long I1 = s_pass_items[0], I2 = s_pass_items[1];
          long long r = s_item, nl1 = 0, nl2 = 0;
          int kind = 0, layer = 0;
          s_step = 0;
          if (r >= I1) {
            r -= I1;
            const long long k = r / (I1 + I2);
            s_step = k;
            r -= k * (I1 + I2);
            if (r < I2) {
              kind = 1;
              layer = 1;
              nl1 = k + 1;
              nl2 = k;
            } else {
              r -= I2;
              kind = k == b.nsteps - 1 ? 3 : 2;
              nl1 = k + 1;
              nl2 = k + 1;
            }
          }
          const int64_t* cum = b.cum + (size_t)layer * (b.ninst + 1);
          int lo = 0, hi = b.ninst - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cum[mid] <= r) lo = mid; else hi = mid - 1;
          }
          i = lo;
          s_inst = i;
          s_pass = kind;
          s_tile = r - cum[i];
          need = (unsigned long long)(nl1 * b.tiles1[i] + nl2 * b.tiles2[i]);
          if (b.unmet && i == 0 && kind == 1 && nl2 == 0) need += 1;  // test hook
        } else {
          const long long k = s_item / b.step_items;
          s_step = k;
          long long r = s_item - k * b.step_items;
          int p = 0;
          while (p + 1 < b.npass && r >= s_pass_items[p]) {
            r -= s_pass_items[p];
            ++p;
          }
          // instance: largest i with cum[p][i] <= r
          const int64_t* cum = b.cum + (size_t)p * (b.ninst + 1);
          int lo = 0, hi = b.ninst - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cum[mid] <= r) lo = mid; else hi = mid - 1;
          }
          i = lo;
          s_inst = i;
          s_pass = p;
          s_tile = r - cum[i];
          // completed tiles of instance i needed before this pass may start
          need = (unsigned long long)(k * b.tiles_step[i]);
          for (int pp = 0; pp < p; ++pp) {
            const int64_t* c2 = b.cum + (size_t)pp * (b.ninst + 1);
            need += (unsigned long long)(c2[i + 1] - c2[i]);
          }
          if (b.unmet && i == 0 && p == 1 && k == 0) need += 1;  // test hook
        }
        const long long t0 = clock64();
        unsigned int spins = 0;
        while (done[i] < need) {
          if (*status != 0) { s_stop = 1; break; }
          if (clock64() - t0 > b.timeout_cycles || ++spins > (1u << 26)) {
            atomicExch(b.status, 1);
            s_stop = 1;
            break;
          }
          __nanosleep(200);
        }
        __threadfence();
      }
    }
    __syncthreads();
    if (s_item < 0 || s_stop) return;
    // per-item arguments: the instance's pass arguments with this step's
    // kinetic units (deterministic) or list and clock (stochastic)
    {
      const int i = s_inst, p = s_pass;
      const int* src = reinterpret_cast<const int*>(s_settle ? b.settle_args + i : b.args + (size_t)p * b.ninst + i);
      int* dst = reinterpret_cast<int*>(&s_args);
      for (int w = threadIdx.x; w < (int)(sizeof(PassArgs) / 4); w += blockDim.x) dst[w] = src[w];
      __syncthreads();
      if (threadIdx.x == 0 && !s_settle && !b.fused) {
        const long long k = s_item / b.step_items;
        if (b.stoch) {
          s_args.list += k * s_args.list_step;
          s_args.now = (int32_t)(k * b.now_mul + s_now_off[p]);
        } else {
          const int var = b.nsteps == 1 ? 3 : (k == 0 ? 0 : (k == b.nsteps - 1 ? 2 : 1));
          s_args.units_pre = s_units[var][p][0];
          s_args.units_post = s_units[var][p][1];
        }
      }
      if (threadIdx.x == 0 && b.ip && !s_settle) s_args.ip_t = s_step * b.ip_step + b.ip_off[p];
      __syncthreads();
    }
    if constexpr (STOCH) {
      if (s_settle) batch_general_tile<Real, BPT, MODE_KIN>(s_args, s_tile, smraw);
      else batch_tile<Real, BPT, MODE_LAZY, KIND>(s_args, s_tile, smraw);
    } else {
      batch_tile<Real, BPT, MODE_STEP, KIND>(s_args, s_tile, smraw);
      if (b.fused && s_pass == 2 && s_args.Khat2 == nullptr) {
        // fused item without a fused tile body: the second factor on the same
        // slices, after the first is complete in this CTA (the barrier orders
        // the CTA's own global writes before its reads)
        __syncthreads();
        const int* src = reinterpret_cast<const int*>(b.args + (size_t)4 * b.ninst + s_inst);
        int* dst = reinterpret_cast<int*>(&s_args);
        for (int w = threadIdx.x; w < (int)(sizeof(PassArgs) / 4); w += blockDim.x) dst[w] = src[w];
        __syncthreads();
        if (threadIdx.x == 0 && b.ip) s_args.ip_t = s_step * b.ip_step + b.ip_off[4];
        __syncthreads();
        batch_tile<Real, BPT, MODE_STEP, KIND>(s_args, s_tile, smraw);
      }
    }
    // every thread's stores precede the barrier; thread 0 then fences at GPU
    // scope and publishes the completed tile to the other CTAs
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd((unsigned long long*)&done[s_inst], 1ull);
    }
  }
}

// Variants (threads per CTA, CTAs per SM the registers are budgeted for):
// KIND 0: (256, 3); KIND 1 (compact-kernel tiles only): (256, 3), (256, 4),
// (128, 6), (128, 8) for complex64 and (256, 3) for complex128.
template <typename Real, int KIND, int MINB, int NTH>
static cudaError_t launch_batch_v(const BatchArgs& b, int nblocks, size_t smem, cudaStream_t st) {
  if (b.stoch) batch_kernel<Real, 2, true, MINB, KIND, NTH><<<nblocks, NTH, smem, st>>>(b);
  else batch_kernel<Real, 2, false, MINB, KIND, NTH><<<nblocks, NTH, smem, st>>>(b);
  return cudaGetLastError();
}

template <typename Real, int KIND, int MINB, int NTH>
static cudaError_t batch_prepare_v(size_t max_smem, size_t smem, int* blocks_per_sm) {
  int a = 0, c = 0;
  cudaError_t e = allow_smem(batch_kernel<Real, 2, false, MINB, KIND, NTH>, max_smem);
  if (e == cudaSuccess) e = allow_smem(batch_kernel<Real, 2, true, MINB, KIND, NTH>, max_smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, batch_kernel<Real, 2, false, MINB, KIND, NTH>, NTH, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, batch_kernel<Real, 2, true, MINB, KIND, NTH>, NTH, smem);
  *blocks_per_sm = a < c ? a : c;
  return e;
}

// Dispatch over the variants; a (kind, minb, nthreads) without a variant
// returns cudaErrorInvalidValue.
#define LS_BATCH_VARIANTS(F, ...)                                                                  \
  if (kind == 0 && minb == 3 && nthreads == 256) return F<Real, 0, 3, 256>(__VA_ARGS__);          \
  if (kind == 1 && minb == 3 && nthreads == 256) return F<Real, 1, 3, 256>(__VA_ARGS__);          \
  if constexpr (sizeof(Real) == 4) {                                                               \
    if (kind == 1 && minb == 4 && nthreads == 256) return F<Real, 1, 4, 256>(__VA_ARGS__);        \
    if (kind == 1 && minb == 6 && nthreads == 128) return F<Real, 1, 6, 128>(__VA_ARGS__);        \
    if (kind == 1 && minb == 8 && nthreads == 128) return F<Real, 1, 8, 128>(__VA_ARGS__);        \
  }                                                                                                \
  return cudaErrorInvalidValue;

template <typename Real> cudaError_t launch_batch(const BatchArgs& b, int nthreads, int nblocks, size_t smem,
                                                  cudaStream_t st) {
  const int kind = b.kind, minb = b.minb;
  LS_BATCH_VARIANTS(launch_batch_v, b, nblocks, smem, st)
}

template <typename Real> cudaError_t batch_prepare(size_t max_smem, int nthreads, size_t smem, int kind, int minb,
                                                   int* blocks_per_sm) {
  LS_BATCH_VARIANTS(batch_prepare_v, max_smem, smem, blocks_per_sm)
}
#undef LS_BATCH_VARIANTS

#define LS_FOR_MODES(X, R, B) \
  X(R, B, MODE_STEP) X(R, B, MODE_LAZY) X(R, B, MODE_MEASURE) X(R, B, MODE_ADJOINT) X(R, B, MODE_KIN)

template <typename Real> cudaError_t pass_prepare(size_t max_smem) {
  cudaError_t e = cudaSuccess;
#define LS_PREP(R, B, MD) \
  if (e == cudaSuccess) e = allow_smem(pass_kernel<R, B, MD>, max_smem);
  LS_FOR_MODES(LS_PREP, Real, 2)
  LS_FOR_MODES(LS_PREP, Real, 4)
#undef LS_PREP
  return e;
}

template <typename Real, int BPT>
static cudaError_t launch_pass_b(const PassArgs& a, int nthreads, int64_t ntiles, size_t smem,
                                 cudaStream_t st) {
  switch (a.mode) {
    case MODE_STEP: pass_kernel<Real, BPT, MODE_STEP><<<(unsigned)ntiles, nthreads, smem, st>>>(a); break;
    case MODE_LAZY: pass_kernel<Real, BPT, MODE_LAZY><<<(unsigned)ntiles, nthreads, smem, st>>>(a); break;
    case MODE_MEASURE: pass_kernel<Real, BPT, MODE_MEASURE><<<(unsigned)ntiles, nthreads, smem, st>>>(a); break;
    case MODE_ADJOINT: pass_kernel<Real, BPT, MODE_ADJOINT><<<(unsigned)ntiles, nthreads, smem, st>>>(a); break;
    case MODE_KIN: pass_kernel<Real, BPT, MODE_KIN><<<(unsigned)ntiles, nthreads, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename Real> cudaError_t launch_pass(const PassArgs& a, int bpt, int nthreads, int64_t ntiles,
                                                 cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  const size_t smem = pass_smem_bytes<Real>(a.g, a.W, a.mode);
  if (bpt == 4) return launch_pass_b<Real, 3>(a, nthreads, ntiles, smem, st);
  return launch_pass_b<Real, 2>(a, nthreads, ntiles, smem, st);
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

// Projection onto the joint cutoff (Sec. 3 index sets): every coefficient
// whose mask byte is 0 is set to zero; members are not touched.
template <typename Real>
__global__ void project_kernel(typename CT<Real>::C* psi, const uint8_t* __restrict__ mask, int64_t M1,
                               int64_t M2, int64_t pitch) {
  using C = typename CT<Real>::C;
  const int64_t total = M1 * M2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[idx]) {
      const int64_t row = idx / M1, col = idx - row * M1;
      psi[row * pitch + col] = czero<C>();
    }
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

#ifdef LS_DEFINE_MISC
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

__global__ void batch_sampler_kernel(BatchSamplerArgs sa, const uint64_t* seed_g0, int32_t* out) {
  extern __shared__ int32_t perm[];  // Smax ints, then Smax flag bytes
  const int64_t per = (int64_t)sa.nsteps * sa.npf;
  const int64_t i = blockIdx.x / per;
  const int64_t rel = blockIdx.x - i * per;
  const int pass = (int)(rel % sa.npf);
  const int S = sa.S[i * sa.npf + pass];
  const int p = sa.p[i * sa.npf + pass];
  unsigned char* flag = reinterpret_cast<unsigned char*>(perm + sa.Smax);
  const uint64_t seed = seed_g0[0] + (uint64_t)i;
  const uint64_t g = seed_g0[1] + (uint64_t)rel;
  for (int q = threadIdx.x; q < S; q += blockDim.x) {
    perm[q] = q;
    flag[q] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t state = seed ^ (g * 0xD1B54A32D192ED03ull);
    for (int q = 0; q < p; ++q) {
      const uint64_t r = splitmix64_next(state);
      const int j = q + (int)(r % (uint64_t)(S - q));
      const int t = perm[q];
      perm[q] = perm[j];
      perm[j] = t;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < p; q += blockDim.x) flag[perm[q]] = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t* o = out + sa.base[i] + (rel / sa.npf) * sa.step_len[i] + sa.pass_off[i * sa.npf + pass];
    int c = 0;
    for (int q = 0; q < S; ++q)
      if (flag[q]) o[c++] = q;
  }
}

__global__ void zero_i32_kernel(int32_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0;
}
__global__ void zero_f64_kernel(double* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0.0;
}

#endif  // LS_DEFINE_MISC

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
cudaError_t launch_project(void* psi, const uint8_t* mask, int64_t M1, int64_t M2, int64_t pitch,
                           cudaStream_t st) {
  project_kernel<Real><<<kReduceBlocks, 256, 0, st>>>(reinterpret_cast<typename CT<Real>::C*>(psi), mask, M1, M2,
                                                      pitch);
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
#ifdef LS_DEFINE_MISC
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
cudaError_t sampler_prepare(size_t smem) { return allow_smem(sampler_kernel, smem); }
cudaError_t launch_batch_sampler(const BatchSamplerArgs& sa, const uint64_t* seed_g0_dev, int64_t blocks,
                                 int32_t* out, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  const size_t smem = (size_t)sa.Smax * 5;
  batch_sampler_kernel<<<(unsigned)blocks, 256, smem, st>>>(sa, seed_g0_dev, out);
  return cudaGetLastError();
}
cudaError_t batch_sampler_prepare(size_t max_block) { return allow_smem(batch_sampler_kernel, max_block); }
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

#endif  // LS_DEFINE_MISC

#define LS_INST(R)                                                                                        \
  template cudaError_t launch_pass<R>(const PassArgs&, int, int, int64_t, cudaStream_t);                 \
  template size_t pass_smem_bytes<R>(const LayerGeom&, int, int);                                        \
  template cudaError_t pass_prepare<R>(size_t);                                                          \
  template cudaError_t launch_gaussian<R>(const ElemArgs&, void*, const double*, double, const double*, \
                                          double*, int, cudaStream_t);                                   \
  template cudaError_t launch_scale<R>(const ElemArgs&, void*, const double*, cudaStream_t);             \
  template cudaError_t launch_project<R>(void*, const uint8_t*, int64_t, int64_t, int64_t, cudaStream_t); \
  template cudaError_t launch_elem_obs<R>(const ElemArgs&, const void*, const void*, double*, int,      \
                                          cudaStream_t);                                                 \
  template cudaError_t launch_fast<R>(const PassArgs&, int64_t, cudaStream_t);                           \
  template size_t fast_smem_bytes<R>(const LayerGeom&, int, int);                                        \
  template cudaError_t fast_prepare<R>(size_t);                                                          \
  template int fast_max_threads<R>();                                                                    \
  template cudaError_t launch_stencil<R>(const PassArgs&, int64_t, cudaStream_t);                        \
  template size_t stencil_smem_bytes<R>(const LayerGeom&, int, int);                                     \
  template cudaError_t stencil_prepare<R>(size_t);                                                       \
  template cudaError_t launch_fast2d<R>(const PassArgs&, int64_t, cudaStream_t);                         \
  template size_t fast2d_smem_bytes<R>(const LayerGeom&);                                                \
  template cudaError_t fast2d_prepare<R>(size_t);
#ifdef LS_INST_REAL
LS_INST(LS_INST_REAL)
#endif
#ifdef LS_INST_BATCH
template cudaError_t launch_batch<float>(const BatchArgs&, int, int, size_t, cudaStream_t);
template cudaError_t batch_prepare<float>(size_t, int, size_t, int, int, int*);
template cudaError_t launch_batch<double>(const BatchArgs&, int, int, size_t, cudaStream_t);
template cudaError_t batch_prepare<double>(size_t, int, size_t, int, int, int*);
#endif

}  // namespace lsk

namespace lsk {
template <typename Real> int pass_max_threads(int bpt) {
  return bpt == 4 ? PassTraits<Real, 4>::kMaxNT : PassTraits<Real, 2>::kMaxNT;
}
#ifdef LS_INST_REAL
template int pass_max_threads<LS_INST_REAL>(int);
#endif
}  // namespace lsk
