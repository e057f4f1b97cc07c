// Tensor-core form of the layer pass for 64 x 64 slices (complex64, the
// contiguous layer): the correction F diag((T - 1)/M) F^{-1} x of Algorithm 3
// as four complex 64 x 64 x 64 matrix products per slice,
//   U = W X, G = U W (to the layer's grid), H = G .* (T - 1)/M,
//   V = conj(W) H, C = V conj(W) (back to coefficients),
// with X[ib][ia] the slice and W[p][k] = exp(+2 pi i p k / 64) (symmetric).
// Every real product runs on the tensor cores in split BF16 (BF16x3): each
// operand is a bf16 high part plus a bf16 low part, and hi*hi + hi*lo + lo*hi
// accumulate in FP32 (mma.sync m16n8k16), about 16 significant bits.  Only the
// correction goes through this arithmetic (y = x + C), so its relative error
// is further scaled by |T - 1| (a few 1e-3 for the workloads' time steps).
//
// One CTA of 8 warps holds one slice at a time in shared memory (persistent
// over slices, so the W planes are read once per CTA):
//   planes 0..3: the current operand (re hi, re lo, im hi, im lo), 4..7: W;
//   each plane is 64 rows of 72 bf16 (rows padded so ldmatrix rows fall on
//   distinct banks); xs: the pre-phased slice in FP32 for the identity term.
// Warp w computes the 16 x 32 output tile (rows 16 (w mod 4), columns
// 32 (w / 4)) of each product.
#include <cuda_bf16.h>

#include "lsplit_kernels.cuh"

namespace lsk {
namespace {

constexpr int kTcRow = 72;
constexpr int kTcPlane = 64 * kTcRow;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void ldsm4t(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void neg4(const uint32_t (&s)[4], uint32_t (&d)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) d[k] = s[k] ^ 0x80008000u;   // both bf16 halves
}

// hi + lo split of a pair of floats, stored as two bf16 pairs (row r, columns c, c+1)
__device__ __forceinline__ void put_split(__nv_bfloat16* hi_plane, __nv_bfloat16* lo_plane, int r, int c, float v0,
                                          float v1) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
  const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
  *reinterpret_cast<__nv_bfloat162*>(hi_plane + r * kTcRow + c) = h;
  *reinterpret_cast<__nv_bfloat162*>(lo_plane + r * kTcRow + c) = l;
}

// Out = Wc * D, Wc = W or conj(W) (planes 4..7), D = planes 0..3 (row-major,
// rows = the contracted index).  Real part Wr Dr - Wi Di, imaginary Wr Di + Wi Dr.
template <bool CONJ>
__device__ __forceinline__ void gemm_left(const __nv_bfloat16* sm, float (&cr)[4][4], float (&ci)[4][4], int rb,
                                          int cb, int lane) {
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int k = 0; k < 4; ++k) cr[t][k] = ci[t][k] = 0.f;
  const int mi = lane >> 3, rr = lane & 7;
#pragma unroll 1
  for (int k0 = 0; k0 < 64; k0 += 16) {
    uint32_t wrh[4], wrl[4], wih[4], wil[4], nih[4], nil[4];
    const int ao = (16 * rb + (mi & 1) * 8 + rr) * kTcRow + k0 + (mi >> 1) * 8;
    ldsm4(su32(sm + 4 * kTcPlane + ao), wrh);
    ldsm4(su32(sm + 5 * kTcPlane + ao), wrl);
    ldsm4(su32(sm + 6 * kTcPlane + ao), wih);
    ldsm4(su32(sm + 7 * kTcPlane + ao), wil);
    if (CONJ) {
      neg4(wih, nih);
      neg4(wil, nil);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t a = wih[k], b = wil[k];
        wih[k] = nih[k];
        wil[k] = nil[k];
        nih[k] = a;
        nil[k] = b;
      }
    } else {
      neg4(wih, nih);
      neg4(wil, nil);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int bo = (k0 + (mi & 1) * 8 + rr) * kTcRow + 32 * cb + 16 * h + (mi >> 1) * 8;
      uint32_t drh[4], drl[4], dih[4], dil[4];
      ldsm4t(su32(sm + 0 * kTcPlane + bo), drh);
      ldsm4t(su32(sm + 1 * kTcPlane + bo), drl);
      ldsm4t(su32(sm + 2 * kTcPlane + bo), dih);
      ldsm4t(su32(sm + 3 * kTcPlane + bo), dil);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        float(&r)[4] = cr[2 * h + u];
        float(&i)[4] = ci[2 * h + u];
        mma16816(r, wrh, drh[2 * u], drh[2 * u + 1]);
        mma16816(r, wrh, drl[2 * u], drl[2 * u + 1]);
        mma16816(r, wrl, drh[2 * u], drh[2 * u + 1]);
        mma16816(r, nih, dih[2 * u], dih[2 * u + 1]);
        mma16816(r, nih, dil[2 * u], dil[2 * u + 1]);
        mma16816(r, nil, dih[2 * u], dih[2 * u + 1]);
        mma16816(i, wrh, dih[2 * u], dih[2 * u + 1]);
        mma16816(i, wrh, dil[2 * u], dil[2 * u + 1]);
        mma16816(i, wrl, dih[2 * u], dih[2 * u + 1]);
        mma16816(i, wih, drh[2 * u], drh[2 * u + 1]);
        mma16816(i, wih, drl[2 * u], drl[2 * u + 1]);
        mma16816(i, wil, drh[2 * u], drh[2 * u + 1]);
      }
    }
  }
}

// Out = D * Wc (D = planes 0..3 as the left operand, Wc = W or conj(W) on the
// right).  Real part Dr Wr - Di Wi, imaginary Dr Wi + Di Wr.
template <bool CONJ>
__device__ __forceinline__ void gemm_right(const __nv_bfloat16* sm, float (&cr)[4][4], float (&ci)[4][4], int rb,
                                           int cb, int lane) {
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int k = 0; k < 4; ++k) cr[t][k] = ci[t][k] = 0.f;
  const int mi = lane >> 3, rr = lane & 7;
#pragma unroll 1
  for (int k0 = 0; k0 < 64; k0 += 16) {
    uint32_t drh[4], drl[4], dih[4], dil[4], nih[4], nil[4];
    const int ao = (16 * rb + (mi & 1) * 8 + rr) * kTcRow + k0 + (mi >> 1) * 8;
    ldsm4(su32(sm + 0 * kTcPlane + ao), drh);
    ldsm4(su32(sm + 1 * kTcPlane + ao), drl);
    ldsm4(su32(sm + 2 * kTcPlane + ao), dih);
    ldsm4(su32(sm + 3 * kTcPlane + ao), dil);
    neg4(dih, nih);
    neg4(dil, nil);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int bo = (k0 + (mi & 1) * 8 + rr) * kTcRow + 32 * cb + 16 * h + (mi >> 1) * 8;
      uint32_t wrh[4], wrl[4], wih[4], wil[4];
      ldsm4t(su32(sm + 4 * kTcPlane + bo), wrh);
      ldsm4t(su32(sm + 5 * kTcPlane + bo), wrl);
      ldsm4t(su32(sm + 6 * kTcPlane + bo), wih);
      ldsm4t(su32(sm + 7 * kTcPlane + bo), wil);
      if (CONJ) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          wih[k] ^= 0x80008000u;
          wil[k] ^= 0x80008000u;
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        float(&r)[4] = cr[2 * h + u];
        float(&i)[4] = ci[2 * h + u];
        mma16816(r, drh, wrh[2 * u], wrh[2 * u + 1]);
        mma16816(r, drh, wrl[2 * u], wrl[2 * u + 1]);
        mma16816(r, drl, wrh[2 * u], wrh[2 * u + 1]);
        mma16816(r, nih, wih[2 * u], wih[2 * u + 1]);
        mma16816(r, nih, wil[2 * u], wil[2 * u + 1]);
        mma16816(r, nil, wih[2 * u], wih[2 * u + 1]);
        mma16816(i, drh, wih[2 * u], wih[2 * u + 1]);
        mma16816(i, drh, wil[2 * u], wil[2 * u + 1]);
        mma16816(i, drl, wih[2 * u], wih[2 * u + 1]);
        mma16816(i, dih, wrh[2 * u], wrh[2 * u + 1]);
        mma16816(i, dih, wrl[2 * u], wrl[2 * u + 1]);
        mma16816(i, dil, wrh[2 * u], wrh[2 * u + 1]);
      }
    }
  }
}

// Write a warp's output tile into the operand planes (hi + lo split).
__device__ __forceinline__ void store_tile(__nv_bfloat16* sm, const float (&cr)[4][4], const float (&ci)[4][4], int rb,
                                           int cb, int lane) {
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int c = 32 * cb + 8 * t + 2 * q;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int r = 16 * rb + g + 8 * hh;
      put_split(sm + 0 * kTcPlane, sm + 1 * kTcPlane, r, c, cr[t][2 * hh], cr[t][2 * hh + 1]);
      put_split(sm + 2 * kTcPlane, sm + 3 * kTcPlane, r, c, ci[t][2 * hh], ci[t][2 * hh + 1]);
    }
  }
}

template <bool FUSED>
__global__ void __launch_bounds__(256, 2) pass_tc2d_kernel(const PassArgs a, const __nv_bfloat16* __restrict__ wpl) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __nv_bfloat16* sm = reinterpret_cast<__nv_bfloat16*>(smraw);
  float2* xs = reinterpret_cast<float2*>(sm + 8 * kTcPlane);
  const LayerGeom& g = a.g;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int rb = warp & 3, cb = warp >> 2;
  const int gq = lane >> 2, qq = lane & 3;
  uint64_t* s_lab = g_tm.la;   // [0] la, [1] lb, [2] c0 of the current slice
  // the W planes, once per CTA (global: 4 planes of 64 x 64, rows unpadded)
  for (int e = t; e < 4 * 64 * 32; e += blockDim.x) {
    const int pl = e / (64 * 32), rem = e - pl * 64 * 32, r = rem >> 5, c2 = rem & 31;
    *reinterpret_cast<uint32_t*>(sm + (4 + pl) * kTcPlane + r * kTcRow + 2 * c2) =
        *reinterpret_cast<const uint32_t*>(wpl + pl * 4096 + r * 64 + 2 * c2);
  }
  float2* psi = reinterpret_cast<float2*>(a.psi);
  const int sub = t & 63, j = t >> 6;
  for (int64_t s = blockIdx.x; s < g.nslices; s += gridDim.x) {
    if (t == 0) {
      const uint64_t ua = (uint64_t)(s % g.oqa + g.olo_a), ub = (uint64_t)(s / g.oqa + g.olo_b);
      s_lab[0] = g.X_aa * ua + g.X_ab * ub;
      s_lab[1] = g.X_ba * ua + g.X_bb * ub;
      s_lab[2] = g.C_aa * (ua * ua) + g.C_ab * (ua * ub) + g.C_bb * (ub * ub);
    }
    __syncthreads();
    const uint64_t la = s_lab[0], lb = s_lab[1], c0 = s_lab[2];
    float2* pp = psi + s * g.slice_stride + sub * g.ea + j * g.eb;
    {
      // load (element ia = sub, ib = j + 4m), kinetic pre-phase, keep and split
      float2 x[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) x[m] = pp[m * 4 * g.eb];
      if (a.units_pre != 0) {
        QuadWalk w(g, sub, j, la, lb, c0);
        w.scale((uint64_t)0 - (uint64_t)a.units_pre);
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          x[m] = apply_phase<float>(x[m], phase_of<float>(w.q));
          w.next();
        }
      }
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int ib = j + 4 * m;
        xs[sub + 64 * ib] = x[m];
        const __nv_bfloat16 hr = __float2bfloat16_rn(x[m].x), hi = __float2bfloat16_rn(x[m].y);
        sm[0 * kTcPlane + ib * kTcRow + sub] = hr;
        sm[1 * kTcPlane + ib * kTcRow + sub] = __float2bfloat16_rn(x[m].x - __bfloat162float(hr));
        sm[2 * kTcPlane + ib * kTcRow + sub] = hi;
        sm[3 * kTcPlane + ib * kTcRow + sub] = __float2bfloat16_rn(x[m].y - __bfloat162float(hi));
      }
    }
    __syncthreads();
    float cr[4][4], ci[4][4];
#pragma unroll 1
    for (int f = 0; f < (FUSED ? 2 : 1); ++f) {
      const float2* T = reinterpret_cast<const float2*>(f == 0 ? a.T : a.T2);
      // to the grid: U = W X, G = U W
      gemm_left<false>(sm, cr, ci, rb, cb, lane);
      __syncthreads();
      store_tile(sm, cr, ci, rb, cb, lane);
      __syncthreads();
      gemm_right<false>(sm, cr, ci, rb, cb, lane);
      __syncthreads();
      // H = G .* (T - 1)/M at grid point (pb, pa) = (row, column)
#pragma unroll
      for (int tt = 0; tt < 4; ++tt) {
        const int c = 32 * cb + 8 * tt + 2 * qq;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int r = 16 * rb + gq + 8 * hh;
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float2 tp = T[(c + e) + 64 * r];
            const float gr = cr[tt][2 * hh + e], gi = ci[tt][2 * hh + e];
            cr[tt][2 * hh + e] = gr * tp.x - gi * tp.y;
            ci[tt][2 * hh + e] = gr * tp.y + gi * tp.x;
          }
        }
      }
      store_tile(sm, cr, ci, rb, cb, lane);
      __syncthreads();
      // back to coefficients: V = conj(W) H, C = V conj(W)
      gemm_left<true>(sm, cr, ci, rb, cb, lane);
      __syncthreads();
      store_tile(sm, cr, ci, rb, cb, lane);
      __syncthreads();
      gemm_right<true>(sm, cr, ci, rb, cb, lane);
      __syncthreads();
      // y = x + C at (ib, ia) = (row, column); then the next factor's input
      // (fused pass: kinetic mid-phase, kept and split) or the post-phase and store
      const bool last = !FUSED || f == 1;
      const int64_t units = last ? a.units_post : a.units_mid;
#pragma unroll
      for (int tt = 0; tt < 4; ++tt) {
        const int ia0 = 32 * cb + 8 * tt + 2 * qq;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int ib = 16 * rb + gq + 8 * hh;
          float2 y[2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float2 x = xs[ia0 + e + 64 * ib];
            y[e] = make_float2(x.x + cr[tt][2 * hh + e], x.y + ci[tt][2 * hh + e]);
            if (units != 0) {
              const uint64_t qd = quad_turns(g, g.lo_a + ia0 + e, g.lo_b + ib, la, lb, c0);
              y[e] = apply_phase<float>(y[e], phase_of<float>((uint64_t)0 - (uint64_t)units * qd));
            }
          }
          if (last) {
            float2* out = psi + s * g.slice_stride + (int64_t)ia0 * g.ea + (int64_t)ib * g.eb;
            out[0] = y[0];
            out[g.ea] = y[1];
          } else {
            xs[ia0 + 64 * ib] = y[0];
            xs[ia0 + 1 + 64 * ib] = y[1];
            put_split(sm + 0 * kTcPlane, sm + 1 * kTcPlane, ib, ia0, y[0].x, y[1].x);
            put_split(sm + 2 * kTcPlane, sm + 3 * kTcPlane, ib, ia0, y[0].y, y[1].y);
          }
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace

size_t tc2d_smem_bytes() { return (size_t)8 * kTcPlane * sizeof(__nv_bfloat16) + (size_t)4096 * sizeof(float2); }

cudaError_t tc2d_prepare(size_t max_smem) {
  cudaError_t e = allow_smem(pass_tc2d_kernel<false>, max_smem);
  if (e == cudaSuccess) e = allow_smem(pass_tc2d_kernel<true>, max_smem);
  return e;
}

cudaError_t launch_tc2d(const PassArgs& a, const void* planes, int nblocks, cudaStream_t st) {
  if (a.g.d != 2 || a.g.qa != 64 || a.g.qb != 64 || a.mode != MODE_STEP || a.list != nullptr || a.g.ea != 1 ||
      a.g.eb != 64)
    return cudaErrorInvalidValue;
  const __nv_bfloat16* w = static_cast<const __nv_bfloat16*>(planes);
  if (a.T2) pass_tc2d_kernel<true><<<nblocks, 256, tc2d_smem_bytes(), st>>>(a, w);
  else pass_tc2d_kernel<false><<<nblocks, 256, tc2d_smem_bytes(), st>>>(a, w);
  return cudaGetLastError();
}

}  // namespace lsk
