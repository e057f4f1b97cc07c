// Internal interface between the host library (lsplit_host.cpp) and the CUDA
// kernels (lsplit_kernels.cu).  Not part of the public C ABI.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include <string>

namespace lsk {

constexpr int kMaxTileSlices = 64;   // W: slices per CTA (upper bound)
constexpr int kMaxThreads = 1024;

// Geometry of one layer's slice passes (P_j acts along layer j's index).
// Fixed-point coefficients are in units of 2^-64 turns per kinetic unit.
struct LayerGeom {
  int d;              // 1 or 2 (slice dimensionality)
  int qa, qb;         // slice extents (qb = 1 in 1D)
  int M;              // qa * qb
  int np;             // FFT length along a (Bluestein length if bluestein)
  int npb;            // FFT length along b (2D), 1 in 1D
  int bluestein;      // 1: 1D slice with q not a power of two
  int buf;            // logical slice buffer length (np in 1D, M in 2D)
  int sb;             // padded slice buffer length in SMEM (elements)
  int64_t nslices;    // number of slices (= size of the other layer's box)
  int64_t slice_stride;  // global element offset between consecutive slices
  int64_t ea, eb;     // global element strides along a and b
  int lo_a, lo_b;     // own box lower bounds: signed index = lo + i
  int oqa, olo_a, olo_b;  // other box: slice index s -> (s % oqa + olo_a, s / oqa + olo_b)
  int shared_b;       // 1: the b index is shared by both layers (three-index lift); the
                      // other layer's slice of element (ia, ib) is then ia alone
  uint64_t A_aa, A_ab, A_bb;           // own quadratic form
  uint64_t X_aa, X_ab, X_ba, X_bb;     // cross: l_a = X_aa nu_a + X_ab nu_b, l_b = X_ba nu_a + X_bb nu_b
  uint64_t C_aa, C_ab, C_bb;           // other quadratic form
  const void* tw;     // np twiddles exp(-2 pi i x / np)
  const void* twb;    // npb twiddles (2D)
  const void* bm;     // Bluestein: FFT_np(b-) / np, b-_j = exp(-i pi j^2 / q)
  const void* bp;     // Bluestein: FFT_np(b+) / np
  const void* chirp;  // Bluestein: exp(+i pi (i^2 mod 2q) / q), q entries
  const double* vgrid;  // v_j(x_p), FP64, M entries
};

enum PassMode { MODE_STEP = 0, MODE_MEASURE = 1, MODE_ADJOINT = 2, MODE_LAZY = 3, MODE_KIN = 4 };

struct PassArgs {
  LayerGeom g;
  void* psi;
  void* lam;               // adjoint: lambda array (same layout)
  const void* T;           // (exp(-i s v_j(x_p)) - 1) / M, M entries (complex Real)
  int64_t units_pre;       // kinetic units before P (MODE_STEP / MODE_ADJOINT)
  int64_t units_post;      // kinetic units after P
  int W;                   // slices per CTA
  int strided;             // 1: slice index fastest in global access
  int mode;
  int64_t pitch;           // row pitch (elements), for touch decoding
  // lazy stochastic mode
  const int32_t* list;     // sampled slice indices for this sub-step (sorted)
  int32_t nlist;
  int32_t* touch_own;      // last kinetic time of own-layer slices (rows for layer 1)
  const int32_t* touch_other;  // last kinetic time of the other layer's slices
  int32_t now;             // kinetic time (units) at which P acts
  // measure / adjoint outputs
  double* partials;        // per-CTA partial sums (MODE_MEASURE)
  double* grad;            // M doubles (MODE_ADJOINT), accumulated atomically
  double sdur;             // duration s of the factor (MODE_ADJOINT)
  // Convolution form of a potential factor (1D slices of length q < N):
  // (P - I) x = c' (*) x, c' = DFT_q(T - 1) / q, as a length-N cyclic
  // convolution through FFT_N; Khat = FFT_N(wrapped c') / N.  With N = 2q - 2
  // the wrapped kernel cannot hold both c'_{q-1} and c'_1 at index q - 1: it
  // keeps c'_{q-1} and output 0 is fixed by fix0 * x_{q-1}, fix0 = c'_1 - c'_{q-1}.
  const void* Khat;        // N entries (complex Real); NULL: Bluestein form
  double fix0_re, fix0_im;
  int64_t list_step;       // batched stochastic runner: list advance per step
  // fused pass (fast path, convolution form): a second factor of the same layer
  // after the kinetic phase units_mid; NULL Khat2 = single factor
  const void* Khat2;
  double fix2_re, fix2_im;
  int64_t units_mid;
  int32_t variant;         // fast pass: 0 two shared buffers (2 CTAs/SM), 1 one buffer (3 CTAs/SM)
  int32_t fast_logn;       // batched runner: tile on the fast pass of length 2^fast_logn (0: general tile)
  const void* T2;          // fused 2D pass: (T - 1)/M table of the second factor
  // Compact-kernel form of a potential factor on 1D slices (sB > 0):
  // (P - I) x = sum_{|d| <= sB} c'_d x_{(i - d) mod q}, the taps c'_d of the
  // circulant kernel c' = DFT_q(T - 1)/q whose l1 tail beyond sB is below the
  // working precision; taps holds 2 sB + 1 complex Real values, d = -sB..sB.
  const void* taps;
  int32_t sB;
  int32_t subtiles;        // batched compact-only kernel: consecutive tiles per work item (0 or 1: one)
  // Interaction frame of a call (MODE_STEP, compact-kernel form, ip = 1): the
  // state is psi~ = K(-t) psi with t the kinetic units applied so far in the
  // call, so P acts as K(-t) P K(t): taps c_d e^{-2 pi i t A d^2} times
  // w_m^d, w_m = e^{2 pi i t (2 A m + l)}; taps holds c'_d / (1 + c'_0) with a
  // zero centre (the scalar 1 + c'_0 of every factor is collected in Lambda).
  // units_pre is 0; units_post, nonzero only in a call's last pass, is the
  // call's total kinetic time T, applied with Lambda: psi = Lambda K(T) psi~.
  int64_t ip_t;            // t: kinetic units before this factor, from the start of the call
  uint64_t lam_turns;      // arg(Lambda) in 2^-64 turns
  double lam_def;          // 1 - |Lambda|
  int32_t ip;              // 1: interaction frame
  int32_t pad_ip;
};

constexpr int kStencilMaxB = 8;       // widest compact kernel (17 taps)
constexpr int kStencilThreads = 256;

struct ElemArgs {          // elementwise kernels over the whole lifted box
  int d;
  int q1a, q1b, lo1a, lo1b;   // layer-1 box
  int q2a, q2b, lo2a, lo2b;   // layer-2 box
  int64_t M1, M2, pitch;
  double B1[4], B2[4];
  double ecut;
};

// ---- launchers (return cudaError_t of the launch) ----
// BPT: butterflies per thread per radix-4 stage (2 or 4); nthreads from
// pass_threads().  MODE_KIN (settle) runs the pass kernel without transforms.
template <typename Real> cudaError_t launch_pass(const PassArgs& a, int bpt, int nthreads,
                                                 int64_t ntiles, cudaStream_t st);
template <typename Real> size_t pass_smem_bytes(const LayerGeom& g, int W, int mode);
template <typename Real> cudaError_t pass_prepare(size_t max_smem);
int pass_threads(const LayerGeom& g, int W, int bpt);
template <typename Real> cudaError_t launch_gaussian(const ElemArgs& e, void* psi, const double* x0,
                                                     double w, const double* k0, double* partials,
                                                     int nblocks, cudaStream_t st);
template <typename Real> cudaError_t launch_scale(const ElemArgs& e, void* psi, const double* sumsq,
                                                  cudaStream_t st);
// Zero every coefficient whose byte in mask (M2 x M1, row-major) is 0.
template <typename Real> cudaError_t launch_project(void* psi, const uint8_t* mask, int64_t M1, int64_t M2,
                                                    int64_t pitch, cudaStream_t st);
template <typename Real> cudaError_t launch_elem_obs(const ElemArgs& e, const void* psi,
                                                     const void* chi, double* partials, int nblocks,
                                                     cudaStream_t st);
cudaError_t launch_reduce(const double* partials, int nparts, int nq, double* out, cudaStream_t st);
// Stochastic slice sampler: block b draws the sample of sub-step g0 + b, whose
// layer is pattern[b % npf].  seed/g0 come from seed_g0_dev[0..1] when that
// pointer is not NULL (so a captured graph can be replayed with new seeds).
struct SamplerArgs {
  int32_t S1, p1, S2, p2, Smax, pmax, npf;
  int32_t pattern[4];
  uint64_t seed, g0;
};
cudaError_t launch_sampler(const SamplerArgs& sa, const uint64_t* seed_g0_dev, int32_t count,
                           int32_t* out, cudaStream_t st);
cudaError_t sampler_prepare(size_t smem);
template <typename Real> int pass_max_threads(int bpt);
// Fast 1D pass (MODE_STEP / MODE_LAZY, power-of-two transform length 256..8192):
// W slices per CTA, W * np / 16 threads.
template <typename Real> cudaError_t launch_fast(const PassArgs& a, int64_t ntiles, cudaStream_t st);
template <typename Real> size_t fast_smem_bytes(const LayerGeom& g, int W, int variant);
template <typename Real> cudaError_t fast_prepare(size_t max_smem);
template <typename Real> int fast_max_threads();
// Fast 2D pass for 64 x 64 slices (MODE_STEP / MODE_LAZY): one slice per
// 256-thread CTA.
template <typename Real> cudaError_t launch_fast2d(const PassArgs& a, int64_t ntiles, cudaStream_t st);
template <typename Real> size_t fast2d_smem_bytes(const LayerGeom& g);
template <typename Real> cudaError_t fast2d_prepare(size_t max_smem);
// Compact-kernel pass (MODE_STEP / MODE_LAZY) over W slices per CTA of
// kStencilThreads threads; the tile (W slices with their wrap halos) sits in
// shared memory.  W must be a power of two for strided slices.
template <typename Real> cudaError_t launch_stencil(const PassArgs& a, int64_t ntiles, cudaStream_t st);
template <typename Real> size_t stencil_smem_bytes(const LayerGeom& g, int W, int B);
template <typename Real> cudaError_t stencil_prepare(size_t max_smem);
// Tensor-core layer pass for contiguous 64 x 64 slices (complex64, MODE_STEP,
// optionally the fused second factor in T2): the DFTs as split-BF16 matrix
// products.  planes: 4 x 64 x 64 bf16 (row-major) with W[p][k] =
// exp(+2 pi i p k / 64): Re hi, Re lo, Im hi, Im lo.  Persistent over the
// slices with nblocks CTAs of 256 threads.
cudaError_t launch_tc2d(const PassArgs& a, const void* planes, int nblocks, cudaStream_t st);
cudaError_t tc2d_prepare(size_t max_smem);
size_t tc2d_smem_bytes();
cudaError_t launch_zero_i32(int32_t* p, int64_t n, cudaStream_t st);
cudaError_t launch_zero_f64(double* p, int64_t n, cudaStream_t st);

// Persistent batched runner: one launch walks the work list of
// (step, pass, instance, slice-tile) items in order, claimed through
// counters[0]; an item waits (bounded) until its instance has completed every
// tile of the previous pass, counted in counters[1 + instance].
struct BatchArgs {
  const PassArgs* args;        // [npass][ninst], units set per step variant below
  const int64_t* cum;          // [npass][ninst + 1] cumulative tile counts per pass
  const int64_t* tiles_step;   // [ninst] tiles of one step of instance i
  int64_t pass_items[4];       // tiles per pass summed over instances
  int64_t step_items;          // tiles per step summed over passes and instances
  int32_t ninst, npass, nsteps;
  int32_t units[4][3][2];      // [variant: first, middle, last, only][pass][pre, post]
  unsigned long long* counters;
  int32_t* status;             // 0 ok, 1 a wait timed out
  long long timeout_cycles;    // clock64() budget of one wait
  int32_t unmet;               // test hook: one wait that nothing can satisfy
  // stochastic schemes: sub-step items walk sampled-slice lists (MODE_LAZY;
  // list of step k = args.list + k * args.list_step, kinetic clock
  // now = k * now_mul + now_off[pass]); a settle phase (MODE_KIN) follows the
  // last step
  int32_t stoch;
  int32_t now_mul, now_off[3];
  const PassArgs* settle_args;  // [ninst]
  const int64_t* settle_cum;    // [ninst + 1]
  int64_t settle_items;
  int32_t minb;                 // CTAs per SM the registers are budgeted for (3, or 4 for KIND 1)
  int32_t kind;                 // 0: any tile kind; 1: compact-kernel tiles only
  // deterministic Strang with fused layer-1 factors (fused != 0): passes of a
  // call are [first L1] then per step [L2, fused L1 (plain L1 in the last
  // step)]; args kinds [5][ninst]: 0 first L1, 1 L2, 2 fused L1 (fused tile
  // when Khat2 is set, else its first factor), 3 last L1, 4 second factor of
  // a fused item without a fused tile; cum rows 0 (layer 1) and 1 (layer 2)
  int32_t fused;
  const int64_t* tiles1;        // [ninst] layer-1 tiles of instance i
  const int64_t* tiles2;        // [ninst] layer-2 tiles of instance i
  // interaction frame (compact-only kernel, deterministic schemes): the factor
  // of an item of step k acts at t = k ip_step + ip_off[pass] kinetic units
  // (fused walk: ip_off[kind], ip_off[4] for the second factor of a fused item)
  int32_t ip;
  int32_t ip_step;
  int32_t ip_off[5];
};

// Slice samples of a batch: block b draws instance i = b / (nsteps * npf),
// sub-step rel = b % (nsteps * npf) with seed + i and g = g0 + rel; writes p
// sorted indices at base[i] + (rel / npf) * step_len[i] + pass_off[i * npf + rel % npf].
struct BatchSamplerArgs {
  const int32_t* S;         // [ninst * npf] slice count of each pass's layer
  const int32_t* p;         // [ninst * npf] samples per sub-step
  const int64_t* base;      // [ninst]
  const int64_t* step_len;  // [ninst]
  const int64_t* pass_off;  // [ninst * npf]
  int32_t npf, nsteps, Smax;
};
cudaError_t launch_batch_sampler(const BatchSamplerArgs& sa, const uint64_t* seed_g0_dev, int64_t blocks,
                                 int32_t* out, cudaStream_t st);
cudaError_t batch_sampler_prepare(size_t max_block);
template <typename Real> cudaError_t launch_batch(const BatchArgs& b, int nthreads, int nblocks, size_t smem,
                                                  cudaStream_t st);
template <typename Real> cudaError_t batch_prepare(size_t max_smem, int nthreads, size_t smem, int kind, int minb,
                                                   int* blocks_per_sm);

// Crank-Nicolson layer factor (Sec. 4.2.1, Eq. (tsCN)) over every slice of
// one layer of a 1D box: (I + i s A/2) y = (I - i s A/2) x, A = diag(|k|^2/4)
// + the banded plane-wave potential matrix (half-width hb), by niter Jacobi
// sweeps on tiles of W slices x (TI + 2 halo) indices.
constexpr int kCnMaxBand = 8;
constexpr int kCnPerThread = 10;      // tile elements per thread (256 threads)
struct CnArgs {
  void* psi;
  int64_t nslices;                    // slices of the layer
  int64_t slice_stride, ea;           // element (slice, i) at slice * slice_stride + i * ea
  int64_t nchunks;                    // index chunks per slice group
  int32_t q;                          // slice length
  int32_t strided;                    // 1: the W slices of a tile are adjacent in memory
  int32_t W, TI, halo, hb, niter;
  double half_s;                      // s / 2
  double b_own, b_oth;                // k = b_own (lo + i) + b_oth (olo + slice)
  int32_t lo, olo;
  // z = (s/2)(|k|^2/4 + Re vhat_0) = za m^2 + zb m n + zc n^2 + zd with
  // m = lo + i, n = olo + slice; each coefficient split into float hi + lo
  float za[2], zb[2], zc[2], zd[2];
  float half_s_f;                     // s / 2 in single precision
  int32_t unitary;                    // 1: vhat_0 real (the diagonal multiplier has modulus 1)
  double v_re[2 * kCnMaxBand + 1], v_im[2 * kCnMaxBand + 1];  // vhat_h at h + kCnMaxBand
};
template <typename Real> cudaError_t launch_cn(const CnArgs& a, cudaStream_t st);
template <typename Real> cudaError_t cn_prepare(size_t max_smem);
size_t cn_smem_bytes(const CnArgs& a, size_t elem_bytes);

// Semi-implicit step (Sec. 4.1, Algorithm 1) and its random batch form
// (Sec. 4.3, Algorithm 4) on a 1D box, out of place:
//   dst = (I + i tau D)^{-1} (src - i tau (w_row V^1 + w_col V^2) src),
// V^j the banded plane-wave potential matrices along m (rows) and n (columns);
// w_row / w_col: 1 (Algorithm 1), or weight on the sampled rows / columns and
// 0 elsewhere (Algorithm 4).
struct SiArgs {
  const void* src;
  void* dst;
  int64_t M1, M2, pitch;
  int32_t hb1, hb2;                   // band half-widths of V^1, V^2
  int32_t lo1, lo2;
  double tau;
  float tau_f;
  float za[2], zb[2], zc[2];          // tau |k|^2 / 2 = za m^2 + zb m n + zc n^2 (float hi + lo)
  double zad, zbd, zcd;               // the same coefficients in double
  double v1_re[2 * kCnMaxBand + 1], v1_im[2 * kCnMaxBand + 1];
  double v2_re[2 * kCnMaxBand + 1], v2_im[2 * kCnMaxBand + 1];
  const int32_t* rows;                // sorted sampled rows (NULL: every row, weight 1)
  const int32_t* cols;                // sorted sampled columns (NULL: every column, weight 1)
  int32_t nrows, ncols;
  double w_row, w_col;                // weights of sampled rows / columns
};
template <typename Real> cudaError_t launch_si(const SiArgs& a, cudaStream_t st);

// Wave function at real-space points: device buffers of the phase tables
// E1 (nx x M1), E2 (nx x M2), the partial sums T (nx x M2) and the output
// (2 nx doubles); f1/f2: B^T x_j / 2 pi as 64-bit fractions per point.
struct DensityArgs {
  const void* psi;
  int64_t M1, M2, pitch, nx;
  int32_t q1a, q2a;                   // first extent of each layer box (the linear index is a + q_a b)
  int32_t lo1a, lo1b, lo2a, lo2b;
  const uint64_t* f1;                 // [2 nx]: (B1^T x_j)_a / 2 pi at j, (B1^T x_j)_b / 2 pi at nx + j
  const uint64_t* f2;                 // [2 nx]: the same with B2
  void *e1, *e2, *t;
  double* out;
  int32_t simt;                       // complex64: 1 forces the CUDA-core contraction
};
template <typename Real> cudaError_t launch_density(const DensityArgs& d, cudaStream_t st);

// Message returned by ls_last_error() on the calling thread.
void set_last_error(const std::string& msg);

constexpr int kObsQ = 8;   // norm, ekin, k0, k1, ovl_re, ovl_im, spare, spare
constexpr int kReduceBlocks = 1024;

}  // namespace lsk
