/*
 * lsplit.h -- C ABI of the GB300 layer-split time stepper for the lifted
 * plane-wave Schroedinger equation of incommensurate bilayers
 * (Wang, Chen, Zhou & Zhou, arXiv 2103.14897).
 *
 * Model.  Two periodic layers with reciprocal lattices B_j = 2 pi A_j^{-T}
 * (Sec. 2).  The wave function is lifted to coefficients phi[n][m] of the
 * plane waves exp(i (B1 m + B2 n) . x) (Sec. 3, Eq. (3.3)); the semidiscrete
 * problem is d phi/dt = -i (D + V^1 + V^2) phi (Eq. (3.4)-(3.7)) with D
 * diagonal, V^1 = I (x) Vc^1 acting on m, V^2 = Vc^2 (x) I acting on n.
 *
 * One step splits exp(-i tau H) into the kinetic factor K(s) = exp(-i s D)
 * and the layer factors P_j(s) = F_j diag(exp(-i s v_j(x_p))) F_j^{-1}
 * along layer j's index for every slice (fixed index of the other layer)
 * (Eq. (4.8), Algorithm 3).  Compositions: Lie (Algorithm 3 order), Strang
 * over H = H1 + H2 (Appendix A), kinetic/potential Strang, and the random
 * batch (Algorithm 4) slice-sampling variants.
 *
 * Conventions for every entry point:
 *   - Return value: LS_OK (0) or a negative LS_ERR_* code; nothing aborts,
 *     no C++ exception crosses the ABI.  ls_last_error() gives a message
 *     (thread-local, valid until the next call on that thread).
 *   - "_dev" pointers are CUDA device memory owned by the caller; "_host"
 *     pointers are host memory owned by the caller.  The library never frees
 *     caller memory and never allocates the wave-function arrays.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued asynchronously unless the function says it syncs.
 *   - Wave-function layout: complex interleaved (re, im), float (LS_C64) or
 *     double (LS_C128).  Element (m, n) is at n_lin * pitch + m_lin, where
 *     m_lin / n_lin are linear box indices with the first component fastest
 *     (m_lin = (m_1 - lo1_1) + q1_1 * (m_2 - lo1_2) in 2D), and pitch >= M1
 *     is given by ls_layout().  Elements in the pitch padding are neither
 *     read nor written.
 */
#ifndef LSPLIT_H
#define LSPLIT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LS_OK = 0,
  LS_ERR_INVALID = -1, /* bad argument or unsupported problem */
  LS_ERR_NOMEM = -2,   /* device or host allocation failed */
  LS_ERR_CUDA = -3,    /* a CUDA runtime call failed */
  LS_ERR_TIMEOUT = -4, /* a bounded device wait expired */
  LS_ERR_STATE = -5    /* call out of order (e.g. destroyed context) */
};

enum { LS_C64 = 0, LS_C128 = 1 };

/* Schemes (one time step tau, factors in application order):
 *   LS_LIE          K(tau), P1(tau), P2(tau)                  (Algorithm 3)
 *   LS_STRANG       L1(tau/2) L2(tau) L1(tau/2),  L_j(s) = K(s/4) P_j(s) K(s/4)
 *                   (Strang over H = H1 + H2, H_j = D/2 + V^j; Appendix A)
 *   LS_STRANG_KP    K(tau/2), P1(tau), P2(tau), K(tau/2)
 *   LS_LIE_STOCH, LS_STRANG_STOCH: as above, but every layer factor acts on
 *                   p = max(1, S/frac_den) seeded random slices out of S with
 *                   duration s*S/p (Algorithm 4); kinetic factors act on all.
 *   LS_YOSHIDA4     fourth order: three LS_STRANG steps of w1 tau, w0 tau, w1 tau,
 *                   w1 = 1/(2 - 2^(1/3)), w0 = -2^(1/3) w1 (the higher-order
 *                   splittings of Sec. 4.2 and Appendix A, by Yoshida's symmetric
 *                   composition); ls_step and ls_adjoint (the batched runner
 *                   returns LS_ERR_INVALID).
 *   LS_CN_STRANG    Crank-Nicolson layer splitting (Sec. 4.2.1, Eq. (tsCN)):
 *                   C1(tau/2) C2(tau) C1(tau/2), C_j(s) = (I + i s H_j/2)^{-1}
 *                   (I - i s H_j/2), H_j = D/2 + V^j with V^j the plane-wave
 *                   potential matrix of Sec. 3 (no wrap at the box ends).  Second
 *                   order and mass conserving.  1D boxes, potentials with
 *                   |h| <= 8 and |tau| sum_{h != 0} |vhat_h| < 1 (each factor is
 *                   solved by Jacobi sweeps to working precision); otherwise
 *                   ls_step returns LS_ERR_INVALID.  ls_step only.
 *   LS_SEMI_IMPLICIT  phi <- (I + i tau D)^{-1} (phi - i tau (V^1 + V^2) phi)
 *                   (Sec. 4.1, Algorithm 1): explicit banded plane-wave potential
 *                   products along both layers, implicit kinetic part.  First
 *                   order; does not conserve the mass.
 *   LS_RANDOM_BATCH Algorithm 4 (Sec. 4.3): as LS_SEMI_IMPLICIT, but the V^1
 *                   product acts on p1 = max(1, M2/frac_den) seeded rows and the
 *                   V^2 product on p2 = max(1, M1/frac_den) seeded columns,
 *                   weighted M2/p1 and M1/p2 (samples: the LS_*_STOCH rule with
 *                   two sub-steps per step, rows first).
 *                   Both: 1D boxes, potentials with |h| <= 8, ls_step only; the
 *                   context allocates a second state array on first use. */
enum { LS_LIE = 0, LS_STRANG = 1, LS_STRANG_KP = 2, LS_LIE_STOCH = 3, LS_STRANG_STOCH = 4, LS_YOSHIDA4 = 5,
       LS_CN_STRANG = 6, LS_SEMI_IMPLICIT = 7, LS_RANDOM_BATCH = 8 };

/* Problem description (Sec. 2-3).  All arrays are read during ls_create only
 * and stay owned by the caller.
 *   d             1 or 2
 *   B1, B2        row-major d x d reciprocal-lattice matrices; k = B1 m + B2 n
 *   lo1, q1       layer-1 box: m_i in [lo1[i], lo1[i] + q1[i]), q1[i] >= 1
 *   lo2, q2       layer-2 box
 *   ecut          energy cutoff Ec of the joint mask |k|^2/2 <= Ec (Sec. 3)
 *   nv1, v1_h, v1_c  nv1 reciprocal indices h (int32, nv1*d) and complex
 *                 Fourier coefficients vhat (re, im pairs, 2*nv1 doubles) of
 *                 v_1 (Eq. (2.2)); v_1(x_p) = Re sum_h vhat_h e^{2 pi i h.p/q1}
 *   nv2, v2_h, v2_c  same for v_2
 *   dtype         LS_C64 (complex float, FP64 phase arithmetic) or LS_C128
 *   frac_den      stochastic sampling denominator (p = max(1, S/frac_den)), >= 1
 *   mask_mode     LS_MASK_INIT_ONLY (0): the joint cutoff shapes the initial
 *                 state and the ls_index_set query only, and the whole box is
 *                 evolved; LS_MASK_PROJECT_EACH_STEP (1): ls_step also zeroes
 *                 every coefficient outside the joint cutoff after each full
 *                 time step (the truncated index set of Sec. 3 enforced during
 *                 the evolution).  The projection is not unitary: ls_adjoint
 *                 and the batched runner return LS_ERR_INVALID for it.
 *   shared        0, or 1 for a three-index lift with an index common to both
 *                 layers (Example 3 of Sec. 5: periodic in y, incommensurate in
 *                 x).  The problem is then given as d = 2 with layer-1 box
 *                 (q1[0], 1) (lo1[1] = 0) and layer-2 box (q2[0], q2[1]); the
 *                 second layer-2 component is the shared index p, so that
 *                 k = B1 (m, 0) + B2 (n, p).  Element (m, n, p) is at
 *                 (n_lin + q2[0] p_lin) * pitch + m_lin.  A layer-1 factor acts
 *                 on the 2D slices (m, p) at fixed n, a layer-2 factor on
 *                 (n, p) at fixed m; potential j has harmonics (h_x, h_y) on the
 *                 grid (q_j[0], q2[1]).  Needs power-of-two q1[0], q2[0], q2[1]
 *                 with q1[0] q2[1] and q2[0] q2[1] at most 4096; the
 *                 Crank-Nicolson and semi-implicit schemes and the batched
 *                 runner return LS_ERR_INVALID.
 * Supported slice shapes: 1D any length (powers of two use a direct radix FFT,
 * others a Bluestein transform of power-of-two length >= 2q-2, at most 8192
 * for LS_C64 and 4096 for LS_C128; ls_create returns LS_ERR_INVALID beyond);
 * 2D slices need power-of-two extents with q_1 * q_2 <= 4096. */
typedef struct ls_problem {
  int32_t d;
  double B1[4];
  double B2[4];
  int32_t lo1[2], q1[2];
  int32_t lo2[2], q2[2];
  double ecut;
  int32_t nv1;
  const int32_t* v1_h;
  const double* v1_c;
  int32_t nv2;
  const int32_t* v2_h;
  const double* v2_c;
  int32_t dtype;
  int32_t frac_den;
  int32_t mask_mode;
  int32_t shared;
} ls_problem;

enum { LS_MASK_INIT_ONLY = 0, LS_MASK_PROJECT_EACH_STEP = 1 };

/* Observables (Eq. (2.4)-(2.5) in the lifted basis, Eq. (3.2) orthonormality),
 * all accumulated in FP64:
 *   norm = sum |phi|^2;  ekin = sum |k|^2/2 |phi|^2;
 *   epot1/epot2 = sum over slices of (1/M_j) sum_p v_j(x_p) |psi(x_p)|^2;
 *   energy = ekin + epot1 + epot2;  kmean[i] = sum k_i |phi|^2;
 *   overlap = sum conj(chi) phi (0 if chi is NULL). */
typedef struct ls_obs {
  double norm, ekin, epot1, epot2, energy;
  double kmean[2];
  double overlap_re, overlap_im;
} ls_obs;

typedef struct ls_ctx ls_ctx;

/* Message for the last failing call on this thread ("" if none). */
const char* ls_last_error(void);

/* Build the index set, device tables (potential grids, transform tables,
 * fixed-point kinetic coefficients) and per-context scratch on the current
 * CUDA device.  *out receives the context.  Errors: LS_ERR_INVALID for an
 * unsupported shape or bad field; LS_ERR_NOMEM / LS_ERR_CUDA. */
int ls_create(const ls_problem* prob, ls_ctx** out);

/* Release the context's device tables and scratch.  Safe on NULL. */
int ls_destroy(ls_ctx* ctx);

/* Layout of the wave-function array: *pitch (elements per layer-1 slice row,
 * >= M1), *rows (= M2), *bytes (pitch * M2 * element size). */
int ls_layout(const ls_ctx* ctx, int64_t* pitch, int64_t* rows, int64_t* bytes);

/* Joint-cutoff index set (Sec. 3 index sets with the joint predicate
 * fl(0.5 * fl(sum_i fl(u_i^2))) <= Ec, u_i = sum_j fl(B1[i][j] m_j) + sum_j
 * fl(B2[i][j] n_j) evaluated left to right in IEEE binary64 without FMA).
 * mask_host: M2*M1 bytes (row n, column m, no padding), may be NULL;
 * *count: number of members. */
int ls_index_set(const ls_ctx* ctx, uint8_t* mask_host, int64_t* count);

/* Initial state (Sec. 5, shifted and scaled): phi = exp(-w^2 |k-k0|^2 / 2)
 * exp(-i k.x0) on the joint mask, zero elsewhere, normalised to unit l2 norm.
 * x0, k0: d doubles (host).  Enqueued on stream. */
int ls_init_gaussian(ls_ctx* ctx, void* psi_dev, const double* x0_host, double w,
                     const double* k0_host, void* stream);

/* Advance psi_dev in place by nsteps steps of tau with the given scheme.
 * seed and step0 fix the stochastic samples (sub-step g = (step0 + k) *
 * factors_per_step + factor index).  Adjacent kinetic factors are merged; each
 * layer factor is one fused pass over the array.  Stochastic schemes apply
 * kinetic factors lazily and finish with a settle pass, so psi_dev is complete
 * on return.  With LS_MASK_PROJECT_EACH_STEP every step ends with the
 * projection onto the joint cutoff.  Enqueued on stream (replays a cached CUDA
 * graph, one per (psi_dev, scheme, tau, nsteps); the graphs keep the tables
 * they use alive, and the table caches are bounded). */
int ls_step(ls_ctx* ctx, void* psi_dev, int64_t nsteps, double tau, int32_t scheme,
            uint64_t seed, uint64_t step0, void* stream);

/* End to end from host memory: copy psi_host (ls_layout()'s bytes; pinned
 * host memory makes the copies asynchronous DMA) into the caller's device
 * buffer psi_dev, run ls_step on it, copy the result back into psi_host and
 * synchronise the stream.  Same arguments and errors as ls_step. */
int ls_step_host(ls_ctx* ctx, void* psi_host, void* psi_dev, int64_t nsteps, double tau, int32_t scheme,
                 uint64_t seed, uint64_t step0, void* stream);

/* Observables of psi_dev (and overlap with chi_dev if not NULL).  Synchronises
 * the stream and writes *out (host). */
int ls_observables(ls_ctx* ctx, const void* psi_dev, const void* chi_dev, ls_obs* out,
                   void* stream);

/* Wave function at real-space points from the plane-wave expansion (Sec. 3;
 * the localisation plots of Sec. 5):
 *   psi(x_j) = sum_{m,n} phi[n][m] exp(i (B1 m + B2 n) . x_j),  j < nx.
 * x_host: nx points of d doubles each; out_host: 2 nx doubles (re, im per
 * point).  The phases are exact (64-bit fixed-point turns); the sum over m
 * runs in the context's precision, the sum over n in FP64.  The points are
 * processed in chunks whose temporary device buffers (chunk * (M1 + 2 M2)
 * complex elements) stay below 512 MB; synchronises the stream.
 * LS_ERR_INVALID for nx beyond 2^22. */
int ls_density(ls_ctx* ctx, const void* psi_dev, const double* x_host, int64_t nx, double* out_host,
               void* stream);

/* Slice samples of the stochastic variant (Algorithm 4) as drawn on the device:
 * for sub-steps g0 .. g0+count-1 of the given layer (1 or 2) writes count * p
 * sorted slice indices to out_host (int32), p = max(1, S/frac_den).
 * Synchronises the stream. */
int ls_samples(ls_ctx* ctx, int32_t layer, uint64_t seed, uint64_t g0, int32_t count,
               int32_t* out_host, int32_t* p_out, void* stream);

/* Reverse sweep for gradients of a real loss L(phi_T) (no stored trajectory).
 * Inputs: psi_dev = phi_T, lam_dev = dL/d conj(phi_T) (Wirtinger).  Runs the
 * inverse of each factor in reverse order on both arrays (the factors are
 * unitary, so phi_T is rebuilt back to phi_0 while lambda is pulled back), and
 * at every layer factor accumulates dL/dv_j(x_p) = 2 s Im(conj(mu_p) psi_p)
 * (mu, psi: unitary grid transforms of lambda and phi after the factor).
 * grad_v1_host and grad_v2_host (one double per point of the layer's grid:
 * M1 and M2, or q_j[0] q2[1] with a shared index) receive the grid
 * gradients; grad_c1_host / grad_c2_host (2*nv doubles, may be NULL) receive
 * (dL/dRe vhat_h, dL/dIm vhat_h) for every coefficient.  On return psi_dev
 * holds the rebuilt phi_0 and lam_dev the gradient with respect to
 * conj(phi_0).  Schemes LS_LIE, LS_STRANG, LS_STRANG_KP, LS_YOSHIDA4 and the
 * stochastic LS_LIE_STOCH and LS_STRANG_STOCH (Algorithm 4): seed and step0
 * must be those of the forward ls_step call, which fix the sampled slices;
 * a sampled factor of duration s acts with duration s*S/p and contributes
 * 2 (s*S/p) Im(conj(mu_p) psi_p) over its sampled slices.  seed and step0 are
 * ignored by the deterministic schemes.  Other schemes, and contexts with
 * LS_MASK_PROJECT_EACH_STEP, return LS_ERR_INVALID.  Synchronises the stream. */
int ls_adjoint(ls_ctx* ctx, void* psi_dev, void* lam_dev, int64_t nsteps, double tau,
               int32_t scheme, uint64_t seed, uint64_t step0, double* grad_v1_host,
               double* grad_v2_host, double* grad_c1_host, double* grad_c2_host, void* stream);

/* ---- batched uneven instances (one persistent launch per call) ----
 * A batch is a set of independent problems (same dtype, any boxes) whose wave
 * functions live in one caller-owned device buffer: instance i starts at
 * element offsets[i] (ls_batch_layout; offsets has count+1 entries, the last
 * being the total element count) with row pitch pitches[i]. */
typedef struct ls_batch ls_batch;

/* Create count instances (an ls_create per problem; 1D problems with the same
 * dtype). */
int ls_batch_create(const ls_problem* probs, int32_t count, ls_batch** out);
int ls_batch_destroy(ls_batch* batch);
/* offsets: count+1 int64 (host), pitches: count int64 (host); either may be NULL. */
int ls_batch_layout(const ls_batch* batch, int64_t* offsets, int64_t* pitches);
/* ls_init_gaussian for every instance (same x0, w, k0). */
int ls_batch_init_gaussian(ls_batch* batch, void* psi_dev, const double* x0_host, double w,
                           const double* k0_host, void* stream);
/* nsteps steps of tau of any scheme for every instance in ONE persistent
 * kernel launch (replayed from a cached CUDA graph): CTAs claim
 * (step, pass, instance, slice-tile) items in order and wait, with a bounded
 * spin, until their instance has finished the previous pass.  Stochastic
 * schemes: instance i draws its samples with seed + i (sub-step g as in
 * ls_step), the sampled-slice lists are drawn on the device in the same graph,
 * kinetic phases are applied lazily and a settle phase ends the call.
 * Synchronises the stream to read the status: LS_ERR_TIMEOUT if a wait
 * expired (psi is then incomplete; the batch stays usable). */
int ls_batch_step(ls_batch* batch, void* psi_dev, int64_t nsteps, double tau, int32_t scheme,
                  uint64_t seed, uint64_t step0, void* stream);
/* ls_batch_step from host memory: psi_host (offsets[count] elements, the
 * ls_batch_layout() layout) is copied into the caller's device buffer
 * psi_dev, advanced, and copied back; synchronises.  Errors as ls_batch_step. */
int ls_batch_step_host(ls_batch* batch, void* psi_host, void* psi_dev, int64_t nsteps, double tau,
                       int32_t scheme, uint64_t seed, uint64_t step0, void* stream);
/* ls_observables for every instance; out: count ls_obs (host).  Synchronises. */
int ls_batch_observables(ls_batch* batch, const void* psi_dev, ls_obs* out_host, void* stream);
/* Configuration of the compact-kernel batched launch (used when every factor
 * of every instance takes the compact-kernel form): *threads per CTA,
 * *ctas_per_sm the registers are budgeted for, *tile_bytes of shared memory
 * per tile, *tiles_per_item consecutive tiles per claimed work item, *tuned = 1
 * once the autotuner has chosen them; *threads = 0 when it chose the transform
 * (FFT) forms instead.  The autotuner runs inside the first ls_batch_step of a
 * (scheme, tau) whose factors all qualify for the compact kernel (complex64
 * batches): it times the configurations (threads, CTAs, tiles per item)
 * (256, 3, 1), (256, 3, 2), (256, 4, 1), (128, 6, 1), (128, 6, 2), (128, 6, 4),
 * (128, 8, 2) and the transform forms, two steps each, on a library-allocated
 * scratch copy of psi, keeps the fastest and records it for the process (same
 * shapes, dtype, scheme and tau reuse it).  tune_ms (may be NULL) receives up
 * to *ntimes of the last tuning's times in ms per two steps, in that order;
 * *ntimes is then set to the number recorded.  Environment: LSPLIT_TUNE=0
 * keeps the default (128, 6, 1); LSPLIT_STENCIL_CFG="threads,ctas[,tiles]"
 * forces one. */
int ls_batch_config(const ls_batch* batch, int32_t* threads, int32_t* ctas_per_sm, int64_t* tile_bytes,
                    int32_t* tiles_per_item, int32_t* tuned, float* tune_ms, int32_t* ntimes);
/* Wait budget of one dependency wait (seconds, default 1) and a test hook that
 * makes one wait unsatisfiable (unmet_dependency != 0) to exercise the
 * timeout path. */
int ls_batch_debug(ls_batch* batch, int32_t unmet_dependency, double timeout_seconds);

/* Mass N = sum |phi|^2 (FP64) of a wave-function array, computed WITHOUT
 * allocating memory: for callers that cannot call cudaMalloc (hosts that hand
 * out all device memory from their own pool and forbid other allocations, and
 * loops that must not pay for or wait on the allocator).  The paper has no
 * counterpart; the same quantity is ls_observables()->norm.
 *   psi_dev   device array, rows x cols used elements, row pitch `pitch`
 *             elements (the ls_layout() layout: rows = M2, cols = M1)
 *   dtype     LS_C64 or LS_C128
 *   out_dev   device double (caller-owned) that receives the mass
 * Scratch is a fixed file-scope device array of 65536 FP64 row sums (512 KB,
 * held by every GPU that loads the library until the process exits); rows >
 * 65536 return LS_ERR_INVALID.  The first call on a device looks up that
 * array's device address (make it before any stream capture).  All calls share
 * the array: calls that overlap on the GPU race and must be ordered by the
 * caller.  Needs no context; enqueued on stream, no synchronisation. */
int ls_mass_noalloc(const void* psi_dev, int32_t dtype, int64_t rows, int64_t cols, int64_t pitch,
                    double* out_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LSPLIT_H */
