/*
 * thc_sox.h - C ABI of the GB300 (sm_103a) library for the imaginary-time
 * second-order-exchange (SOX) self-energy in tensor-hypercontraction (THC)
 * form and its screened variants (arXiv 2412.18829, Sec. II B-C).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an int status (SOX_OK = 0 on success).  On failure
 *   sox_last_error(h) returns a message; nothing is written to outputs that
 *   failed validation.
 * - Pointers are owned by the caller.  Tensor pointers may be DEVICE or HOST
 *   memory (detected per pointer).  Host inputs are staged through the
 *   handle's workspace; when any output is in host memory the call
 *   synchronises `stream` before returning.  The library never keeps a caller
 *   pointer past the call.
 * - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL
 *   is the legacy default stream) when all tensors are device pointers.
 * - The handle owns a device workspace that grows on demand with cudaMalloc.
 *   A call that needs more workspace than any earlier call allocates, so
 *   capture calls into a CUDA graph only after one un-captured call of the
 *   same (or larger) size, or after sox_reserve.
 * - Layouts are row-major, contiguous, outermost index first:
 *     G, Sigma  [n_spin][n_k][n_tau][n][n]
 *     X         [n_k][N][n]         X[k][P][p] = X^k_{pP}
 *     V, W0     [n_q][N][N]         U^q_{PQ}   (n_q = n_k)
 *   Real data (SOX_REAL64) are doubles; complex data (SOX_COMPLEX128) are
 *   interleaved (re, im) doubles.  Molecules are SOX_REAL64 with n_k = 1.
 *   Solids (any k-mesh) are SOX_COMPLEX128: sox_sigma, sox_sigma_general,
 *   sosex_static_sigma and sosex_dynamic_sigma accept them and run the
 *   momentum-resolved chain, in FP64 complex on CUDA cores (SOX_PREC_FP64) or
 *   with every contraction as complex FP16-pair GEMMs on the tensor cores
 *   (SOX_PREC_F16X2; projections, D accumulation over v and the final orbital
 *   sum in FP64).  The other entry points return SOX_ERR_UNSUPPORTED for
 *   complex data.
 * - k labels run row-major over the mesh (k = 2 pi m / nk, m in [0, nk)^3);
 *   V[q] is the THC metric of momentum transfer q = k_i - k_j (Sec. II C).
 * - The tau grid must be mirror-symmetric, tau_{n_tau-1-j} = beta - tau_j
 *   (Chebyshev-Lobatto, see sox_tau_grid): G(-tau_j) is taken as
 *   -G(tau_{n_tau-1-j}) (fermionic antiperiodicity of Eq. G_def).
 * - Same-spin only (Sec. II C): spin blocks are independent.
 */
#ifndef THC_SOX_H
#define THC_SOX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SOX_API __attribute__((visibility("default")))
#else
#define SOX_API
#endif

/* status codes */
#define SOX_OK 0
#define SOX_ERR_INVALID_ARG 1  /* null pointer, bad enum, bad handle          */
#define SOX_ERR_SHAPE 2        /* sizes out of range or inconsistent           */
#define SOX_ERR_UNSUPPORTED 3  /* valid request this build does not implement  */
#define SOX_ERR_OOM 4          /* device or pinned allocation failed           */
#define SOX_ERR_CUDA 5         /* a CUDA runtime/driver call failed            */
#define SOX_ERR_TIMEOUT 6      /* a device-side wait hit its iteration cap     */

/* arithmetic of the contractions (projections, back-projection, Phi: FP64) */
#define SOX_PREC_FP64 0   /* every step in FP64 on CUDA cores (reference path)          */
#define SOX_PREC_F16X2 1  /* B/C/A/U contractions as 2-piece FP16 splits with per-row
                             power-of-two scaling on tcgen05 tensor cores, FP32 accumulate */

#define SOX_REAL64 0
#define SOX_COMPLEX128 1

/* limits checked by every entry point */
#define SOX_MAX_N_AO 1024
#define SOX_MAX_N_THC 16384
#define SOX_MAX_N_TAU 4096

typedef struct sox_context *sox_handle;

typedef struct {
  int precision;        /* SOX_PREC_*                                           */
  int device;           /* CUDA device ordinal the handle is bound to            */
  long long spin_limit; /* iteration cap for device-side waits; 0 = default      */
  long long workspace_limit; /* bytes of chunked intermediates each entry point
                          * sizes its tau / v chunks for; 0 = the library's
                          * defaults (12-32 GiB per path; 64 GiB for the
                          * split-precision adjoint, 128 GiB for the uneven
                          * batch).  A chunk of one tau
                          * point (or one v) is used even when it exceeds the
                          * limit; fixed-size tensors (mixed tensors, the D
                          * array of the dynamic paths) are not counted.      */
  int no_autotune;      /* 0: on the first call for a new shape, the split path
                         * times its fused-kernel variants on the call's own
                         * data (one extra launch each, a host synchronisation)
                         * and keeps the fastest for that shape on the handle;
                         * skipped while the stream is being captured.
                         * nonzero: fixed choice, no timing.                   */
} sox_options;

typedef struct {
  int n;      /* orbitals per k-point (n_AO), 1..SOX_MAX_N_AO                    */
  int N;      /* THC interpolation points, 1..SOX_MAX_N_THC                       */
  int n_tau;  /* imaginary-time points, 2..SOX_MAX_N_TAU, mirror-symmetric grid   */
  int n_spin; /* 1 (restricted) or 2 (unrestricted, independent blocks)           */
  int nk[3];  /* k-mesh; {1,1,1} for molecules                                    */
  int dtype;  /* SOX_REAL64 or SOX_COMPLEX128                                     */
  double beta;/* inverse temperature (Ha^-1), > 0                                 */
} sox_problem;

/* Library version (major*10000 + minor*100 + patch). */
SOX_API int sox_version(void);

/* Create a handle bound to opt->device (NULL opt: FP64, device 0).
 * Allocates nothing on the device until the first call needs workspace. */
SOX_API int sox_create(sox_handle *out, const sox_options *opt);

/* Destroy a handle and free its workspace (synchronises the device). */
SOX_API int sox_destroy(sox_handle h);

/* Message for the last failed call on this handle ("" if none).  Valid until
 * the next call on the same handle. */
SOX_API const char *sox_last_error(sox_handle h);

/* Launch accounting for measurement.  While enabled, every kernel the
 * handle launches is counted, and the launches of the named hot kernels are
 * bracketed by CUDA events on their launch stream.  sox_profile_read
 * synchronises the device, then returns for `kernel` (e.g. "sox_bcd") the
 * number of timed launches and their summed device time in ms; kernel = NULL
 * returns the total number of kernels launched since enabling (ms = 0).
 * Enabling resets the counters. */
SOX_API int sox_profile_enable(sox_handle h, int enable);
SOX_API int sox_profile_read(sox_handle h, const char *kernel, long long *launches, double *ms);

/* Synchronise the handle's device and report device-side wait failures:
 * SOX_ERR_TIMEOUT if any kernel of an earlier call on this handle gave up a
 * bounded wait (its results are then invalid; the status is cleared). */
SOX_API int sox_check_device(sox_handle h);

/* Partial builds for a split over GPUs (no paper passage: the partition of Sec. II C's
 * sums over the orbital index v, which the paper moves to the outside loop of the dynamic
 * algorithm for the same purpose).  After sox_set_v_range(h, v0, v1) every self-energy
 * call on h keeps only the terms of Eq. (sox) whose index v (the column of G(-tau) in
 * G_sv(-tau)) lies in [v0, v1): sox_sigma, sox_sigma_general, sosex_static_sigma,
 * g3w2_static_sigma, sosex2_static_sigma and sosex_dynamic_sigma (static and dynamic parts,
 * molecules and solids, both precisions) return the partial Sigma, phi_sox the partial Phi
 * and phi_sox_backward the gradients dX, dV of that partial Phi.  Every chain is linear in
 * that sum, so the partial results of a partition of [0, n), summed (one all-reduce),
 * equal the whole build.  v1 <= 0 (or v1 >= n) means up to n; (0, 0) restores the whole
 * build.  With a partial range phi_sox_backward refuses dG (SOX_ERR_UNSUPPORTED: the
 * identity dPhi/dG = -w Sigma(beta - tau)^T needs the whole Sigma), and the projections,
 * sox_pi0, sox_w_static and sox_w_dynamic are not affected.  Batch plans keep the range of
 * their handle at creation.  Returns SOX_ERR_INVALID_ARG for v0 < 0 or 0 < v1 < v0. */
SOX_API int sox_set_v_range(sox_handle h, int v0, int v1);

/* Fused B/C/Hadamard kernel of the split-precision molecular chain (Sec. II C, the B, C
 * and D steps; used by sox_sigma, sox_sigma_general, sosex_static_sigma, phi_sox and the
 * batch calls on an SOX_PREC_F16X2 handle).  SOX_KERNEL_AUTO (the default) times the
 * variants on the first call per shape and keeps the fastest (outside a stream capture
 * and unless sox_options.no_autotune; else resident for n <= 128, streamed above);
 * the others force one variant for every later call on h:
 *   SOX_KERNEL_RESIDENT  G_Rq / G_wP^T tiles resident in shared memory (n <= 128 only;
 *                        larger n run the streamed kernel),
 *   SOX_KERNEL_STREAMED  all four operands streamed through a 3-stage TMA pipeline,
 *   SOX_KERNEL_PAIR      streamed on CTA pairs (tcgen05 cta_group::2, 256 x 128 tiles,
 *                        each SM loading half of the R-side operand).
 * Every variant computes the same Sigma up to FP32 accumulation order.  Returns
 * SOX_ERR_INVALID_ARG for another value. */
enum { SOX_KERNEL_AUTO = 0, SOX_KERNEL_RESIDENT = 1, SOX_KERNEL_STREAMED = 2, SOX_KERNEL_PAIR = 3 };
SOX_API int sox_set_kernel_variant(sox_handle h, int variant);

/* Grow the workspace for problem p now (outside any graph capture). */
SOX_API int sox_reserve(sox_handle h, const sox_problem *p);

/* Host helper: Chebyshev-Lobatto nodes tau_j = (beta/2)(1 - cos(pi j/(n_tau-1)))
 * and Clenshaw-Curtis weights w_j (sum_j w_j f(tau_j) ~ int_0^beta f).  The
 * paper uses sparse-ir grids (Sec. III A); any mirror-symmetric grid with
 * symmetric weights may be passed instead.  tau, w: host arrays [n_tau]. */
SOX_API int sox_tau_grid(int n_tau, double beta, double *tau, double *w);

/* THC projections of G (Sec. II C, the G_Rq and G_wP steps after
 * Eq. U_contraction; full projection G^PQ = X G X^T used by Pi and Phi):
 *   G_Rq[s][k][t][R][q] = sum_u X_{uR} G_{uq}(tau_t)
 *   G_wP[s][k][t][w][P] = sum_p G_{wp}(tau_t) X_{pP}
 *   G_PQ[s][k][t][P][Q] = sum_pq X_{pP} G_{pq}(tau_t) X_{qQ}   (may be NULL)
 * All FP64 regardless of precision. */
SOX_API int thc_project_G(sox_handle h, const sox_problem *p, const double *G, const double *X,
                  double *G_Rq, double *G_wP, double *G_PQ, void *stream);

/* Bare SOX self-energy, Eq. (sox) with U(1) = U(2) = v in THC form and the
 * static time collapse (Sec. II C).  For a solid, with momentum transfers
 * q1, q2 of the two interactions,
 *   Sigma^k_tr = -1/N_k^2 sum_{q1,q2} U1^{q1}_(pr|qs) U2^{q2}_(tu|vw)
 *                G^{k+q1}_wp(tau) G^{k-q2}_uq(tau) G^{k+q1-q2}_sv(-tau).
 * Molecules:
 *   Sigma_tr(tau) = -sum U1_(pr|qs) U2_(tu|vw) G_wp(tau) G_uq(tau) G_sv(-tau).
 * Computed by the THC chain U_Pqs -> A -> (B o C summed over v) -> D ->
 * Sigma_RP = -D_PR -> Sigma_tr = sum_PR X_tR Sigma_RP X_rP.
 * G, Sigma [n_spin][1][n_tau][n][n]; X [1][N][n]; V [1][N][N]. */
SOX_API int sox_sigma(sox_handle h, const sox_problem *p, const double *G, const double *X,
              const double *V, double *Sigma, void *stream);

/* Statically screened SOSEX (Sec. II B): SOX with one interaction replaced by
 * the screened W(i Omega = 0).  slot = 1: U(1) = W0, U(2) = V (the screened
 * first interaction of Sec. II B and the dynamic algorithm); slot = 2:
 * U(1) = V, U(2) = W0 (the form written in the G3W2 decomposition, Sec. III C).
 * W0 [1][N][N]. */
SOX_API int sosex_static_sigma(sox_handle h, const sox_problem *p, const double *G, const double *X,
                       const double *V, const double *W0, int slot, double *Sigma,
                       void *stream);

/* Compositions of statically screened SOX (Sec. III C, the G3W2 decomposition
 * with W_d = W(0) - v):
 *   g3w2_static_sigma:   Sigma^G3W2stat = SOX(W0, W0), both interactions screened;
 *   sosex2_static_sigma: Sigma^2SOSEXstat = SOX(v, v) + SOX(v, W_d) + SOX(W_d, v),
 *                        computed as SOX(v, W0) + SOX(W0 - v, v).
 * Layouts and precision as sox_sigma (molecules and solids; V, W0 [n_q][N][N]).
 * sosex2_static_sigma keeps its partial result, W_d and any host tensors it
 * stages in a second buffer of the handle that grows on demand (the growth
 * synchronises the device); with a host Sigma it synchronises the stream at
 * the end.  It costs two SOX builds. */
SOX_API int g3w2_static_sigma(sox_handle h, const sox_problem *p, const double *G, const double *X,
                              const double *W0, double *Sigma, void *stream);
SOX_API int sosex2_static_sigma(sox_handle h, const sox_problem *p, const double *G, const double *X,
                                const double *V, const double *W0, double *Sigma, void *stream);

/* General static SOX(U1, U2) (Eq. sox with two static interactions). */
SOX_API int sox_sigma_general(sox_handle h, const sox_problem *p, const double *G, const double *X,
                      const double *U1, const double *U2, double *Sigma, void *stream);

/* Static polarisability in THC form for the statically screened interaction:
 *   Pi0[s][P][Q] = sum_j w_j G^PQ(tau_j) G^QP(-tau_j)   (FP64)
 * w: tau weights [n_tau] (host or device).  Pi0 [n_spin][N][N]. */
SOX_API int sox_pi0(sox_handle h, const sox_problem *p, const double *G, const double *X,
            const double *w, double *Pi0, void *stream);

/* Screened interaction W0 = V^1/2 (1 - V^1/2 Pi V^1/2)^-1 V^1/2, computed as
 * the equal (1 - V Pi)^-1 V by Gauss-Jordan elimination with partial
 * pivoting in FP64.  Pi is the total polarisability [N][N] (sum the spin
 * blocks of sox_pi0 first if desired).  Returns SOX_ERR_INVALID_ARG for a
 * singular system. */
SOX_API int sox_w_static(sox_handle h, const sox_problem *p, const double *V, const double *Pi,
                 double *W0, void *stream);

/* Luttinger-Ward functional of bare SOX per spin block:
 *   phi[s] = 1/4 sum_j w_j Tr[Sigma(tau_j) G(-tau_j)]          (FP64 trace)
 * (the tau form of the SOX part of E_dyn, Eq. E2b, divided by 4).
 * Sigma_out [n_spin][1][n_tau][n][n] may be NULL; phi [n_spin]. */
SOX_API int phi_sox(sox_handle h, const sox_problem *p, const double *G, const double *X,
            const double *V, const double *w, double *phi, double *Sigma_out, void *stream);

/* Adjoint of phi_sox: given dphi [n_spin] (the cotangent of phi), returns
 *   dG[s][0][j][r][t] = dphi[s] * dPhi_s/dG_rt(tau_j)  = -dphi[s] w_j Sigma_tr(beta - tau_j)
 *   dX[0][P][p]       = sum_s dphi[s] dPhi_s/dX_pP
 *   dV[0][P][Q]       = sum_s dphi[s] dPhi_s/dV_PQ
 * with respect to the unsymmetrised entries.  Any of dG, dX, dV may be NULL.
 * dG follows from Sigma by the identity above (computed in the handle's
 * precision); dX and dV come from a reverse pass through the THC chain in FP64
 * that recomputes B_v and C_v per tau chunk instead of storing them. */
SOX_API int phi_sox_backward(sox_handle h, const sox_problem *p, const double *G, const double *X,
                     const double *V, const double *w, const double *dphi, double *dG,
                     double *dX, double *dV, void *stream);

/* The G part of the adjoint from a Sigma the caller already holds (for example
 * the Sigma_out of phi_sox), without recomputing it:
 *   dG[s][0][j][r][t] = -dphi[s] w_j Sigma[s][0][n_tau-1-j][t][r]
 * (the conserving identity dPhi/dG_rt(tau_j) = -w_j Sigma_tr(beta - tau_j) on a
 * mirror-symmetric grid, Sec. II C with Eq. E2b).  Sigma and dG
 * [n_spin][1][n_tau][n][n], w [n_tau], dphi [n_spin]; FP64, molecules only.
 * dG must not alias Sigma. */
SOX_API int phi_sox_grad_G(sox_handle h, const sox_problem *p, const double *Sigma, const double *w,
                   const double *dphi, double *dG, void *stream);

/* Dynamically screened SOSEX for molecules (Sec. II C, Eq. GG and the steps
 * after it):
 *   Sigma = SOX(v, v) + Sigma_d with
 *   Sigma_d,tr(tau_i) = -sum v_(tu|vw) G_wp(tau_i)
 *        sum_m T_inv[i][m] sum_j T_fwd[m][j] Wd_(pr|qs)(i Omega_m) G_uq(tau_j) G_sv(-tau_j)
 * Wd [n_omega][N][N] real: W(i Omega_m) - v, real and even in Omega for a real
 * molecule; T_fwd [n_omega][n_tau] and T_inv [n_tau][n_omega] complex
 * (interleaved).  The transform pair is the caller's (the paper uses sparse-ir,
 * Sec. II C).  SOX(v, v) runs in the handle's precision, Sigma_d in FP64 with v in
 * the outer loop (GG, transform, W_d product, inverse transform, then the fused
 * B/C/D kernel with X in place of G_Rq).
 * Solids (dtype SOX_COMPLEX128, any k-mesh; Sec. II C with momenta): Wd is
 * complex [n_q][n_omega][N][N], W_d^q(i Omega_m) for every transfer q in the
 * k-mesh order of V; W_d sits in the first interaction slot and carries the
 * transfer q1 of that slot,
 *   Sigma_d^k(tau_i) = -1/N_k^2 sum_{q1,q2} X_k^H D_d^k(tau_i)^T X_k,
 * where D_d is the static chain's D with B built from
 *   A^{q1,ks}_Puv(tau_i) = sum_m T_inv[i][m] sum_Q W_d^{q1}_PQ(i Omega_m)
 *        sum_j T_fwd[m][j] G^{ks-q1}_uQ(tau_j) G^{ks}_Qv(-tau_j).
 * Solids run in the handle's precision (see the layout notes above).  G, X, V
 * and Sigma use the solid layouts of sox_sigma. */
SOX_API int sosex_dynamic_sigma(sox_handle h, const sox_problem *p, const double *G, const double *X,
                        const double *V, const double *Wd, const double *T_fwd,
                        const double *T_inv, int n_omega, double *Sigma, void *stream);

/* RPA screened interaction on the transform's bosonic frequencies: the W_d input of
 * sosex_dynamic_sigma built on the GPU from G (Sec. III C, W = v^1/2 (1 - v^1/2 Pi
 * v^1/2)^-1 v^1/2, with the THC form of the bubble, Sec. II C):
 *   Pi(tau_j)_PQ    = sum_s G_s^PQ(tau_j) G_s^QP(-tau_j),   G^PQ = sum_pp' X_Pp G_pp' X_Qp'
 *   Pi(i Omega_m)   = sum_j T_fwd[m][j] Pi(tau_j)
 *   Wd(i Omega_m)   = (1 - V Pi(i Omega_m))^-1 V - V
 * (the same W as the symmetric form for positive semidefinite V), with
 * G(-tau_j) = -G(tau_{n_tau-1-j}) on the mirror-symmetric grid and the spin blocks of
 * G summed.  Molecules (SOX_REAL64): the real part of Pi(i Omega_m), symmetrised; Wd
 * [n_omega][N][N] real.  Solids (SOX_COMPLEX128, mesh sides <= 8): per transfer q,
 *   Pi^q(tau_j)_PQ = 1/N_k sum_k G^PQ_{k+q}(tau_j) G^QP_k(-tau_j),  G^PQ_k = X^k G^k X^k^H,
 * and Wd [n_q][n_omega][N][N] complex, the layout sosex_dynamic_sigma reads.
 * T_fwd [n_omega][n_tau] complex (interleaved).  FP64 throughout; the solve is
 * Gauss-Jordan with partial pivoting batched over (q, m).  When the rows of T_fwd pair
 * up as +-Omega (row n_omega-1-m the conjugate of row m) and G is Hermitian (a real
 * molecule: the pairs suffice), Wd(-Omega) = Wd(Omega)^H and only m < (n_omega+1)/2 is
 * solved.  Synchronises `stream`.
 * Returns SOX_ERR_INVALID_ARG if some 1 - V Pi is singular, SOX_ERR_SHAPE for a mesh
 * side above 8 or more than 65535 (q, m) systems. */
SOX_API int sox_w_dynamic(sox_handle h, const sox_problem *p, const double *G, const double *X,
                          const double *V, const double *T_fwd, int n_omega, double *Wd, void *stream);

/* Batch of independent bare-SOX problems (uneven sizes allowed), Eq. (sox) for each, on one
 * stream.  probs, G, X, V, Sigma are HOST arrays of `count` entries; the tensors they point
 * to follow the single-problem rules (device or host memory).  On an SOX_PREC_F16X2 handle a
 * batch of molecules shares its tau chunks: each instance's chain up to A and after D runs on
 * its own, and the fused B / C / Hadamard step of one chunk of every instance is ONE
 * persistent launch over all their (P, R) tiles, largest instances first (at most 24
 * instances per launch; more take several).  Solids and FP64 handles run the instances in
 * turn.  The first instance that fails stops the batch (its index in sox_last_error). */
SOX_API int sox_sigma_batch(sox_handle h, int count, const sox_problem *probs,
                    const double *const *G, const double *const *X, const double *const *V,
                    double *const *Sigma, void *stream);


/* phi_sox over a batch of molecules (Sec. II C chain; Phi := 1/4 sum_j w_j Tr[Sigma(tau_j)
 * G(-tau_j)] per spin), with the batched fused launch of sox_sigma_batch.  w[i] [n_tau],
 * phi[i] [n_spin] and Sigma[i] (required) are the arrays of phi_sox for instance i.  Solids:
 * SOX_ERR_UNSUPPORTED. */
SOX_API int phi_sox_batch(sox_handle h, int count, const sox_problem *probs, const double *const *G,
                          const double *const *X, const double *const *V, const double *const *w,
                          double *const *phi, double *const *Sigma, void *stream);

/* Batch plan (graph form of sox_sigma_batch).  The whole launch sequence of
 * `count` independent bare-SOX problems (uneven sizes allowed; molecules,
 * SOX_REAL64) is run once eagerly and then recorded once into a CUDA graph;
 * sox_plan_launch replays it with a single graph launch, reading the current
 * contents of the same G, X, V and writing the same Sigma.  No paper passage:
 * this is the batching of Sec. II C's per-instance chains, as an execution plan.
 *   - h: supplies precision, device and limits; the plan owns its own handle and
 *     workspace (sized for the largest instance at creation, never regrown), so
 *     other calls on h cannot invalidate it.  Creation synchronises its device.
 *   - probs, G, X, V, Sigma: HOST arrays of `count` entries; every tensor must be
 *     device memory on h's GPU and stay allocated, at the same address, for the
 *     plan's lifetime.  Host tensors and solids: SOX_ERR_INVALID_ARG /
 *     SOX_ERR_UNSUPPORTED.
 *   - sox_plan_launch is asynchronous on `stream`; launches on one stream run in
 *     order; launches of one plan on different streams at once race (they share
 *     the plan's workspace).  sox_plan_check_device synchronises the device and
 *     reports a device-side wait that timed out, like sox_check_device.
 *   - sox_plan_destroy synchronises the device and frees the plan. */
typedef struct sox_plan_s *sox_plan;
SOX_API int sox_sigma_batch_plan(sox_handle h, int count, const sox_problem *probs, const double *const *G,
                                 const double *const *X, const double *const *V, double *const *Sigma,
                                 sox_plan *out);
SOX_API int sox_plan_launch(sox_plan plan, void *stream);
SOX_API int sox_plan_check_device(sox_plan plan);
SOX_API const char *sox_plan_last_error(sox_plan plan);
SOX_API int sox_plan_destroy(sox_plan plan);

/* ------------------------------------------------------------------------
 * The self-consistent loop around Sigma for molecules (Sec. II A): its device steps.
 * Real molecular data (SOX_REAL64, n_k = 1); layouts as above plus
 *   omegas  [n_w]                        fermionic Matsubara frequencies w = (2m+1) pi / beta
 *   F, Sigma_hf, gamma, tails             [n_spin][n][n] real (tails: [n_spin][3][n][n])
 *   Sigma_iw, G_iw                        [n_spin][n_w][n][n] complex (interleaved)
 *   G_tau, Sigma_tau                      [n_spin][n_tau][n][n] real
 * Host or device pointers like the other calls (sox_mix_green: device only).  FP64.
 * ------------------------------------------------------------------------ */

/* Dyson equation on the Matsubara frequencies (Eqs. Dyson and G0, S = 1):
 *   G_iw[s][w] = [(i w + mu) 1 - F[s] - Sigma_iw[s][w]]^-1
 * with F = H0 + Sigma_HF (the static part) and Sigma_iw the dynamic part (NULL: zero).
 * Complex Gauss-Jordan with partial pivoting, one CUDA block per (spin, frequency).
 * Synchronises `stream`; SOX_ERR_INVALID_ARG for a singular system. */
SOX_API int sox_dyson(sox_handle h, const sox_problem *p, int n_w, const double *omegas, double mu, const double *F,
                      const double *Sigma_iw, double *G_iw, void *stream);

/* High-frequency coefficients of G = [i w - (F - mu) - Sigma(i w)]^-1:
 *   tails[s] = {1, F[s] - mu, (F[s] - mu)^2 + Sigma_1[s]},  Sigma_1 = -(Sigma(tau_{n_tau-1}) + Sigma(tau_0))
 * (the jump of the antiperiodic Sigma(tau); Sigma_tau NULL: zero). */
SOX_API int sox_green_tails(sox_handle h, const sox_problem *p, double mu, const double *F, const double *Sigma_tau,
                            double *tails, void *stream);

/* Back to imaginary time with the tails summed exactly:
 *   G_tau[s][t] = Re[(1/beta) sum_w e^{-i w tau_t} (G(i w) - c1/(i w) - c2/(i w)^2 - c3/(i w)^3)]
 *                 - c1/2 + (2 tau_t - beta)/4 c2 + tau_t (beta - tau_t)/4 c3
 * (the closed-form tau images of the three tail powers summed over all fermionic w), at the
 * caller's n_t points tau [n_t] of [0, beta] (end points read as 0^+ and beta^-). */
SOX_API int sox_iw_to_tau(sox_handle h, const sox_problem *p, int n_w, const double *omegas, const double *G_iw,
                          const double *tails, int n_t, const double *tau, double *G_tau, void *stream);

/* To the Matsubara frequencies with the caller's transform (the paper takes its transforms
 * from sparse-ir; any quadrature of F(i w) = int_0^beta e^{i w tau} F(tau) d tau for the
 * interpolant on the tau grid): F_iw[s][w] = sum_j T_w[w][j] F_tau[s][j], T_w [n_w][n_tau] complex. */
SOX_API int sox_tau_to_iw(sox_handle h, const sox_problem *p, int n_w, const double *T_w, const double *F_tau,
                          double *F_iw, void *stream);

/* Chemical potential for the target electron count (Sec. II A): bisection on [lo, hi] of
 *   count(mu) = sum_s Tr gamma^s(mu),  gamma = -G(beta^-)^T  from the Dyson G at mu
 * until hi - lo < tol or max_iter steps; *mu (host) receives the midpoint.  Synchronises. */
SOX_API int sox_find_mu(sox_handle h, const sox_problem *p, int n_w, const double *omegas, double target,
                        const double *F, const double *Sigma_iw, const double *Sigma_tau, double lo, double hi,
                        double tol, int max_iter, double *mu);

/* Correlated density matrix gamma_pq = G_qp(0^-) = -G_qp(beta^-) from G_tau's last point
 * (the sign reading of Sec. II A's gamma that gives positive occupations). */
SOX_API int sox_density_matrix(sox_handle h, const sox_problem *p, const double *G_tau, double *gamma, void *stream);

/* Hartree-Fock self-energy in THC form, (pq|rs) = sum_PQ X_Pp X_Pq V_PQ X_Qr X_Qs:
 *   Sigma_hf[s] = J - K[s],  J_pq = sum_rs (pq|rs) rho_rs (rho = sum_s gamma[s]),
 *   K[s]_pq = sum_rs (pr|sq) gamma[s]_rs,
 * and, when F is not NULL, the static part of the Dyson equation F[s] = H0 + Sigma_hf[s]
 * (H0 [n][n], needed then).  X [N][n], V [N][N]. */
SOX_API int sox_sigma_hf(sox_handle h, const sox_problem *p, const double *X, const double *V, const double *gamma,
                         const double *H0, double *Sigma_hf, double *F, void *stream);

/* Galitskii-Migdal energies summed over spin blocks (Eqs. E1b and E2b, the latter in
 * imaginary time on the mirror-symmetric grid with weights w [n_tau]):
 *   E[0] = E_inf = sum_s sum_pq (H0 + Sigma_hf[s] / 2)_pq gamma[s]_pq
 *   E[1] = E_dyn = -sum_s sum_j w_j Tr[Sigma[s](tau_{n_tau-1-j}) G[s](tau_j)]
 * H0 [n][n]; E [2] (host or device). */
SOX_API int sox_gm_energies(sox_handle h, const sox_problem *p, const double *H0, const double *Sigma_hf,
                            const double *gamma, const double *Sigma_tau, const double *G_tau, const double *w,
                            double *E, void *stream);

/* Linear mixing of the iteration (the paper's CDIIS is not part of this library):
 *   G = (1 - a) G + a G_new over `count` doubles (device), *change (host) = max |G_new - G|
 * before the update.  Synchronises `stream`. */
SOX_API int sox_mix_green(sox_handle h, long long count, double a, double *G, const double *G_new, double *change,
                          void *stream);

/* ------------------------------------------------------------------------
 * Allocation-free variant (the paper has no counterpart; this is a service to
 * callers of the library).
 *
 * Some callers cannot allocate device memory at all: a process whose device
 * memory is handed to another runtime's fixed pool at start-up, or a component
 * that may only work inside buffers it was given.  They cannot create a
 * sox_handle, because a handle allocates its workspace and status word with
 * cudaMalloc.  sox_sigma_fp64_noalloc computes the same bare SOX self-energy as
 * sox_sigma on an FP64 handle (same kernels, same layouts) without a handle and
 * without calling cudaMalloc, cudaFree or any allocating library routine.
 *
 * - Scratch: a fixed device array of SOX_NOALLOC_SCRATCH_BYTES (64 MiB) in the
 *   library, held by every GPU that loads the library until the process exits.
 *   A problem needs 8 * (N n^2 + c (N n^2 + 3 N n + N^2)) bytes (plus 256-byte
 *   padding per slice) for c = 1 tau point at least; larger problems are
 *   rejected with SOX_ERR_SHAPE.  n = 80 with N = 480 fits, n = 90 with N = 540
 *   does not.
 * - The first call on each device looks up the array's device address (with
 *   that device current); make that first call before any stream capture.  The
 *   address is kept per device with the id of the context it belongs to; after a
 *   cudaDeviceReset the next call on that device looks it up again (set-up again),
 *   so that call too should come before any capture.
 * - Every call shares the one array, and it keeps the last call's contents
 *   (nothing in it needs to start at zero: every element is written before it
 *   is read).  Calls that overlap on the GPU race on the array: run them on
 *   one stream or serialise them.
 * - G, X, V, Sigma must be device (or managed) pointers of the current device:
 *   host pointers and device memory of another GPU return SOX_ERR_INVALID_ARG
 *   (staging them would need memory).
 * - A launch error left pending by the caller's earlier work on this thread is
 *   cleared on entry and not reported; SOX_ERR_CUDA reports this call's launches.
 * - Returns SOX_OK, SOX_ERR_INVALID_ARG, SOX_ERR_SHAPE, SOX_ERR_UNSUPPORTED
 *   (solids / complex data) or SOX_ERR_CUDA; asynchronous on `stream`.
 * ------------------------------------------------------------------------ */
#define SOX_NOALLOC_SCRATCH_BYTES (64ull << 20)
SOX_API int sox_sigma_fp64_noalloc(const sox_problem *p, const double *G, const double *X, const double *V,
                                   double *Sigma, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* THC_SOX_H */
