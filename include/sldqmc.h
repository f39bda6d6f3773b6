/*
 * sldqmc.h -- C ABI of the GB300 (sm_103a) self-learning determinantal QMC
 * library.  Every entry point returns an int status: SLDQMC_OK (0) or a
 * negative SLDQMC_ERR_* code; sldqmc_strerror() names it.
 *
 * Paper: X. Y. Xu, Y. Qi, J. Liu, L. Fu, Z. Y. Meng, "Self-Learning
 * Determinantal Quantum Monte Carlo Method", arXiv:1612.03804 (PRB 96,
 * 041119 (2017)).  Sections cited below: "Basics of DQMC" (Eq. 1 and the
 * local update), "Formalism of SLDQMC" (Eqs. 2-4, steps i-iv), "Results"
 * (Eq. 6, the model and the fit score R^2).
 *
 * Conventions shared by every call:
 *   - Lattice: Lx x Ly periodic square lattice, N = Lx*Ly, site
 *     i = x + Lx*y.  A direction of length 1 has no bond; a direction of
 *     length 2 carries its bond twice (both wrap directions).
 *   - Imaginary time: M = round(beta/dtau) slices; beta must equal M*dtau to
 *     1e-12 relative.
 *   - Field configuration s: int8 array of M*N values in {-1,+1},
 *     tau-major (s[tau*N + i]); tau = 0..M-1 is slice tau+1.  Any other
 *     value is rejected with SLDQMC_ERR_ARG (host-pointer calls) or flagged
 *     as SLDQMC_ERR_ARG by the device checks (device-pointer calls).
 *   - Slice matrix (Eq. 1 with K the hopping of Eq. 6):
 *       B_tau = exp(-dtau K) diag(exp(eta dtau xi s_tau)),  K = -t A - mu I,
 *     for flavour eta = +1 or -1.  The bilayer of Eq. 6 has two flavours of
 *     each eta, so the fermion weight is
 *       log omega_F = 2 ld(+1) + 2 ld(-1),  ld(eta) = log|det(1 + B_M..B_1)|.
 *   - Matrices are row-major double, N x N.
 *
 * Ownership and threading: a context owns all device memory it allocates
 * (at create time, and the exact log weight's second workspace on its first
 * use, see sldqmc_log_weight_batch_dev) and one CUDA stream (the caller's, or
 * the legacy default stream when NULL).  Host-pointer calls copy in, run and copy out, and
 * return after the stream has finished (synchronous).  Device-pointer calls
 * (suffix _dev) take caller-owned device memory, are ordered on the
 * context's stream and return before completion; their error flags are
 * reported by sldqmc_sync().  A context is not thread-safe: use one per host
 * thread / stream.  On any error the caller's output buffers are left
 * unchanged by host-pointer calls.
 */
#ifndef SLDQMC_H
#define SLDQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SLDQMC_OK 0
#define SLDQMC_ERR_ARG (-1)       /* invalid argument or field value */
#define SLDQMC_ERR_OOM (-2)       /* device allocation failed */
#define SLDQMC_ERR_CUDA (-3)      /* a CUDA runtime call failed */
#define SLDQMC_ERR_NUMERICAL (-4) /* non-positive Cholesky pivot, zero LU pivot or non-finite value */
#define SLDQMC_ERR_TIMEOUT (-5)   /* a bounded device-side wait ran out */
#define SLDQMC_ERR_UNSUPPORTED (-6)

/* Arithmetic of the slice products inside a stabilisation block.  The
 * stabilisation (QR), the final determinant, the Green's function and every
 * Monte Carlo decision are FP64 in all modes. */
typedef enum {
    SLDQMC_FP64 = 0,   /* FP64 FMA products */
    SLDQMC_3XTF32 = 1, /* split-TF32 tensor-core products: the running product in two TF32
                          parts, exp(-dtau K) in three (five MMAs per K-step), FP32
                          accumulation spread over eight tensor-memory accumulators */
    SLDQMC_BF16 = 2,   /* BF16 tensor-core products, FP32 accumulate */
    SLDQMC_BF16X3 = 3  /* split-BF16 tensor-core products: both operands in three BF16 parts,
                          six MMAs per 16-wide K-step, FP32 accumulation spread over eight
                          tensor-memory accumulators */
} sldqmc_prec;

typedef struct {
    int Lx, Ly;         /* lattice */
    double t, mu, xi;   /* hopping, chemical potential, Ising-fermion coupling (Eq. 6) */
    double beta, dtau;  /* inverse temperature and Trotter step */
    int n_wrap;         /* slices per stabilisation block (>= 1) */
    double J_ising, h;  /* Ising exchange and transverse field of H_s (Eq. 6) */
    int prec;           /* sldqmc_prec */
    int max_batch;      /* configurations evaluated together (workspace size), >= 1 */
} sldqmc_params;

typedef struct sldqmc_ctx sldqmc_ctx;

typedef struct {
    long long accepted;      /* accepted local flips */
    long long proposed;      /* proposed local flips */
    long long margin_events; /* decisions with |log r - log u| <= 1e-8 */
    double max_drift;        /* max |G_wrapped - G_fresh| at re-computation */
} sldqmc_stats;

/* Create a context: validates params, allocates the workspace for
 * max_batch configurations and builds exp(-dtau K) and exp(+dtau K) on the
 * device.  stream: a cudaStream_t, or NULL for the default stream. */
int sldqmc_create(const sldqmc_params *p, void *stream, sldqmc_ctx **out);
void sldqmc_destroy(sldqmc_ctx *ctx);
const char *sldqmc_strerror(int status);
/* N and M of the context. */
int sldqmc_dims(const sldqmc_ctx *ctx, int *N, int *M);
/* Waits for the context's stream and returns the first device-side error
 * flag raised since the last call (then clears it). */
int sldqmc_sync(sldqmc_ctx *ctx);

/* build_K ("Basics of DQMC": K the hopping matrix; Eq. 6 fixes
 * K = -t A - mu I).  Copies K, exp(-dtau K) and exp(+dtau K) (each N x N,
 * row-major) to host buffers; any pointer may be NULL. */
int sldqmc_build_K(sldqmc_ctx *ctx, double *K, double *expmK, double *exppK);

/* weight (Eq. 1): log|det(1 + B_M..B_1)| and its sign for flavour eta
 * (+1/-1).  eta = 0 returns the bilayer fermion weight
 * log omega_F = 2 ld(+1) + 2 ld(-1) with sign +1.  s: host, M*N int8. */
int sldqmc_weight(sldqmc_ctx *ctx, const int8_t *s, int eta, double *logabsdet, int *sign);

/* Batched weight over B configurations (host buffers, synchronous).
 * s: B*M*N int8; logabsdet: B doubles; sign: B ints (may be NULL).
 * B may exceed max_batch (processed in chunks). */
int sldqmc_weight_batch(sldqmc_ctx *ctx, const int8_t *s, int B, int eta, double *logabsdet,
                        int *sign);

/* Same on device buffers, stream-ordered.  eta must be +1 or -1. */
int sldqmc_weight_batch_dev(sldqmc_ctx *ctx, const int8_t *d_s, int B, int eta,
                            double *d_logabsdet, int *d_sign);

/* green ("Basics of DQMC": the equal-time Green's function the local update
 * needs): G(tau) = (1 + B_tau..B_1 B_M..B_{tau+1})^{-1}, N x N, for
 * 0 <= tau <= M (tau = 0 and tau = M both give (1 + B_M..B_1)^{-1}), with
 * the log|det| and sign of the same cyclic product.  Host buffers. */
int sldqmc_green(sldqmc_ctx *ctx, const int8_t *s, int eta, int tau, double *G,
                 double *logabsdet, int *sign);
int sldqmc_green_batch_dev(sldqmc_ctx *ctx, const int8_t *d_s, int B, int eta, int tau,
                           double *d_G, double *d_logabsdet, int *d_sign);

/* Bare Ising weight phi(C) ("Basics of DQMC": the bare part including the
 * transformation constant), read as the Trotter map of H_s of Eq. 6:
 *   log phi = dtau J sum_tau sum_<ij> s s + Kt sum_i sum_tau s_{i,tau} s_{i,tau+1},
 *   Kt = -ln(tanh(dtau h))/2, periodic in tau, configuration-independent
 * constant dropped.  Host s. */
int sldqmc_log_bare_weight(sldqmc_ctx *ctx, const int8_t *s, double *log_phi);

/* Local DQMC sweeps ("Basics of DQMC"): flips s(i,tau) one by one in
 * order tau = 1..M, i = 0..N-1; O(1) ratio from the Green's function
 * (both flavours, each squared, times the phi ratio), O(N^2) Sherman-Morrison
 * update on acceptance, slice-to-slice wrapping and a fresh Green's function
 * every n_wrap slices.  Uniforms come from Philox-4x32-10 with key = seed and
 * counter (i, tau, sweep0 + k, 1); accept iff log u < log r.
 * s: host, M*N int8, updated in place.  stats may be NULL. */
int sldqmc_local_sweep(sldqmc_ctx *ctx, int8_t *s, uint64_t seed, uint64_t sweep0, int n_sweeps,
                       sldqmc_stats *stats);
/* Batched over B independent chains on device buffers (chain b uses key
 * seed + (b << 32)); stats: host array of B (may be NULL). */
int sldqmc_local_sweep_batch_dev(sldqmc_ctx *ctx, int8_t *d_s, int B, uint64_t seed,
                                 uint64_t sweep0, int n_sweeps, sldqmc_stats *stats);

/* Delayed local updates ("Basics of DQMC": the O(N^2) Sherman-Morrison
 * update per accepted flip).  k = 1 (default): every accepted flip updates
 * both Green's functions at once (rank 1).  2 <= k <= 32: the sites of a
 * slice are taken in blocks of k; inside a block the Green's function is
 * kept as G0 - U V with one column/row pair per accepted flip (each site's
 * diagonal element and each new pair cost O(N k) instead of O(N^2)), and
 * after the block the rank-k correction is applied to every chain by one
 * batched GEMM per flavour.  The flips, decisions and random numbers are
 * those of k = 1; only the rounding of the Green's function differs (the
 * decisions agree outside the 1e-8 margin). */
int sldqmc_set_local_update_rank(sldqmc_ctx *ctx, int k);

/* Effective model (Eq. 2): H_eff = E0 + sum_c J_c f_c(C),
 * f_c(C) = sum_x sum_{o in class c} s_x s_{x+o}.  Class c has n_off[c]
 * offsets (dx, dy, dtau), stored consecutively as int triples in offsets
 * (each unordered pair once: give one of o and -o).  Self-pairs count 1.
 * At most 32 classes and 64 offsets in total. */
int sldqmc_set_effective_model(sldqmc_ctx *ctx, int n_class, const int *n_off, const int *offsets,
                               const double *J, double E0);

/* Features f_c for n_cfg configurations (host): F[n_cfg * n_class]. */
int sldqmc_features(sldqmc_ctx *ctx, const int8_t *cfgs, int n_cfg, int64_t *F);

/* Training, step ii / Eq. 3: regress y = ln omega = log phi + log omega_F on
 * [1, f_1..f_nc] by least squares in FP64; -beta H_eff = ln omega gives
 * E0 = -a_0/beta, J_c = -a_c/beta.  R^2 = 1 - SS_res/SS_tot (the score of
 * "Results").  cfgs: host n_cfg*M*N; logw: host n_cfg (if NULL, the library
 * evaluates ln omega itself).  The fitted model becomes the context's
 * effective model.  J: n_class doubles. */
int sldqmc_fit_effective_action(sldqmc_ctx *ctx, const int8_t *cfgs, const double *logw, int n_cfg,
                                double *J, double *E0, double *r2);

/* Effective-model sweeps (step iii): n_sweeps colour-ordered single-spin
 * Metropolis sweeps on H_eff (log acceptance 2 beta s sum_c J_c n_c), colour
 * order forward (dir = 0) or reversed (dir = 1).  Uniforms: Philox key seed,
 * counter (i, tau, step, 2 | sweep << 8).  Host s in place. */
int sldqmc_eff_sweeps(sldqmc_ctx *ctx, int8_t *s, int n_sweeps, uint64_t seed, uint32_t step,
                      int dir, long long *n_accept);

/* Batched effective-model sweeps on device buffers (stream-ordered): chain
 * b of d_s (B*M*N) uses key seed + (b << 32); dir = 0/1 fixes the colour
 * order, dir = -1 draws it per chain from counter (0,0,step,3).
 * d_accepts: B long longs incremented by the accepted flips (may be NULL). */
int sldqmc_eff_sweeps_batch_dev(sldqmc_ctx *ctx, int8_t *d_s, int B, int n_sweeps, uint64_t seed,
                                uint32_t step, int dir, long long *d_accepts);

/* Cumulative update (steps iii + iv, acceptance Eq. 4): proposes C' by
 * n_eff effective sweeps from C (direction bit from Philox counter
 * (0,0,step,3)), evaluates log omega(C') exactly (two flavours, FP64
 * finalisation) and accepts iff log u < log r with
 *   log r = [log omega(C') - log omega(C)] + beta sum_c J_c (f_c(C') - f_c(C)),
 * u from counter (0,0,step,4).  logw: log omega(C), cached, in/out. */
int sldqmc_cumulative_update(sldqmc_ctx *ctx, int8_t *s, double *logw, int n_eff, uint64_t seed,
                             uint32_t step, int *accepted, double *log_r);

/* n_steps cumulative updates for B chains on device buffers, stream-ordered
 * and free of host synchronisation (capturable in a CUDA graph).  Chain b
 * uses key seed + (b << 32) and steps step0 .. step0+n_steps-1.
 * d_s: B*M*N, d_logw: B (in/out), d_accepts: B ints incremented per
 * accepted step, d_log_r: B doubles (last step's log r; may be NULL). */
int sldqmc_cumulative_batch_dev(sldqmc_ctx *ctx, int8_t *d_s, double *d_logw, int B, int n_eff,
                                uint64_t seed, uint32_t step0, int n_steps, int *d_accepts,
                                double *d_log_r);

/* Host-buffer form of sldqmc_cumulative_batch_dev (synchronous): copies
 * s (B*M*N) and logw (B) in, runs n_steps updates, copies s, logw and the
 * per-chain accept counts (accepts: B ints, added to) back.  B <= max_batch. */
int sldqmc_cumulative_batch(sldqmc_ctx *ctx, int8_t *s, double *logw, int B, int n_eff, uint64_t seed,
                            uint32_t step0, int n_steps, int *accepts);

/* Batched uneven chains in one CUDA graph.  Captures one cumulative update
 * of every member -- context ctxs[i] (its own lattice, beta, precision and
 * n_wrap) with chains d_s[i] (B[i]*M_i*N_i), cached log weights d_logw[i]
 * and accept counters d_accepts[i] -- into a single graph whose branches run
 * concurrently on streams of their own, forked from and joined to `stream`
 * (NULL: the graph creates a stream).  Each member keeps a device step
 * counter starting at step0 that the graph advances, so every replay is the
 * next step of every chain, identical to sldqmc_cumulative_batch_dev with
 * seeds[i] and steps step0, step0+1, ...  While a graph exists its members
 * must not be used elsewhere concurrently. */
typedef struct sldqmc_graph sldqmc_graph;
int sldqmc_graph_create(sldqmc_ctx *const *ctxs, int n, int8_t *const *d_s, double *const *d_logw, const int *B,
                        int n_eff, const uint64_t *seeds, int *const *d_accepts, uint32_t step0, void *stream,
                        sldqmc_graph **out);
/* Replays the graph n_steps times on its stream (stream-ordered). */
int sldqmc_graph_launch(sldqmc_graph *g, int n_steps);
/* Waits for the graph's stream; returns the first error flag of any member. */
int sldqmc_graph_sync(sldqmc_graph *g);
void sldqmc_graph_destroy(sldqmc_graph *g);

/* log omega = log phi + 2 ld(+1) + 2 ld(-1) for B configurations on device
 * buffers (the exact weight a cumulative update needs).  The first call
 * creates a second workspace of twice max_batch with its own stream, if it
 * takes under a third of the free device memory.  With it, a batch whose
 * 2B items fit in one wave of CTAs (2B <= the device's SMs) runs both
 * flavours as one batch [s; -s] at eta = +1 (B_tau(-1) for s is B_tau(+1)
 * for -s, Eq. 1), so that every launch of the chain serves both; a larger
 * batch runs the two flavours on the two streams at once.  Without it the
 * flavours run in sequence on the context.  The results are the same bit
 * for bit.  B may exceed max_batch (processed in chunks). */
int sldqmc_log_weight_batch_dev(sldqmc_ctx *ctx, const int8_t *d_s, int B, double *d_logw);

/* Form in which the kinetic propagator exp(-dtau K) enters the slice
 * products of every weight and Green's-function evaluation of the context
 * (weight, green, log weight, fresh Green's functions of the local sweep,
 * cumulative updates).  The paper's cost of a cumulative update assumes a B
 * matrix applied in O(N^2) per slice and column rather than a dense product
 * ("Formalism of SLDQMC", the complexity paragraph).
 *   SLDQMC_KINETIC_DENSE (default): dense N x N products (the slice GEMMs of
 *     sldqmc_prec).
 *   SLDQMC_KINETIC_SEPARABLE: the exact factorisation of the periodic
 *     lattice, exp(-dtau K) = e^{dtau mu} E1x (x) E1y with E1 the ring
 *     propagator of each direction, applied as two circular convolutions of
 *     every row of the running product: 2 N^2 (Lx + Ly) flops per slice and
 *     configuration instead of 2 N^3.  It is not a Trotter splitting of K: the
 *     result equals the dense form up to rounding.  Arithmetic: FP64 in the
 *     FP64 mode; split FP32 (each value a pair of floats, 48 significant bits,
 *     FP32 accumulation) in the mixed modes.  The stabilisation and everything
 *     after it are unchanged.  Requires N <= about 14500 (a row of the
 *     product in shared memory); SLDQMC_ERR_UNSUPPORTED otherwise.
 * The wrapping of the Green's function between slices in local sweeps keeps
 * the dense products. */
#define SLDQMC_KINETIC_DENSE 0
#define SLDQMC_KINETIC_SEPARABLE 1
int sldqmc_set_kinetic_form(sldqmc_ctx *ctx, int form);

/* Output tile of the tensor-core slice products of the mixed modes:
 * 128 x 64 (bn = 64, default) with the FP32 accumulation spread over eight
 * tensor-memory accumulators, or 128 x 128 (bn = 128) with four, which reads
 * fewer shared-memory operand bytes per flop.  Four accumulators over the
 * whole K would take three times as many MMAs each, so a 128-wide tile
 * drains its accumulators into registers after each third of K; its log|det|
 * error is still larger (split-TF32, 16x16, M = 160: 1.0e-6 against 6.7e-7
 * with bn = 64; 100x100 uniform field: 8.4e-7 against 4.6e-7).  The
 * autotuner picks the faster tile whose error meets the mode's bound.  FP64
 * mode: only 64 is accepted. */
int sldqmc_set_tile_n(sldqmc_ctx *ctx, int bn);

/* Number of this library's kernels launched on the context since create. */
long long sldqmc_kernel_launches(const sldqmc_ctx *ctx);

/* Allocation-free exact weight.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc or cudaFree, such as
 * code running under a host framework that owns the whole device heap and
 * forbids direct allocations, or code on a latency-critical path that must
 * not take the implicit device synchronisation of cudaFree.
 *
 * Computes the same log|det(1 + B_M..B_1)| and sign as
 * sldqmc_weight_batch_dev (FP64 products only; prec must be SLDQMC_FP64),
 * for B configurations d_s (device, B*M*N int8) into d_logabsdet and d_sign
 * (device; d_sign may be NULL), on `stream` (NULL = legacy default stream),
 * without a context and without allocating: its workspace is one 16 MiB
 * file-scope device array that every device loading the library keeps until
 * the process exits.  Problems whose workspace exceeds 16 MiB are rejected
 * with SLDQMC_ERR_UNSUPPORTED (about 50 configurations at 8x8, 2 at 16x16;
 * no 32x32; lattices above 16384 sites or more than 100000 slices are
 * rejected the same way).  The first call on a device looks up the array's
 * device address (once per device, with that device current).  The call
 * waits for its stream and reads the status flag back before returning, so
 * it cannot be called while its stream is being captured into a CUDA graph.
 * All calls share the one array and each call overwrites what the previous
 * one left there: calls that overlap on the GPU (other host threads, other
 * streams) race and must be serialised by the caller. */
int sldqmc_weight_noalloc(const sldqmc_params *p, void *stream, const int8_t *d_s, int B, int eta,
                          double *d_logabsdet, int *d_sign);

/* Gram matrices W_b = X_b X_b^T of the Cholesky-QR stabilisation (the first
 * step of each re-orthogonalisation, whose accuracy bounds the condition
 * number Cholesky-QR can take: kappa(X)^2 eps_W < 1).  d_X holds B row-major
 * N x N FP64 matrices (item stride N*N), d_W receives B row-major N x N FP64
 * matrices of which every element on or above the diagonal is written (the
 * rest is unspecified).  Computed exactly as the context's stabilisation does:
 * in the mixed-precision modes with N >= 128 on the BF16 tensor cores by
 * error-free digit splitting (FP64 accuracy: error below ~2^-52 of
 * sqrt(W_ii W_jj)), otherwise by the FP64 GEMM.  1 <= B <= max_batch.
 * Stream-ordered on the context's stream; caller-owned device buffers. */
int sldqmc_gram_batch_dev(sldqmc_ctx *ctx, const double *d_X, int B, double *d_W);

/* Failure-path self-test of the bounded device waits used by the
 * tensor-core kernels: launches a kernel that waits on an mbarrier nothing
 * arrives at, for at most max_polls polls (1 .. 2^24), so the wait runs out
 * and raises the timeout flag; sldqmc_sync then returns SLDQMC_ERR_TIMEOUT
 * and the context stays usable. */
int sldqmc_wait_selftest(sldqmc_ctx *ctx, int max_polls);

/* Kernel classes for the timing hooks below. */
#define SLDQMC_KC_GEMM_F64 0   /* FP64 GEMM (slice products in FP64 mode, Gram, trailing updates) */
#define SLDQMC_KC_GEMM_TC 1    /* tensor-core slice products (3xTF32 / BF16) */
#define SLDQMC_KC_PANEL_F64 2  /* FP64 panel kernels (32x32 Cholesky blocks and inverses, LU panels, triangular solves, pivot sort) */
#define SLDQMC_KC_EFF 3        /* effective-model sweeps */
#define SLDQMC_KC_LOCAL 4      /* local-update flips */
#define SLDQMC_KC_OTHER 5      /* everything else */
#define SLDQMC_KC_GEMM_OZ 6    /* FP64-accurate digit-split products on the BF16 tensor cores (mixed modes): Gram matrices, Cholesky-QR updates and panels, R2 R1, V update, LU updates */
#define SLDQMC_KC_SEP 7        /* slice products with the separable exp(-dtau K) (sldqmc_set_kinetic_form) */
#define SLDQMC_KC_COUNT 8

/* Timing hooks (off by default): when on, every launch on the context's
 * stream is bracketed by CUDA events and tagged with its class and its
 * algorithmic FP64/tensor flops.  sldqmc_profile_read synchronises the
 * stream and returns, per class, the launch count, the summed event time
 * (ms) and the summed algorithmic flops, then clears the record. */
int sldqmc_profile_enable(sldqmc_ctx *ctx, int on);
int sldqmc_profile_read(sldqmc_ctx *ctx, long long *launches, double *ms, double *flops);
/* Same record by launch site instead of by class: one text line per site,
 * "site class launches ms flops", into buf (len bytes, NUL-terminated;
 * lines that do not fit are dropped), then clears the record. */
int sldqmc_profile_read_sites(sldqmc_ctx *ctx, char *buf, int len);

#ifdef __cplusplus
}
#endif
#endif /* SLDQMC_H */
