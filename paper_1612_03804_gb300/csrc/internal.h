// internal.h -- shared declarations of the sldqmc CUDA library (not part of
// the public C ABI).  All kernels are written for sm_103a (GB300).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

struct sldqmc_ctx;

#include "sldqmc.h"

namespace sldqmc {

// Error bits raised by kernels into the context's device flag word.
enum : int {
    FLAG_NUMERICAL = 1,  // non-positive Cholesky pivot, zero LU pivot or non-finite value
    FLAG_ARG = 2,        // field value outside {-1, +1}
    FLAG_TIMEOUT = 4,    // a bounded device wait ran out
};

// Batched FP64 GEMM description: for each batch item b,
//   C = alpha * op(A) * diag(kscale) * op(B) * diag(nscale) * diag(mscale) + beta * C
// op(A) is M x K: A[m*lda + k] (TA = false) or A[k*lda + m] (TA = true).
// op(B) is K x N: B[k*ldb + n] (TB = false) or B[n*ldb + k] (TB = true).
// kscale/nscale/(s_m row scale) come from a field slice: value cu where s > 0, cd otherwise.
// mscale is a double vector (or its reciprocal when ms_recip).
// a_upper: A is upper triangular (op(A)[m][k] = 0 for k < m): skip those k.
// c_upper: only tiles touching the upper triangle of C (n >= m) are written.
struct GemmF64 {
    int M, N, K;
    const double *A;
    long long lda, sA;
    const double *B;
    long long ldb, sB;
    double *C;
    long long ldc, sC;
    double alpha, beta;
    const int8_t *s_k;
    long long sSk;
    const int8_t *s_n;
    long long sSn;
    const int8_t *s_m;  // row scale of C from a field slice
    long long sSm;
    double cu, cd;
    const double *ms;
    long long sMs;
    int ms_recip;
    int a_upper;
    int b_upper;  // op(B) upper triangular (op(B)[k][n] = 0 for k > n): skip those k
    int c_upper;
    int batch;
};

void gemm_f64(const GemmF64 &g, bool TA, bool TB, cudaStream_t st);
// Algorithmic flops of a GEMM description (triangles counted once).
double gemm_flops(const GemmF64 &g);
GemmF64 gemm_desc(int M, int N, int K, const double *A, long long lda, long long sA,
                  const double *B, long long ldb, long long sB, double *C, long long ldc,
                  long long sC, int batch);

// Mixed-precision modes, N >= 128: W = X X^T to FP64 accuracy on the
// BF16 tensor cores (Ozaki splitting; X row stride N, batch stride sX; W row
// stride ldw, batch stride sW; tiles on or above the diagonal written).
// oz_prepare leaves c->oz_ws null outside that range.  Defined in oz_gram.cu.
int oz_prepare(sldqmc_ctx *c);
void oz_release(sldqmc_ctx *c);
void oz_gram(sldqmc_ctx *c, const double *X, long long sX, double *W, long long sW, int ldw, int B);
// Left-looking Cholesky-QR on the tensor cores (mixed modes, same N range):
// oz_chol_begin fixes the digit exponents of R's columns from diag(W);
// oz_chol_update subtracts the contributions of the finished rows
// kstart..k0-1 from rows k0..k0+kb of W and of Y = Q^T (k0 - kstart a
// multiple of 32 and > 0); oz_chol_panel factors the
// panel's diagonal block, forms its rows of R and Q^T as products with the
// block's inverse and splits them for the later panels.  W row stride N,
// item stride sW; R, Y row stride N, item stride N*N.
void oz_chol_begin(sldqmc_ctx *c, const double *W, long long sW, int B);
void oz_chol_update(sldqmc_ctx *c, int k0, int kb, int kstart, double *W, long long sW, double *Y, int B);
void oz_chol_panel(sldqmc_ctx *c, int k0, int kb, const double *W, long long sW, double *Y, double *R, int B);
// Trailing update of the finalisation's blocked LU without a right-hand side
// (A row stride lda, item stride sA; panel k0..k0+kb with kb = 32), FP64-
// accurate on the tensor cores.
void oz_lu_update(sldqmc_ctx *c, double *A, long long sA, int lda, int k0, int kb, int B);
// R = R2 R1 of the two passes on the tensor cores (tiles on or above the
// diagonal written); oz_keep_bounds saves the first pass's column bounds of R
// before the second pass replaces them.
void oz_keep_bounds(sldqmc_ctx *c, int B);
// V <- (D^-1 R D_p) P^T V, FP64-accurate on the tensor cores (R upper
// triangular; D, D_p, P from the context; Ts an N x N FP64 scratch per item).
void oz_update_V(sldqmc_ctx *c, const double *R, double *V, double *Ts, int B);
void oz_r2r1(sldqmc_ctx *c, const double *R2, const double *R1, double *R, int B);

// Slice products with the separable exp(-dtau K) (sep.cu): X^T_out =
// U^T D_t0 E D_t0+1 E ... for nb slices, one row per CTA in shared memory.
bool sep_supported(int Lx, int Ly);
void sep_set_limits();
void sep_chain_block(sldqmc_ctx *c, const double *Ut, const int8_t *d_s, int B, double cu, double cd, int t0,
                     int nb, const double *ring, double *Xt_out);

// Event-bracketed timing of launches (sldqmc_profile_*).
struct ProfRec {
    cudaEvent_t a, b;
    int cls;
    double flops;
    const char *site;  // the launch site (a static string)
};
struct Prof {
    bool on = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    int open_cls = -1;
    double open_flops = 0.0;
};
void prof_begin(sldqmc_ctx *c, int cls, double flops, const char *site = nullptr);
void prof_end(sldqmc_ctx *c);
// Launch an FP64 GEMM on the context's stream (counted and, when on, timed).
void gemm_ctx(sldqmc_ctx *c, const GemmF64 &g, bool TA, bool TB);

}  // namespace sldqmc

// The context (opaque in the public header).
struct sldqmc_ctx {
    sldqmc_params p;
    int N, M;
    cudaStream_t st;
    long long launches;
    int *d_flag;  // device error bits
    // constants
    double *d_K, *d_E, *d_Einv;  // N x N
    float *d_Ehi, *d_Elo;        // split-TF32 copies of E (3xTF32 mode)
    void *d_Ebf;                 // BF16 copy of E (BF16 mode)
    double ex_scale[2][2];       // [eta==-1][s<0]: exp(eta*dtau*xi*s)
    double dtauJ, Ktau;          // bare-weight constants
    // stabilisation workspace, cap items each
    int cap;
    long long nn;      // N*N
    double *buf[9];    // Ut, V, X1, X2, W(2*nn), Y, R1, R2, Vg
    double *d_D, *d_Dp, *d_logacc;
    int *d_perm, *d_sgn, *d_piv;
    int *d_tslu;       // row nominations of the tournament-pivoting LU panels (24 * 32 per item)
    void *tc_ws;       // tensor-core operand workspace (split copies)
    void *oz_ws;       // digit planes of the tensor-core Gram and Cholesky-QR (mixed modes, N >= 128)
    // Monte Carlo state
    int8_t *d_s_tmp;   // cap * M * N proposal buffer
    int8_t *d_s_one;   // staging for host calls
    double *d_G[2];    // Gt for the local sweep: cap items per flavour
    double *d_U, *d_V; // pending pairs of the delayed local update: 2 flavours x cap x 32 N each
    int local_rank;    // sites per delayed-update block (1: immediate rank-1 updates)
    int tile_n;        // output tile width of the tensor-core slice products (64 or 128)
    double *d_ld_tmp, *d_ld_tmp2;
    int *d_sg_tmp;
    long long *d_stats; // cap * 4 (accepted, proposed, margin, drift bits)
    // effective model
    int n_class, n_off_total;
    int h_n_off[32];
    int h_offsets[64 * 3];
    double h_J[32];
    double E0;
    int have_model;
    int n_colors;
    int *d_col_start, *d_col_sites;
    long long *d_feat0, *d_feat1;
    double *d_Jdev;
    int *d_offdev, *d_noffdev;
    sldqmc::Prof *prof;
    const uint32_t *step_dev;  // when set (graph capture), kernels read the MC step from here
    uint32_t *d_step;          // this context's device step counter
    sldqmc_ctx *twin;          // second workspace (twice the capacity) + stream for the exact log weight
    cudaEvent_t ev_fork, ev_join;
    int no_twin;               // set on a twin itself, or when the twin could not be created
    int num_sms;               // streaming multiprocessors of the context's device
    int kinetic;               // SLDQMC_KINETIC_*: form in which exp(-dtau K) enters the slice products
};
