// stab.cu -- FP64 kernels of the stabilised determinant: pre-pivoted
// Cholesky-QR re-factorisation of the running U D V product, and the
// blocked LU finalisation det(1 + U D V) = det(U) det(D_b) det(M_mid).
//
// The paper uses the numerically stable B-chain evaluation of DQMC (the
// scheme of Loh et al. it cites in "Basics of DQMC") without spelling it
// out.  On GB300 the stabilisation is FP64 work on a ~1.1 TFLOP/s pipe, so
// it is arranged as GEMM-shaped batched work with small panel kernels:
//
//   X = B_block .. U  (the block's slice products),
//   sort the columns of X diag(D) by norm (pre-pivoting, permutation P),
//   X P = Q R by Cholesky-QR applied twice (Gram matrix, Cholesky, a
//   triangular solve; the second pass restores orthogonality to O(eps)),
//   U <- Q,  D <- |diag R| * D_P,  V <- D^{-1} R D_P P^T V.
//
// Cholesky-QR needs kappa(X)^2 * eps < 1; the block products are applied
// to an orthonormal U and hold the field's scales in D, so
// kappa(X) <= exp(n_wrap * dtau * (8t + 2 xi)), checked by the host.
// Every matrix is stored row-major; the chain works on X^T so that columns
// of X are contiguous rows.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "internal.h"

namespace sldqmc {

// ---------------------------------------------------------------- helpers
__global__ void k_init_udv(double *Ut, double *V, long long nn, int N, double *D, int *sgn,
                           double *logacc, int cap)
{
    const int b = blockIdx.y;
    const long long off = (long long)b * nn;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e / N), j = (int)(e % N);
        double v = (i == j) ? 1.0 : 0.0;
        Ut[off + e] = v;
        V[off + e] = v;
        if (j == 0) D[(long long)b * N + i] = 1.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sgn[b] = 1;
        sgn[cap + b] = 1;
        logacc[b] = 0.0;
    }
}

// Sort the columns of X diag(D) by decreasing norm (bitonic network in
// shared memory).  key_j = sqrt(W_jj) D_j where W = X^T X.  Padding keys
// -1, -2, ... keep the pads in place so the swap-count parity is the
// parity of the real permutation.  perm[k] = column at position k.
__global__ void k_sort_pivot(const double *W, long long sW, int ldw, const double *D, int N,
                             int Npad, int *perm, double *Dp, int *sgn)
{
    extern __shared__ unsigned char smem_raw[];
    double *key = reinterpret_cast<double *>(smem_raw);
    int *idx = reinterpret_cast<int *>(key + Npad);
    __shared__ int par;
    const int b = blockIdx.x;
    const double *Wb = W + (long long)b * sW;
    const double *Db = D + (long long)b * N;
    if (threadIdx.x == 0) par = 0;
    for (int j = threadIdx.x; j < Npad; j += blockDim.x) {
        key[j] = (j < N) ? sqrt(Wb[(long long)j * ldw + j]) * Db[j] : -(1.0 + (double)(j - N));
        idx[j] = j;
    }
    __syncthreads();
    int swaps = 0;
    for (int k = 2; k <= Npad; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < Npad; t += blockDim.x) {
                int u = t ^ j;
                if (u > t) {
                    bool desc = (t & k) == 0;
                    double a = key[t], c = key[u];
                    bool sw = desc ? (a < c) : (a > c);
                    if (sw) {
                        key[t] = c; key[u] = a;
                        int q = idx[t]; idx[t] = idx[u]; idx[u] = q;
                        swaps ^= 1;
                    }
                }
            }
            __syncthreads();
        }
    if (swaps) atomicXor(&par, 1);
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        perm[(long long)b * N + j] = idx[j];
        Dp[(long long)b * N + j] = Db[idx[j]];
    }
    if (threadIdx.x == 0 && par) sgn[b] = -sgn[b];
}

// Wc[a][c] = W[p_a][p_c] for c >= a (W holds its upper triangle) and
// Y[a][:] = Xt[p_a][:]  (the columns of X P as rows).
__global__ void k_gather_pivot(const double *W, long long sW, const double *Xt, double *Wc, double *Y,
                               long long nn, int N, int ldw, const int *perm)
{
    const int b = blockIdx.z;
    const int a = blockIdx.y;
    const int *p = perm + (long long)b * N;
    const int pa = p[a];
    const double *Wb = W + (long long)b * sW;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        Y[(long long)b * nn + (long long)a * N + c] = Xt[(long long)b * nn + (long long)pa * N + c];
        if (c >= a) {
            int pc = p[c];
            int r0 = pa < pc ? pa : pc, c0 = pa < pc ? pc : pa;
            Wc[(long long)b * nn + (long long)a * N + c] = Wb[(long long)r0 * ldw + c0];
        }
    }
}

// One block row of the stacked Cholesky-QR: factor the kb x kb diagonal
// block W_kk = R_kk^T R_kk (in shared memory, every CTA redundantly), then
// solve R_kk^T y = w for each column: W-columns right of the block give
// R's block row, Y-columns give Q^T's block row (in place).
template <int KB, int CPT>
__global__ void __launch_bounds__(128) k_chol_panel(const double *W, long long sW, int ldw, double *Y,
                                                    long long sY, double *R, long long sR, int N,
                                                    int k0, int kb, int *flag)
{
    __shared__ double Rk[KB][KB + 1];
    const int b = blockIdx.y;
    const double *Wb = W + (long long)b * sW;
    for (int e = threadIdx.x; e < KB * KB; e += blockDim.x) {
        int r = e / KB, c = e % KB;
        double v = 0.0;
        if (r < kb && c < kb) {
            if (c >= r) v = Wb[(long long)(k0 + r) * ldw + k0 + c];
        } else if (r == c) {
            v = 1.0;
        }
        Rk[r][c] = v;
    }
    __syncthreads();
    // Factor the KB x KB block (right-looking, all threads of the CTA); the
    // reciprocals of the pivots are kept so that every later division is a
    // multiplication (FP64 division is many times slower than an FMA here).
    __shared__ double rinv[KB];
    for (int j = 0; j < KB; ++j) {
        if (threadIdx.x == 0) {
            double d = Rk[j][j];
            if (!(d > 0.0) || !isfinite(d)) {
                if (j < kb) atomicOr(flag, FLAG_NUMERICAL);
                d = 1.0;
            }
            d = sqrt(d);
            Rk[j][j] = d;
            rinv[j] = 1.0 / d;
        }
        __syncthreads();
        const double ri = rinv[j];
        for (int c = j + 1 + threadIdx.x; c < KB; c += blockDim.x) Rk[j][c] *= ri;
        __syncthreads();
        for (int e = threadIdx.x; e < KB * KB; e += blockDim.x) {
            int r = e / KB, c = e % KB;
            if (r > j && c >= r) Rk[r][c] -= Rk[j][r] * Rk[j][c];
        }
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        double *Rb = R + (long long)b * sR;
        for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
            int r = e / kb, c = e % kb;
            Rb[(long long)(k0 + r) * N + k0 + c] = (c >= r) ? Rk[r][c] : 0.0;
        }
    }
    const int nW = N - (k0 + kb);
    // CPT columns per thread (blockDim.x apart, so each load and store
    // instruction stays coalesced); every shared-memory load of R_kk then feeds
    // CPT independent FMA chains.
    double w[CPT][KB];
    double *dst[CPT];
    int cc[CPT];
    long long ldd[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int col = (blockIdx.x * CPT + q) * blockDim.x + threadIdx.x;
        const double *src = nullptr;
        long long lds = 0;
        cc[q] = -1;
        dst[q] = nullptr;
        ldd[q] = 0;
        if (col < nW) {
            cc[q] = k0 + kb + col;
            src = Wb; lds = ldw;
            dst[q] = R + (long long)b * sR; ldd[q] = N;
        } else if (col < nW + N) {
            cc[q] = col - nW;
            src = Y + (long long)b * sY; lds = N;
            dst[q] = Y + (long long)b * sY; ldd[q] = N;
        }
#pragma unroll
        for (int r = 0; r < KB; ++r) w[q][r] = (cc[q] >= 0 && r < kb) ? src[(long long)(k0 + r) * lds + cc[q]] : 0.0;
    }
    // Column-oriented order: once w[l] is final, its contribution is
    // subtracted from every later w[r] -- up to KB - 1 independent FMAs per
    // step.  Each w[r] receives the same operations in the same order as in
    // the row-oriented form (r's terms l = 0, 1, ..., r - 1, then the scale).
#pragma unroll
    for (int l = 0; l < KB; ++l) {
#pragma unroll
        for (int q = 0; q < CPT; ++q) w[q][l] *= rinv[l];
#pragma unroll
        for (int r = 0; r < KB; ++r) {
            if (r > l) {
                const double rl = Rk[l][r];
#pragma unroll
                for (int q = 0; q < CPT; ++q) w[q][r] -= rl * w[q][l];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q)
        if (cc[q] >= 0)
#pragma unroll
            for (int r = 0; r < KB; ++r)
                if (r < kb) dst[q][(long long)(k0 + r) * ldd[q] + cc[q]] = w[q][r];
}

// D_new[k] = R_kk * D_p[k]  (R from Cholesky has a positive diagonal).
__global__ void k_new_D(const double *R, long long nn, int N, const double *Dp, double *D, int *flag)
{
    const int b = blockIdx.y;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        double v = R[(long long)b * nn + (long long)k * N + k] * Dp[(long long)b * N + k];
        if (!(v > 0.0) || !isfinite(v)) {
            atomicOr(flag, FLAG_NUMERICAL);
            v = 1.0;
        }
        D[(long long)b * N + k] = v;
    }
}

// Vg[a][:] = D_p[a] * V[p_a][:]
__global__ void k_gather_V(const double *V, double *Vg, long long nn, int N, const int *perm,
                           const double *Dp)
{
    const int b = blockIdx.z, a = blockIdx.y;
    const int pa = perm[(long long)b * N + a];
    const double s = Dp[(long long)b * N + a];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
        Vg[(long long)b * nn + (long long)a * N + c] = s * V[(long long)b * nn + (long long)pa * N + c];
}

// M_mid = D_b^{-1} U^T + D_s V, written with row stride ldo; when rhs, the
// right-hand side D_b^{-1} U^T of the Green's function follows in columns
// N..2N-1.  D_b = max(D,1), D_s = min(D,1).
__global__ void k_mmid(const double *Ut, const double *V, const double *D, double *Out, long long nn,
                       int N, int ldo, int rhs)
{
    const int b = blockIdx.z, i = blockIdx.y;
    const double d = D[(long long)b * N + i];
    const double ds = d > 1.0 ? 1.0 : d;
    // 1 / D_b once per row (FP64 division is a long chain on this pipe)
    __shared__ double s_rdb;
    if (threadIdx.x == 0) s_rdb = d > 1.0 ? 1.0 / d : 1.0;
    __syncthreads();
    const double rdb = s_rdb;
    const double *u = Ut + (long long)b * nn + (long long)i * N;
    const double *v = V + (long long)b * nn + (long long)i * N;
    double *o = Out + (long long)b * N * ldo + (long long)i * ldo;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        double uu = u[j] * rdb;
        o[j] = uu + ds * v[j];
        if (rhs) o[N + j] = uu;
    }
}

// Row interchanges of one LU panel, as the rows of its block row receive
// them.  Partial pivoting swaps row j with row p_j >= j for j = 0..kb-1 (rows
// relative to k0).  Composed, the new row j < kb is the original row src_j
// (any row), and a row i >= kb changes only if it is some p_j, when it
// receives an original row below kb.  The panel kernels record this per item
// in the kb + kb ints of piv from position k0: src_j for j < kb, then one
// entry i * 64 + src(i) per changed row i >= kb (ascending i), closed by -1
// when the list ends before N.  Only the columns right of the panel still
// need the interchange (those left of it hold L factors whose trailing
// updates are done; nothing reads them again), and k_lu_trsm_row applies it
// as it loads the block row.
__device__ __forceinline__ bool lu_key_better(unsigned long long k, int i, unsigned long long bk, int bi)
{
    return k > bk || (k == bk && i < bi);
}

// |v| as an integer key: for non-negative doubles the bit pattern orders as
// the value, so the pivot search runs on the integer pipe.  The largest |v|
// wins, the lowest row on ties.
__device__ __forceinline__ unsigned long long lu_key(double v)
{
    return (unsigned long long)__double_as_longlong(fabs(v));
}

__device__ __forceinline__ void lu_warp_argmax(unsigned long long &k, int &i)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_down_sync(0xffffffffu, k, o);
        const int oi = __shfl_down_sync(0xffffffffu, i, o);
        if (lu_key_better(ok, oi, k, i)) { k = ok; i = oi; }
    }
}

// Logarithm, sign and the interchange record of a factored panel (pr[j]: the
// pivot row of step j, src[j]: the original row now at j; changed rows >= kb
// listed by warp 0 in ascending order from org[]).
__device__ void lu_panel_close(int *pv_out, int R, int kb, const int *org, const double *pvv, const int *pr,
                               double *logacc, int *lusgn, int b, int N, int k0)
{
    __shared__ double lg[32];
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane < kb) {
            lg[lane] = log(fabs(pvv[lane]));
            pv_out[lane] = org[lane];
        }
        int e = 0;
        for (int i0 = kb; i0 < R; i0 += 32) {
            const int i = i0 + lane;
            const bool ch = i < R && org[i] != i;
            const unsigned m = __ballot_sync(0xffffffffu, ch);
            if (ch) pv_out[kb + e + __popc(m & ((1u << lane) - 1u))] = i * 64 + org[i];
            e += __popc(m);
        }
        if (lane == 0 && k0 + kb + e < N) pv_out[kb + e] = -1;
        __syncwarp();
        if (lane == 0) {
            double acc = logacc[b];
            int sg = 1;
            for (int j = 0; j < kb; ++j) {
                acc += lg[j];
                if (pr[j] != j) sg = -sg;
                if (pvv[j] < 0.0) sg = -sg;
            }
            logacc[b] = acc;
            lusgn[b] *= sg;
        }
    }
}

// Panel of the right-looking blocked LU with partial pivoting, one CTA of
// 256 threads per matrix, the panel (rows k0..N-1, kb <= 32 columns) in
// shared memory.  Per column j: the pivot (found during the previous
// column's update, integer keys), the swap of rows j and p inside the panel
// by warp 0 with one reciprocal of the pivot, then one pass in which each
// thread scales its rows' multipliers and updates their remaining columns.
// Dynamic shared memory: (N - k0) * 33 doubles + (N - k0) ints.
constexpr int LU_SMEM_MAX_ROWS = 800;
constexpr int LU_THREADS = 256;
__global__ void __launch_bounds__(LU_THREADS) k_lu_panel_smem(double *A, long long sA, int lda, int N, int k0,
                                                              int kb, int *piv, double *logacc, int *lusgn,
                                                              int *flag)
{
    extern __shared__ double P[];  // [R][33], then org[R]
    __shared__ unsigned long long wk[LU_THREADS / 32];
    __shared__ int wi[LU_THREADS / 32];
    __shared__ double pvv[32];
    __shared__ int pr[32];
    __shared__ double s_vinv;
    const int b = blockIdx.x;
    double *Ab = A + (long long)b * sA;
    const int R = N - k0;
    int *org = reinterpret_cast<int *>(P + (size_t)R * 33);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int e = tid; e < R * 32; e += LU_THREADS) {
        const int r = e >> 5, l = e & 31;
        P[r * 33 + l] = l < kb ? Ab[(long long)(k0 + r) * lda + k0 + l] : 0.0;
    }
    for (int i = tid; i < R; i += LU_THREADS) org[i] = i;
    __syncthreads();
    unsigned long long bk = 0;
    int bi = R;
    for (int r = tid; r < R; r += LU_THREADS) {
        const unsigned long long k = lu_key(P[r * 33]);
        if (lu_key_better(k, r, bk, bi)) { bk = k; bi = r; }
    }
    for (int j = 0; j < kb; ++j) {
        lu_warp_argmax(bk, bi);
        if (lane == 0) { wk[wid] = bk; wi[wid] = bi; }
        __syncthreads();
        if (wid == 0) {
            unsigned long long k = lane < LU_THREADS / 32 ? wk[lane] : 0ull;
            int i = lane < LU_THREADS / 32 ? wi[lane] : R;
            lu_warp_argmax(k, i);
            const int p = __shfl_sync(0xffffffffu, i, 0) < R ? __shfl_sync(0xffffffffu, i, 0) : j;
            if (p != j) {
                const double t = P[j * 33 + lane];
                P[j * 33 + lane] = P[p * 33 + lane];
                P[p * 33 + lane] = t;
                if (lane == 0) {
                    const int o = org[j];
                    org[j] = org[p];
                    org[p] = o;
                }
            }
            __syncwarp();
            if (lane == 0) {
                double v = P[j * 33 + j];
                if (v == 0.0 || !isfinite(v)) {
                    atomicOr(flag, FLAG_NUMERICAL);
                    v = 1.0;
                    P[j * 33 + j] = 1.0;
                }
                pvv[j] = v;
                pr[j] = p;
                s_vinv = 1.0 / v;
            }
        }
        __syncthreads();
        const double vinv = s_vinv;
        bk = 0;
        bi = R;
        for (int r = j + 1 + tid; r < R; r += LU_THREADS) {
            double *row = P + r * 33;
            const double m = row[j] * vinv;
            row[j] = m;
#pragma unroll 4
            for (int l = j + 1; l < kb; ++l) row[l] -= m * P[j * 33 + l];
            if (j + 1 < kb) {
                const unsigned long long k = lu_key(row[j + 1]);
                if (lu_key_better(k, r, bk, bi)) { bk = k; bi = r; }
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < R * 32; e += LU_THREADS) {
        const int r = e >> 5, l = e & 31;
        if (l < kb) Ab[(long long)(k0 + r) * lda + k0 + l] = P[r * 33 + l];
    }
    lu_panel_close(piv + (long long)b * N + k0, R, kb, org, pvv, pr, logacc, lusgn, b, N, k0);
}

// ---------------------------------------------------------------------------
// Panels taller than LU_SMEM_MAX_ROWS: tournament pivoting.  The panel's rows
// are cut into up to TSLU_BLOCKS balanced row blocks; each block (one CTA)
// runs partial pivoting on its own rows in shared memory and nominates the
// kb rows it pivoted on; one CTA then runs partial pivoting on the
// nominated rows (at most TSLU_BLOCKS * 32 of them), whose pivot rows, in
// order, become the panel's block row: their factors are the panel's L11
// and U11.  The block row's former rows move into the rows the pivots left,
// giving the same interchange record as one partial-pivoting pass (the
// source of each new row j < kb, then the changed rows below), and every
// other row gets its multipliers from L21 = A21 U11^{-1}.  Any pivot choice
// with bounded growth gives the same determinant and solve; this one keeps
// a panel's serial pivot chain inside shared memory and spreads the row
// work over many CTAs, where a single CTA would stream a tall panel from
// global memory 32 times.
constexpr int TSLU_BLOCKS = 24;   // nominated rows 24 * 32 <= LU_SMEM_MAX_ROWS
constexpr int TSLU_MIN_ROWS = 256;

// Partial pivoting on R rows of kb columns in shared memory (row stride 33),
// org[] permuted with the rows: afterwards rows 0..min(kb, R)-1 hold the
// pivot rows in order with their L multipliers and U entries.
__device__ void lu_gepp_rows(double *P, int *org, int R, int kb, double *pvv, int *pr, int *flag,
                             unsigned long long *wk, int *wi, double *s_vinv)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int steps = kb < R ? kb : R;
    unsigned long long bk = 0;
    int bi = R;
    for (int r = tid; r < R; r += LU_THREADS) {
        const unsigned long long k = lu_key(P[r * 33]);
        if (lu_key_better(k, r, bk, bi)) { bk = k; bi = r; }
    }
    for (int j = 0; j < steps; ++j) {
        lu_warp_argmax(bk, bi);
        if (lane == 0) { wk[wid] = bk; wi[wid] = bi; }
        __syncthreads();
        if (wid == 0) {
            unsigned long long k = lane < LU_THREADS / 32 ? wk[lane] : 0ull;
            int i = lane < LU_THREADS / 32 ? wi[lane] : R;
            lu_warp_argmax(k, i);
            const int p = __shfl_sync(0xffffffffu, i, 0) < R ? __shfl_sync(0xffffffffu, i, 0) : j;
            if (p != j) {
                const double t = P[j * 33 + lane];
                P[j * 33 + lane] = P[p * 33 + lane];
                P[p * 33 + lane] = t;
                if (lane == 0) {
                    const int o = org[j];
                    org[j] = org[p];
                    org[p] = o;
                }
            }
            __syncwarp();
            if (lane == 0) {
                double v = P[j * 33 + j];
                if (v == 0.0 || !isfinite(v)) {
                    atomicOr(flag, FLAG_NUMERICAL);
                    v = 1.0;
                    P[j * 33 + j] = 1.0;
                }
                pvv[j] = v;
                pr[j] = p;
                *s_vinv = 1.0 / v;
            }
        }
        __syncthreads();
        const double vinv = *s_vinv;
        bk = 0;
        bi = R;
        for (int r = j + 1 + tid; r < R; r += LU_THREADS) {
            double *row = P + r * 33;
            const double m = row[j] * vinv;
            row[j] = m;
#pragma unroll 4
            for (int l = j + 1; l < kb; ++l) row[l] -= m * P[j * 33 + l];
            if (j + 1 < kb) {
                const unsigned long long k = lu_key(row[j + 1]);
                if (lu_key_better(k, r, bk, bi)) { bk = k; bi = r; }
            }
        }
    }
    __syncthreads();
}

// Tournament stage 1: row block g of the panel of item b nominates its pivot rows
// (panel-relative row numbers) into cand[(b * nblk + g) * 32 + j].
__global__ void __launch_bounds__(LU_THREADS) k_lu_tslu_local(const double *A, long long sA, int lda, int N, int k0,
                                                              int kb, int nblk, int *cand, int *flag)
{
    extern __shared__ double P[];
    __shared__ unsigned long long wk[LU_THREADS / 32];
    __shared__ int wi[LU_THREADS / 32];
    __shared__ double pvv[32], s_vinv;
    __shared__ int pr[32];
    const int b = blockIdx.y, g = blockIdx.x;
    const int R = N - k0;
    const int r0 = (int)((long long)g * R / nblk), r1 = (int)((long long)(g + 1) * R / nblk), nr = r1 - r0;
    int *org = reinterpret_cast<int *>(P + (size_t)nr * 33);
    const double *Ab = A + (long long)b * sA + (long long)(k0 + r0) * lda + k0;
    for (int e = threadIdx.x; e < nr * 32; e += LU_THREADS) {
        const int r = e >> 5, l = e & 31;
        P[r * 33 + l] = l < kb ? Ab[(long long)r * lda + l] : 0.0;
    }
    for (int r = threadIdx.x; r < nr; r += LU_THREADS) org[r] = r0 + r;
    __syncthreads();
    lu_gepp_rows(P, org, nr, kb, pvv, pr, flag, wk, wi, &s_vinv);
    if (threadIdx.x < kb) cand[((long long)b * nblk + g) * 32 + threadIdx.x] = threadIdx.x < nr ? org[threadIdx.x] : -1;
}

// Tournament stage 2: partial pivoting on the nominated rows; the pivot rows become
// the block row (factored), the block row's former rows move into the rows
// the pivots left (original values), and the interchange record, the log
// of the pivots and the sign are written as by the one-pass panel kernels.
__global__ void __launch_bounds__(LU_THREADS) k_lu_tslu_final(double *A, long long sA, int lda, int N, int k0,
                                                              int kb, int nblk, const int *cand, int *piv,
                                                              double *logacc, int *lusgn, int *flag)
{
    extern __shared__ double P[];
    __shared__ double top[32 * 33];
    __shared__ unsigned long long wk[LU_THREADS / 32];
    __shared__ int wi[LU_THREADS / 32];
    __shared__ double pvv[32], s_vinv;
    __shared__ int pr[32], dst_q[32], src_t[32], s_nq;
    const int b = blockIdx.x;
    double *Ab = A + (long long)b * sA + (long long)k0 * lda + k0;
    const int *cb = cand + (long long)b * nblk * 32;
    // nominated rows, in block order (blocks with fewer than kb rows leave -1)
    int nc = 0;
    for (int g = 0; g < nblk; ++g)
        for (int j = 0; j < kb; ++j) nc += cb[g * 32 + j] >= 0;
    int *org = reinterpret_cast<int *>(P + (size_t)nc * 33);
    if (threadIdx.x == 0) {
        int c = 0;
        for (int g = 0; g < nblk; ++g)
            for (int j = 0; j < kb; ++j)
                if (cb[g * 32 + j] >= 0) org[c++] = cb[g * 32 + j];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nc * 32; e += LU_THREADS) {
        const int r = e >> 5, l = e & 31;
        P[r * 33 + l] = l < kb ? Ab[(long long)org[r] * lda + l] : 0.0;
    }
    for (int e = threadIdx.x; e < kb * 32; e += LU_THREADS) {
        const int r = e >> 5, l = e & 31;
        top[r * 33 + l] = l < kb ? Ab[(long long)r * lda + l] : 0.0;
    }
    __syncthreads();
    lu_gepp_rows(P, org, nc, kb, pvv, pr, flag, wk, wi, &s_vinv);
    if (threadIdx.x == 0) {
        // pivots p_j = org[j]; block-row rows not chosen move, in ascending
        // order, into the chosen rows below the block row, in ascending order
        unsigned chosen_top = 0u;
        int nq = 0;
        for (int j = 0; j < kb; ++j) {
            const int p = org[j];
            if (p < kb) chosen_top |= 1u << p;
            else dst_q[nq++] = p;
        }
        for (int x = 1; x < nq; ++x)  // insertion sort of at most 32 rows
            for (int y = x; y > 0 && dst_q[y - 1] > dst_q[y]; --y) {
                const int t = dst_q[y];
                dst_q[y] = dst_q[y - 1];
                dst_q[y - 1] = t;
            }
        int nd = 0;
        for (int t = 0; t < kb; ++t)
            if (!(chosen_top & (1u << t))) src_t[nd++] = t;
        s_nq = nq;
        int *out = piv + (long long)b * N + k0;
        for (int j = 0; j < kb; ++j) out[j] = org[j];
        for (int m = 0; m < nq; ++m) out[kb + m] = dst_q[m] * 64 + src_t[m];
        if (k0 + kb + nq < N) out[kb + nq] = -1;
        // parity of the permutation: position j < kb receives row p_j, position
        // dst_q[m] receives row src_t[m]; count the cycles over the moved positions
        int pos[64], img[64], n = 0;
        for (int j = 0; j < kb; ++j) { pos[n] = j; img[n] = org[j]; ++n; }
        for (int m = 0; m < nq; ++m) { pos[n] = dst_q[m]; img[n] = src_t[m]; ++n; }
        unsigned long long seen = 0ull;
        int cycles = 0;
        for (int s0 = 0; s0 < n; ++s0) {
            if (seen & (1ull << s0)) continue;
            ++cycles;
            int cur = s0;
            while (!(seen & (1ull << cur))) {
                seen |= 1ull << cur;
                int nxt = -1;
                for (int u = 0; u < n; ++u)
                    if (pos[u] == img[cur]) { nxt = u; break; }
                if (nxt < 0) break;
                cur = nxt;
            }
        }
        double acc = logacc[b];
        int sg = ((n - cycles) & 1) ? -1 : 1;
        for (int j = 0; j < kb; ++j) {
            acc += log(fabs(pvv[j]));
            if (pvv[j] < 0.0) sg = -sg;
        }
        logacc[b] = acc;
        lusgn[b] *= sg;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kb * 32; e += LU_THREADS) {
        const int r = e >> 5, l = e & 31;
        if (l < kb) Ab[(long long)r * lda + l] = P[r * 33 + l];
    }
    const int nq = s_nq;
    for (int e = threadIdx.x; e < nq * 32; e += LU_THREADS) {
        const int m = e >> 5, l = e & 31;
        if (l < kb) Ab[(long long)dst_q[m] * lda + l] = top[src_t[m] * 33 + l];
    }
}

// Tournament stage 3: multipliers of the rows below the block row, L21 = A21 U11^{-1},
// one thread per row.
__global__ void __launch_bounds__(128) k_lu_tslu_l21(double *A, long long sA, int lda, int N, int k0, int kb)
{
    __shared__ double U[32][33];
    __shared__ double uinv[32];
    const int b = blockIdx.y;
    double *Ab = A + (long long)b * sA + (long long)k0 * lda + k0;
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int r = e >> 5, c = e & 31;
        U[r][c] = (r < kb && c < kb && c >= r) ? Ab[(long long)r * lda + c] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < 32) uinv[threadIdx.x] = threadIdx.x < kb ? 1.0 / U[threadIdx.x][threadIdx.x] : 0.0;
    __syncthreads();
    const int R = N - k0;
    const int i = kb + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R) return;
    double *row = Ab + (long long)i * lda;
    double x[32];
#pragma unroll
    for (int l = 0; l < 32; ++l) x[l] = l < kb ? row[l] : 0.0;
#pragma unroll
    for (int l = 0; l < 32; ++l) {
        double acc = x[l];
#pragma unroll
        for (int m = 0; m < l; ++m) acc -= x[m] * U[m][l];
        x[l] = acc * uinv[l];
    }
#pragma unroll
    for (int l = 0; l < 32; ++l)
        if (l < kb) row[l] = x[l];
}

// U12 = L11^{-1} A12 for the block row k0..k0+kb (L11 unit lower), with the
// panel's row interchanges applied to these columns on the way (the record
// in piv, see above): each thread owns one column, reads the kb source rows
// and the sources of the changed rows below the block before it writes.
template <int KB>
__global__ void __launch_bounds__(128) k_lu_trsm_row(double *A, long long sA, int lda, int N, int ncols, int k0,
                                                     int kb, const int *piv)
{
    __shared__ double Lk[KB][KB + 1];
    __shared__ int src[KB], edst[KB], esrc[KB];
    __shared__ int s_E;
    const int b = blockIdx.y;
    double *Ab = A + (long long)b * sA;
    const int *rec = piv + (long long)b * N + k0;
    for (int e = threadIdx.x; e < KB * KB; e += blockDim.x) {
        int r = e / KB, c = e % KB;
        Lk[r][c] = (r < kb && c < r) ? Ab[(long long)(k0 + r) * lda + k0 + c] : 0.0;
    }
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        src[lane] = lane < kb ? rec[lane] : 0;
        const int v = (lane < KB && k0 + kb + lane < N) ? rec[kb + lane] : -1;
        const unsigned m = __ballot_sync(0xffffffffu, v >= 0);
        const int E = ~m ? __ffs(~m) - 1 : 32;
        if (lane < E) {
            edst[lane] = v >> 6;
            esrc[lane] = v & 63;
        }
        if (lane == 0) s_E = E;
    }
    __syncthreads();
    const int c = k0 + kb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const int E = s_E;
    double *col = Ab + (long long)k0 * lda + c;
    double w[KB], x[KB];
#pragma unroll
    for (int r = 0; r < KB; ++r) w[r] = (r < kb) ? col[(long long)src[r] * lda] : 0.0;
#pragma unroll
    for (int e = 0; e < KB; ++e)
        if (e < E) x[e] = col[(long long)esrc[e] * lda];
#pragma unroll
    for (int r = 0; r < KB; ++r) {
        double acc = w[r];
#pragma unroll
        for (int l = 0; l < r; ++l) acc -= Lk[r][l] * w[l];
        w[r] = acc;
    }
#pragma unroll
    for (int e = 0; e < KB; ++e)
        if (e < E) col[(long long)edst[e] * lda] = x[e];
#pragma unroll
    for (int r = 0; r < KB; ++r)
        if (r < kb) col[(long long)r * lda] = w[r];
}

// X_k = U_kk^{-1} Y_k for the block row k0..k0+kb of the right-hand side
// held in columns N..2N-1 (back substitution of the Green's function).
template <int KB>
__global__ void __launch_bounds__(128) k_trsm_upper_rhs(double *A, long long sA, int lda, int N, int k0, int kb)
{
    __shared__ double Uk[KB][KB + 1];
    __shared__ double uinv[KB];
    const int b = blockIdx.y;
    double *Ab = A + (long long)b * sA;
    for (int e = threadIdx.x; e < KB * KB; e += blockDim.x) {
        int r = e / KB, c = e % KB;
        double v = 0.0;
        if (r < kb && c < kb && c >= r) v = Ab[(long long)(k0 + r) * lda + k0 + c];
        else if (r == c) v = 1.0;
        Uk[r][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < KB) uinv[threadIdx.x] = 1.0 / Uk[threadIdx.x][threadIdx.x];
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    double w[KB];
#pragma unroll
    for (int r = 0; r < KB; ++r) w[r] = (r < kb) ? Ab[(long long)(k0 + r) * lda + N + c] : 0.0;
#pragma unroll
    for (int r = KB - 1; r >= 0; --r) {
        double acc = w[r];
#pragma unroll
        for (int l = r + 1; l < KB; ++l) acc -= Uk[r][l] * w[l];
        w[r] = acc * uinv[r];
    }
#pragma unroll
    for (int r = 0; r < KB; ++r)
        if (r < kb) Ab[(long long)(k0 + r) * lda + N + c] = w[r];
}

// log|det(1 + U D V)| = sum log D_b + log|det M_mid|, sign = det(U) sign * LU sign.
__global__ void k_finalize(const double *D, int N, const double *logacc, const int *sgn, int cap,
                           double *ld_out, int *sign_out, double scale, int accumulate)
{
    const int b = blockIdx.x;
    __shared__ double part[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double d = D[(long long)b * N + i];
        if (d > 1.0) s += log(d);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        double ld = t + logacc[b];
        int sg = sgn[b] * sgn[cap + b];
        if (accumulate) {
            ld_out[b] += scale * ld;
        } else {
            ld_out[b] = scale * ld;
            if (sign_out) sign_out[b] = sg;
        }
    }
}

__global__ void k_copy_rhs(const double *A, long long sA, int lda, int N, double *G)
{
    const int b = blockIdx.z, i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x)
        G[(long long)b * N * N + (long long)i * N + j] = A[(long long)b * sA + (long long)i * lda + N + j];
}

// ------------------------------------------------------------ launchers
static inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

void stab_set_limits(int Npad)
{
    // Function attributes belong to the current device's context, so the
    // limits reached so far are kept per device.  They only grow, so that a
    // smaller context never lowers a larger one's limit.
    constexpr int MAX_DEV = 64;
    static std::mutex mu;
    static size_t sort_max[MAX_DEV];
    static bool lu_set[MAX_DEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) {
        cudaGetLastError();
        dev = -1;
    }
    std::lock_guard<std::mutex> lk(mu);
    // always raised from its default: the sort kernel also has static shared
    // memory, so a dynamic size of exactly 48 KB (Npad = 4096) is already too much
    const size_t sh = (size_t)Npad * (sizeof(double) + sizeof(int));
    if (dev < 0 || sh > sort_max[dev]) {
        cudaFuncSetAttribute(k_sort_pivot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (dev >= 0) sort_max[dev] = sh;
    }
    if (dev < 0 || !lu_set[dev]) {
        const int lu_sh = (int)((sizeof(double) * 33 + sizeof(int)) * LU_SMEM_MAX_ROWS);
        cudaFuncSetAttribute(k_lu_panel_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, lu_sh);
        cudaFuncSetAttribute(k_lu_tslu_local, cudaFuncAttributeMaxDynamicSharedMemorySize, lu_sh);
        cudaFuncSetAttribute(k_lu_tslu_final, cudaFuncAttributeMaxDynamicSharedMemorySize, lu_sh);
        if (dev >= 0) lu_set[dev] = true;
    }
}

void launch_init_udv(sldqmc_ctx *c, double *Ut, double *V, int B)
{
    dim3 grid(cdiv(c->nn, 256) < 64 ? cdiv(c->nn, 256) : 64, B);
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_init_udv");
    k_init_udv<<<grid, 256, 0, c->st>>>(Ut, V, c->nn, c->N, c->d_D, c->d_sgn, c->d_logacc, c->cap);
    prof_end(c);
    c->launches++;
}

constexpr int CHOL_CPT = 2;      // columns per thread of the panel solves
constexpr int CHOL_BLOCK = 256;  // rows per block of the left-looking tensor-core Cholesky-QR
constexpr int CHOL_THREADS = 128; // threads per CTA of the panel kernel

static void chol_pass(sldqmc_ctx *c, double *W, long long sW, double *Y, double *R, int B)
{
    const int N = c->N;
    const long long nn = c->nn;
    cudaMemsetAsync(R, 0, sizeof(double) * nn * B, c->st);
    // Tensor-core path (mixed modes): left-looking, the panel's rows of W and
    // Y are brought up to date just before the panel, the panel's rows of R
    // and Q^T are its rows of W and Y multiplied by the inverse of the
    // diagonal block's factor (all FP64-accurate digit splitting), and that
    // product also splits the finished rows for the later panels.  Otherwise
    // right-looking with FP64 triangular solves and trailing updates.
    const bool oz = c->oz_ws != nullptr;
    if (oz) {
        // blocks of CHOL_BLOCK rows: one update of the block's rows with every
        // earlier row (CHOL_BLOCK output columns: CHOL_BLOCK / 32 times the tiles
        // of a panel's update, that fraction of the long-K launches), then per
        // 32-row panel an update with the block's own finished rows (K < CHOL_BLOCK)
        // and the panel itself
        oz_chol_begin(c, W, sW, B);
        for (int K0 = 0; K0 < N; K0 += CHOL_BLOCK) {
            const int KB = N - K0 < CHOL_BLOCK ? N - K0 : CHOL_BLOCK;
            if (K0 > 0) oz_chol_update(c, K0, KB, 0, W, sW, Y, B);
            for (int k0 = K0; k0 < K0 + KB; k0 += 32) {
                const int kb = N - k0 < 32 ? N - k0 : 32;
                if (k0 > K0) oz_chol_update(c, k0, kb, K0, W, sW, Y, B);
                oz_chol_panel(c, k0, kb, W, sW, Y, R, B);
            }
        }
        return;
    }
    for (int k0 = 0; k0 < N; k0 += 32) {
        int kb = N - k0 < 32 ? N - k0 : 32;
        int nW = N - (k0 + kb);
        {
            dim3 grid(cdiv(nW + N, CHOL_THREADS * CHOL_CPT), B);
            // algorithmic flops: factor of the kb x kb block, triangular solves of nW + N columns
            prof_begin(c, SLDQMC_KC_PANEL_F64, (double)B * ((double)kb * kb * kb / 3.0 + (double)(nW + N) * kb * kb), "chol_panel_f64");
            k_chol_panel<32, CHOL_CPT><<<grid, CHOL_THREADS, 0, c->st>>>(W, sW, N, Y, nn, R, nn, N, k0, kb, c->d_flag);
            prof_end(c);
            c->launches++;
        }
        if (nW == 0) continue;
        // W[k0+kb:, k0+kb:] -= R_blk^T R_blk   (upper triangle only)
        GemmF64 g = gemm_desc(nW, nW, kb, R + (long long)k0 * N + k0 + kb, N, nn,
                              R + (long long)k0 * N + k0 + kb, N, nn,
                              W + (long long)(k0 + kb) * N + k0 + kb, N, sW, B);
        g.alpha = -1.0; g.beta = 1.0; g.c_upper = 1;
        gemm_ctx(c, g, true, false);
        // Y[k0+kb:, :] -= R_blk^T Qt_blk
        GemmF64 h = gemm_desc(nW, N, kb, R + (long long)k0 * N + k0 + kb, N, nn,
                              Y + (long long)k0 * N, N, nn, Y + (long long)(k0 + kb) * N, N, nn, B);
        h.alpha = -1.0; h.beta = 1.0;
        gemm_ctx(c, h, true, false);
    }
}

// Re-factorise X (given as Xt = X^T) against the running D and V.
// On return: the new U^T is in *Y (caller swaps buffers), D and V updated.
// passes = 1: one Cholesky-QR pass, Q orthogonal to O(kappa(X)^2 eps).  The
// U D V representation stays exact whatever the orthogonality of U; only the
// final U must be orthogonal to working precision (the finalisation uses
// U^T as U^{-1}), so the last block of a chain takes passes = 2.
void stabilize(sldqmc_ctx *c, double *Xt, double *Wc, double *Y, int B, int passes)
{
    const int N = c->N;
    const long long nn = c->nn;
    double *W = c->buf[4];
    double *R1 = c->buf[6], *R2 = c->buf[7], *Vg = c->buf[8], *V = c->buf[1];
    // W = Xt Xt^T (upper triangle): FP64, or FP64-accurate on the tensor cores
    if (c->oz_ws) {
        oz_gram(c, Xt, nn, W, 2 * nn, N, B);
    } else {
        GemmF64 g = gemm_desc(N, N, N, Xt, N, nn, Xt, N, nn, W, N, 2 * nn, B);
        g.c_upper = 1;
        gemm_ctx(c, g, false, true);
    }
    int Npad = 1;
    while (Npad < N) Npad <<= 1;
    size_t sh = (size_t)Npad * (sizeof(double) + sizeof(int));
    prof_begin(c, SLDQMC_KC_PANEL_F64, 0.0, "sort_pivot");
    k_sort_pivot<<<B, 1024, sh, c->st>>>(W, 2 * nn, N, c->d_D, N, Npad, c->d_perm, c->d_Dp, c->d_sgn);
    prof_end(c);
    dim3 gg(cdiv(N, 256), N, B);
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_gather_pivot");
    k_gather_pivot<<<gg, 256, 0, c->st>>>(W, 2 * nn, Xt, Wc, Y, nn, N, N, c->d_perm);
    prof_end(c);
    c->launches += 2;
    chol_pass(c, Wc, nn, Y, R1, B);
    const double *R = R1;
    if (passes == 2) {
        // second pass: W = Q1^T Q1 (as Y Y^T), upper triangle; Q = Q1 R2^{-1}, R = R2 R1
        if (c->oz_ws) {
            oz_keep_bounds(c, B);
            oz_gram(c, Y, nn, W, 2 * nn, N, B);
        } else {
            GemmF64 g2 = gemm_desc(N, N, N, Y, N, nn, Y, N, nn, W, N, 2 * nn, B);
            g2.c_upper = 1;
            gemm_ctx(c, g2, false, true);
        }
        chol_pass(c, W, 2 * nn, Y, R2, B);
        if (c->oz_ws) {
            oz_r2r1(c, R2, R1, Xt, B);
        } else {
            GemmF64 g3 = gemm_desc(N, N, N, R2, N, nn, R1, N, nn, Xt, N, nn, B);
            g3.a_upper = 1;
            g3.b_upper = 1;
            gemm_ctx(c, g3, false, false);
        }
        R = Xt;
    }
    dim3 gd(cdiv(N, 256), B);
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_new_D");
    k_new_D<<<gd, 256, 0, c->st>>>(R, nn, N, c->d_Dp, c->d_D, c->d_flag);
    prof_end(c);
    c->launches++;
    if (c->oz_ws) {
        // mixed-precision modes: V = (D^{-1} R D_p) P^T V, FP64-accurate on the tensor cores
        oz_update_V(c, R, V, Vg, B);
        return;
    }
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_gather_V");
    k_gather_V<<<gg, 256, 0, c->st>>>(V, Vg, nn, N, c->d_perm, c->d_Dp);
    prof_end(c);
    // V = D^{-1} R Vg
    GemmF64 g4 = gemm_desc(N, N, N, R, N, nn, Vg, N, nn, V, N, nn, B);
    g4.a_upper = 1;
    g4.ms = c->d_D; g4.sMs = N; g4.ms_recip = 1;
    gemm_ctx(c, g4, false, false);
    c->launches++;
}

// Final determinant (and optionally G) from the running U^T, D, V.
void finalize(sldqmc_ctx *c, const double *Ut, int B, double *d_ld, int *d_sign, double *d_G,
              double scale, int accumulate)
{
    const int N = c->N;
    const long long nn = c->nn;
    const int rhs = d_G != nullptr;
    const int lda = rhs ? 2 * N : N;
    const int ncols = lda;
    double *A = c->buf[4];  // 2*nn per item
    dim3 gm(cdiv(N, 256), N, B);
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_mmid");
    k_mmid<<<gm, 256, 0, c->st>>>(Ut, c->buf[1], c->d_D, A, nn, N, lda, rhs);
    prof_end(c);
    c->launches++;
    // note: k_mmid writes item b at offset b*N*lda; with lda = N the items
    // are packed at stride nn, with lda = 2N at stride 2nn.
    const long long sItem = (long long)N * lda;
    for (int k0 = 0; k0 < N; k0 += 32) {
        int kb = N - k0 < 32 ? N - k0 : 32;
        prof_begin(c, SLDQMC_KC_PANEL_F64, (double)B * (N - k0) * kb * kb, N - k0 <= LU_SMEM_MAX_ROWS ? "lu_panel_smem" : "lu_panel_tournament");
        if (N - k0 <= LU_SMEM_MAX_ROWS) {
            k_lu_panel_smem<<<B, LU_THREADS, (sizeof(double) * 33 + sizeof(int)) * (N - k0), c->st>>>(
                A, sItem, lda, N, k0, kb, c->d_piv, c->d_logacc, c->d_sgn + c->cap, c->d_flag);
            c->launches++;
        } else {
            // tournament pivoting: nominations by row blocks, the final choice, the multipliers
            const int R = N - k0;
            int nblk = R / TSLU_MIN_ROWS;
            if (nblk > TSLU_BLOCKS) nblk = TSLU_BLOCKS;
            const int rmax = (R + nblk - 1) / nblk;
            int *cand = c->d_tslu;  // TSLU_BLOCKS * 32 nominations per item
            k_lu_tslu_local<<<dim3(nblk, B), LU_THREADS, (sizeof(double) * 33 + sizeof(int)) * rmax, c->st>>>(
                A, sItem, lda, N, k0, kb, nblk, cand, c->d_flag);
            k_lu_tslu_final<<<B, LU_THREADS, (sizeof(double) * 33 + sizeof(int)) * nblk * 32, c->st>>>(
                A, sItem, lda, N, k0, kb, nblk, cand, c->d_piv, c->d_logacc, c->d_sgn + c->cap, c->d_flag);
            k_lu_tslu_l21<<<dim3(cdiv(R - kb, 128), B), 128, 0, c->st>>>(A, sItem, lda, N, k0, kb);
            c->launches += 3;
        }
        prof_end(c);
        int rest = ncols - (k0 + kb);
        if (rest > 0) {
            dim3 gt(cdiv(rest, 128), B);
            prof_begin(c, SLDQMC_KC_PANEL_F64, (double)B * rest * kb * kb, "lu_trsm_row");
            k_lu_trsm_row<32><<<gt, 128, 0, c->st>>>(A, sItem, lda, N, ncols, k0, kb, c->d_piv);
            prof_end(c);
            c->launches++;
            int m2 = N - (k0 + kb);
            if (m2 > 0 && c->oz_ws && !rhs) {
                oz_lu_update(c, A, sItem, lda, k0, kb, B);
            } else if (m2 > 0) {
                GemmF64 g = gemm_desc(m2, rest, kb, A + (long long)(k0 + kb) * lda + k0, lda, sItem,
                                      A + (long long)k0 * lda + k0 + kb, lda, sItem,
                                      A + (long long)(k0 + kb) * lda + k0 + kb, lda, sItem, B);
                g.alpha = -1.0; g.beta = 1.0;
                gemm_ctx(c, g, false, false);
            }
        }
    }
    if (rhs) {
        int nblk = (N + 31) / 32;
        for (int kbi = nblk - 1; kbi >= 0; --kbi) {
            int k0 = kbi * 32;
            int kb = N - k0 < 32 ? N - k0 : 32;
            dim3 gt(cdiv(N, 128), B);
            prof_begin(c, SLDQMC_KC_PANEL_F64, (double)B * N * kb * kb, "trsm_upper_rhs");
            k_trsm_upper_rhs<32><<<gt, 128, 0, c->st>>>(A, sItem, lda, N, k0, kb);
            prof_end(c);
            c->launches++;
            if (k0 > 0) {
                GemmF64 g = gemm_desc(k0, N, kb, A + k0, lda, sItem, A + (long long)k0 * lda + N, lda,
                                      sItem, A + N, lda, sItem, B);
                g.alpha = -1.0; g.beta = 1.0;
                gemm_ctx(c, g, false, false);
            }
        }
        dim3 gc(cdiv(N, 256), N, B);
        prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_copy_rhs");
        k_copy_rhs<<<gc, 256, 0, c->st>>>(A, sItem, lda, N, d_G);
        prof_end(c);
        c->launches++;
    }
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_finalize");
    k_finalize<<<B, 256, 0, c->st>>>(c->d_D, N, c->d_logacc, c->d_sgn, c->cap, d_ld, d_sign, scale,
                                     accumulate);
    prof_end(c);
    c->launches++;
}

}  // namespace sldqmc
