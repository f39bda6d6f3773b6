// oz_gram.cu -- FP64-accurate products on the BF16 tensor cores (Ozaki's
// error-free splitting) for the stabilisation and the determinant of the
// mixed-precision modes: Gram matrices, the left-looking Cholesky-QR updates
// and panel products (with the inverse of each 32 x 32 diagonal factor,
// formed here in FP64), R = R2 R1, the V update and the trailing updates of
// the determinant's LU.  The Gram matrix shows the scheme:
//
// W = X X^T for the rows x_i of X (N x N per batch item).  Each row is
// scaled by a power of two, 2^-E_i with |x_ik| < 2^E_i, and written as eight
// balanced base-2^7 digits,
//   x_ik 2^-E_i = sum_{p=1..8} a_p,ik 2^-7p   (|a_1| <= 128, |a_p| <= 64, p > 1),
// exact up to the rounding of x_ik 2^-E_i to a multiple of 2^-56.  Then
//   W_ij 2^-(E_i+E_j) = sum_{p,q} 2^-7(p+q) sum_k a_p,ik a_q,jk,
// of which the 36 products with p + q <= 9 are kept: each dropped term is
// below 2^-56 of the row maxima, the same order as FP64's own rounding of the
// sum.  The digit planes are BF16 integers; the products of one group
// g = p + q share one FP32 tensor-memory accumulator, and every partial sum
// of a group is an integer of magnitude < K (2 * 8192 + 6 * 4096) < 2^24 for
// K <= 384, so the tensor-core accumulation is exact.  Longer contractions
// run in chunks of at most 384: the epilogue converts each chunk's eight
// group sums to integers, combines them in two 64-bit integers, forms the
// chunk's FP64 value with one rounding and adds the chunks in FP64.
//
// One persistent CTA per SM walks the 128 x 32 output tiles of every item
// (for a Gram matrix only those on or above the diagonal; a launch may carry
// two parts with their own A rows and outputs): warp 0 streams the 8 + 8
// digit-plane tiles of a 32-wide K-block by TMA (64-byte swizzle), warp 1
// issues the 36 digit products per 16-wide K-step as eight MMAs (A's plane p
// against B's planes 0..7-p at once), and eight epilogue warps drain one
// of two tensor-memory buffers (8 groups x 32 columns each) while the next
// tile accumulates into the other.  Every mbarrier wait is bounded; a wait
// that runs out raises the context's timeout flag and the CTA frees its
// tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_common.cuh"

namespace sldqmc {

namespace {

using namespace tcx;

constexpr int OZ_S = 8;           // digit planes
constexpr int OZ_BETA = 7;        // bits per digit
constexpr int OZ_G = 8;           // groups p + q = 2..9
constexpr int OZ_KCHUNK = 12;     // K-blocks (of 32) per exactly accumulated chunk: K <= 384
constexpr int OBM = 128, OBN = 32;
constexpr int OKE = 32;           // BF16 elements per K-block (64-byte rows)
constexpr int OSTAGES = 2;
constexpr int OTILE_A = OBM * 64;  // one digit plane of A per stage
constexpr int OTILE_B = OBN * 64;
constexpr int OSTAGE = OZ_S * (OTILE_A + OTILE_B);
constexpr int OEPI = 8;            // epilogue warps, two per TMEM lane quarter
constexpr int OTHREADS = 64 + 32 * OEPI;
constexpr int OTMEM = 2 * OZ_G * OBN;  // two buffers of eight 32-column accumulators

constexpr size_t oz_smem_bytes() { return (size_t)OSTAGES * OSTAGE + 1024 + 256; }

// Shared-memory descriptor of a K-major BF16 operand with 64-byte rows and the
// 64-byte swizzle (8-row atoms of 512 bytes).
__device__ __forceinline__ uint64_t smem_desc64(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(512u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)4u << 61;
    return d;
}

// kind::f16 with BF16 operands, FP32 accumulator, K-major A and B, M = 128,
// N = n (a multiple of 32 up to 256).
__device__ __forceinline__ constexpr uint32_t oz_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(OBM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Balanced base-2^7 digits of v = round(|x| 2^(56 - E)) < 2^56 for a double x
// with |x| < 2^E (E the frexp exponent of its row's maximum, ef_max its
// biased exponent, 0 for a row of zeros or subnormals): x 2^-E = sum_p
// dg[p] 2^-7(p+1), p = 0..7.
__device__ __forceinline__ void oz_digits(double x, int E, int ef_max, int dg[OZ_S])
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((u >> 52) & 0x7FF);
    long long v = 0;
    if (ef > 0 && ef_max > 0) {
        // x = m 2^(ef - 1075)
        const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = ef - 1075 + 56 - E;
        if (sh >= 0) v = (long long)(m << sh);  // sh <= 3 since |x| < 2^E
        else if (sh > -60) v = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
    }
#pragma unroll
    for (int p = OZ_S - 1; p >= 1; --p) {
        int d = (int)(v & ((1 << OZ_BETA) - 1));
        v >>= OZ_BETA;
        if (d >= (1 << (OZ_BETA - 1))) {
            d -= 1 << OZ_BETA;
            v += 1;
        }
        dg[p] = d;
    }
    dg[0] = (int)v;  // 0..128
    if (u >> 63)
#pragma unroll
        for (int p = 0; p < OZ_S; ++p) dg[p] = -dg[p];
}

// Digits of the rows of X (rows x cols, row stride ld, item stride sX): row i
// becomes plane row i (prow plane rows per item, leading dimension ldp) with
// K positions 0..cols-1 and exponent E[b * prow + i]; the planes' columns
// beyond cols are left as they are (zero pads of the buffer).  One warp per
// row, eight rows per CTA: the row's maximum by warp shuffles, then each lane
// converts pairs of adjacent entries and stores each plane's pair as one
// BF16x2.
__global__ void __launch_bounds__(256) k_oz_slice(const double *X, long long sX, int rows, int cols, int ld, int prow,
                                                  int ldp, long long plane_stride, __nv_bfloat16 *planes, int *E)
{
    const int b = blockIdx.y, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= rows) return;  // whole warps
    const int N = cols;
    const double *x = X + (long long)b * sX + (long long)i * ld;
    // the largest |x_ik| (non-negative doubles order like their bit patterns)
    unsigned long long mx = 0;
    for (int k = lane; k < N; k += 32) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(x[k]) & 0x7FFFFFFFFFFFFFFFull;
        mx = u > mx ? u : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
    }
    const int ef_max = (int)(mx >> 52);
    const int Ei = ef_max > 0 ? ef_max - 1022 : 0;
    if (lane == 0) E[(long long)b * prow + i] = Ei;
    const long long row = ((long long)b * prow + i) * ldp;
    for (int k = 2 * lane; k < N; k += 64) {
        int d0[OZ_S], d1[OZ_S];
        oz_digits(x[k], Ei, ef_max, d0);
        oz_digits(k + 1 < N ? x[k + 1] : 0.0, Ei, ef_max, d1);
#pragma unroll
        for (int p = 0; p < OZ_S; ++p)
            *reinterpret_cast<__nv_bfloat162 *>(planes + (long long)p * plane_stride + row + k) =
                __floats2bfloat162_rn((float)d0[p], (float)d1[p]);
    }
}

// Digits of krows rows of a row-major matrix (row stride ld), in blocks of 32
// rows (blockIdx.z), stored from K-block koff/32 of the planes on: plane row
// j (j0 <= j < Nc) gets src[l * ld + j] at K position koff + l (0 beyond
// krows within the last block).
// The exponents are given (Ej[b * sE + j]; sE = 0 for one shared row of
// exponents), chosen by the caller as bounds known before the values exist;
// a value at or above its bound raises the numerical flag.  LOCAL: krows <=
// 32 (one block), and each plane row takes the exponent of its own largest
// entry, written to Ej.  One CTA converts 32 plane rows; eight threads share
// a row.
template <bool LOCAL>
__device__ __forceinline__ void oz_slice_block(int bx, const double *src, long long sS, long long ld, int j0, int Nc,
                                               int krows, int koff, long long plane_stride, int rows_cap, int ldk,
                                               __nv_bfloat16 *planes, int *Ej, long long sE, int *flag,
                                               const int *rowidx, long long sR)
{
    __shared__ double tile[32][33];
    const int b = blockIdx.y, c0 = j0 + bx * 32;
    // blockIdx.z: the 32-row block of the krows source rows (K positions koff + 32 z ..);
    // source row l is rowidx[b * sR + l] when a row index is given
    const int kz = 32 * blockIdx.z;
    const int kb = krows - kz < 32 ? krows - kz : 32;
    koff += kz;
    const double *s = src + (long long)b * sS;
    const int *ri = rowidx ? rowidx + (long long)b * sR + kz : nullptr;
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
        const int l = idx >> 5, r = idx & 31;
        double v = 0.0;
        if (l < kb && c0 + r < Nc) v = s[(long long)(ri ? ri[l] : kz + l) * ld + c0 + r];
        tile[l][r] = v;
    }
    __syncthreads();
    const int r = threadIdx.x >> 3, q = threadIdx.x & 7;
    const int j = c0 + r;
    int dg[4][OZ_S];
    if (LOCAL) {
        // the row's largest |entry| over its eight threads (lanes 8r'..8r'+7)
        unsigned long long mx = 0;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const unsigned long long u =
                (unsigned long long)__double_as_longlong(tile[4 * q + jj][r]) & 0x7FFFFFFFFFFFFFFFull;
            mx = u > mx ? u : mx;
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = v > mx ? v : mx;
        }
        if (j >= Nc) return;
        const int ef_max = (int)(mx >> 52);
        const int E = ef_max > 0 ? ef_max - 1022 : 0;
        if (q == 0) Ej[(long long)b * sE + j] = E;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) oz_digits(tile[4 * q + jj][r], E, ef_max, dg[jj]);
    } else {
        if (j >= Nc) return;
        const int E = Ej[(long long)b * sE + j];
        const unsigned long long bound = (unsigned long long)(E + 1023) << 52;  // bit pattern of 2^E
        bool over = false;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const double x = tile[4 * q + jj][r];
            over |= ((unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull) >= bound;
            oz_digits(x, E, 1, dg[jj]);
        }
        if (over) atomicOr(flag, FLAG_NUMERICAL);
    }
    const long long row = ((long long)b * rows_cap + j) * ldk + koff + 4 * q;
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) {
        __nv_bfloat162 h2[2] = {__floats2bfloat162_rn((float)dg[0][p], (float)dg[1][p]),
                                __floats2bfloat162_rn((float)dg[2][p], (float)dg[3][p])};
        *reinterpret_cast<uint2 *>(planes + (long long)p * plane_stride + row) = *reinterpret_cast<const uint2 *>(h2);
    }
}

__global__ void __launch_bounds__(256) k_oz_slice_fixed(const double *src, long long sS, long long ld, int j0, int Nc,
                                                        int krows, int koff, long long plane_stride, int rows_cap,
                                                        int ldk, __nv_bfloat16 *planes, int *Ej, long long sE,
                                                        int *flag, const int *rowidx = nullptr, long long sR = 0)
{
    oz_slice_block<false>(blockIdx.x, src, sS, ld, j0, Nc, krows, koff, plane_stride, rows_cap, ldk, planes, Ej, sE,
                          flag, rowidx, sR);
}

// The unsolved rows k0..k0+kb of a Cholesky-QR panel in one launch, each
// plane row with its own maximum (LOCAL): blocks x < nb0 split Y's rows (all
// N columns, into the Q^T planes), the others W's (columns j0.., into the R
// planes).
struct OzPanelSlice {
    const double *src[2];
    long long sS[2];
    int j0[2], nb0;
    __nv_bfloat16 *planes[2];
    int *E[2];
};

__global__ void __launch_bounds__(256) k_oz_slice_panel(OzPanelSlice a, int N, int ld, int kb, int koff,
                                                        long long plane_stride, int ldk, int *flag)
{
    const int part = blockIdx.x < a.nb0 ? 0 : 1;
    const int bx = part ? blockIdx.x - a.nb0 : blockIdx.x;
    oz_slice_block<true>(bx, part ? a.src[1] : a.src[0], part ? a.sS[1] : a.sS[0], ld, part ? a.j0[1] : a.j0[0], N,
                         kb, koff, plane_stride, N, ldk, part ? a.planes[1] : a.planes[0], part ? a.E[1] : a.E[0], N,
                         flag, nullptr, 0);
}

// Bounds for the entries of R's columns in a Cholesky factorisation of the
// Gram matrix W: sum_l R_lj^2 = W_jj, so |R_lj| <= sqrt(W_jj) < 2^E_j with
// E_j = ceil(e/2) + 1, W_jj < 2^e (one bit of margin for rounding).
__global__ void k_oz_col_exponents(const double *W, long long sW, int ldw, int N, int *E)
{
    const int b = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const unsigned long long u =
            (unsigned long long)__double_as_longlong(W[(long long)b * sW + (long long)j * ldw + j]) & 0x7FFFFFFFFFFFFFFFull;
        const int ef = (int)(u >> 52);
        const int e = ef > 0 ? ef - 1022 : -1022;
        E[(long long)b * N + j] = ((e + 1) >> 1) + 1;
    }
}

// E[b][j] = frexp exponent of max_r |src[r][j]| (|src[r][j]| < 2^E; 0 for a
// zero column).  A CTA covers 32 columns with eight row groups (each warp
// reads one 256-byte row segment per row); the eight partial maxima meet in
// shared memory.
__global__ void __launch_bounds__(256) k_oz_col_max_exponents(const double *src, long long sS, int rows, int cols,
                                                              int *E)
{
    __shared__ unsigned long long part[8][32];
    const int b = blockIdx.y, lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;
    const double *s = src + (long long)b * sS;
    unsigned long long mx = 0;
    if (j < cols) {
#pragma unroll 4
        for (int r = g; r < rows; r += 8) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(s[(long long)r * cols + j]) & 0x7FFFFFFFFFFFFFFFull;
            mx = u > mx ? u : mx;
        }
    }
    part[g][lane] = mx;
    __syncthreads();
    if (g == 0 && j < cols) {
#pragma unroll
        for (int q = 1; q < 8; ++q) mx = part[q][lane] > mx ? part[q][lane] : mx;
        const int ef = (int)(mx >> 52);
        E[(long long)b * cols + j] = ef > 0 ? ef - 1022 : 0;
    }
}

// T[m][k] = R[m][k] Dp[k] / D[m] for k >= m, 0 below (FP64), the triangular
// factor of the V update V <- T P^T V.
__global__ void k_oz_make_T(const double *R, long long nn, int N, const double *D, const double *Dp, double *T)
{
    const int b = blockIdx.z, m = blockIdx.y;
    __shared__ double s_rd;  // one division per row (FP64 division is a long chain on this pipe)
    if (threadIdx.x == 0) s_rd = 1.0 / D[(long long)b * N + m];
    __syncthreads();
    const double rd = s_rd;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x)
        T[(long long)b * nn + (long long)m * N + k] =
            k >= m ? R[(long long)b * nn + (long long)m * N + k] * Dp[(long long)b * N + k] * rd : 0.0;
}

// Row j of the diagonal block's factor and of its inverse, finalised by one
// warp: y = 1/sqrt(d) of the updated pivot d, R_jc = W_jc y (c > j), R_jj =
// d y, and row j of T scaled by y (it has received its terms l < j).
__device__ __forceinline__ void oz_chol_finalise_row(double (*Rk)[33], double (*Tm)[33], int j, int lane, int kb,
                                                     int *flag)
{
    double d = Rk[j][j];
    if (!(d > 0.0) || !isfinite(d)) {
        if (lane == 0 && j < kb) atomicOr(flag, FLAG_NUMERICAL);
        d = 1.0;
    }
    const double y = rsqrt(d);
    if (lane > j) Rk[j][lane] *= y;
    if (lane <= j) Tm[j][lane] *= y;
    __syncwarp();  // every lane has read the pivot
    if (lane == j) Rk[j][j] = d * y;
    __syncwarp();
}

// Rows r > j of R (upper part c >= r) and of T (finished columns c <= j)
// lose row j's share: one FMA per warp and row.
__device__ __forceinline__ void oz_chol_update_row(double (*Rk)[33], double (*Tm)[33], int j, int r, int lane)
{
    const double rjr = Rk[j][r];
    if (lane >= r) Rk[r][lane] -= rjr * Rk[j][lane];
    else if (lane <= j) Tm[r][lane] -= rjr * Tm[j][lane];
}

// Cholesky factor of a panel's diagonal block, W_kk = R_kk^T R_kk (R_kk
// upper triangular, written to R), and the digit planes of T = R_kk^-T
// (lower triangular; each row with its own maximum as exponent, ET) for the
// panel's product [R_k,k+ | Q_k^T] = T [W_k,k+ | Y_k] on the tensor cores.
// One CTA of 128 threads per item; rows and columns kb..31 of R_kk are the
// identity.  Right-looking: once row j of R and of T is final (T by forward
// substitution of R_kk^T T = I), every later row loses row j's share.  Warp 0
// updates row j + 1 first and finalises it (the chain of pivots: update,
// rsqrt, scale) while warps 1..3 update the rows below, so each step costs one
// barrier and the pivot chain overlaps the other rows' updates.  Every FP64
// instruction occupies the pipe for a whole warp, so the work is grouped by
// rows.
__global__ void __launch_bounds__(128) k_oz_chol_factor(const double *W, long long sW, int ldw, double *R, long long sR,
                                                        int N, int k0, int kb, __nv_bfloat16 *tplanes, long long tps,
                                                        int *ET, int *flag)
{
    __shared__ double Rk[32][33];
    __shared__ double Tm[32][33];
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const double *Wb = W + (long long)b * sW;
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
        const int r = e >> 5, c = e & 31;
        double v = 0.0;
        if (r < kb && c < kb) {
            if (c >= r) v = Wb[(long long)(k0 + r) * ldw + k0 + c];
        } else if (r == c) {
            v = 1.0;
        }
        Rk[r][c] = v;
        Tm[r][c] = r == c ? 1.0 : 0.0;
    }
    __syncthreads();
    if (wid == 0) oz_chol_finalise_row(Rk, Tm, 0, lane, kb, flag);
    __syncthreads();
    for (int j = 0; j < 31; ++j) {
        if (wid == 0) {
            oz_chol_update_row(Rk, Tm, j, j + 1, lane);
            __syncwarp();
            oz_chol_finalise_row(Rk, Tm, j + 1, lane, kb, flag);
        } else {
            for (int r = j + 1 + wid; r < 32; r += 3) oz_chol_update_row(Rk, Tm, j, r, lane);
        }
        __syncthreads();
    }
    double *Rb = R + (long long)b * sR;
    for (int e = tid; e < kb * kb; e += blockDim.x) {
        const int r = e / kb, c = e % kb;
        Rb[(long long)(k0 + r) * N + k0 + c] = c >= r ? Rk[r][c] : 0.0;
    }
    // digits of T's rows: four threads per row, eight K positions each
    const int r = tid >> 2, q = tid & 3;
    unsigned long long mx = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(Tm[r][8 * q + i]) & 0x7FFFFFFFFFFFFFFFull;
        mx = u > mx ? u : mx;
    }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
    }
    const int ef_max = (int)(mx >> 52);
    const int E = ef_max > 0 ? ef_max - 1022 : 0;
    if (q == 0) ET[b * 32 + r] = E;
    int dg[8][OZ_S];
#pragma unroll
    for (int i = 0; i < 8; ++i) oz_digits(Tm[r][8 * q + i], E, ef_max, dg[i]);
    const long long row = ((long long)b * 32 + r) * 32 + 8 * q;
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) {
        __nv_bfloat162 h2[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) h2[i] = __floats2bfloat162_rn((float)dg[2 * i][p], (float)dg[2 * i + 1][p]);
        *reinterpret_cast<uint4 *>(tplanes + (long long)p * tps + row) = *reinterpret_cast<const uint4 *>(h2);
    }
}

// One part of a product's rows: rows m of C (rows of A, starting at plane row
// arow0 of the part's A map), their exponents, and where C goes; with SLICE,
// where the digits of C's values go as well (plane rows srow0 + m, K
// positions skoff + n, exponents SE[b * sSE + srow0 + m]).
struct OzPart {
    int M, arow0;
    const int *EA;
    long long sEA;
    double *C;
    long long sC;
    int ldc;
    __nv_bfloat16 *sp;
    const int *SE;
    long long sSE;
    int srow0;
};

// x 2^e, exact: through the exponent field while the result stays normal
// (integer arithmetic, off the FP64 pipe), otherwise scalbn.
__device__ __forceinline__ double oz_scale2(double x, int e)
{
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex != 0 && ex + e > 0 && ex + e < 2047) return __longlong_as_double(bits + ((long long)e << 52));
    return scalbn(x, e);
}

struct OzArgs {
    OzPart pt[2];           // pt[1] only with nparts = 2 (its A rows through the second A map)
    int nparts;
    int Nn, brow0;          // rows of B (columns of C), first plane row of B
    int batch, nk;          // items, 32-wide K-blocks
    int kA0, kB0;           // first K positions (elements) of A and B in their planes
    const int *EB;          // row exponents of B
    long long sEB;
    long long splane_stride;  // SLICE: plane stride, leading dimension, plane rows per item,
    int sldp, srows, skoff;   // and the K position of n = 0
    int a_tri, b_tri;         // A upper triangular (A[m][k] = 0 for k < m) / B^T upper triangular
                              // (B[n][k] = 0 for k > n): a tile's K-blocks start at m0 / 32 / end
                              // after the one holding n0 + 31 (kA0 = kB0 = 0)
    int *flag;
};

// K-blocks [k_lo, k_hi) that can hold nonzero products for the tile at (m0, n0).
__device__ __forceinline__ void oz_krange(const OzArgs &a, int m0, int n0, int &k_lo, int &k_hi)
{
    k_lo = a.a_tri ? m0 / OKE : 0;
    k_hi = a.nk;
    if (a.b_tri) {
        const int e = (n0 + OBN + OKE - 1) / OKE;
        if (e < k_hi) k_hi = e;
    }
    if (k_hi < k_lo) k_hi = k_lo;
}

// Tile t of the persistent walk -> (item, first row, first column).
// Without UPPER every tile, row strip by row strip, columns fastest (a wave
// of CTAs shares one row strip of A; the tiles of a strip have the same K
// range, which keeps the triangular products balanced).  UPPER: the
// 128 x 32 tiles on or above the diagonal (tile (tm, tn) with tn >= 4 tm)
// of a Gram matrix, in groups of OZ_GROUP_M row strips, column-major inside
// a group, so that the CTAs of one wave share a few row strips of A and a
// few of B: walking columns first, every CTA of a wave read its own B strip,
// and at N = 10^4 the digit planes (16 bytes per element) far exceed L2 (at
// N = 4096 the grouped walk reads 2.7 instead of 5.3 GB from DRAM per Gram,
// in the same time).  In a group of gm strips starting at m_first, the walk
// first meets the ramp of columns 4 (m_first + j) .. + 3 with j + 1 rows
// (j < gm - 1), then columns with all gm rows.
constexpr int OZ_GROUP_M = 8;

// Upper tiles of the group of gm row strips starting at m_first.
__host__ __device__ inline int oz_group_tiles(int m_first, int gm, int tiles_n)
{
    const int T = tiles_n - 4 * m_first, F = T / 4, R = T % 4;
    const int S = F <= gm ? F * (F + 1) / 2 : gm * (gm + 1) / 2 + (F - gm) * gm;
    return 4 * S + R * (F + 1 < gm ? F + 1 : gm);
}

template <bool UPPER>
__device__ __forceinline__ void oz_tile(int t, int tiles_m, int tiles_n, int per_item, int &b, int &m0, int &n0)
{
    b = t / per_item;
    int r = t - b * per_item;
    if (!UPPER) {
        m0 = (r / tiles_n) * OBM;
        n0 = (r % tiles_n) * OBN;
        return;
    }
    int m_first = 0, gm = 0;
    for (; m_first < tiles_m; m_first += OZ_GROUP_M) {
        gm = tiles_m - m_first < OZ_GROUP_M ? tiles_m - m_first : OZ_GROUP_M;
        const int cnt = oz_group_tiles(m_first, gm, tiles_n);
        if (r < cnt) break;
        r -= cnt;
    }
    for (int j = 0; j < gm - 1; ++j) {
        const int cols = tiles_n - 4 * (m_first + j) < 4 ? tiles_n - 4 * (m_first + j) : 4;
        const int n_in = cols * (j + 1);
        if (r < n_in) {
            m0 = (m_first + r % (j + 1)) * OBM;
            n0 = (4 * (m_first + j) + r / (j + 1)) * OBN;
            return;
        }
        r -= n_in;
    }
    m0 = (m_first + r % gm) * OBM;
    n0 = (4 * (m_first + gm - 1) + r / gm) * OBN;
}

template <bool UPPER>
__host__ __device__ inline int oz_per_item(int tiles_m, int tiles_n)
{
    if (!UPPER) return tiles_m * tiles_n;
    int n = 0;
    for (int tm = 0; tm < tiles_m; ++tm) n += tiles_n - 4 * tm;
    return n;
}

// Tiles of the whole launch: part 0's for all items, then part 1's.
template <bool UPPER>
__host__ __device__ inline int oz_part_tiles(const OzArgs &a, int part)
{
    const int M = part ? a.pt[1].M : a.pt[0].M;
    return oz_per_item<UPPER>((M + OBM - 1) / OBM, (a.Nn + OBN - 1) / OBN) * a.batch;
}

template <bool UPPER>
__device__ __forceinline__ void oz_locate(const OzArgs &a, int t, int tiles0, int &part, int &b, int &m0, int &n0)
{
    part = t < tiles0 ? 0 : 1;
    if (part) t -= tiles0;
    const int M = part ? a.pt[1].M : a.pt[0].M;
    const int tiles_m = (M + OBM - 1) / OBM, tiles_n = (a.Nn + OBN - 1) / OBN;
    oz_tile<UPPER>(t, tiles_m, tiles_n, oz_per_item<UPPER>(tiles_m, tiles_n), b, m0, n0);
}

// UPPER: only the tiles on or above the diagonal (C square, A and B the same
// rows); SUB: C -= A B^T, otherwise C = A B^T; TRANS: element (m, n) of the
// product lives at C[n * ldc + m] (a warp's 32 rows m are then contiguous);
// SLICE (with TRANS, not SUB): the results are also split into digit planes
// with given exponents, the value (m, n) at K position skoff + n of plane row
// srow0 + m (zero digits for n >= Nn up to the tile's 32).
template <bool UPPER, bool SUB, bool TRANS = false, bool SLICE = false>
__global__ void __launch_bounds__(OTHREADS, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
              const __grid_constant__ CUtensorMap tB, OzArgs a)
{
    static_assert(!SLICE || (TRANS && !SUB), "SLICE needs TRANS and C = A B^T");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(base + OSTAGES * OSTAGE);
    uint64_t *empty = full + OSTAGES;
    uint64_t *tmem_full = empty + OSTAGES;  // [2]
    uint64_t *tmem_free = tmem_full + 2;    // [2]
    uint32_t *tmem_slot = (uint32_t *)(tmem_free + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles0 = oz_part_tiles<UPPER>(a, 0);
    const int tiles = tiles0 + (a.nparts > 1 ? oz_part_tiles<UPPER>(a, 1) : 0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < OSTAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int u = 0; u < 2; ++u) {
            mbar_init(&tmem_full[u], 1);
            mbar_init(&tmem_free[u], 32 * OEPI);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(OTMEM)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                int part, b, m0, n0;
                oz_locate<UPPER>(a, t, tiles0, part, b, m0, n0);
                const CUtensorMap *mA = part ? &tA1 : &tA0;
                const int arow0 = part ? a.pt[1].arow0 : a.pt[0].arow0;
                int k_lo, k_hi;
                oz_krange(a, m0, n0, k_lo, k_hi);
                for (int kb = k_lo; kb < k_hi; ++kb, ++it) {
                    const int s = it % OSTAGES;
                    if (it >= OSTAGES && !mbar_wait(&empty[s], ((it / OSTAGES) - 1) & 1, a.flag)) { ok = false; break; }
                    mbar_expect_tx(&full[s], OSTAGE);
                    uint8_t *st = base + s * OSTAGE;
                    const int k0 = kb * OKE;
#pragma unroll
                    for (int p = 0; p < OZ_S; ++p) {
                        tma_load_4d(st + p * OTILE_A, mA, a.kA0 + k0, arow0 + m0, b, p, &full[s]);
                        tma_load_4d(st + OZ_S * OTILE_A + p * OTILE_B, &tB, a.kB0 + k0, a.brow0 + n0, b, p, &full[s]);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, cc = 0;  // K-block and chunk counters of this CTA
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                int part, b, m0, n0, k_lo, k_hi;
                oz_locate<UPPER>(a, t, tiles0, part, b, m0, n0);
                oz_krange(a, m0, n0, k_lo, k_hi);
                for (int kc0 = k_lo; kc0 < k_hi && ok; kc0 += OZ_KCHUNK, ++cc) {
                    const int u = cc & 1;
                    // the epilogue must have drained this buffer (used two chunks ago)
                    if (cc >= 2 && !mbar_wait(&tmem_free[u], ((cc >> 1) - 1) & 1, a.flag)) { ok = false; break; }
                    fence_after();
                    const uint32_t acc0 = tmem + (uint32_t)(u * OZ_G * OBN);
                    const int kc1 = kc0 + OZ_KCHUNK < k_hi ? kc0 + OZ_KCHUNK : k_hi;
                    for (int kb = kc0; kb < kc1; ++kb, ++it) {
                        const int s = it % OSTAGES;
                        if (!mbar_wait(&full[s], (it / OSTAGES) & 1, a.flag)) { ok = false; break; }
                        fence_after();
                        const uint32_t sa = smem_u32(base + s * OSTAGE);
                        const uint32_t sb = sa + OZ_S * OTILE_A;
                        // The B planes of a stage lie one after another (32 rows each), so
                        // planes 0..7-p form one K-major operand of 32 (8 - p) rows: a single
                        // MMA multiplies A's plane p with all of them, and with its output
                        // starting at column 32 p the product with plane q lands in group
                        // p + q's accumulator.  Eight MMAs per K-step instead of 36, each
                        // reading A's plane from shared memory once.  The first MMA of a
                        // chunk (p = 0) spans every group and initialises all eight.
#pragma unroll
                        for (int k = 0; k < OKE / 16; ++k) {
#pragma unroll
                            for (int p = 0; p < OZ_S; ++p) {
                                mma_bf16(acc0 + (uint32_t)(p * OBN), smem_desc64(sa + p * OTILE_A + k * 32),
                                         smem_desc64(sb + k * 32), oz_idesc(OBN * (OZ_S - p)),
                                         (kb != kc0 || k != 0 || p != 0) ? 1u : 0u);
                            }
                        }
                        mma_commit(&empty[s]);
                    }
                    if (ok) mma_commit(&tmem_full[u]);
                }
            }
        }
    } else {
        // epilogue: warp w drains lane quarter w % 4, columns [hc, hc + 16)
        const int q4 = warp & 3;
        const int hc = ((warp - 2) >> 2) * 16;
        int cc = 0;  // chunk counter, in step with the MMA thread's
        bool ok = true;
        for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
            int part, b, m0, n0;
            oz_locate<UPPER>(a, t, tiles0, part, b, m0, n0);
            const int M = part ? a.pt[1].M : a.pt[0].M;
            const int *EA = part ? a.pt[1].EA : a.pt[0].EA;
            const long long sEA = part ? a.pt[1].sEA : a.pt[0].sEA;
            double *C = part ? a.pt[1].C : a.pt[0].C;
            const long long sC = part ? a.pt[1].sC : a.pt[0].sC;
            const int ldc = part ? a.pt[1].ldc : a.pt[0].ldc;
            const int mm = m0 + q4 * 32 + lane;
            const int Ei = mm < M ? EA[(long long)b * sEA + mm] : 0;
            // element (mm, n) at o[n * cs]; for an update, the old values of this
            // thread's row segment, fetched while the MMAs run
            double *o = C + (long long)b * sC + (TRANS ? (long long)mm : (long long)mm * ldc);
            const long long cs = TRANS ? ldc : 1;
            const int nb = n0 + hc;
            const int *eb = a.EB + (long long)b * a.sEB;
            double cold[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) cold[j] = (SUB && mm < M && nb + j < a.Nn) ? o[(nb + j) * cs] : 0.0;
            // the columns' exponents, also fetched while the MMAs run (not for an
            // update, whose old values already take those registers)
            int ebv[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) ebv[j] = (!SUB && nb + j < a.Nn) ? eb[nb + j] : 0;
            // sum over K-chunks of the exactly accumulated chunk products
            double w[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) w[j] = 0.0;
            int k_lo, k_hi;
            oz_krange(a, m0, n0, k_lo, k_hi);
            for (int kc0 = k_lo; kc0 < k_hi; kc0 += OZ_KCHUNK, ++cc) {
                const int u = cc & 1;
                ok = mbar_wait(&tmem_full[u], (cc >> 1) & 1, a.flag);
                fence_after();
                const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(u * OZ_G * OBN + hc);
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    // group sums as exact integers, folded as they arrive: groups 0..3
                    // (p + q = 2..5) into h, 4..7 (6..9) into l, so that
                    // sum_g acc_g 2^-7(g+2) = h 2^-35 + l 2^-63
                    long long h[8], l[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) h[j] = l[j] = 0;
#pragma unroll
                    for (int gg = 0; gg < OZ_G; gg += 2) {
                        uint32_t r0[8], r1[8];
                        tmem_ld8_nowait(lane_base + (uint32_t)(gg * OBN + half * 8), r0);
                        tmem_ld8_nowait(lane_base + (uint32_t)((gg + 1) * OBN + half * 8), r1);
                        tmem_wait_ld8x2(r0, r1);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const long long v0 = (long long)__float2int_rn(__uint_as_float(r0[j]));
                            const long long v1 = (long long)__float2int_rn(__uint_as_float(r1[j]));
                            if (gg < 4) h[j] += (v0 << (OZ_BETA * (3 - gg))) + (v1 << (OZ_BETA * (2 - gg)));
                            else l[j] += (v0 << (OZ_BETA * (7 - gg))) + (v1 << (OZ_BETA * (6 - gg)));
                        }
                    }
                    // the chunk's value (one rounding); the first chunk needs no addition
                    if (kc0 == k_lo) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) w[half * 8 + j] = fma((double)l[j], 0x1p-28, (double)h[j]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j) w[half * 8 + j] += fma((double)l[j], 0x1p-28, (double)h[j]);
                    }
                }
                fence_before();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tmem_free[u])) : "memory");
                if (!ok) break;
            }
            if (!ok) break;
            if (mm >= M) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = nb + j;
                double v = 0.0;
                if (n < a.Nn) {
                    v = oz_scale2(w[j], Ei + (SUB ? eb[n] : ebv[j]) - 35);
                    o[n * cs] = SUB ? cold[j] - v : v;
                }
                if (SLICE) w[j] = v;
            }
            if (SLICE) {
                const int srow = (part ? a.pt[1].srow0 : a.pt[0].srow0) + mm;
                const int *SE = part ? a.pt[1].SE : a.pt[0].SE;
                const long long sSE = part ? a.pt[1].sSE : a.pt[0].sSE;
                __nv_bfloat16 *sp = part ? a.pt[1].sp : a.pt[0].sp;
                const int E = SE[(long long)b * sSE + srow];
                const unsigned long long bound = (unsigned long long)(E + 1023) << 52;  // bit pattern of 2^E
                bool over = false;
                __nv_bfloat16 *dst = sp + ((long long)b * a.srows + srow) * a.sldp + a.skoff + nb;
                // eight K positions per 16-byte store: each lane writes its own plane row,
                // so the stores cannot coalesce across lanes; wider stores halve the
                // sector writes
#pragma unroll
                for (int g8 = 0; g8 < 2; ++g8) {
                    int dg[8][OZ_S];
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        const double x = w[8 * g8 + jj];
                        over |= ((unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull) >= bound;
                        oz_digits(x, E, 1, dg[jj]);
                    }
#pragma unroll
                    for (int p = 0; p < OZ_S; ++p) {
                        __nv_bfloat162 h2[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            h2[i] = __floats2bfloat162_rn((float)dg[2 * i][p], (float)dg[2 * i + 1][p]);
                        *reinterpret_cast<uint4 *>(dst + (long long)p * a.splane_stride + 8 * g8) =
                            *reinterpret_cast<const uint4 *>(h2);
                    }
                }
                if (over) atomicOr(a.flag, FLAG_NUMERICAL);
            }
        }
    }
    __syncwarp();
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OTMEM) : "memory");
}

struct OzWs {
    int ldp;
    long long plane_stride;
    __nv_bfloat16 *planes;  // digit planes of the Gram operand; in the Cholesky-QR, of Q's finished rows
    int *E;
    CUtensorMap mapA, mapB;
    // Cholesky-QR: digit planes of R's finished rows, stored by column of R
    // (plane row j holds R[l][j] at K position l), with fixed exponents ER
    // (bounds from the Gram diagonal) and EQ = 1 for Q's rows (|Q_lj| < 2)
    __nv_bfloat16 *rplanes;
    int *ER, *EQ;
    int *ER1;  // column bounds of the first pass's R (kept for R = R2 R1)
    CUtensorMap mapRA, mapRB;  // 128-row and 32-row boxes
    // Cholesky-QR panels: digit planes of T = R_kk^-T (32 x 32 per item) and
    // their row exponents; column exponents of the unsolved panel rows of Y
    // (EPY) and of W (EPW)
    __nv_bfloat16 *tplanes;
    long long tplane_stride;
    int *ET, *EPY, *EPW;
    CUtensorMap mapT;
    int num_sms;
};

bool encode4(CUtensorMap *map, void *ptr, int ldp, int rows, int batch, int box_rows)
{
    auto fn = get_encode();
    if (!fn) return false;
    cuuint64_t dims[4] = {(cuuint64_t)ldp, (cuuint64_t)rows, (cuuint64_t)batch, (cuuint64_t)OZ_S};
    cuuint64_t strides[3] = {(cuuint64_t)ldp * 2, (cuuint64_t)ldp * rows * 2, (cuuint64_t)ldp * rows * batch * 2};
    cuuint32_t box[4] = {(cuuint32_t)OKE, (cuuint32_t)box_rows, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

int oz_prepare(sldqmc_ctx *c)
{
    c->oz_ws = nullptr;
    if (c->N < OBM) return SLDQMC_OK;  // tiles are 128 rows
    OzWs *w = new OzWs();
    const int N = c->N;
    w->ldp = (N + 63) / 64 * 64;
    w->plane_stride = (long long)c->cap * N * w->ldp;
    const size_t pbytes = (size_t)OZ_S * w->plane_stride * sizeof(__nv_bfloat16);
    const size_t ebytes = sizeof(int) * (size_t)c->cap * N;
    w->tplane_stride = (long long)c->cap * 32 * 32;
    const size_t tbytes = (size_t)OZ_S * w->tplane_stride * sizeof(__nv_bfloat16);
    const size_t tebytes = sizeof(int) * (size_t)c->cap * 32;
    const size_t eoff = 2 * pbytes + tbytes;  // the int arrays follow the planes
    void *mem = nullptr;
    if (cudaMalloc(&mem, eoff + 5 * ebytes + tebytes + sizeof(int) * N) != cudaSuccess) {
        cudaGetLastError();
        delete w;
        return SLDQMC_ERR_OOM;
    }
    w->planes = (__nv_bfloat16 *)mem;
    w->rplanes = (__nv_bfloat16 *)((uint8_t *)mem + pbytes);
    w->tplanes = (__nv_bfloat16 *)((uint8_t *)mem + 2 * pbytes);
    w->E = (int *)((uint8_t *)mem + eoff);
    w->ER = w->E + (size_t)c->cap * N;
    w->ER1 = w->ER + (size_t)c->cap * N;
    w->EPY = w->ER1 + (size_t)c->cap * N;
    w->EPW = w->EPY + (size_t)c->cap * N;
    w->ET = w->EPW + (size_t)c->cap * N;
    w->EQ = w->ET + (size_t)c->cap * 32;
    cudaMemsetAsync(mem, 0, eoff + 5 * ebytes + tebytes, c->st);  // zero pads: never written
    {
        std::vector<int> ones((size_t)N, 1);
        if (cudaMemcpyAsync(w->EQ, ones.data(), sizeof(int) * N, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
            cudaStreamSynchronize(c->st) != cudaSuccess) {
            cudaFree(mem);
            delete w;
            return SLDQMC_ERR_CUDA;
        }
    }
    if (!encode4(&w->mapA, w->planes, w->ldp, N, c->cap, OBM) || !encode4(&w->mapB, w->planes, w->ldp, N, c->cap, OBN) ||
        !encode4(&w->mapRA, w->rplanes, w->ldp, N, c->cap, OBM) ||
        !encode4(&w->mapRB, w->rplanes, w->ldp, N, c->cap, OBN) ||
        !encode4(&w->mapT, w->tplanes, 32, 32, c->cap, OBN)) {
        cudaFree(mem);
        delete w;
        return SLDQMC_ERR_CUDA;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&w->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || w->num_sms < 1)
        w->num_sms = 148;
    cudaFuncSetAttribute(k_oz_gemm<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes());
    cudaFuncSetAttribute(k_oz_gemm<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes());
    cudaFuncSetAttribute(k_oz_gemm<false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)oz_smem_bytes());
    cudaFuncSetAttribute(k_oz_gemm<false, false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)oz_smem_bytes());
    cudaFuncSetAttribute(k_oz_gemm<false, true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)oz_smem_bytes());
    c->oz_ws = w;
    return SLDQMC_OK;
}

void oz_release(sldqmc_ctx *c)
{
    OzWs *w = (OzWs *)c->oz_ws;
    if (!w) return;
    cudaFree(w->planes);
    delete w;
    c->oz_ws = nullptr;
}

namespace {

OzPart oz_part(int M, int arow0, const int *EA, long long sEA, double *C, long long sC, int ldc)
{
    OzPart p{};
    p.M = M;
    p.arow0 = arow0;
    p.EA = EA;
    p.sEA = sEA;
    p.C = C;
    p.sC = sC;
    p.ldc = ldc;
    return p;
}

template <bool UPPER>
int oz_grid(const OzWs *w, const OzArgs &a)
{
    const int tiles = oz_part_tiles<UPPER>(a, 0) + (a.nparts > 1 ? oz_part_tiles<UPPER>(a, 1) : 0);
    return tiles < w->num_sms ? tiles : w->num_sms;
}

}  // namespace

// W = X X^T (rows of X: row stride N, batch stride sX); W row stride ldw,
// batch stride sW.  Tiles on or above the diagonal are written in full.
void oz_gram(sldqmc_ctx *c, const double *X, long long sX, double *W, long long sW, int ldw, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    const int N = c->N;
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_oz_slice");
    k_oz_slice<<<dim3((N + 7) / 8, B), 256, 0, c->st>>>(X, sX, N, N, N, N, w->ldp, w->plane_stride, w->planes,
                                                         w->E);
    prof_end(c);
    OzArgs a{};
    a.pt[0] = oz_part(N, 0, w->E, N, W, sW, ldw);
    a.nparts = 1;
    a.Nn = N;
    a.batch = B;
    a.nk = w->ldp / OKE;
    a.EB = w->E;
    a.sEB = N;
    a.flag = c->d_flag;
    prof_begin(c, SLDQMC_KC_GEMM_OZ, (double)N * N * (N + 1) * B, "oz_gram");
    k_oz_gemm<true, false><<<oz_grid<true>(w, a), OTHREADS, oz_smem_bytes(), c->st>>>(w->mapA, w->mapA, w->mapB, a);
    prof_end(c);
    c->launches += 2;
}

// Left-looking Cholesky-QR of W = X X^T (row stride N, item stride sW) that
// forms Q^T = R^-T X^T in Y (row stride N, item stride N*N): before the rows
// k0..k0+kb the products of the finished rows kstart..k0-1 are subtracted
// from them (the caller runs it once per block of up to 128 rows with all
// earlier rows, then per 32-row panel with the block's own finished rows),
//   Y[k0+r][n]    -= sum_{l<k0} Q^T[l][n] R[l][k0+r],
//   W[k0+r][k0+n] -= sum_{l<k0} R[l][k0+n] R[l][k0+r],
// FP64-accurate on the tensor cores in one launch of two parts (the product
// computed with rows n and columns r, stored transposed so that a warp's
// stores are contiguous); the panel then splits its finished rows of R and
// Q^T into K-block k0/32 of the digit planes.  oz_chol_begin fixes the
// exponents of R's columns from W's diagonal.
void oz_chol_begin(sldqmc_ctx *c, const double *W, long long sW, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    const int N = c->N;
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_oz_col_exponents");
    k_oz_col_exponents<<<dim3((N + 255) / 256, B), 256, 0, c->st>>>(W, sW, N, N, w->ER);
    prof_end(c);
    c->launches++;
}

void oz_chol_update(sldqmc_ctx *c, int k0, int kb, int kstart, double *W, long long sW, double *Y, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    const int N = c->N;
    OzArgs a{};
    a.pt[0] = oz_part(N, 0, w->EQ, 0, Y + (long long)k0 * N, c->nn, N);                    // rows n: columns of Q^T
    a.pt[1] = oz_part(N - k0, k0, w->ER + k0, N, W + (long long)k0 * N + k0, sW, N);      // rows n: columns k0.. of R
    a.nparts = 2;
    a.Nn = kb;
    a.brow0 = k0;
    a.batch = B;
    a.kA0 = kstart;
    a.kB0 = kstart;
    a.nk = (k0 - kstart) / OKE;
    a.EB = w->ER + k0;
    a.sEB = N;
    a.flag = c->d_flag;
    prof_begin(c, SLDQMC_KC_GEMM_OZ, 2.0 * (2 * N - k0) * kb * (k0 - kstart) * B,
               kstart ? "oz_chol_update_inner" : "oz_chol_update");
    k_oz_gemm<false, true, true>
        <<<oz_grid<false>(w, a), OTHREADS, oz_smem_bytes(), c->st>>>(w->mapA, w->mapRA, w->mapRB, a);
    prof_end(c);
    c->launches++;
}

// The panel of rows k0..k0+kb once its rows of W and Y are up to date: the
// unsolved rows are split with each column's own maximum, the diagonal block
// is factored and inverted (FP64, one CTA per item), and
//   Y[k0+n][j] = sum_l T[n][l] Y[k0+l][j]   (all j: the rows of Q^T),
//   R[k0+n][j] = sum_l T[n][l] W[k0+l][j]   (j >= k0 + kb),
// run FP64-accurate on the tensor cores (K = 32, one exactly accumulated
// chunk) in place of the triangular solves, in one launch of two parts whose
// epilogue also splits the finished rows into K-block k0/32 of the digit
// planes (fixed exponents: EQ for Q^T, ER for R) for the later panels.
void oz_chol_panel(sldqmc_ctx *c, int k0, int kb, const double *W, long long sW, double *Y, double *R, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    const int N = c->N;
    const int j0 = k0 + kb, nW = N - j0;
    OzPanelSlice sl{};
    sl.src[0] = Y + (long long)k0 * N;
    sl.sS[0] = c->nn;
    sl.j0[0] = 0;
    sl.planes[0] = w->planes;
    sl.E[0] = w->EPY;
    sl.nb0 = (N + 31) / 32;
    sl.src[1] = W + (long long)k0 * N;
    sl.sS[1] = sW;
    sl.j0[1] = j0;
    sl.planes[1] = w->rplanes;
    sl.E[1] = w->EPW;
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_oz_slice_panel");
    k_oz_slice_panel<<<dim3(sl.nb0 + (nW + 31) / 32, B), 256, 0, c->st>>>(sl, N, N, kb, k0, w->plane_stride,
                                                                           w->ldp, c->d_flag);
    prof_end(c);
    prof_begin(c, SLDQMC_KC_PANEL_F64, (double)B * 2.0 * kb * kb * kb / 3.0, "oz_chol_factor");
    k_oz_chol_factor<<<B, 128, 0, c->st>>>(W, sW, N, R, c->nn, N, k0, kb, w->tplanes, w->tplane_stride, w->ET,
                                           c->d_flag);
    prof_end(c);
    OzArgs a{};
    a.pt[0] = oz_part(N, 0, w->EPY, N, Y + (long long)k0 * N, c->nn, N);
    a.pt[0].sp = w->planes;
    a.pt[0].SE = w->EQ;
    a.pt[0].sSE = 0;
    a.pt[0].srow0 = 0;
    a.pt[1] = oz_part(nW, j0, w->EPW + j0, N, R + (long long)k0 * N + j0, c->nn, N);
    a.pt[1].sp = w->rplanes;
    a.pt[1].SE = w->ER;
    a.pt[1].sSE = N;
    a.pt[1].srow0 = j0;
    a.nparts = nW > 0 ? 2 : 1;
    a.Nn = kb;
    a.brow0 = 0;
    a.batch = B;
    a.nk = 1;
    a.kA0 = k0;
    a.kB0 = 0;
    a.EB = w->ET;
    a.sEB = 32;
    a.splane_stride = w->plane_stride;
    a.sldp = w->ldp;
    a.srows = N;
    a.skoff = k0;
    a.flag = c->d_flag;
    prof_begin(c, SLDQMC_KC_GEMM_OZ, 2.0 * (N + nW) * kb * kb * B, "oz_chol_panel");
    k_oz_gemm<false, false, true, true>
        <<<oz_grid<false>(w, a), OTHREADS, oz_smem_bytes(), c->st>>>(w->mapA, w->mapRA, w->mapT, a);
    prof_end(c);
    c->launches += 3;
}

// Trailing update of the finalisation's blocked LU without a right-hand
// side, A[i][j] -= sum_l L[i][k0+l] U[k0+l][j] for i, j >= k0 + kb (A row
// stride lda, item stride sA), FP64-accurate on the tensor cores: the rows of
// L21 and the columns of U12 each split with their own maximum (K = kb = 32,
// one exactly accumulated chunk).
void oz_lu_update(sldqmc_ctx *c, double *A, long long sA, int lda, int k0, int kb, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    const int N = c->N;
    const int j0 = k0 + kb, M = N - j0;
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_oz_slice");
    k_oz_slice<<<dim3((M + 7) / 8, B), 256, 0, c->st>>>(A + (long long)j0 * lda + k0, sA, M, kb, lda, N, w->ldp,
                                                         w->plane_stride, w->planes, w->E);
    prof_end(c);
    OzPanelSlice sl{};
    sl.src[0] = A + (long long)k0 * lda;
    sl.sS[0] = sA;
    sl.j0[0] = j0;
    sl.planes[0] = w->rplanes;
    sl.E[0] = w->EPW;
    sl.nb0 = (M + 31) / 32;
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_oz_slice_panel");
    k_oz_slice_panel<<<dim3(sl.nb0, B), 256, 0, c->st>>>(sl, N, lda, kb, 0, w->plane_stride, w->ldp, c->d_flag);
    prof_end(c);
    OzArgs a{};
    a.pt[0] = oz_part(M, 0, w->E, N, A + (long long)j0 * lda + j0, sA, lda);
    a.nparts = 1;
    a.Nn = M;
    a.brow0 = j0;
    a.batch = B;
    a.nk = 1;
    a.EB = w->EPW + j0;
    a.sEB = N;
    a.flag = c->d_flag;
    prof_begin(c, SLDQMC_KC_GEMM_OZ, 2.0 * M * M * kb * B, "oz_lu_update");
    k_oz_gemm<false, true, false, false>
        <<<oz_grid<false>(w, a), OTHREADS, oz_smem_bytes(), c->st>>>(w->mapA, w->mapA, w->mapRB, a);
    prof_end(c);
    c->launches += 3;
}

// V <- T P^T V with T = D^-1 R D_p (upper triangular; R row stride N),
// FP64-accurate on the tensor cores: T's rows split with their own maxima,
// the gathered rows V[p_k] split column-wise with each column's maximum.
// Ts: an N x N FP64 scratch per item (item stride N*N).
void oz_update_V(sldqmc_ctx *c, const double *R, double *V, double *Ts, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    const int N = c->N;
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_oz_make_T");
    k_oz_make_T<<<dim3((N + 255) / 256, N, B), 256, 0, c->st>>>(R, c->nn, N, c->d_D, c->d_Dp, Ts);
    prof_end(c);
    k_oz_slice<<<dim3((N + 7) / 8, B), 256, 0, c->st>>>(Ts, c->nn, N, N, N, N, w->ldp, w->plane_stride, w->planes,
                                                         w->E);
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_oz_col_max_exponents");
    k_oz_col_max_exponents<<<dim3((N + 31) / 32, B), 256, 0, c->st>>>(V, c->nn, N, N, w->ER1);
    prof_end(c);
    k_oz_slice_fixed<<<dim3((N + 31) / 32, B, (N + 31) / 32), 256, 0, c->st>>>(
        V, c->nn, N, 0, N, N, 0, w->plane_stride, N, w->ldp, w->rplanes, w->ER1, N, c->d_flag, c->d_perm, N);
    OzArgs a{};
    a.pt[0] = oz_part(N, 0, w->E, N, V, c->nn, N);
    a.nparts = 1;
    a.Nn = N;
    a.batch = B;
    a.nk = w->ldp / OKE;
    a.EB = w->ER1;
    a.sEB = N;
    a.a_tri = 1;  // T is upper triangular: tile rows m0.. need K >= m0 only
    a.flag = c->d_flag;
    prof_begin(c, SLDQMC_KC_GEMM_OZ, (double)N * N * (N + 1) * B, "oz_update_V");
    k_oz_gemm<false, false><<<oz_grid<false>(w, a), OTHREADS, oz_smem_bytes(), c->st>>>(w->mapA, w->mapA, w->mapRB, a);
    prof_end(c);
    c->launches += 5;
}

// Keeps the current column bounds of R (a first Cholesky-QR pass) for the
// product R = R2 R1 after the second pass.
void oz_keep_bounds(sldqmc_ctx *c, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    cudaMemcpyAsync(w->ER1, w->ER, sizeof(int) * (size_t)B * c->N, cudaMemcpyDeviceToDevice, c->st);
}

// R = R2 R1 of the two Cholesky-QR passes (upper triangular, row stride N,
// item stride N*N; only the tiles on or above the diagonal of R are
// written), FP64-accurate on the tensor cores: R2's rows with their own
// maxima as exponents, R1's columns with the first pass's bounds.
void oz_r2r1(sldqmc_ctx *c, const double *R2, const double *R1, double *R, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    const int N = c->N;
    prof_begin(c, SLDQMC_KC_OTHER, 0.0, "k_oz_slice");
    k_oz_slice<<<dim3((N + 7) / 8, B), 256, 0, c->st>>>(R2, c->nn, N, N, N, N, w->ldp, w->plane_stride, w->planes,
                                                         w->E);
    prof_end(c);
    k_oz_slice_fixed<<<dim3((N + 31) / 32, B, (N + 31) / 32), 256, 0, c->st>>>(
        R1, c->nn, N, 0, N, N, 0, w->plane_stride, N, w->ldp, w->rplanes, w->ER1, N, c->d_flag);
    OzArgs a{};
    a.pt[0] = oz_part(N, 0, w->E, N, R, c->nn, N);
    a.nparts = 1;
    a.Nn = N;
    a.batch = B;
    a.nk = w->ldp / OKE;
    a.EB = w->ER1;
    a.sEB = N;
    a.a_tri = 1;  // R2[m][l] = 0 for l < m and R1[l][n] = 0 for l > n
    a.b_tri = 1;
    a.flag = c->d_flag;
    prof_begin(c, SLDQMC_KC_GEMM_OZ, (double)N * N * N / 3.0 * B, "oz_r2r1");
    k_oz_gemm<true, false><<<oz_grid<true>(w, a), OTHREADS, oz_smem_bytes(), c->st>>>(w->mapA, w->mapA, w->mapRB, a);
    prof_end(c);
    c->launches += 3;
}

}  // namespace sldqmc
