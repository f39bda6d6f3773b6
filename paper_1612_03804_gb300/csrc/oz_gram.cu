// oz_gram.cu -- FP64-accurate Gram matrices on the BF16 tensor cores
// (Ozaki's error-free splitting), for the Cholesky-QR of the mixed-precision
// modes.
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
// One persistent CTA per SM walks the 128 x 32 tiles on or above the
// diagonal of every item: warp 0 streams the 8 + 8 digit-plane tiles of a
// 32-wide K-block by TMA (64-byte swizzle), warp 1 issues the 36 MMAs per
// 16-wide K-step, and eight epilogue warps drain one of two tensor-memory
// buffers (8 groups x 32 columns each) while the next tile accumulates into
// the other.
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

// kind::f16 with BF16 operands, FP32 accumulator, K-major A and B, M = 128, N = 32.
constexpr uint32_t OZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OBN >> 3) << 17) |
                              ((uint32_t)(OBM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(OZ_IDESC), "r"(acc));
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

// Digits of every row of X (row-major N x N per item): E[b][i] and the planes
// (plane p at p * plane_stride, leading dimension ldp; columns N..ldp-1 stay
// zero).
__global__ void __launch_bounds__(128) k_oz_slice(const double *X, long long sX, int N, int ldp,
                                                  long long plane_stride, __nv_bfloat16 *planes, int *E)
{
    const int b = blockIdx.y, i = blockIdx.x;
    const double *x = X + (long long)b * sX + (long long)i * N;
    // the largest |x_ik| (non-negative doubles order like their bit patterns)
    unsigned long long mx = 0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(x[k]) & 0x7FFFFFFFFFFFFFFFull;
        mx = u > mx ? u : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
    }
    __shared__ unsigned long long red[4];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = red[w] > mx ? red[w] : mx;
    const int ef_max = (int)(mx >> 52);
    const int Ei = ef_max > 0 ? ef_max - 1022 : 0;
    if (threadIdx.x == 0) E[(long long)b * N + i] = Ei;
    const long long row = (long long)b * N * ldp + (long long)i * ldp;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        int dg[OZ_S];
        oz_digits(x[k], Ei, ef_max, dg);
#pragma unroll
        for (int p = 0; p < OZ_S; ++p)
            planes[(long long)p * plane_stride + row + k] = __float2bfloat16_rn((float)dg[p]);
    }
}

// Digits of krows rows of a row-major matrix (row stride ld), in blocks of 32
// rows (blockIdx.z), stored from K-block koff/32 of the planes on: plane row
// j (j0 <= j < Nc) gets src[l * ld + j] at K position koff + l (0 beyond
// krows within the last block).
// The exponents are given (Ej[b * sE + j]; sE = 0 for one shared row of
// exponents), chosen by the caller as bounds known before the values exist;
// a value at or above its bound raises the numerical flag.  One CTA converts
// 32 plane rows; eight threads share a row.
__global__ void __launch_bounds__(256) k_oz_slice_fixed(const double *src, long long sS, long long ld, int j0, int Nc,
                                                        int krows, int koff, long long plane_stride, int rows_cap,
                                                        int ldk, __nv_bfloat16 *planes, const int *Ej, long long sE,
                                                        int *flag, const int *rowidx = nullptr, long long sR = 0)
{
    __shared__ double tile[32][33];
    const int b = blockIdx.y, c0 = j0 + blockIdx.x * 32;
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
    if (j >= Nc) return;
    const int E = Ej[(long long)b * sE + j];
    const unsigned long long bound = (unsigned long long)(E + 1023) << 52;  // bit pattern of 2^E
    int dg[4][OZ_S];
    bool over = false;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
        const double x = tile[4 * q + jj][r];
        over |= ((unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull) >= bound;
        oz_digits(x, E, 1, dg[jj]);
    }
    if (over) atomicOr(flag, FLAG_NUMERICAL);
    const long long row = ((long long)b * rows_cap + j) * ldk + koff + 4 * q;
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) {
        __nv_bfloat162 h2[2] = {__floats2bfloat162_rn((float)dg[0][p], (float)dg[1][p]),
                                __floats2bfloat162_rn((float)dg[2][p], (float)dg[3][p])};
        *reinterpret_cast<uint2 *>(planes + (long long)p * plane_stride + row) = *reinterpret_cast<const uint2 *>(h2);
    }
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
// zero column): one thread per column, rows read coalesced across threads.
__global__ void k_oz_col_max_exponents(const double *src, long long sS, int rows, int cols, int *E)
{
    const int b = blockIdx.y;
    const double *s = src + (long long)b * sS;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cols; j += gridDim.x * blockDim.x) {
        unsigned long long mx = 0;
        for (int r = 0; r < rows; ++r) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(s[(long long)r * cols + j]) & 0x7FFFFFFFFFFFFFFFull;
            mx = u > mx ? u : mx;
        }
        const int ef = (int)(mx >> 52);
        E[(long long)b * cols + j] = ef > 0 ? ef - 1022 : 0;
    }
}

// T[m][k] = R[m][k] Dp[k] / D[m] for k >= m, 0 below (FP64), the triangular
// factor of the V update V <- T P^T V.
__global__ void k_oz_make_T(const double *R, long long nn, int N, const double *D, const double *Dp, double *T)
{
    const int b = blockIdx.z, m = blockIdx.y;
    const double rd = 1.0 / D[(long long)b * N + m];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x)
        T[(long long)b * nn + (long long)m * N + k] =
            k >= m ? R[(long long)b * nn + (long long)m * N + k] * Dp[(long long)b * N + k] * rd : 0.0;
}

struct OzArgs {
    int M, Nn;              // rows of A (rows of C) and rows of B (columns of C)
    int arow0, brow0;       // first plane rows of A and B (tensor-map row coordinates)
    int batch, nk;          // items, 32-wide K-blocks
    const int *EA, *EB;     // row exponents of A and B
    long long sEA, sEB;     // their item strides
    double *C;              // result: row stride ldc, item stride sC
    long long sC;
    int ldc;
    int *flag;
};

// Tile t of the persistent walk -> (item, first row, first column).  UPPER:
// the 128 x 32 tiles on or above the diagonal; otherwise every tile, columns
// fastest.
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
    int tm = 0;
    for (; tm < tiles_m; ++tm) {
        const int cnt = tiles_n - 4 * tm;
        if (r < cnt) break;
        r -= cnt;
    }
    m0 = tm * OBM;
    n0 = (4 * tm + r) * OBN;
}

template <bool UPPER>
__host__ __device__ inline int oz_per_item(int tiles_m, int tiles_n)
{
    if (!UPPER) return tiles_m * tiles_n;
    int n = 0;
    for (int tm = 0; tm < tiles_m; ++tm) n += tiles_n - 4 * tm;
    return n;
}

// UPPER: only the tiles on or above the diagonal (C square, A and B the same
// rows); SUB: C -= A B^T, otherwise C = A B^T; TRANS: element (m, n) of the
// product lives at C[n * ldc + m] (a warp's 32 rows m are then contiguous).
template <bool UPPER, bool SUB, bool TRANS = false>
__global__ void __launch_bounds__(OTHREADS, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, OzArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(base + OSTAGES * OSTAGE);
    uint64_t *empty = full + OSTAGES;
    uint64_t *tmem_full = empty + OSTAGES;  // [2]
    uint64_t *tmem_free = tmem_full + 2;    // [2]
    uint32_t *tmem_slot = (uint32_t *)(tmem_free + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = (a.M + OBM - 1) / OBM, tiles_n = (a.Nn + OBN - 1) / OBN;
    const int per_item = oz_per_item<UPPER>(tiles_m, tiles_n);
    const int tiles = per_item * a.batch;

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
                int b, m0, n0;
                oz_tile<UPPER>(t, tiles_m, tiles_n, per_item, b, m0, n0);
                for (int kb = 0; kb < a.nk; ++kb, ++it) {
                    const int s = it % OSTAGES;
                    if (it >= OSTAGES && !mbar_wait(&empty[s], ((it / OSTAGES) - 1) & 1, a.flag)) { ok = false; break; }
                    mbar_expect_tx(&full[s], OSTAGE);
                    uint8_t *st = base + s * OSTAGE;
                    const int k0 = kb * OKE;
#pragma unroll
                    for (int p = 0; p < OZ_S; ++p) {
                        tma_load_4d(st + p * OTILE_A, &tA, k0, a.arow0 + m0, b, p, &full[s]);
                        tma_load_4d(st + OZ_S * OTILE_A + p * OTILE_B, &tB, k0, a.brow0 + n0, b, p, &full[s]);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, cc = 0;  // K-block and chunk counters of this CTA
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                for (int kc0 = 0; kc0 < a.nk && ok; kc0 += OZ_KCHUNK, ++cc) {
                    const int u = cc & 1;
                    // the epilogue must have drained this buffer (used two chunks ago)
                    if (cc >= 2 && !mbar_wait(&tmem_free[u], ((cc >> 1) - 1) & 1, a.flag)) { ok = false; break; }
                    fence_after();
                    const uint32_t acc0 = tmem + (uint32_t)(u * OZ_G * OBN);
                    uint32_t started = 0;
                    const int kc1 = kc0 + OZ_KCHUNK < a.nk ? kc0 + OZ_KCHUNK : a.nk;
                    for (int kb = kc0; kb < kc1; ++kb, ++it) {
                        const int s = it % OSTAGES;
                        if (!mbar_wait(&full[s], (it / OSTAGES) & 1, a.flag)) { ok = false; break; }
                        fence_after();
                        const uint32_t sa = smem_u32(base + s * OSTAGE);
                        const uint32_t sb = sa + OZ_S * OTILE_A;
#pragma unroll
                        for (int k = 0; k < OKE / 16; ++k) {
#pragma unroll
                            for (int p = 0; p < OZ_S; ++p) {
                                const uint64_t da = smem_desc64(sa + p * OTILE_A + k * 32);
#pragma unroll
                                for (int q = 0; q < OZ_S - p; ++q) {
                                    const int g = p + q;
                                    mma_bf16(acc0 + (uint32_t)(g * OBN), da, smem_desc64(sb + q * OTILE_B + k * 32),
                                             (started >> g) & 1u);
                                    started |= 1u << g;
                                }
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
            int b, m0, n0;
            oz_tile<UPPER>(t, tiles_m, tiles_n, per_item, b, m0, n0);
            const int mm = m0 + q4 * 32 + lane;
            const int Ei = mm < a.M ? a.EA[(long long)b * a.sEA + mm] : 0;
            // element (mm, n) at o[n * cs]; for an update, the old values of this
            // thread's row segment, fetched while the MMAs run
            double *o = a.C + (long long)b * a.sC + (TRANS ? (long long)mm : (long long)mm * a.ldc);
            const long long cs = TRANS ? a.ldc : 1;
            const int nb = n0 + hc;
            const int *eb = a.EB + (long long)b * a.sEB;
            double cold[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) cold[j] = (SUB && mm < a.M && nb + j < a.Nn) ? o[(nb + j) * cs] : 0.0;
            // sum over K-chunks of the exactly accumulated chunk products
            double w[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) w[j] = 0.0;
            for (int kc0 = 0; kc0 < a.nk; kc0 += OZ_KCHUNK, ++cc) {
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
#pragma unroll
                    for (int j = 0; j < 8; ++j) w[half * 8 + j] += fma((double)l[j], 0x1p-28, (double)h[j]);
                }
                fence_before();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tmem_free[u])) : "memory");
                if (!ok) break;
            }
            if (!ok) break;
            if (mm >= a.M) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = nb + j;
                if (n < a.Nn) {
                    const int e = Ei + eb[n] - 35;
                    const double v = (e > -1000 && e < 1000) ? w[j] * __longlong_as_double((long long)(e + 1023) << 52)
                                                             : scalbn(w[j], e);
                    o[n * cs] = SUB ? cold[j] - v : v;
                }
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
    void *mem = nullptr;
    if (cudaMalloc(&mem, 2 * pbytes + 3 * ebytes + sizeof(int) * N) != cudaSuccess) {
        cudaGetLastError();
        delete w;
        return SLDQMC_ERR_OOM;
    }
    w->planes = (__nv_bfloat16 *)mem;
    w->rplanes = (__nv_bfloat16 *)((uint8_t *)mem + pbytes);
    w->E = (int *)((uint8_t *)mem + 2 * pbytes);
    w->ER = w->E + (size_t)c->cap * N;
    w->ER1 = w->ER + (size_t)c->cap * N;
    w->EQ = w->ER1 + (size_t)c->cap * N;
    cudaMemsetAsync(mem, 0, 2 * pbytes + 3 * ebytes, c->st);  // zero pads: never written
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
        !encode4(&w->mapRB, w->rplanes, w->ldp, N, c->cap, OBN)) {
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

// W = X X^T (rows of X: row stride N, batch stride sX); W row stride ldw,
// batch stride sW.  Tiles on or above the diagonal are written in full.
void oz_gram(sldqmc_ctx *c, const double *X, long long sX, double *W, long long sW, int ldw, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    const int N = c->N;
    k_oz_slice<<<dim3(N, B), 128, 0, c->st>>>(X, sX, N, w->ldp, w->plane_stride, w->planes, w->E);
    OzArgs a{};
    a.M = N;
    a.Nn = N;
    a.batch = B;
    a.nk = w->ldp / OKE;
    a.EA = w->E;
    a.EB = w->E;
    a.sEA = N;
    a.sEB = N;
    a.C = W;
    a.sC = sW;
    a.ldc = ldw;
    a.flag = c->d_flag;
    const int tiles = oz_per_item<true>((N + OBM - 1) / OBM, (N + OBN - 1) / OBN) * B;
    const int grid = tiles < w->num_sms ? tiles : w->num_sms;
    prof_begin(c, SLDQMC_KC_GEMM_OZ, (double)N * N * (N + 1) * B);
    k_oz_gemm<true, false><<<grid, OTHREADS, oz_smem_bytes(), c->st>>>(w->mapA, w->mapB, a);
    prof_end(c);
    c->launches += 2;
}

// Left-looking Cholesky-QR of W = X X^T (row stride N, item stride sW) that
// forms Q^T = R^-T X^T in Y (row stride N, item stride N*N): before the panel
// of rows k0..k0+kb the products of all finished rows are subtracted from the
// panel's rows,
//   W[k0+r][k0+n] -= sum_{l<k0} R[l][k0+n] R[l][k0+r],
//   Y[k0+r][n]    -= sum_{l<k0} Q^T[l][n] R[l][k0+r],
// both FP64-accurate on the tensor cores (the product computed with rows n and
// columns r, stored transposed so that a warp's stores are contiguous); after
// the panel its rows of R and Q^T are split into K-block k0/32 of the digit
// planes.  oz_chol_begin fixes the exponents of R's columns from W's diagonal.
void oz_chol_begin(sldqmc_ctx *c, const double *W, long long sW, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    const int N = c->N;
    k_oz_col_exponents<<<dim3((N + 255) / 256, B), 256, 0, c->st>>>(W, sW, N, N, w->ER);
    c->launches++;
}

void oz_chol_update(sldqmc_ctx *c, int k0, int kb, double *W, long long sW, double *Y, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    const int N = c->N;
    OzArgs a{};
    a.batch = B;
    a.nk = k0 / OKE;
    a.flag = c->d_flag;
    a.brow0 = k0;
    a.EB = w->ER + k0;
    a.sEB = N;
    a.Nn = kb;
    // Y rows k0.. : product rows n = columns of Q^T (all N)
    a.M = N;
    a.arow0 = 0;
    a.EA = w->EQ;
    a.sEA = 0;
    a.C = Y + (long long)k0 * N;
    a.sC = c->nn;
    a.ldc = N;
    int tiles = oz_per_item<false>((N + OBM - 1) / OBM, 1) * B;
    int grid = tiles < w->num_sms ? tiles : w->num_sms;
    prof_begin(c, SLDQMC_KC_GEMM_OZ, 2.0 * N * kb * k0 * B);
    k_oz_gemm<false, true, true><<<grid, OTHREADS, oz_smem_bytes(), c->st>>>(w->mapA, w->mapRB, a);
    prof_end(c);
    // W rows k0.. : product rows n = columns k0.. of R
    const int M = N - k0;
    a.M = M;
    a.arow0 = k0;
    a.EA = w->ER + k0;
    a.sEA = N;
    a.C = W + (long long)k0 * N + k0;
    a.sC = sW;
    tiles = oz_per_item<false>((M + OBM - 1) / OBM, 1) * B;
    grid = tiles < w->num_sms ? tiles : w->num_sms;
    prof_begin(c, SLDQMC_KC_GEMM_OZ, 2.0 * M * kb * k0 * B);
    k_oz_gemm<false, true, true><<<grid, OTHREADS, oz_smem_bytes(), c->st>>>(w->mapRA, w->mapRB, a);
    prof_end(c);
    c->launches += 2;
}

// V <- T P^T V with T = D^-1 R D_p (upper triangular; R row stride N),
// FP64-accurate on the tensor cores: T's rows split with their own maxima,
// the gathered rows V[p_k] split column-wise with each column's maximum.
// Ts: an N x N FP64 scratch per item (item stride N*N).
void oz_update_V(sldqmc_ctx *c, const double *R, double *V, double *Ts, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    const int N = c->N;
    k_oz_make_T<<<dim3((N + 255) / 256, N, B), 256, 0, c->st>>>(R, c->nn, N, c->d_D, c->d_Dp, Ts);
    k_oz_slice<<<dim3(N, B), 128, 0, c->st>>>(Ts, c->nn, N, w->ldp, w->plane_stride, w->planes, w->E);
    k_oz_col_max_exponents<<<dim3((N + 127) / 128, B), 128, 0, c->st>>>(V, c->nn, N, N, w->ER1);
    k_oz_slice_fixed<<<dim3((N + 31) / 32, B, (N + 31) / 32), 256, 0, c->st>>>(
        V, c->nn, N, 0, N, N, 0, w->plane_stride, N, w->ldp, w->rplanes, w->ER1, N, c->d_flag, c->d_perm, N);
    OzArgs a{};
    a.M = N;
    a.Nn = N;
    a.batch = B;
    a.nk = w->ldp / OKE;
    a.EA = w->E;
    a.EB = w->ER1;
    a.sEA = N;
    a.sEB = N;
    a.C = V;
    a.sC = c->nn;
    a.ldc = N;
    a.flag = c->d_flag;
    const int tiles = oz_per_item<false>((N + OBM - 1) / OBM, (N + OBN - 1) / OBN) * B;
    const int grid = tiles < w->num_sms ? tiles : w->num_sms;
    prof_begin(c, SLDQMC_KC_GEMM_OZ, (double)N * N * (N + 1) * B);
    k_oz_gemm<false, false><<<grid, OTHREADS, oz_smem_bytes(), c->st>>>(w->mapA, w->mapRB, a);
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
    k_oz_slice<<<dim3(N, B), 128, 0, c->st>>>(R2, c->nn, N, w->ldp, w->plane_stride, w->planes, w->E);
    k_oz_slice_fixed<<<dim3((N + 31) / 32, B, (N + 31) / 32), 256, 0, c->st>>>(
        R1, c->nn, N, 0, N, N, 0, w->plane_stride, N, w->ldp, w->rplanes, w->ER1, N, c->d_flag);
    OzArgs a{};
    a.M = N;
    a.Nn = N;
    a.batch = B;
    a.nk = w->ldp / OKE;
    a.EA = w->E;
    a.EB = w->ER1;
    a.sEA = N;
    a.sEB = N;
    a.C = R;
    a.sC = c->nn;
    a.ldc = N;
    a.flag = c->d_flag;
    const int tiles = oz_per_item<true>((N + OBM - 1) / OBM, (N + OBN - 1) / OBN) * B;
    const int grid = tiles < w->num_sms ? tiles : w->num_sms;
    prof_begin(c, SLDQMC_KC_GEMM_OZ, (double)N * N * N / 3.0 * B);
    k_oz_gemm<true, false><<<grid, OTHREADS, oz_smem_bytes(), c->st>>>(w->mapA, w->mapRB, a);
    prof_end(c);
    c->launches += 3;
}

void oz_chol_slice(sldqmc_ctx *c, int k0, int kb, const double *R, const double *Y, int B)
{
    OzWs *w = (OzWs *)c->oz_ws;
    const int N = c->N;
    // R's rows k0..k0+kb, columns k0+kb.. (the ones later panels read)
    const int j0 = k0 + kb;
    k_oz_slice_fixed<<<dim3((N - j0 + 31) / 32, B), 256, 0, c->st>>>(R + (long long)k0 * N, c->nn, N, j0, N, kb, k0,
                                                                    w->plane_stride, N, w->ldp, w->rplanes, w->ER, N,
                                                                    c->d_flag);
    // Q^T's rows k0..k0+kb, all columns
    k_oz_slice_fixed<<<dim3((N + 31) / 32, B), 256, 0, c->st>>>(Y + (long long)k0 * N, c->nn, N, 0, N, kb, k0,
                                                               w->plane_stride, N, w->ldp, w->planes, w->EQ, 0,
                                                               c->d_flag);
    c->launches += 2;
}

}  // namespace sldqmc
