// tc_gemm.cu -- tensor-core slice products for the mixed-precision modes.
//
// Inside one stabilisation block the running product is X^T <- X^T E
// diag(d_next), with E = exp(-dtau K) (symmetric) and d the field scale of
// the next slice (B_tau = E diag(exp(eta dtau xi s_tau))).  Both operands are
// K-major, so the product maps directly onto tcgen05.mma:
//
//   split TF32 ("3xTF32" mode): the running product is split in two TF32
//           parts A = A_h + A_l; E, which every slice reuses, in three
//           (E_h + E_m + E_l) so that its representation error (systematic
//           across slices) falls to 2^-33; A E ~ A_h E_h + A_h E_m + A_l E_h
//           + A_h E_l + A_l E_m, five kind::tf32 products per K-step;
//   split BF16 ("bf16x3" mode): both operands in three BF16 parts, the six
//           products a0e0 + a0e1 + a1e0 + a0e2 + a1e1 + a2e0 as kind::f16 MMAs;
//   BF16:   one kind::f16 MMA with BF16 operands.
//
// The tensor cores accumulate in FP32 with a rounding that is not
// round-to-nearest, so the error of one accumulator grows with the number
// of MMAs it receives.  Each CTA therefore spreads its K-steps round-robin
// over several accumulators in tensor memory (512 columns) and adds them in
// the epilogue.  The leading products use all accumulators but the last,
// which the small correction products share (seven and one with 128 x 64
// tiles, three and one with 128 x 128).
//
// A persistent CTA per SM walks the 128 x 64 output tiles of the batch:
// warp 0 drives TMA (128-byte swizzled boxes, mbarrier completion) without
// stopping at tile boundaries, warp 1 issues the MMAs from one thread, and
// eight epilogue warps drain the accumulators with tcgen05.ld, hand tensor
// memory back, and then apply the next slice's column scaling (as a float
// pair, so that the scale constant adds no systematic error) while
// re-splitting the result into the operand format of the next product (or
// FP64 for the stabilisation at the end of the block).  Every mbarrier wait
// is bounded; a wait that runs out raises the context's timeout flag and the
// CTA frees its tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_common.cuh"

namespace sldqmc {

namespace {

using namespace tcx;

// Output tiles are BM x BN with BN = 64 (eight accumulators) or BN = 128
// (four accumulators: half the shared-memory operand reads per flop, one
// accumulator for every three leading products instead of every seven).
// Both fill the 512 tensor-memory columns.
constexpr int BM = 128, BN = 64;
constexpr int TILE_A = BM * 128;  // one A part of one stage: 128 rows x 128 bytes
constexpr int TMEM_COLS = 512;
template <int BNT> struct TileCfg {
    static constexpr int NACC = TMEM_COLS / BNT;  // accumulators
    static constexpr int TILE_B = BNT * 128;      // one B part of one stage: BNT rows x 128 bytes
};

struct TcArgs {
    int N, ldp, nk, batch;
    int kseg;      // K-blocks per accumulation segment: the epilogue drains and sums the
                   // accumulators after each segment (bounds the MMAs per accumulator)
    void *out[3];  // next operand, split in parts (FP32 for split TF32, BF16 otherwise)
    double *out_f64;
    long long s_out, s_f64;
    const int8_t *s_n;
    long long sSn;
    float cu_h, cu_l, cd_h, cd_l;  // scale constants as float pairs
    int *flag;
};

// Exercises the bounded-wait path: waits on an mbarrier that nothing
// arrives at, so the wait must run out, raise the flag and return.
__global__ void k_wait_selftest(int *flag, int limit)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, flag, limit);
}

// Shared-memory matrix descriptor for a K-major operand stored as 128-byte
// rows with the 128-byte swizzle (8-row atoms of 1024 bytes).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address
    d |= (uint64_t)1u << 16;                   // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;         // stride byte offset: 8 rows x 128 bytes
    d |= (uint64_t)1u << 46;                   // descriptor version
    d |= (uint64_t)2u << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulator, K-major A and B, M = 128, N = BNT.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t ab_format, int BNT)
{
    return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(BNT >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    if (MODE == 0)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Modes: 0 = split TF32 (A in 2 parts, E in 3, five kind::tf32 MMAs per
// 8-wide K-step); 1 = BF16 (one kind::f16 MMA per 16-wide K-step); 2 = split
// BF16 (A and E in 3 BF16 parts each, six kind::f16 MMAs per 16-wide K-step).
template <int MODE> struct ModeCfg;
template <> struct ModeCfg<0> { static constexpr int NPA = 2, NPB = 3, KELEM = 32; static constexpr uint32_t FMT = 2; };
template <> struct ModeCfg<1> { static constexpr int NPA = 1, NPB = 1, KELEM = 64; static constexpr uint32_t FMT = 1; };
template <> struct ModeCfg<2> { static constexpr int NPA = 3, NPB = 3, KELEM = 64; static constexpr uint32_t FMT = 1; };

template <int MODE, int BNT>
__host__ __device__ constexpr int stage_bytes() { return ModeCfg<MODE>::NPA * TILE_A + ModeCfg<MODE>::NPB * TileCfg<BNT>::TILE_B; }
// pipeline stages: 64-wide tiles 3 (split modes) or 5 (BF16), measured best;
// 128-wide tiles as many as fit in 227 KB, at most five
template <int MODE, int BNT>
__host__ __device__ constexpr int stages()
{
    return BNT == 64 ? (MODE == 1 ? 5 : 3)
                     : ((227 * 1024 - 1024 - 256) / stage_bytes<MODE, BNT>() < 5
                            ? (227 * 1024 - 1024 - 256) / stage_bytes<MODE, BNT>()
                            : 5);
}

// Persistent kernel: one CTA per SM loops over the 128 x 64 output tiles of
// the whole batch (tile t = blockIdx.x, blockIdx.x + gridDim.x, ...).
// Warp 0 (one thread) streams TMA stages continuously across tile
// boundaries; warp 1 (one thread) issues the MMAs of a tile once the
// epilogue has handed tensor memory back; the epilogue warps (two per TMEM
// lane quarter, each owning half of the tile's columns) drain the
// accumulators into registers, hand tensor memory back at once, and then
// scale, re-split and store while the MMAs of the next tile run.
constexpr int EPI_WARPS = 8;                     // epilogue warps: EPI_WARPS / 4 per TMEM lane quarter
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;

__device__ __forceinline__ __nv_bfloat16 bf16_rn(float x) { return __float2bfloat16_rn(x); }

// Stores one 16-column row segment of an operand part: FP32 (split TF32) or
// BF16 (rounded here; the leading parts are BF16 values already).  `full`
// segments are 16-element aligned; a ragged one writes its first `rem`.
template <int MODE>
__device__ __forceinline__ void store_part(void *base, long long o, const float (&pp)[16], bool full, int rem)
{
    if (MODE == 0) {
        float *dst = static_cast<float *>(base) + o;
        if (full) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                reinterpret_cast<float4 *>(dst)[k] = make_float4(pp[4 * k], pp[4 * k + 1], pp[4 * k + 2], pp[4 * k + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (j < rem) dst[j] = pp[j];
        }
    } else {
        __nv_bfloat16 *dst = static_cast<__nv_bfloat16 *>(base) + o;
        if (full) {
            uint4 w[2];
            __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(w);
#pragma unroll
            for (int k = 0; k < 8; ++k) h2[k] = __floats2bfloat162_rn(pp[2 * k], pp[2 * k + 1]);
            reinterpret_cast<uint4 *>(dst)[0] = w[0];
            reinterpret_cast<uint4 *>(dst)[1] = w[1];
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (j < rem) dst[j] = bf16_rn(pp[j]);
        }
    }
}

// Tile t of the persistent walk -> (item, row strip, column strip).  Within
// an item the tiles go in groups of TILE_GROUP_M row strips, column-major
// inside a group: the CTAs of one wave (consecutive t) then share a few
// 128-row strips of the running product and a few strips of E, rather than
// one strip of the first and a different strip of E each.  At N = 10^4 the
// three parts of E (1.2 GB) far exceed L2, and walking columns first
// streamed E from HBM about once per row strip: at N = 4096 (two items) the
// grouped walk reads 2.7 instead of 5.8 GB from DRAM per product, in the
// same time (the kernel is bound by its shared-memory operand traffic).
constexpr int TILE_GROUP_M = 8;

__device__ __forceinline__ void tc_tile(int t, int tiles_m, int tiles_n, int &b, int &tm, int &tn)
{
    const int per_item = tiles_m * tiles_n;
    b = t / per_item;
    const int r = t - b * per_item;
    const int g = r / (TILE_GROUP_M * tiles_n);
    const int m_first = g * TILE_GROUP_M;
    const int gm = tiles_m - m_first < TILE_GROUP_M ? tiles_m - m_first : TILE_GROUP_M;
    const int rr = r - g * TILE_GROUP_M * tiles_n;
    tm = m_first + rr % gm;
    tn = rr / gm;
}

template <int MODE, int BNT>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
              const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tB0,
              const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB2, TcArgs a)
{
    using C = ModeCfg<MODE>;
    constexpr int BN = BNT;
    constexpr int NACC = TileCfg<BNT>::NACC;
    constexpr int TILE_B = TileCfg<BNT>::TILE_B;
    constexpr int EPI_COLS = BN * 4 / EPI_WARPS;  // accumulator columns drained by one epilogue warp
    static_assert(EPI_COLS % 16 == 0 && EPI_COLS <= 64, "epilogue warps drain 16-column chunks");
    constexpr int STAGE_BYTES = stage_bytes<MODE, BNT>();
    constexpr int STAGES = stages<MODE, BNT>();
    constexpr int KSTEPS = 4;  // 128-byte row / 32 bytes per MMA K-step (8 TF32 or 16 BF16)
    constexpr uint32_t IDESC = instr_desc(C::FMT, BNT);
    constexpr bool SPLIT = MODE != 1;  // leading products on accumulators 0..NACC-2, corrections on the last

    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(base + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tmem_full = empty + STAGES;
    uint64_t *tmem_free = tmem_full + 1;
    uint32_t *tmem_slot = (uint32_t *)(tmem_free + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_n = (a.N + BN - 1) / BN, tiles_m = (a.N + BM - 1) / BM;
    const int tiles = tiles_n * tiles_m * a.batch;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tmem_full, 1);
        mbar_init(tmem_free, 32 * EPI_WARPS);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;  // global k-block counter of this CTA
            bool ok = true;
            const CUtensorMap *mA[3] = {&tA0, &tA1, &tA2};
            const CUtensorMap *mB[3] = {&tB0, &tB1, &tB2};
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                int b, tm, tn;
                tc_tile(t, tiles_m, tiles_n, b, tm, tn);
                const int n0 = tn * BN, m0 = tm * BM;
                for (int kb = 0; kb < a.nk; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (it >= STAGES && !mbar_wait(&empty[s], ((it / STAGES) - 1) & 1, a.flag)) { ok = false; break; }
                    mbar_expect_tx(&full[s], STAGE_BYTES);
                    uint8_t *st = base + s * STAGE_BYTES;
                    const int k0 = kb * C::KELEM;
#pragma unroll
                    for (int p = 0; p < C::NPA; ++p) tma_load_3d(st + p * TILE_A, mA[p], k0, m0, b, &full[s]);
#pragma unroll
                    for (int q = 0; q < C::NPB; ++q) {
                        tma_load_2d(st + C::NPA * TILE_A + q * TILE_B, mB[q], k0, n0, &full[s]);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, sc = 0;  // K-block and segment counters of this CTA
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
              for (int s0 = 0; s0 < a.nk && ok; s0 += a.kseg, ++sc) {
                // the epilogue must have drained the previous segment's accumulators
                if (sc > 0 && !mbar_wait(tmem_free, (sc - 1) & 1, a.flag)) { ok = false; break; }
                fence_after();
                const int s1 = s0 + a.kseg < a.nk ? s0 + a.kseg : a.nk;
                for (int kb = s0; kb < s1; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!mbar_wait(&full[s], (it / STAGES) & 1, a.flag)) { ok = false; break; }
                    fence_after();
                    const uint32_t sa = smem_u32(base + s * STAGE_BYTES);
                    const uint32_t sb = sa + C::NPA * TILE_A;
#pragma unroll
                    for (int k = 0; k < KSTEPS; ++k) {
                        const uint32_t off = k * 32;
                        const int g = (kb - s0) * KSTEPS + k;  // step within the segment
                        if (SPLIT) {
                            // The leading product round-robin over accumulators 0..NACC-2;
                            // the small correction products all go to the last accumulator,
                            // where their rounding is relative to a much smaller sum.
                            const uint32_t acc_main = tmem + (uint32_t)((g % (NACC - 1)) * BN);
                            const uint32_t acc_small = tmem + (uint32_t)((NACC - 1) * BN);
                            const uint64_t a0 = smem_desc(sa + off), a1 = smem_desc(sa + TILE_A + off);
                            const uint64_t e0 = smem_desc(sb + off), e1 = smem_desc(sb + TILE_B + off),
                                           e2 = smem_desc(sb + 2 * TILE_B + off);
                            mma<MODE == 0 ? 0 : 1>(acc_main, a0, e0, IDESC, g < NACC - 1 ? 0u : 1u);
                            mma<MODE == 0 ? 0 : 1>(acc_small, a0, e1, IDESC, g == 0 ? 0u : 1u);
                            mma<MODE == 0 ? 0 : 1>(acc_small, a1, e0, IDESC, 1u);
                            mma<MODE == 0 ? 0 : 1>(acc_small, a0, e2, IDESC, 1u);
                            mma<MODE == 0 ? 0 : 1>(acc_small, a1, e1, IDESC, 1u);
                            if (MODE == 2) {
                                const uint64_t a2 = smem_desc(sa + 2 * TILE_A + off);
                                mma<1>(acc_small, a2, e0, IDESC, 1u);
                            }
                        } else {
                            const uint32_t acc_t = tmem + (uint32_t)((g % NACC) * BN);
                            mma<1>(acc_t, smem_desc(sa + off), smem_desc(sb + off), IDESC, g < NACC ? 0u : 1u);
                        }
                    }
                    mma_commit(&empty[s]);
                }
                if (ok) mma_commit(tmem_full);
              }
            }
        }
    } else {
        // epilogue warps: warp w drains TMEM lane quarter w % 4 (rows), columns
        // [cb, cb + EPI_COLS) of the tile; each thread owns one row.
        const int q4 = warp & 3;
        const int cb = ((warp - 2) >> 2) * EPI_COLS;
        int sc = 0;  // segment counter, in step with the MMA thread's
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            int b, tm, tn;
            tc_tile(t, tiles_m, tiles_n, b, tm, tn);
            const int n0 = tn * BN, m0 = tm * BM;
            // Column scale signs of this warp's columns as a 64-bit mask,
            // fetched before the accumulators are ready.
            uint64_t up_mask = 0;
            const int8_t *sn = a.s_n ? a.s_n + (long long)b * a.sSn : nullptr;
            if (sn) {
                const int c0w = n0 + cb;
                const bool u0 = lane < EPI_COLS && c0w + lane < a.N && sn[c0w + lane] > 0;
                const bool u1 = 32 + lane < EPI_COLS && c0w + 32 + lane < a.N && sn[c0w + 32 + lane] > 0;
                up_mask = (uint64_t)__ballot_sync(0xffffffffu, u0) | ((uint64_t)__ballot_sync(0xffffffffu, u1) << 32);
            }
            // Drain this warp's accumulator columns into registers after every
            // segment (summed over the accumulators; each received MMAs in every
            // segment), handing tensor memory back each time, so that the next
            // segment's or tile's MMAs run while this tile is scaled, split and
            // stored.
            float v[EPI_COLS / 16][16];
#pragma unroll
            for (int c = 0; c < EPI_COLS / 16; ++c)
#pragma unroll
                for (int j = 0; j < 16; ++j) v[c][j] = 0.0f;
            bool ok = true;
            for (int s0 = 0; s0 < a.nk; s0 += a.kseg, ++sc) {
                ok = mbar_wait(tmem_full, sc & 1, a.flag);
                fence_after();
#pragma unroll
                for (int c = 0; c < EPI_COLS / 16; ++c) {
                    const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(cb + c * 16);
#pragma unroll
                    for (int q = 0; q < NACC; q += 2) {
                        uint32_t r0[16], r1[16];
                        tmem_ld16_nowait(lane_base + (uint32_t)(q * BN), r0);
                        tmem_ld16_nowait(lane_base + (uint32_t)((q + 1) * BN), r1);
                        tmem_wait_ld32(r0, r1);
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[c][j] += __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
                    }
                }
                fence_before();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tmem_free)) : "memory");
                if (!ok) break;
            }
            if (!ok) break;  // a wait ran out: the flag is raised, stop instead of waiting per tile
            const int mm = m0 + q4 * 32 + lane;
#pragma unroll
            for (int c = 0; c < EPI_COLS / 16; ++c) {
                const int c0 = cb + c * 16;
                const int nb = n0 + c0;
                if (nb >= a.N || mm >= a.N) continue;
                const bool full = nb + 16 <= a.N;
                if (a.out_f64) {
                    const long long off = (long long)b * a.s_f64 + (long long)mm * a.N + nb;
                    double *o = a.out_f64 + off;
                    if (full && (off & 1) == 0) {  // 16-byte aligned (the buffer itself is)
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            reinterpret_cast<double2 *>(o)[k] = make_double2((double)v[c][2 * k], (double)v[c][2 * k + 1]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (nb + j < a.N) o[j] = (double)v[c][j];
                    }
                    continue;
                }
                float p0[16], p1[16], p2[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    // y = v * d with d = dh + dl: yh = fl(v dh), ye = the rounding error of
                    // that product (exact by FMA) plus v dl.
                    const float x = v[c][j];
                    float yh = x, ye = 0.0f;
                    if (sn) {
                        const bool up = (up_mask >> (c * 16 + j)) & 1u;
                        const float dh = up ? a.cu_h : a.cd_h, dl = up ? a.cu_l : a.cd_l;
                        yh = x * dh;
                        ye = fmaf(x, dh, -yh) + x * dl;
                    }
                    if (MODE == 0) {
                        p0[j] = to_tf32(yh);
                        p1[j] = to_tf32((yh - p0[j]) + ye);
                    } else if (MODE == 1) {
                        p0[j] = yh + ye;
                    } else {
                        p0[j] = __bfloat162float(bf16_rn(yh));
                        const float r1 = (yh - p0[j]) + ye;
                        p1[j] = __bfloat162float(bf16_rn(r1));
                        p2[j] = r1 - p1[j];
                    }
                }
                const long long o = (long long)b * a.s_out + (long long)mm * a.ldp + nb;
                store_part<MODE>(a.out[0], o, p0, full, a.N - nb);
                if (MODE != 1) store_part<MODE>(a.out[1], o, p1, full, a.N - nb);
                if (MODE == 2) store_part<MODE>(a.out[2], o, p2, full, a.N - nb);
            }
        }
    }
    __syncwarp();
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Split of an FP64 matrix (times an optional K-index field scale) into the
// operand parts of a mode: the first product of a block (Ut diag(d_first))
// and, once per context, E itself.
template <int MODE>
__global__ void k_tc_split(const double *X, long long sX, int N, int ldp, const int8_t *s_k, long long sSk, double cu,
                           double cd, void *o0, void *o1, void *o2, long long s_out, int e_parts)
{
    const int b = blockIdx.z, m = blockIdx.y;
    const int8_t *sk = s_k ? s_k + (long long)b * sSk : nullptr;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        double v = X[(long long)b * sX + (long long)m * N + k];
        if (sk) v *= (sk[k] > 0 ? cu : cd);
        const long long o = (long long)b * s_out + (long long)m * ldp + k;
        if (MODE == 0) {
            const float h = to_tf32((float)v);
            const double r1 = v - (double)h;
            const float mid = to_tf32((float)r1);
            static_cast<float *>(o0)[o] = h;
            static_cast<float *>(o1)[o] = mid;
            if (e_parts == 3) static_cast<float *>(o2)[o] = to_tf32((float)(r1 - (double)mid));
        } else if (MODE == 1) {
            static_cast<__nv_bfloat16 *>(o0)[o] = bf16_rn((float)v);
        } else {
            const __nv_bfloat16 p0 = bf16_rn((float)v);
            const double r1 = v - (double)__bfloat162float(p0);
            const __nv_bfloat16 p1 = bf16_rn((float)r1);
            const __nv_bfloat16 p2 = bf16_rn((float)(r1 - (double)__bfloat162float(p1)));
            static_cast<__nv_bfloat16 *>(o0)[o] = p0;
            static_cast<__nv_bfloat16 *>(o1)[o] = p1;
            static_cast<__nv_bfloat16 *>(o2)[o] = p2;
        }
    }
}

struct TcWs {
    int mode, ldp, npa, npb, esz;
    size_t part_elems;       // per operand part: cap * N * ldp
    void *op[2][3];          // [ping-pong buffer][part]
    void *Ep[3];             // E in parts
    CUtensorMap mapA[2][3];  // [buffer][part]
    CUtensorMap mapB[3];     // [part], 64-row boxes
    CUtensorMap mapB128[3];  // [part], 128-row boxes
    int bn;                  // output tile width of the slice products: 64 or 128
    void *mem;
    int num_sms;
};

bool encode(CUtensorMap *map, void *ptr, bool bf16, int rank, int ldp, int rows, int batch, int box_rows)
{
    auto fn = get_encode();
    if (!fn) return false;
    const int esz = bf16 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)ldp, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)ldp * esz, (cuuint64_t)ldp * rows * esz};
    cuuint32_t box[3] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank,
                    ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int MODE, int BNT>
constexpr size_t smem_bytes()
{
    // stages, alignment, barriers
    return (size_t)stages<MODE, BNT>() * stage_bytes<MODE, BNT>() + 1024 + 256;
}

int mode_of(const sldqmc_ctx *c) { return c->p.prec == SLDQMC_3XTF32 ? 0 : (c->p.prec == SLDQMC_BF16 ? 1 : 2); }

template <int MODE>
void launch_split(sldqmc_ctx *c, const TcWs *w, const double *X, long long sX, int B, const int8_t *s_k, long long sSk,
                  double cu, double cd, void *const *o, long long s_out, int e_parts)
{
    dim3 g((c->N + 255) / 256, c->N, B);
    k_tc_split<MODE><<<g, 256, 0, c->st>>>(X, sX, c->N, w->ldp, s_k, sSk, cu, cd, o[0], o[1], o[2], s_out, e_parts);
    c->launches++;
}

template <int MODE>
void launch_gemm(sldqmc_ctx *c, const TcWs *w, int src, int grid, const TcArgs &a)
{
    const CUtensorMap *A = w->mapA[src];
    if (w->bn == 128) {
        const CUtensorMap *E = w->mapB128;
        k_tc_gemm<MODE, 128><<<grid, NTHREADS, smem_bytes<MODE, 128>(), c->st>>>(A[0], A[1], A[2], E[0], E[1], E[2], a);
    } else {
        const CUtensorMap *E = w->mapB;
        k_tc_gemm<MODE, 64><<<grid, NTHREADS, smem_bytes<MODE, 64>(), c->st>>>(A[0], A[1], A[2], E[0], E[1], E[2], a);
    }
}

}  // namespace

void launch_wait_selftest(sldqmc_ctx *c, int limit)
{
    k_wait_selftest<<<1, 32, 0, c->st>>>(c->d_flag, limit);
    c->launches++;
}

int tc_prepare(sldqmc_ctx *c)
{
    if (c->N < BM) return SLDQMC_ERR_UNSUPPORTED;  // tensor-core tiles are 128 rows
    TcWs *w = new TcWs();
    c->tc_ws = w;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        w->num_sms = 0;
        if (cudaDeviceGetAttribute(&w->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || w->num_sms < 1)
            w->num_sms = 148;
    }
    const int N = c->N;
    w->mode = mode_of(c);
    w->ldp = (N + 63) / 64 * 64;
    w->npa = w->mode == 0 ? 2 : (w->mode == 1 ? 1 : 3);
    w->npb = w->mode == 0 ? 3 : (w->mode == 1 ? 1 : 3);
    w->esz = w->mode == 0 ? 4 : 2;
    const bool bf = w->mode != 0;
    w->part_elems = (size_t)c->cap * N * w->ldp;
    const size_t bytes = (size_t)w->esz * (2 * w->npa * w->part_elems + (size_t)w->npb * N * w->ldp);
    if (cudaMalloc(&w->mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        w->mem = nullptr;
        return SLDQMC_ERR_OOM;
    }
    // zero pads (columns N..ldp-1 are never written), ordered before the
    // context's first kernels on its own stream
    cudaMemsetAsync(w->mem, 0, bytes, c->st);
    uint8_t *q = (uint8_t *)w->mem;
    for (int i = 0; i < 2; ++i)
        for (int p = 0; p < 3; ++p) {
            if (p < w->npa) {
                w->op[i][p] = q;
                q += w->esz * w->part_elems;
                if (!encode(&w->mapA[i][p], w->op[i][p], bf, 3, w->ldp, N, c->cap, BM)) return SLDQMC_ERR_CUDA;
            } else {
                w->op[i][p] = nullptr;
                w->mapA[i][p] = w->mapA[i][0];
            }
        }
    for (int p = 0; p < 3; ++p) {
        if (p < w->npb) {
            w->Ep[p] = q;
            q += (size_t)w->esz * N * w->ldp;
            if (!encode(&w->mapB[p], w->Ep[p], bf, 2, w->ldp, N, 1, 64)) return SLDQMC_ERR_CUDA;
            if (!encode(&w->mapB128[p], w->Ep[p], bf, 2, w->ldp, N, 1, 128)) return SLDQMC_ERR_CUDA;
        } else {
            w->Ep[p] = nullptr;
            w->mapB[p] = w->mapB[0];
            w->mapB128[p] = w->mapB128[0];
        }
    }
    w->bn = 64;
    cudaFuncSetAttribute(k_tc_gemm<0, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<0, 64>());
    cudaFuncSetAttribute(k_tc_gemm<1, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<1, 64>());
    cudaFuncSetAttribute(k_tc_gemm<2, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<2, 64>());
    cudaFuncSetAttribute(k_tc_gemm<0, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<0, 128>());
    cudaFuncSetAttribute(k_tc_gemm<1, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<1, 128>());
    cudaFuncSetAttribute(k_tc_gemm<2, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<2, 128>());
    return SLDQMC_OK;
}

void tc_release(sldqmc_ctx *c)
{
    TcWs *w = (TcWs *)c->tc_ws;
    if (!w) return;
    cudaFree(w->mem);
    delete w;
    c->tc_ws = nullptr;
}

void tc_convert_E(sldqmc_ctx *c)
{
    TcWs *w = (TcWs *)c->tc_ws;
    void *o[3] = {w->Ep[0], w->Ep[1], w->Ep[2]};
    if (w->mode == 0) launch_split<0>(c, w, c->d_E, 0, 1, nullptr, 0, 1.0, 1.0, o, 0, 3);
    else if (w->mode == 1) launch_split<1>(c, w, c->d_E, 0, 1, nullptr, 0, 1.0, 1.0, o, 0, 1);
    else launch_split<2>(c, w, c->d_E, 0, 1, nullptr, 0, 1.0, 1.0, o, 0, 3);
}

// X^T = Ut D_{s0} E D_{s1} E ... D_{s_{nb-1}} E for one block; result (FP64)
// in Xt_out.
void tc_chain_block(sldqmc_ctx *c, const double *Ut, const int8_t *d_s, int B, double cu, double cd,
                    const int *slices, int nb, double *Xt_out, double *, double *)
{
    TcWs *w = (TcWs *)c->tc_ws;
    const int N = c->N, M = c->M;
    const long long sS = (long long)M * N;
    const long long s_out = (long long)N * w->ldp;
    {
        prof_begin(c, SLDQMC_KC_OTHER, 0.0, "tc_split");
        void *o[3] = {w->op[0][0], w->op[0][1], w->op[0][2]};
        const int8_t *sk = d_s + (long long)slices[0] * N;
        if (w->mode == 0) launch_split<0>(c, w, Ut, c->nn, B, sk, sS, cu, cd, o, s_out, 2);
        else if (w->mode == 1) launch_split<1>(c, w, Ut, c->nn, B, sk, sS, cu, cd, o, s_out, 1);
        else launch_split<2>(c, w, Ut, c->nn, B, sk, sS, cu, cd, o, s_out, 3);
        prof_end(c);
    }
    const int tiles = ((N + w->bn - 1) / w->bn) * ((N + BM - 1) / BM) * B;
    const int grid = tiles < w->num_sms ? tiles : w->num_sms;
    for (int j = 0; j < nb; ++j) {
        const int src = j & 1, dst = src ^ 1;
        TcArgs a{};
        a.N = N;
        a.ldp = w->ldp;
        a.nk = w->ldp / (w->mode == 0 ? 32 : 64);
        a.batch = B;
        a.s_out = s_out;
        a.s_f64 = c->nn;
        a.flag = c->d_flag;
        // 128-wide tiles (four accumulators) drain after each third of K, so that
        // an accumulator takes no more MMAs than in a 64-wide tile (eight
        // accumulators, one segment)
        a.kseg = w->bn == 128 ? (a.nk + 2) / 3 : a.nk;
        if (j == nb - 1) {
            a.out_f64 = Xt_out;
        } else {
            a.s_n = d_s + (long long)slices[j + 1] * N;
            a.sSn = sS;
            a.cu_h = (float)cu;
            a.cu_l = (float)(cu - (double)a.cu_h);
            a.cd_h = (float)cd;
            a.cd_l = (float)(cd - (double)a.cd_h);
            for (int p = 0; p < 3; ++p) a.out[p] = w->op[dst][p];
        }
        prof_begin(c, SLDQMC_KC_GEMM_TC, 2.0 * (double)N * N * N * B, "tc_gemm");
        if (w->mode == 0) launch_gemm<0>(c, w, src, grid, a);
        else if (w->mode == 1) launch_gemm<1>(c, w, src, grid, a);
        else launch_gemm<2>(c, w, src, grid, a);
        prof_end(c);
        c->launches++;
    }
}

}  // namespace sldqmc

namespace sldqmc {
int tc_set_tile_n(sldqmc_ctx *c, int bn)
{
    TcWs *w = (TcWs *)c->tc_ws;
    if (!w) return SLDQMC_ERR_UNSUPPORTED;
    if (bn != 64 && bn != 128) return SLDQMC_ERR_ARG;
    w->bn = bn;
    return SLDQMC_OK;
}
}  // namespace sldqmc
