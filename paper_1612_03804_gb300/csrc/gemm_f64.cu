// gemm_f64.cu -- batched FP64 GEMM on the FP64 FMA pipe of sm_103a.
//
// GB300 executes FP64 at roughly 1.1 TFLOP/s (about two DFMA per clock per
// SM), some 60x below its FP32 FMA rate and three orders of magnitude below
// its tensor cores.  An FP64 GEMM is therefore bound by the DFMA issue rate
// alone: a 64x64 tile with a 4x4 register block per thread needs one 8-byte
// shared-memory read per two DFMAs, far inside the SM's bandwidth.  What
// matters is keeping every SM's FP64 units busy, so the grid is
// (N/64, M/64, batch) with several CTAs resident per SM, and the next K-slab
// is prefetched into registers while the current one is consumed.
//
// The same kernel serves the slice products of the FP64 mode (with the
// field scalings of B_tau = exp(-dtau K) diag(exp(eta dtau xi s)) fused in:
// the first slice of a block scales the K index, later slices scale the
// output columns), the Gram matrices and trailing updates of the
// stabilisation, and the LU updates of the final determinant.
#include <cuda_runtime.h>

#include "internal.h"

namespace sldqmc {

namespace {

constexpr int BK = 16;

// Tile BMt x BNt, BMt*BNt/16 threads, each owning a 4 x 4 register block
// (rows ty + (BMt/4) i, columns tx + (BNt/4) j).
template <bool TA, bool TB, int BMt, int BNt>
__global__ void __launch_bounds__(BMt * BNt / 16) k_gemm_f64(GemmF64 g)
{
    constexpr int BM = BMt, BN = BNt, NT = BMt * BNt / 16;
    constexpr int TXN = BNt / 4, TYN = BMt / 4;
    constexpr int LA = BMt * BK / NT, LB = BNt * BK / NT;
    const int b = blockIdx.z;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (g.c_upper && n0 + BN - 1 < m0) return;  // tile strictly below the diagonal
    const double *A = g.A + (long long)b * g.sA;
    const double *B = g.B + (long long)b * g.sB;
    double *C = g.C + (long long)b * g.sC;
    const int8_t *sk = g.s_k ? g.s_k + (long long)b * g.sSk : nullptr;

    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];

    const int tid = threadIdx.x;
    const int tx = tid % TXN, ty = tid / TXN;

    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    int kbeg = 0;
    if (g.a_upper) kbeg = (m0 / BK) * BK;
    int K = g.K;
    if (g.b_upper && n0 + BN < K) K = n0 + BN;

    double ra[LA], rb[LB];
    auto load = [&](int k0) {
#pragma unroll
        for (int e = 0; e < LA; ++e) {
            int idx = tid + NT * e;
            int m, k;
            if (!TA) { m = idx / BK; k = idx % BK; } else { k = idx / BM; m = idx % BM; }
            int gm = m0 + m, gk = k0 + k;
            double v = 0.0;
            if (gm < g.M && gk < K) {
                v = TA ? A[(long long)gk * g.lda + gm] : A[(long long)gm * g.lda + gk];
                if (sk) v *= (sk[gk] > 0 ? g.cu : g.cd);
            }
            ra[e] = v;
        }
#pragma unroll
        for (int e = 0; e < LB; ++e) {
            int idx = tid + NT * e;
            int n, k;
            if (!TB) { k = idx / BN; n = idx % BN; } else { n = idx / BK; k = idx % BK; }
            int gn = n0 + n, gk = k0 + k;
            double v = 0.0;
            if (gn < g.N && gk < K) v = TB ? B[(long long)gn * g.ldb + gk] : B[(long long)gk * g.ldb + gn];
            rb[e] = v;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int e = 0; e < LA; ++e) {
            int idx = tid + NT * e;
            int m, k;
            if (!TA) { m = idx / BK; k = idx % BK; } else { k = idx / BM; m = idx % BM; }
            As[k][m] = ra[e];
        }
#pragma unroll
        for (int e = 0; e < LB; ++e) {
            int idx = tid + NT * e;
            int n, k;
            if (!TB) { k = idx / BN; n = idx % BN; } else { n = idx / BK; k = idx % BK; }
            Bs[k][n] = rb[e];
        }
    };

    if (kbeg < K) load(kbeg);
    for (int k0 = kbeg; k0 < K; k0 += BK) {
        __syncthreads();
        store();
        __syncthreads();
        if (k0 + BK < K) load(k0 + BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            double a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + TYN * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[k][tx + TXN * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
    }

    const int8_t *sn = g.s_n ? g.s_n + (long long)b * g.sSn : nullptr;
    const double *ms = g.ms ? g.ms + (long long)b * g.sMs : nullptr;
    const int8_t *sm = g.s_m ? g.s_m + (long long)b * g.sSm : nullptr;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty + TYN * i;
        if (gm >= g.M) continue;
        double rsc = 1.0;
        if (ms) rsc = g.ms_recip ? 1.0 / ms[gm] : ms[gm];
        if (sm) rsc *= (sm[gm] > 0 ? g.cu : g.cd);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx + TXN * j;
            if (gn >= g.N) continue;
            if (g.c_upper && gn < gm) continue;
            double v = g.alpha * acc[i][j];
            if (sn) v *= (sn[gn] > 0 ? g.cu : g.cd);
            v *= rsc;
            double *cp = C + (long long)gm * g.ldc + gn;
            if (g.beta != 0.0) v = fma(g.beta, *cp, v);
            *cp = v;
        }
    }
}

}  // namespace

GemmF64 gemm_desc(int M, int N, int K, const double *A, long long lda, long long sA,
                  const double *B, long long ldb, long long sB, double *C, long long ldc,
                  long long sC, int batch)
{
    GemmF64 g{};
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.sA = sA;
    g.B = B; g.ldb = ldb; g.sB = sB;
    g.C = C; g.ldc = ldc; g.sC = sC;
    g.alpha = 1.0; g.beta = 0.0;
    g.cu = g.cd = 1.0;
    g.batch = batch;
    return g;
}

double gemm_flops(const GemmF64 &g)
{
    const double M = g.M, N = g.N, K = g.K;
    double f;
    if (g.c_upper) f = K * M * (M + 1.0);       // upper triangle of a square C
    else if (g.a_upper && g.b_upper) f = K * (K + 1.0) * (K + 2.0) / 3.0;  // upper x upper
    else if (g.a_upper) f = N * K * (K + 1.0);  // triangular A (square)
    else f = 2.0 * M * N * K;
    return f * g.batch;
}

template <int BMt, int BNt>
static void launch_tiles(const GemmF64 &g, bool TA, bool TB, cudaStream_t st)
{
    dim3 grid((g.N + BNt - 1) / BNt, (g.M + BMt - 1) / BMt, g.batch);
    constexpr int NT = BMt * BNt / 16;
    if (!TA && !TB) k_gemm_f64<false, false, BMt, BNt><<<grid, NT, 0, st>>>(g);
    else if (!TA && TB) k_gemm_f64<false, true, BMt, BNt><<<grid, NT, 0, st>>>(g);
    else if (TA && !TB) k_gemm_f64<true, false, BMt, BNt><<<grid, NT, 0, st>>>(g);
    else k_gemm_f64<true, true, BMt, BNt><<<grid, NT, 0, st>>>(g);
}

void gemm_f64(const GemmF64 &g, bool TA, bool TB, cudaStream_t st)
{
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
    // 64 x 64 tiles when they give every SM several CTAs, else 32 x 32 tiles:
    // the FP64 pipe is saturated inside a CTA either way, so what matters is
    // that no SM idles (triangular operands make tile work uneven).
    const long long tiles64 = (long long)((g.N + 63) / 64) * ((g.M + 63) / 64) * g.batch;
    if (tiles64 >= 8LL * 152) launch_tiles<64, 64>(g, TA, TB, st);
    else launch_tiles<32, 32>(g, TA, TB, st);
}

}  // namespace sldqmc
