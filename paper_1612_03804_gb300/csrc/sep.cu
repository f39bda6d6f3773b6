// sep.cu -- slice products with the separable form of exp(-dtau K).
//
// On the periodic Lx x Ly square lattice the hopping matrix splits into two
// commuting parts, K = -t (A_x (x) 1 + 1 (x) A_y) - mu 1, so the kinetic
// propagator factorises exactly:
//   exp(-dtau K)[i][j] = e^{dtau mu} E1x(x_i - x_j) E1y(y_i - y_j),
// with E1 the ring propagator exp(dtau t A_1) (a symmetric circulant, L
// distinct values).  The paper's cost of one cumulative update assumes a
// B matrix applied in O(N^2) instead of a dense O(N^3) product ("Formalism
// of SLDQMC", the complexity paragraph); this is the exact form of that
// structure (no Trotter splitting of K, so the result equals the dense
// product up to rounding).
//
// The block chain works on X^T = U^T D_0 E D_1 E ... D_{nb-1} E.  Every row
// of X^T evolves on its own, so one CTA keeps a row in shared memory for the
// whole block: per slice a field scale and two circular convolutions of the
// row seen as an Ly x Lx image (along x with E1x, then along y with
// e^{dtau mu} E1y), 2 N (Lx + Ly) flops per row and slice instead of 2 N^2,
// and one read and one write of the row per block instead of one per slice.
//
// Two arithmetics:
//   FP64 (the FP64 mode): plain FP64 FMAs.
//   split FP32 (the mixed modes): the row as an unevaluated pair hi + lo of
//   floats (48 significant bits), E1 likewise; each product term is
//   hi*e_hi + hi*e_lo + lo*e_hi on the FP32 pipe, the leading terms spread
//   over two accumulators, and the pair is renormalised after each
//   convolution.  FP64 only to load and store the row once per block.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "internal.h"

namespace sldqmc {

namespace {

constexpr int SEP_THREADS = 512;

struct SepArgs {
    const double *Ut;     // B items of N x N (row stride N, item stride nn)
    double *Xt;
    const int8_t *s;      // field, item stride sS, slice stride N
    long long sS;
    long long nn;
    int N, Lx, Ly, M, B;
    int t0, nb;           // slices t0, t0+1, ... (mod M)
    double cu, cd;        // d = cu where s > 0, cd otherwise
    const double *ex;     // ring propagators E1x (Lx), E1y (Ly)
    const double *ey;
    double emu;           // e^{dtau mu}
};

__device__ __forceinline__ double field_scale(const SepArgs &a, const int8_t *sl, int i)
{
    return sl[i] > 0 ? a.cu : a.cd;
}

// FP64: one row per CTA iteration, persistent over the B*N rows.
__global__ void __launch_bounds__(SEP_THREADS) k_sep_block_f64(SepArgs a)
{
    extern __shared__ double sm[];
    double *v = sm, *z = sm + a.N, *ex = z + a.N, *ey = ex + a.Lx;
    const int tid = threadIdx.x;
    for (int i = tid; i < a.Lx; i += SEP_THREADS) ex[i] = a.ex[i];
    for (int i = tid; i < a.Ly; i += SEP_THREADS) ey[i] = a.emu * a.ey[i];
    const long long rows = (long long)a.B * a.N;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int b = (int)(row / a.N);
        const double *src = a.Ut + b * a.nn + (row - (long long)b * a.N) * a.N;
        const int8_t *fs = a.s + b * a.sS;
        const int8_t *sl0 = fs + (long long)(a.t0 % a.M) * a.N;
        __syncthreads();  // the previous row is stored, ex/ey are loaded
        for (int i = tid; i < a.N; i += SEP_THREADS) v[i] = src[i] * field_scale(a, sl0, i);
        __syncthreads();
        for (int j = 0; j < a.nb; ++j) {
            // along x: z[y][xo] = sum_d E1x(d) v[y][(xo + d) mod Lx]
            for (int o = tid; o < a.N; o += SEP_THREADS) {
                const int y = o / a.Lx, xo = o - y * a.Lx;
                const double *vr = v + y * a.Lx;
                double acc = 0.0;
                int x = xo;
                for (int d = 0; d < a.Lx; ++d) {
                    acc = fma(vr[x], ex[d], acc);
                    if (++x == a.Lx) x = 0;
                }
                z[o] = acc;
            }
            __syncthreads();
            // along y, with e^{dtau mu} and the next slice's field scale:
            // v[yo][x] = d_next * sum_d e^{dtau mu} E1y(d) z[(yo + d) mod Ly][x]
            const int8_t *sln = j + 1 < a.nb ? fs + (long long)((a.t0 + j + 1) % a.M) * a.N : nullptr;
            for (int o = tid; o < a.N; o += SEP_THREADS) {
                const int yo = o / a.Lx, x = o - yo * a.Lx;
                double acc = 0.0;
                int y = yo;
                for (int d = 0; d < a.Ly; ++d) {
                    acc = fma(z[y * a.Lx + x], ey[d], acc);
                    if (++y == a.Ly) y = 0;
                }
                v[o] = sln ? acc * field_scale(a, sln, o) : acc;
            }
            __syncthreads();
        }
        double *dst = a.Xt + b * a.nn + (row - (long long)b * a.N) * a.N;
        for (int i = tid; i < a.N; i += SEP_THREADS) dst[i] = v[i];
    }
}

// (hi, lo) <- hi + lo renormalised so that |lo| <= ulp(hi)/2 (Fast2Sum; |hi| >= |lo|).
__device__ __forceinline__ float2 renorm(float hi, float lo)
{
    const float s = hi + lo;
    return make_float2(s, lo - (s - hi));
}

// Error-free sum of two floats (TwoSum), returned as (sum, error).
__device__ __forceinline__ float2 two_sum(float a, float b)
{
    const float s = a + b;
    const float bp = s - a;
    return make_float2(s, (a - (s - bp)) + (b - bp));
}

__device__ __forceinline__ float2 split_pair(double x)
{
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

// pair * pair (scale by a field factor): hi*hi exactly (FMA residual) plus the cross terms.
__device__ __forceinline__ float2 mul_pair(float2 v, float2 d)
{
    const float p = v.x * d.x;
    const float e = fmaf(v.x, d.x, -p);
    return renorm(p, fmaf(v.x, d.y, fmaf(v.y, d.x, e)));
}

// One circular convolution of length L of pair data: acc over d of
// w[(o0 + d) mod L] * e[d], w at stride `stride`; leading terms on two
// accumulators, cross terms on a third, combined without FP64.
__device__ __forceinline__ float2 conv_pair(const float2 *w, int stride, int o0, int L, const float2 *e)
{
    float a0 = 0.0f, a1 = 0.0f, c = 0.0f;
    int k = o0;
    int d = 0;
    for (; d + 1 < L; d += 2) {
        const float2 w0 = w[k * stride];
        const float2 e0 = e[d];
        if (++k == L) k = 0;
        const float2 w1 = w[k * stride];
        const float2 e1 = e[d + 1];
        if (++k == L) k = 0;
        a0 = fmaf(w0.x, e0.x, a0);
        c = fmaf(w0.x, e0.y, c);
        c = fmaf(w0.y, e0.x, c);
        a1 = fmaf(w1.x, e1.x, a1);
        c = fmaf(w1.x, e1.y, c);
        c = fmaf(w1.y, e1.x, c);
    }
    if (d < L) {
        const float2 w0 = w[k * stride];
        const float2 e0 = e[d];
        a0 = fmaf(w0.x, e0.x, a0);
        c = fmaf(w0.x, e0.y, c);
        c = fmaf(w0.y, e0.x, c);
    }
    const float2 s = two_sum(a0, a1);
    return renorm(s.x, s.y + c);
}

__global__ void __launch_bounds__(SEP_THREADS) k_sep_block_f32x2(SepArgs a)
{
    extern __shared__ float2 sm2[];
    float2 *v = sm2, *z = sm2 + a.N, *ex = z + a.N, *ey = ex + a.Lx;
    const int tid = threadIdx.x;
    for (int i = tid; i < a.Lx; i += SEP_THREADS) ex[i] = split_pair(a.ex[i]);
    for (int i = tid; i < a.Ly; i += SEP_THREADS) ey[i] = split_pair(a.emu * a.ey[i]);
    const float2 du = split_pair(a.cu), dd = split_pair(a.cd);
    const long long rows = (long long)a.B * a.N;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int b = (int)(row / a.N);
        const double *src = a.Ut + b * a.nn + (row - (long long)b * a.N) * a.N;
        const int8_t *fs = a.s + b * a.sS;
        const int8_t *sl0 = fs + (long long)(a.t0 % a.M) * a.N;
        __syncthreads();
        for (int i = tid; i < a.N; i += SEP_THREADS) v[i] = split_pair(src[i] * field_scale(a, sl0, i));
        __syncthreads();
        for (int j = 0; j < a.nb; ++j) {
            for (int o = tid; o < a.N; o += SEP_THREADS) {
                const int y = o / a.Lx, xo = o - y * a.Lx;
                z[o] = conv_pair(v + y * a.Lx, 1, xo, a.Lx, ex);
            }
            __syncthreads();
            const int8_t *sln = j + 1 < a.nb ? fs + (long long)((a.t0 + j + 1) % a.M) * a.N : nullptr;
            for (int o = tid; o < a.N; o += SEP_THREADS) {
                const int yo = o / a.Lx, x = o - yo * a.Lx;
                const float2 r = conv_pair(z + x, a.Lx, yo, a.Ly, ey);
                v[o] = sln ? mul_pair(r, sln[o] > 0 ? du : dd) : r;
            }
            __syncthreads();
        }
        double *dst = a.Xt + b * a.nn + (row - (long long)b * a.N) * a.N;
        for (int i = tid; i < a.N; i += SEP_THREADS) dst[i] = (double)v[i].x + (double)v[i].y;
    }
}

size_t sep_smem_bytes(int N, int Lx, int Ly)
{
    return sizeof(double) * (2 * (size_t)N + Lx + Ly);
}

}  // namespace

// Largest lattice the shared-memory row kernel takes (two rows of 8-byte
// values and the ring propagators within 227 KB).
bool sep_supported(int Lx, int Ly)
{
    return sep_smem_bytes(Lx * Ly, Lx, Ly) <= 227 * 1024;
}

void sep_set_limits()
{
    cudaFuncSetAttribute(k_sep_block_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_sep_block_f32x2, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

// X^T_out = U^T D_{t0} E D_{t0+1} E ... D_{t0+nb-1} E for B items, E applied
// in its separable form; FP64 arithmetic in the FP64 mode, split FP32 in the
// mixed modes.  ring: E1x (Lx values) then E1y (Ly values).
void sep_chain_block(sldqmc_ctx *c, const double *Ut, const int8_t *d_s, int B, double cu, double cd, int t0,
                     int nb, const double *ring, double *Xt_out)
{
    SepArgs a{};
    a.Ut = Ut;
    a.Xt = Xt_out;
    a.s = d_s;
    a.sS = (long long)c->M * c->N;
    a.nn = c->nn;
    a.N = c->N;
    a.Lx = c->p.Lx;
    a.Ly = c->p.Ly;
    a.M = c->M;
    a.B = B;
    a.t0 = t0;
    a.nb = nb;
    a.cu = cu;
    a.cd = cd;
    a.ex = ring;
    a.ey = ring + c->p.Lx;
    a.emu = exp(c->p.dtau * c->p.mu);
    const size_t sh = sep_smem_bytes(c->N, c->p.Lx, c->p.Ly);
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool f64 = c->p.prec == SLDQMC_FP64;
    if (f64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sep_block_f64, SEP_THREADS, sh);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sep_block_f32x2, SEP_THREADS, sh);
    if (per_sm < 1) per_sm = 1;
    const long long rows = (long long)B * c->N;
    const long long cap = (long long)sms * per_sm;
    const int grid = (int)(rows < cap ? rows : cap);
    const double flops = 2.0 * (double)c->N * c->N * (c->p.Lx + c->p.Ly) * nb * B;
    prof_begin(c, SLDQMC_KC_SEP, flops);
    if (f64) k_sep_block_f64<<<grid, SEP_THREADS, sh, c->st>>>(a);
    else k_sep_block_f32x2<<<grid, SEP_THREADS, sh, c->st>>>(a);
    prof_end(c);
    c->launches++;
}

}  // namespace sldqmc
