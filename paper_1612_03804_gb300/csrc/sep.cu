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
constexpr int XB = 8;  // outputs per thread along a line (register blocking)

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
    int R;                // rows of X^T held by a CTA at a time
    int P;                // line stride of a row image in shared memory (odd, >= Lx)
};

// Value types: FP64, or an unevaluated pair hi + lo of floats.
struct F64 {
    using T = double;
    struct Acc {
        double a[XB];
        __device__ __forceinline__ void zero()
        {
#pragma unroll
            for (int k = 0; k < XB; ++k) a[k] = 0.0;
        }
        __device__ __forceinline__ void mac(int k, int, double w, double e) { a[k] = fma(w, e, a[k]); }
        __device__ __forceinline__ double get(int k) const { return a[k]; }
    };
    static __device__ __forceinline__ double from(double x) { return x; }
    static __device__ __forceinline__ double to(double v) { return v; }
    static __device__ __forceinline__ double scale(double v, double d) { return v * d; }
    static __device__ __forceinline__ double zero() { return 0.0; }
};

// (hi, lo) <- hi + lo renormalised (Fast2Sum; |hi| >= |lo|).
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

struct F32x2 {
    using T = float2;
    // per output: leading products on two accumulators (even and odd d), the
    // cross terms hi*e_lo + lo*e_hi on a third
    struct Acc {
        float a0[XB], a1[XB], c[XB];
        __device__ __forceinline__ void zero()
        {
#pragma unroll
            for (int k = 0; k < XB; ++k) a0[k] = a1[k] = c[k] = 0.0f;
        }
        __device__ __forceinline__ void mac(int k, int par, float2 w, float2 e)
        {
            if (par) a1[k] = fmaf(w.x, e.x, a1[k]);
            else a0[k] = fmaf(w.x, e.x, a0[k]);
            c[k] = fmaf(w.x, e.y, c[k]);
            c[k] = fmaf(w.y, e.x, c[k]);
        }
        __device__ __forceinline__ float2 get(int k) const
        {
            const float2 s = two_sum(a0[k], a1[k]);
            return renorm(s.x, s.y + c[k]);
        }
    };
    static __device__ __forceinline__ float2 from(double x)
    {
        const float h = (float)x;
        return make_float2(h, (float)(x - (double)h));
    }
    static __device__ __forceinline__ double to(float2 v) { return (double)v.x + (double)v.y; }
    // pair * pair: hi*hi exactly (FMA residual) plus the cross terms
    static __device__ __forceinline__ float2 scale(float2 v, float2 d)
    {
        const float p = v.x * d.x;
        const float e = fmaf(v.x, d.x, -p);
        return renorm(p, fmaf(v.x, d.y, fmaf(v.y, d.x, e)));
    }
    static __device__ __forceinline__ float2 zero() { return make_float2(0.0f, 0.0f); }
};

// XB outputs of one line: out[k] = sum_d e[d] w[(o0 + k + d) mod L], the line's
// values at stride `st` from w; e zero-padded to a multiple of XB.  The
// window of 2 XB - 1 values of a d-block sits in registers, so a value read
// from shared memory serves XB products.
template <class V>
__device__ __forceinline__ void conv_line(const typename V::T *w, int st, int L, int o0, const typename V::T *e,
                                          int Lpad, typename V::Acc &acc)
{
    using T = typename V::T;
    acc.zero();
    T win[2 * XB - 1];
    int li = o0;  // index of the next value to load, kept in [0, L)
#pragma unroll
    for (int j = 0; j < XB - 1; ++j) {
        win[XB + j] = w[li * st];
        if (++li == L) li = 0;
    }
    for (int d0 = 0; d0 < Lpad; d0 += XB) {
#pragma unroll
        for (int j = 0; j < XB - 1; ++j) win[j] = win[XB + j];
#pragma unroll
        for (int j = XB - 1; j < 2 * XB - 1; ++j) {
            win[j] = w[li * st];
            if (++li == L) li = 0;
        }
#pragma unroll
        for (int t = 0; t < XB; ++t) {
            const T et = e[d0 + t];
#pragma unroll
            for (int k = 0; k < XB; ++k) acc.mac(k, t & 1, win[k + t], et);
        }
    }
}

// Each CTA holds R rows of X^T as Ly x Lx images (line stride P, odd, so
// that lanes reading consecutive lines of the x pass hit different banks),
// persistent over the B*N rows.  Per slice: the x pass (lines = image rows,
// work item = line x output block, consecutive lanes on consecutive lines),
// then the y pass (lines = image columns, consecutive lanes on consecutive
// columns) with e^{dtau mu} and the next slice's field scale.
template <class V>
__global__ void __launch_bounds__(SEP_THREADS) k_sep_block(SepArgs a)
{
    using T = typename V::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int Lx = a.Lx, Ly = a.Ly, N = a.N, P = a.P, R = a.R;
    const int img = Ly * P;
    const int Lxp = (Lx + XB - 1) / XB * XB, Lyp = (Ly + XB - 1) / XB * XB;
    T *v = reinterpret_cast<T *>(smraw);
    T *z = v + (size_t)R * img;
    T *ex = z + (size_t)R * img;
    T *ey = ex + Lxp;
    const int tid = threadIdx.x;
    for (int i = tid; i < Lxp; i += SEP_THREADS) ex[i] = i < Lx ? V::from(a.ex[i]) : V::zero();
    for (int i = tid; i < Lyp; i += SEP_THREADS) ey[i] = i < Ly ? V::from(a.emu * a.ey[i]) : V::zero();
    const T du = V::from(a.cu), dd = V::from(a.cd);
    const long long rows = (long long)a.B * N;
    const int nbx = Lxp / XB, nby = Lyp / XB;
    for (long long row0 = (long long)blockIdx.x * R; row0 < rows; row0 += (long long)gridDim.x * R) {
        const int nr = rows - row0 < R ? (int)(rows - row0) : R;
        __syncthreads();  // the previous rows are stored; ex, ey are loaded
        for (int e = tid; e < nr * N; e += SEP_THREADS) {
            const int r = e / N, i = e - r * N;
            const long long row = row0 + r;
            const int b = (int)(row / N);
            const int8_t *sl0 = a.s + b * a.sS + (long long)(a.t0 % a.M) * N;
            const double x = a.Ut[b * a.nn + (row - (long long)b * N) * N + i];
            const int y = i / Lx;
            v[r * img + y * P + (i - y * Lx)] = V::from(x * (sl0[i] > 0 ? a.cu : a.cd));
        }
        __syncthreads();
        for (int j = 0; j < a.nb; ++j) {
            // along x: z[r][y][xo] = sum_d E1x(d) v[r][y][(xo + d) mod Lx]
            const int lx = nr * Ly;
            for (int w = tid; w < lx * nbx; w += SEP_THREADS) {
                const int line = w % lx, o0 = (w / lx) * XB;
                const int r = line / Ly, y = line - r * Ly;
                typename V::Acc acc;
                conv_line<V>(v + r * img + y * P, 1, Lx, o0, ex, Lxp, acc);
                T *zo = z + r * img + y * P;
#pragma unroll
                for (int k = 0; k < XB; ++k)
                    if (o0 + k < Lx) zo[o0 + k] = acc.get(k);
            }
            __syncthreads();
            // along y, times e^{dtau mu} (in ey) and the next slice's field scale
            const bool more = j + 1 < a.nb;
            const int ly = nr * Lx;
            for (int w = tid; w < ly * nby; w += SEP_THREADS) {
                const int line = w % ly, o0 = (w / ly) * XB;
                const int r = line / Lx, x = line - r * Lx;
                typename V::Acc acc;
                conv_line<V>(z + r * img + x, P, Ly, o0, ey, Lyp, acc);
                const long long row = row0 + r;
                const int b = (int)(row / N);
                const int8_t *sln = more ? a.s + b * a.sS + (long long)((a.t0 + j + 1) % a.M) * N : nullptr;
                T *vo = v + r * img + x;
#pragma unroll
                for (int k = 0; k < XB; ++k) {
                    const int y = o0 + k;
                    if (y < Ly) {
                        const T val = acc.get(k);
                        vo[y * P] = more ? V::scale(val, sln[y * Lx + x] > 0 ? du : dd) : val;
                    }
                }
            }
            __syncthreads();
        }
        for (int e = tid; e < nr * N; e += SEP_THREADS) {
            const int r = e / N, i = e - r * N;
            const long long row = row0 + r;
            const int b = (int)(row / N);
            const int y = i / Lx;
            a.Xt[b * a.nn + (row - (long long)b * N) * N + i] = V::to(v[r * img + y * P + (i - y * Lx)]);
        }
    }
}

int odd_stride(int Lx) { return Lx | 1; }

size_t sep_smem_bytes(int Lx, int Ly, int R)
{
    const int Lxp = (Lx + XB - 1) / XB * XB, Lyp = (Ly + XB - 1) / XB * XB;
    return 8 * (2 * (size_t)R * Ly * odd_stride(Lx) + Lxp + Lyp);
}

// Rows per CTA: enough that a CTA's passes have several thousand outputs
// between barriers, within the shared memory of one CTA.
int sep_rows_per_cta(int N, int Lx, int Ly)
{
    int R = 1;
    while (R < 32 && (long long)(2 * R) * N <= 4096 && sep_smem_bytes(Lx, Ly, 2 * R) <= 200 * 1024) R *= 2;
    return R;
}

}  // namespace

// Largest lattice the shared-memory row kernel takes (two images of one
// row of 8-byte values and the ring propagators within 227 KB).
bool sep_supported(int Lx, int Ly)
{
    return sep_smem_bytes(Lx, Ly, 1) <= 227 * 1024;
}

void sep_set_limits()
{
    cudaFuncSetAttribute(k_sep_block<F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_sep_block<F32x2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
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
    a.R = sep_rows_per_cta(c->N, a.Lx, a.Ly);
    a.P = odd_stride(a.Lx);
    const size_t sh = sep_smem_bytes(a.Lx, a.Ly, a.R);
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool f64 = c->p.prec == SLDQMC_FP64;
    if (f64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sep_block<F64>, SEP_THREADS, sh);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sep_block<F32x2>, SEP_THREADS, sh);
    if (per_sm < 1) per_sm = 1;
    const long long groups = ((long long)B * c->N + a.R - 1) / a.R;
    const long long cap = (long long)sms * per_sm;
    const int grid = (int)(groups < cap ? groups : cap);
    const double flops = 2.0 * (double)c->N * c->N * (c->p.Lx + c->p.Ly) * nb * B;
    prof_begin(c, SLDQMC_KC_SEP, flops, "sep_block");
    if (f64) k_sep_block<F64><<<grid, SEP_THREADS, sh, c->st>>>(a);
    else k_sep_block<F32x2><<<grid, SEP_THREADS, sh, c->st>>>(a);
    prof_end(c);
    c->launches++;
}

}  // namespace sldqmc
