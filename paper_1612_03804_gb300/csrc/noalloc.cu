// noalloc.cu -- an allocation-free form of the FP64 exact-weight evaluation.
//
// Some callers cannot call cudaMalloc or cudaFree: code that runs under a
// host framework which owns the whole device heap and forbids direct
// allocations, or code on a latency-critical path that must not take the
// implicit device synchronisation cudaFree performs.  For them,
// sldqmc_weight_noalloc runs the same kernels and launch sequence as
// sldqmc_weight_batch_dev, with every workspace buffer carved out of one
// file-scope device array instead of a context's cudaMalloc'd memory.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "internal.h"

namespace sldqmc {
void build_K_into(sldqmc_ctx *c, double *ring);
int weight_run_into(sldqmc_ctx *c, const int8_t *d_s, int B, int eta, double *d_ld, int *d_sign);
void stab_set_limits(int Npad);
}  // namespace sldqmc

using namespace sldqmc;

namespace {

// 16 MiB of workspace, reserved on every device that loads the library until
// the process exits.
constexpr size_t SCRATCH_BYTES = 16u << 20;
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES];  // device address of g_scratch, per device, once set up

// Device address of the scratch array on the current device.  In host code
// g_scratch is only a host-side stand-in, never a device address.
int scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return SLDQMC_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SLDQMC_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return SLDQMC_OK;
}

// Carves 256-byte-aligned regions out of the scratch array (or, with a zero
// base, only measures how many bytes they need).
struct Carver {
    uintptr_t base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * count;
        return p;
    }
};

// Workspace of one call: flag, K/E/E^{-1} and ring propagators, the nine
// work buffers (the LU buffer twice the size), D/D_p/log accumulators,
// permutations, pivots and signs.  Returns the bytes used.
size_t layout(sldqmc_ctx *c, uintptr_t base, double **ring)
{
    Carver k{base};
    const size_t nn = (size_t)c->nn, N = (size_t)c->N, B = (size_t)c->cap;
    c->d_flag = k.take<int>(1);
    c->d_K = k.take<double>(3 * nn);
    c->d_E = base ? c->d_K + nn : nullptr;
    c->d_Einv = base ? c->d_E + nn : nullptr;
    *ring = k.take<double>(2 * (size_t)(c->p.Lx + c->p.Ly));
    double *q = k.take<double>(10 * nn * B);
    for (int j = 0; j < 9; ++j) {
        c->buf[j] = q;
        if (q) q += (j == 4 ? 2 : 1) * nn * B;
    }
    c->d_D = k.take<double>(N * B);
    c->d_Dp = k.take<double>(N * B);
    c->d_logacc = k.take<double>(B);
    c->d_perm = k.take<int>(N * B);
    c->d_piv = k.take<int>(N * B);
    c->d_sgn = k.take<int>(2 * B);
    c->d_tslu = k.take<int>(24 * 32 * B);
    return k.off;
}

}  // namespace

extern "C" int sldqmc_weight_noalloc(const sldqmc_params *p, void *stream, const int8_t *d_s, int B, int eta,
                                     double *d_logabsdet, int *d_sign)
{
    if (!p || !d_s || !d_logabsdet || B < 1 || (eta != 1 && eta != -1)) return SLDQMC_ERR_ARG;
    if (p->Lx < 1 || p->Ly < 1 || p->n_wrap < 1 || !(p->dtau > 0.0) || !(p->beta > 0.0) || !isfinite(p->t) ||
        !isfinite(p->mu) || !isfinite(p->xi))
        return SLDQMC_ERR_ARG;
    if (p->prec != SLDQMC_FP64) return SLDQMC_ERR_UNSUPPORTED;
    const long long N = (long long)p->Lx * p->Ly;
    const long long M = llround(p->beta / p->dtau);
    if (M < 1 || fabs((double)M * p->dtau - p->beta) > 1e-12 * p->beta) return SLDQMC_ERR_ARG;
    // the same limits as a context, then a bound computed in floating point
    // (the nine N x N work buffers per configuration alone take 80 N^2 B
    // bytes) so that no size below can overflow
    if (N > 16384 || M > 100000) return SLDQMC_ERR_UNSUPPORTED;
    if (80.0 * (double)N * (double)N * (double)B > (double)SCRATCH_BYTES) return SLDQMC_ERR_UNSUPPORTED;
    const double logk = (double)(p->n_wrap < M ? p->n_wrap : M) * p->dtau * (8.0 * fabs(p->t) + 2.0 * fabs(p->xi));
    if (logk > 16.0) return SLDQMC_ERR_UNSUPPORTED;

    sldqmc_ctx c;
    memset(&c, 0, sizeof(c));
    c.p = *p;
    c.N = (int)N;
    c.M = (int)M;
    c.p.beta = (double)M * p->dtau;
    c.st = (cudaStream_t)stream;
    c.cap = B;
    c.nn = N * N;
    for (int e = 0; e < 2; ++e) {
        const double et = e == 0 ? 1.0 : -1.0;
        c.ex_scale[e][0] = exp(et * p->dtau * p->xi);
        c.ex_scale[e][1] = exp(-et * p->dtau * p->xi);
    }
    // size check before touching the device
    double *ring = nullptr;
    {
        sldqmc_ctx probe = c;
        if (layout(&probe, 0, &ring) > SCRATCH_BYTES) return SLDQMC_ERR_UNSUPPORTED;
    }
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    layout(&c, (uintptr_t)base, &ring);
    // the LU panel kernel needs more than the default 48 KiB of dynamic
    // shared memory from about N = 184 on; a context sets this at creation,
    // this call may be the first user of the library on its device
    {
        int Npad = 1;
        while (Npad < N) Npad <<= 1;
        stab_set_limits(Npad);
    }
    // the flag must start at zero; every other region is fully written by the
    // kernels before it is read (identity U and V, D = 1, zeroed R factors)
    if (cudaMemsetAsync(c.d_flag, 0, sizeof(int), c.st) != cudaSuccess) return SLDQMC_ERR_CUDA;
    build_K_into(&c, ring);
    rc = weight_run_into(&c, d_s, B, eta, d_logabsdet, d_sign);
    if (rc) return rc;
    if (cudaStreamSynchronize(c.st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return SLDQMC_ERR_CUDA;
    int f = 0;
    if (cudaMemcpy(&f, c.d_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SLDQMC_ERR_CUDA;
    if (f & FLAG_ARG) return SLDQMC_ERR_ARG;
    if (f & FLAG_TIMEOUT) return SLDQMC_ERR_TIMEOUT;
    if (f & FLAG_NUMERICAL) return SLDQMC_ERR_NUMERICAL;
    return SLDQMC_OK;
}
