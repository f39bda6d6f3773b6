// mc.cu -- Monte Carlo kernels: the DQMC local update ("Basics of DQMC"),
// the effective-model sweeps and features of the self-learned action
// (Eq. 2, step iii), the bare Ising weight and the cumulative-update
// acceptance (Eq. 4).  Every decision is taken in FP64 with explicitly
// rounded operations so that it matches a plain IEEE evaluation.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "internal.h"

namespace sldqmc {

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products with the Weyl key schedule between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

// Uniform in [0,1) from the top 53 bits of (x1:x0); key = 64-bit seed.
__device__ __forceinline__ double philox_uniform(uint64_t seed, uint32_t a, uint32_t b, uint32_t c,
                                                 uint32_t purpose)
{
    uint32_t x[4] = {a, b, c, purpose};
    philox4x32_10(x, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t w = ((uint64_t)x[1] << 32) | (uint64_t)x[0];
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ uint32_t philox_word(uint64_t seed, uint32_t a, uint32_t b, uint32_t c,
                                                uint32_t purpose)
{
    uint32_t x[4] = {a, b, c, purpose};
    philox4x32_10(x, (uint32_t)seed, (uint32_t)(seed >> 32));
    return x[0];
}

enum : uint32_t { PURPOSE_LOCAL = 1, PURPOSE_EFF = 2, PURPOSE_DIR = 3, PURPOSE_ACCEPT = 4 };
constexpr double MARGIN = 1e-8;

__device__ __forceinline__ int wrapi(int a, int L)
{
    a %= L;
    return a < 0 ? a + L : a;
}

// Flags any field value outside {-1, +1}.
__global__ void k_check_field(const int8_t *s, long long n, int *flag)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        int v = s[e];
        if (v != 1 && v != -1) atomicOr(flag, FLAG_ARG);
    }
}

// ------------------------------------------------------- bare weight phi
// log phi = dtau J sum_tau sum_<ij> s s + Kt sum_i sum_tau s_{i,tau} s_{i,tau+1}.
// Integer sums per configuration, then one FP64 combination.
__global__ void k_log_bare(const int8_t *s, int Lx, int Ly, int M, double dtauJ, double Kt, double *out,
                           int accumulate)
{
    const int b = blockIdx.x;
    const int N = Lx * Ly;
    const int8_t *sb = s + (long long)b * M * N;
    long long sp = 0, tm = 0;
    for (int v = threadIdx.x; v < M * N; v += blockDim.x) {
        int tau = v / N, i = v % N, x = i % Lx, y = i / Lx;
        int si = sb[v];
        if (Lx > 1) sp += si * sb[tau * N + wrapi(x + 1, Lx) + Lx * y];
        if (Ly > 1) sp += si * sb[tau * N + x + Lx * wrapi(y + 1, Ly)];
        tm += si * sb[((tau + 1) % M) * N + i];
    }
    __shared__ long long a1[32], a2[32];
    for (int o = 16; o > 0; o >>= 1) {
        sp += __shfl_down_sync(0xffffffffu, sp, o);
        tm += __shfl_down_sync(0xffffffffu, tm, o);
    }
    if ((threadIdx.x & 31) == 0) { a1[threadIdx.x >> 5] = sp; a2[threadIdx.x >> 5] = tm; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t1 = 0, t2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t1 += a1[w]; t2 += a2[w]; }
        double v = dtauJ * (double)t1 + Kt * (double)t2;
        if (accumulate) out[b] += v; else out[b] = v;
    }
}

// --------------------------------------------------------- local update
// Flips every site of slice tau in order i = 0..N-1 for one chain per CTA.
// Gt_f = E^{-1} G(tau) E for flavour f (eta = +1, -1): flipping s_{tau,i}
// gives R_f = 1 + Delta_f (1 - Gt_f[i][i]), Delta_f = exp(-2 eta dtau xi s) - 1;
// the Metropolis ratio is R_+^2 R_-^2 phi'/phi; on acceptance
// Gt_f <- Gt_f - (Delta_f / R_f) Gt_f[:,i] (e_i^T - Gt_f[i,:]).
struct LocalArgs {
    double *Gp, *Gm;   // per chain N x N (stride nn)
    long long nn;
    int8_t *s;         // per chain M x N
    int Lx, Ly, M, tau;
    uint32_t sweep;
    uint64_t seed;
    double dtxi;       // dtau * xi
    double dtauJ, Kt;
    long long *stats;  // per chain: accepted, proposed, margin
};

__global__ void __launch_bounds__(512) k_local_flips(LocalArgs a)
{
    const int b = blockIdx.x;
    const int N = a.Lx * a.Ly;
    double *G[2] = {a.Gp + (long long)b * a.nn, a.Gm + (long long)b * a.nn};
    int8_t *s = a.s + (long long)b * a.M * N;
    extern __shared__ double sh[];
    double *col = sh;           // 2N
    double *row = sh + 2 * N;   // 2N
    double *lus = sh + 4 * N;   // N: log u of every site of the slice
    __shared__ double coef[2], dls[2][2];
    __shared__ int accept;
    const uint64_t seed = a.seed + ((uint64_t)b << 32);
    long long n_acc = 0, n_mg = 0;
    const int tau = a.tau;
    // off the serial chain: the uniforms of all sites, and Delta_f for both field values
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        lus[i] = log(philox_uniform(seed, (uint32_t)i, (uint32_t)tau, a.sweep, PURPOSE_LOCAL));
    if (threadIdx.x < 4) {
        const int f = threadIdx.x >> 1, sp = threadIdx.x & 1;
        const double eta = f == 0 ? 1.0 : -1.0;
        dls[f][sp] = exp(-2.0 * eta * a.dtxi * (sp ? 1.0 : -1.0)) - 1.0;
    }
    __syncthreads();
    for (int i = 0; i < N; ++i) {
        if (threadIdx.x == 0) {
            const int sold = s[tau * N + i];
            const int x = i % a.Lx, y = i / a.Lx;
            int nsp = 0;
            if (a.Lx > 1) nsp += s[tau * N + wrapi(x + 1, a.Lx) + a.Lx * y] + s[tau * N + wrapi(x - 1, a.Lx) + a.Lx * y];
            if (a.Ly > 1) nsp += s[tau * N + x + a.Lx * wrapi(y + 1, a.Ly)] + s[tau * N + x + a.Lx * wrapi(y - 1, a.Ly)];
            const int ntm = s[wrapi(tau + 1, a.M) * N + i] + s[wrapi(tau - 1, a.M) * N + i];
            double logr = __dmul_rn(-2.0 * (double)sold,
                                    __dadd_rn(__dmul_rn(a.dtauJ, (double)nsp), __dmul_rn(a.Kt, (double)ntm)));
            double R[2], Dl[2];
            for (int f = 0; f < 2; ++f) {
                Dl[f] = dls[f][sold > 0];
                R[f] = __dadd_rn(1.0, __dmul_rn(Dl[f], __dadd_rn(1.0, -G[f][(long long)i * N + i])));
                logr = __dadd_rn(logr, __dmul_rn(2.0, log(fabs(R[f]))));
            }
            const double lu = lus[i];
            if (fabs(logr - lu) <= MARGIN) n_mg++;
            const int acc = lu < logr;
            accept = acc;
            if (acc) {
                coef[0] = Dl[0] / R[0];
                coef[1] = Dl[1] / R[1];
                s[tau * N + i] = (int8_t)(-sold);
                n_acc++;
            }
        }
        __syncthreads();
        const int acc_i = accept;
        __syncthreads();  // every thread has read the decision before thread 0 writes the next
        if (acc_i) {
            for (int e = threadIdx.x; e < 2 * N; e += blockDim.x) {
                const int f = e / N, k = e % N;
                col[e] = G[f][(long long)k * N + i];
                row[e] = (k == i ? 1.0 : 0.0) - G[f][(long long)i * N + k];
            }
            __syncthreads();
            // warp w takes rows w, w + nwarps, ...; its lanes walk the row's
            // columns (coalesced, no index division)
            const int nwarps = blockDim.x >> 5, wl = threadIdx.x & 31;
            for (int fr = threadIdx.x >> 5; fr < 2 * N; fr += nwarps) {
                const int f = fr >= N, rr = fr - f * N;
                const double cf = coef[f] * col[f * N + rr];
                double *g = G[f] + (long long)rr * N;
                const double *rw = row + f * N;
                for (int k = wl; k < N; k += 32) g[k] -= cf * rw[k];
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        a.stats[b * 4 + 0] += n_acc;
        a.stats[b * 4 + 1] += N;
        a.stats[b * 4 + 2] += n_mg;
    }
}

// ------------------------------------------------- delayed (rank-k) update
// The same sequence of flips, decisions and Green's functions with the
// Sherman-Morrison updates delayed: within a block of k <= 32 sites of slice
// tau the current Green's function of flavour f is
//   Gt_f = G0_f - U_f V_f,   U_f = [u_0 .. u_{n-1}] (N x n),  V_f = [v_0; ..; v_{n-1}] (n x N),
// one column/row pair per accepted flip so far.  A site needs only
// Gt_f[i][i] = G0_f[i][i] - U_f[i,:] V_f[:,i] (n terms); an accepted flip
// at i appends u_n = (Delta_f / R_f) Gt_f[:, i] and v_n = e_i^T - Gt_f[i, :],
// each formed from G0 and the n earlier pairs (2 N n multiply-adds instead
// of the N^2 of an immediate update).  After the block the pending rank-k
// correction G0 -= U V is applied by one batched GEMM over every chain
// (unused pairs are zero), so the N^2 work per accepted flip runs as a GEMM
// on all SMs instead of as rank-1 passes on one SM per chain.
// U: per chain N x 32 (row stride 32), V: per chain 32 x N; flavour f of
// chain b at U + (f * cap + b) * 32 N.
struct DelayArgs {
    LocalArgs l;
    double *U, *V;
    int cap;
    int i0, ns;   // sites i0 .. i0 + ns - 1 of slice tau (ns <= 32)
};

__global__ void __launch_bounds__(512) k_local_flips_delayed(DelayArgs d)
{
    const LocalArgs &a = d.l;
    const int b = blockIdx.x;
    const int N = a.Lx * a.Ly;
    const double *G[2] = {a.Gp + (long long)b * a.nn, a.Gm + (long long)b * a.nn};
    double *U[2], *V[2];
    for (int f = 0; f < 2; ++f) {
        U[f] = d.U + ((long long)f * d.cap + b) * 32 * N;
        V[f] = d.V + ((long long)f * d.cap + b) * 32 * N;
    }
    int8_t *s = a.s + (long long)b * a.M * N;
    __shared__ double ui[2][32], vi[2][32];  // U[i, :n] and V[:n, i] of the current site
    __shared__ double coef[2], dls[2][2], lus[32];
    __shared__ int accept;
    const uint64_t seed = a.seed + ((uint64_t)b << 32);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    long long n_acc = 0, n_mg = 0;
    const int tau = a.tau;
    int n = 0;  // pending pairs
    // off the serial chain: the block's uniforms, and Delta_f for both field values
    if (tid < d.ns)
        lus[tid] = log(philox_uniform(seed, (uint32_t)(d.i0 + tid), (uint32_t)tau, a.sweep, PURPOSE_LOCAL));
    if (tid >= 32 && tid < 36) {
        const int f = (tid - 32) >> 1, sp = tid & 1;
        const double eta = f == 0 ? 1.0 : -1.0;
        dls[f][sp] = exp(-2.0 * eta * a.dtxi * (sp ? 1.0 : -1.0)) - 1.0;
    }
    __syncthreads();
    for (int q = 0; q < d.ns; ++q) {
        const int i = d.i0 + q;
        if (wid == 0) {
            // U[i, j] and V[j, i] for j < n, and the current diagonals
            double dg[2];
            for (int f = 0; f < 2; ++f) {
                const double uu = lane < n ? U[f][(long long)i * 32 + lane] : 0.0;
                const double vv = lane < n ? V[f][(long long)lane * N + i] : 0.0;
                ui[f][lane] = uu;
                vi[f][lane] = vv;
                double p = uu * vv;
                for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
                dg[f] = G[f][(long long)i * N + i] - p;
            }
            if (lane == 0) {
                const int sold = s[tau * N + i];
                const int x = i % a.Lx, y = i / a.Lx;
                int nsp = 0;
                if (a.Lx > 1) nsp += s[tau * N + wrapi(x + 1, a.Lx) + a.Lx * y] + s[tau * N + wrapi(x - 1, a.Lx) + a.Lx * y];
                if (a.Ly > 1) nsp += s[tau * N + x + a.Lx * wrapi(y + 1, a.Ly)] + s[tau * N + x + a.Lx * wrapi(y - 1, a.Ly)];
                const int ntm = s[wrapi(tau + 1, a.M) * N + i] + s[wrapi(tau - 1, a.M) * N + i];
                double logr = __dmul_rn(-2.0 * (double)sold,
                                        __dadd_rn(__dmul_rn(a.dtauJ, (double)nsp), __dmul_rn(a.Kt, (double)ntm)));
                double R[2], Dl[2];
                for (int f = 0; f < 2; ++f) {
                    Dl[f] = dls[f][sold > 0];
                    R[f] = __dadd_rn(1.0, __dmul_rn(Dl[f], __dadd_rn(1.0, -dg[f])));
                    logr = __dadd_rn(logr, __dmul_rn(2.0, log(fabs(R[f]))));
                }
                const double lu = lus[q];
                if (fabs(logr - lu) <= MARGIN) n_mg++;
                const int acc = lu < logr;
                accept = acc;
                if (acc) {
                    coef[0] = Dl[0] / R[0];
                    coef[1] = Dl[1] / R[1];
                    s[tau * N + i] = (int8_t)(-sold);
                    n_acc++;
                }
            }
        }
        __syncthreads();
        if (accept) {
            // u_n = coef (G0[:, i] - U[:, :n] V[:n, i]),  v_n = e_i - (G0[i, :] - U[i, :n] V[:n, :])
            for (int e = tid; e < 2 * N; e += blockDim.x) {
                const int f = e >= N, r = e - f * N;
                double c = G[f][(long long)r * N + i];
                const double *ur = U[f] + (long long)r * 32;
                double w = G[f][(long long)i * N + r];
                for (int j = 0; j < n; ++j) {
                    c -= ur[j] * vi[f][j];
                    w -= ui[f][j] * V[f][(long long)j * N + r];
                }
                U[f][(long long)r * 32 + n] = coef[f] * c;
                V[f][(long long)n * N + r] = (r == i ? 1.0 : 0.0) - w;
            }
            ++n;
        }
        __syncthreads();
    }
    // unused pairs are zero for the batched correction
    for (int f = 0; f < 2; ++f) {
        for (long long e = tid; e < (long long)N * (32 - n); e += blockDim.x) {
            const int r = (int)(e / (32 - n)), j = n + (int)(e % (32 - n));
            U[f][(long long)r * 32 + j] = 0.0;
        }
        for (long long e = tid; e < (long long)(32 - n) * N; e += blockDim.x) V[f][(long long)n * N + e] = 0.0;
    }
    if (tid == 0) {
        a.stats[b * 4 + 0] += n_acc;
        a.stats[b * 4 + 1] += d.ns;
        a.stats[b * 4 + 2] += n_mg;
    }
}

void launch_local_flips_delayed(sldqmc_ctx *c, double *Gp, double *Gm, double *U, double *V, int8_t *d_s, int B,
                                int tau, int i0, int ns, uint32_t sweep, uint64_t seed, long long *stats)
{
    DelayArgs d;
    LocalArgs &a = d.l;
    a.Gp = Gp; a.Gm = Gm; a.nn = c->nn; a.s = d_s;
    a.Lx = c->p.Lx; a.Ly = c->p.Ly; a.M = c->M; a.tau = tau; a.sweep = sweep; a.seed = seed;
    a.dtxi = c->p.dtau * c->p.xi; a.dtauJ = c->dtauJ; a.Kt = c->Ktau; a.stats = stats;
    d.U = U; d.V = V; d.cap = c->cap; d.i0 = i0; d.ns = ns;
    prof_begin(c, SLDQMC_KC_LOCAL, 0.0, "local_flips_delayed");
    k_local_flips_delayed<<<B, 512, 0, c->st>>>(d);
    prof_end(c);
    c->launches++;
}

// Gt <- D_tau Gt D_tau^{-1} applied after the two wrap GEMMs is fused into
// the GEMM epilogues; the drift check compares a wrapped Gt with a fresh one.
__global__ void k_drift(const double *Gw, const double *Gf, long long nn, long long *stats, int B2)
{
    const int b = blockIdx.y;
    double m = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
         e += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(Gw[(long long)b * nn + e] - Gf[(long long)b * nn + e]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) {
        // non-negative doubles order like their bit patterns
        const int chain = b % B2;
        atomicMax(reinterpret_cast<unsigned long long *>(&stats[chain * 4 + 3]),
                  (unsigned long long)__double_as_longlong(m));
    }
}

// ------------------------------------------------------ effective model
// The model of one context travels with each launch as a kernel parameter
// (constant bank): class c has noff[c] offset triples (dx, dy, dtau), listed
// class after class in off, and coupling J[c].
struct EffModel {
    int n_class;
    int noff[32];
    int off[64 * 3];
    double J[32];
};

static EffModel eff_model_of(const sldqmc_ctx *c)
{
    EffModel m;
    m.n_class = c->n_class;
    memcpy(m.noff, c->h_n_off, sizeof(m.noff));
    memcpy(m.off, c->h_offsets, sizeof(m.off));
    memcpy(m.J, c->h_J, sizeof(m.J));
    return m;
}

__device__ __forceinline__ int shift_site(int v, int N, int Lx, int Ly, int M, const int *o, int sg)
{
    const int tau = v / N, i = v % N, x = i % Lx, y = i / Lx;
    return wrapi(tau + sg * o[2], M) * N + wrapi(x + sg * o[0], Lx) + Lx * wrapi(y + sg * o[1], Ly);
}

// n_sweeps colour-ordered Metropolis sweeps on H_eff for one chain per CTA.
// log acceptance a = ((2 beta) * sum_c J_c n_c) * s with n_c the integer
// neighbour sums (self-pairs excluded), accumulated in class order.
template <bool SMEM>
__global__ void __launch_bounds__(1024) k_eff_sweeps(int8_t *s_all, int Lx, int Ly, int M, double beta,
                                                     const __grid_constant__ EffModel em, const int *col_start,
                                                     const int *col_sites, int n_colors, int n_sweeps,
                                                     uint64_t seed, uint32_t step, int dir_fixed,
                                                     long long *n_accept, long long *n_margin,
                                                     const uint32_t *d_step)
{
    if (d_step) step = *d_step;  // graph replays read the step from device memory
    const int b = blockIdx.x;
    const int N = Lx * Ly;
    const int V = N * M;
    extern __shared__ int8_t sm8[];
    int8_t *gs = s_all + (long long)b * V;
    int8_t *s = SMEM ? sm8 : gs;
    const uint64_t key = seed + ((uint64_t)b << 32);
    if (SMEM) {
        for (int v = threadIdx.x; v < V; v += blockDim.x) s[v] = gs[v];
        __syncthreads();
    }
    int dir = dir_fixed;
    if (dir < 0) dir = (int)(philox_word(key, 0, 0, step, PURPOSE_DIR) & 1u);
    long long acc = 0, mg = 0;
    const double twob = 2.0 * beta;
    for (int sw = 0; sw < n_sweeps; ++sw)
        for (int cc = 0; cc < n_colors; ++cc) {
            const int col = dir ? (n_colors - 1 - cc) : cc;
            for (int q = col_start[col] + threadIdx.x; q < col_start[col + 1]; q += blockDim.x) {
                const int v = col_sites[q];
                double sum = 0.0;
                int oi = 0;
                for (int c = 0; c < em.n_class; ++c) {
                    int n = 0;
                    for (int t = 0; t < em.noff[c]; ++t, ++oi) {
                        const int b1 = shift_site(v, N, Lx, Ly, M, em.off + 3 * oi, 1);
                        const int b2 = shift_site(v, N, Lx, Ly, M, em.off + 3 * oi, -1);
                        if (b1 != v) n += s[b1];
                        if (b2 != v) n += s[b2];
                    }
                    sum = __dadd_rn(sum, __dmul_rn(em.J[c], (double)n));
                }
                const int sv = s[v];
                const double av = __dmul_rn(__dmul_rn(twob, sum), (double)sv);
                const int tau = v / N, i = v % N;
                const double u = philox_uniform(key, (uint32_t)i, (uint32_t)tau, step,
                                                PURPOSE_EFF | ((uint32_t)sw << 8));
                const double lu = log(u);
                if (fabs(av - lu) <= MARGIN) mg++;
                if (lu < av) {
                    s[v] = (int8_t)(-sv);
                    acc++;
                }
            }
            __syncthreads();
        }
    if (SMEM) {
        for (int v = threadIdx.x; v < V; v += blockDim.x) gs[v] = s[v];
    }
    __shared__ long long r1[32], r2[32];
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_down_sync(0xffffffffu, acc, o);
        mg += __shfl_down_sync(0xffffffffu, mg, o);
    }
    if ((threadIdx.x & 31) == 0) { r1[threadIdx.x >> 5] = acc; r2[threadIdx.x >> 5] = mg; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t1 = 0, t2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t1 += r1[w]; t2 += r2[w]; }
        if (n_accept) n_accept[b] += t1;
        if (n_margin) n_margin[b] += t2;
    }
}

// f_c(C) = sum_x sum_{o in c} s_x s_{x+o} (self-pairs give 1), one CTA per
// configuration; out[b*n_class + c].
__global__ void k_features(const int8_t *s_all, int Lx, int Ly, int M, const __grid_constant__ EffModel em,
                           long long *out)
{
    const int b = blockIdx.x;
    const int N = Lx * Ly, V = N * M;
    const int8_t *s = s_all + (long long)b * V;
    __shared__ long long red[32];
    const int n_class = em.n_class;
    int oi = 0;
    for (int c = 0; c < n_class; ++c) {
        long long acc = 0;
        for (int t = 0; t < em.noff[c]; ++t, ++oi)
            for (int v = threadIdx.x; v < V; v += blockDim.x)
                acc += s[v] * s[shift_site(v, N, Lx, Ly, M, em.off + 3 * oi, 1)];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            out[(long long)b * n_class + c] = t;
        }
        __syncthreads();
    }
}

// Eq. 4 in log form, per chain:
//   log r = [lw1 - lw0] - [-beta sum_c J_c (f1_c - f0_c)],  accept iff log u < log r.
__global__ void k_cumulative_accept(const double *lw1, double *lw0, const long long *f0, const long long *f1,
                                    const __grid_constant__ EffModel em, double beta, uint64_t seed, uint32_t step, int B,
                                    int *accepted, int *accept_count, double *log_r, long long *margin,
                                    const uint32_t *d_step)
{
    if (d_step) step = *d_step;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int n_class = em.n_class;
    double acc = 0.0;
    for (int c = 0; c < n_class; ++c)
        acc = __dadd_rn(acc, __dmul_rn(em.J[c], (double)(f1[(long long)b * n_class + c] - f0[(long long)b * n_class + c])));
    const double dlweff = __dmul_rn(-beta, acc);
    const double lr = __dadd_rn(__dadd_rn(lw1[b], -lw0[b]), -dlweff);
    const uint64_t key = seed + ((uint64_t)b << 32);
    const double u = philox_uniform(key, 0, 0, step, PURPOSE_ACCEPT);
    const double lu = log(u);
    if (margin && fabs(lr - lu) <= MARGIN) margin[b]++;
    const int a = lu < lr;
    accepted[b] = a;
    if (a) lw0[b] = lw1[b];
    if (accept_count) accept_count[b] += a;
    if (log_r) log_r[b] = lr;
}

// s[b] <- s'[b] where accepted[b]
__global__ void k_commit(int8_t *s, const int8_t *sp, const int *accepted, long long V)
{
    const int b = blockIdx.y;
    if (!accepted[b]) return;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < V;
         e += (long long)gridDim.x * blockDim.x)
        s[(long long)b * V + e] = sp[(long long)b * V + e];
}

// ------------------------------------------------------------ launchers
static inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

void launch_check_field(sldqmc_ctx *c, const int8_t *d_s, long long n)
{
    int g = cdiv(n, 256);
    if (g > 1024) g = 1024;
    if (g < 1) g = 1;
    k_check_field<<<g, 256, 0, c->st>>>(d_s, n, c->d_flag);
    c->launches++;
}

void launch_log_bare(sldqmc_ctx *c, const int8_t *d_s, int B, double *out, int accumulate)
{
    k_log_bare<<<B, 256, 0, c->st>>>(d_s, c->p.Lx, c->p.Ly, c->M, c->dtauJ, c->Ktau, out, accumulate);
    c->launches++;
}

void launch_local_flips(sldqmc_ctx *c, double *Gp, double *Gm, int8_t *d_s, int B, int tau,
                        uint32_t sweep, uint64_t seed, long long *stats)
{
    LocalArgs a;
    a.Gp = Gp; a.Gm = Gm; a.nn = c->nn; a.s = d_s;
    a.Lx = c->p.Lx; a.Ly = c->p.Ly; a.M = c->M; a.tau = tau; a.sweep = sweep; a.seed = seed;
    a.dtxi = c->p.dtau * c->p.xi; a.dtauJ = c->dtauJ; a.Kt = c->Ktau; a.stats = stats;
    size_t sh = sizeof(double) * 5 * (size_t)c->N;
    int nt = c->N * c->N >= 512 ? 512 : 256;
    prof_begin(c, SLDQMC_KC_LOCAL, 0.0, "local_flips");
    k_local_flips<<<B, nt, sh, c->st>>>(a);
    prof_end(c);
    c->launches++;
}

void launch_drift(sldqmc_ctx *c, const double *Gw, const double *Gf, int B2x, int B, long long *stats)
{
    dim3 g(cdiv(c->nn, 256) < 32 ? cdiv(c->nn, 256) : 32, B2x);
    k_drift<<<g, 256, 0, c->st>>>(Gw, Gf, c->nn, stats, B);
    c->launches++;
}

void launch_eff_sweeps(sldqmc_ctx *c, int8_t *d_s, int B, int n_sweeps, uint64_t seed, uint32_t step,
                       int dir, long long *n_accept, long long *n_margin)
{
    const long long V = (long long)c->N * c->M;
    const int nt = 1024;
    const EffModel em = eff_model_of(c);
    prof_begin(c, SLDQMC_KC_EFF, 0.0, "eff_sweeps");
    if (V <= 200 * 1024) {
        k_eff_sweeps<true><<<B, nt, (size_t)V, c->st>>>(d_s, c->p.Lx, c->p.Ly, c->M, c->p.beta,
                                                        em, c->d_col_start, c->d_col_sites,
                                                        c->n_colors, n_sweeps, seed, step, dir,
                                                        n_accept, n_margin, c->step_dev);
    } else {
        k_eff_sweeps<false><<<B, nt, 0, c->st>>>(d_s, c->p.Lx, c->p.Ly, c->M, c->p.beta, em,
                                                 c->d_col_start, c->d_col_sites, c->n_colors, n_sweeps,
                                                 seed, step, dir, n_accept, n_margin, c->step_dev);
    }
    prof_end(c);
    c->launches++;
}

void launch_features(sldqmc_ctx *c, const int8_t *d_s, int B, long long *out)
{
    k_features<<<B, 512, 0, c->st>>>(d_s, c->p.Lx, c->p.Ly, c->M, eff_model_of(c), out);
    c->launches++;
}

void launch_cumulative_accept(sldqmc_ctx *c, const double *lw1, double *lw0, const long long *f0,
                              const long long *f1, uint64_t seed, uint32_t step, int B, int *accepted,
                              int *accept_count, double *log_r, long long *margin)
{
    k_cumulative_accept<<<cdiv(B, 128), 128, 0, c->st>>>(lw1, lw0, f0, f1, eff_model_of(c), c->p.beta, seed,
                                                        step, B, accepted, accept_count, log_r, margin,
                                                        c->step_dev);
    c->launches++;
}

void launch_commit(sldqmc_ctx *c, int8_t *d_s, const int8_t *d_sp, const int *accepted, int B)
{
    const long long V = (long long)c->N * c->M;
    dim3 g(cdiv(V, 256) < 64 ? cdiv(V, 256) : 64, B);
    k_commit<<<g, 256, 0, c->st>>>(d_s, d_sp, accepted, V);
    c->launches++;
}

__global__ void k_step_advance(uint32_t *d_step) { *d_step += 1u; }

void launch_step_advance(sldqmc_ctx *c, uint32_t *d_step)
{
    k_step_advance<<<1, 1, 0, c->st>>>(d_step);
    c->launches++;
}

void set_eff_smem_limits()
{
    cudaFuncSetAttribute(k_eff_sweeps<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_local_flips, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace sldqmc
