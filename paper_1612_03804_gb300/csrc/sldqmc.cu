// sldqmc.cu -- context management and the C ABI of include/sldqmc.h.
//
// Everything numerical runs in this library's kernels on the context's
// stream; the host side only validates arguments, sizes workspaces, orders
// launches and copies inputs and results.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace sldqmc {
// stab.cu
void launch_init_udv(sldqmc_ctx *c, double *Ut, double *V, int B);
void stabilize(sldqmc_ctx *c, double *Xt, double *Wc, double *Y, int B, int passes);
void finalize(sldqmc_ctx *c, const double *Ut, int B, double *d_ld, int *d_sign, double *d_G,
              double scale, int accumulate);
// mc.cu
void launch_check_field(sldqmc_ctx *c, const int8_t *d_s, long long n);
void launch_log_bare(sldqmc_ctx *c, const int8_t *d_s, int B, double *out, int accumulate);
void launch_local_flips(sldqmc_ctx *c, double *Gp, double *Gm, int8_t *d_s, int B, int tau,
                        uint32_t sweep, uint64_t seed, long long *stats);
void launch_drift(sldqmc_ctx *c, const double *Gw, const double *Gf, int B2x, int B, long long *stats);
void launch_local_flips_delayed(sldqmc_ctx *c, double *Gp, double *Gm, double *U, double *V, int8_t *d_s, int B,
                                int tau, int i0, int ns, uint32_t sweep, uint64_t seed, long long *stats);
void launch_eff_sweeps(sldqmc_ctx *c, int8_t *d_s, int B, int n_sweeps, uint64_t seed, uint32_t step,
                       int dir, long long *n_accept, long long *n_margin);
void launch_features(sldqmc_ctx *c, const int8_t *d_s, int B, long long *out);
void launch_cumulative_accept(sldqmc_ctx *c, const double *lw1, double *lw0, const long long *f0,
                              const long long *f1, uint64_t seed, uint32_t step, int B, int *accepted,
                              int *accept_count, double *log_r, long long *margin);
void launch_commit(sldqmc_ctx *c, int8_t *d_s, const int8_t *d_sp, const int *accepted, int B);
void set_eff_smem_limits();
void launch_step_advance(sldqmc_ctx *c, uint32_t *d_step);
void stab_set_limits(int Npad);
// tc_gemm.cu
void tc_convert_E(sldqmc_ctx *c);
void launch_wait_selftest(sldqmc_ctx *c, int limit);
int tc_prepare(sldqmc_ctx *c);
void tc_release(sldqmc_ctx *c);
void tc_chain_block(sldqmc_ctx *c, const double *Ut, const int8_t *d_s, int B, double cu, double cd,
                    const int *slices, int nb, double *Xt_out, double *scratch_a, double *scratch_b);
int tc_set_tile_n(sldqmc_ctx *c, int bn);
}  // namespace sldqmc

using namespace sldqmc;

namespace sldqmc {

void prof_begin(sldqmc_ctx *c, int cls, double flops, const char *site)
{
    Prof *p = c->prof;
    if (!p || !p->on) return;
    while (p->pool.size() < p->used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { p->on = false; return; }
        p->pool.push_back(e);
    }
    cudaEvent_t a = p->pool[p->used], b = p->pool[p->used + 1];
    p->used += 2;
    cudaEventRecord(a, c->st);
    p->recs.push_back(ProfRec{a, b, cls, flops, site});
    p->open_cls = cls;
}

void prof_end(sldqmc_ctx *c)
{
    Prof *p = c->prof;
    if (!p || !p->on || p->open_cls < 0) return;
    cudaEventRecord(p->recs.back().b, c->st);
    p->open_cls = -1;
}

void gemm_ctx(sldqmc_ctx *c, const GemmF64 &g, bool TA, bool TB)
{
    const bool timed = c->prof && c->prof->on;
    if (timed) prof_begin(c, SLDQMC_KC_GEMM_F64, gemm_flops(g), "gemm_f64");
    gemm_f64(g, TA, TB, c->st);
    if (timed) prof_end(c);
    c->launches++;
}

}  // namespace sldqmc

namespace {

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Ring propagator e^{c A_1} on a ring of length L by its Fourier sum
// E1(d) = (1/L) sum_n exp(2c cos k_n) cos(k_n d), k_n = 2 pi n / L; L = 1
// has no bond.  One thread per distance d.
__global__ void k_ring(int L, double c, double *E1)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= L) return;
    if (L == 1) { E1[0] = 1.0; return; }
    double acc = 0.0;
    for (int n = 0; n < L; ++n) {
        const double k = 2.0 * M_PI * (double)n / (double)L;
        acc += exp(2.0 * c * cos(k)) * cos(k * (double)d);
    }
    E1[d] = acc / (double)L;
}

// K = -t A - mu I and the separable exp(-+dtau K) = e^{+-dtau mu} Ex (x) Ey.
__global__ void k_build_K(int Lx, int Ly, double t, double mu, double dtau, const double *ex_p,
                          const double *ey_p, const double *ex_m, const double *ey_m, double *K,
                          double *E, double *Einv)
{
    const int N = Lx * Ly;
    const long long nn = (long long)N * N;
    const double sp = exp(dtau * mu), sm = exp(-dtau * mu);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / N), j = (int)(e % N);
        const int xi = i % Lx, yi = i / Lx, xj = j % Lx, yj = j / Lx;
        int dx = (xi - xj) % Lx; if (dx < 0) dx += Lx;
        int dy = (yi - yj) % Ly; if (dy < 0) dy += Ly;
        E[e] = sp * ex_p[dx] * ey_p[dy];
        Einv[e] = sm * ex_m[dx] * ey_m[dy];
        double k = (i == j) ? -mu : 0.0;
        if (Lx > 1) {
            int dxa = (xj - xi) % Lx; if (dxa < 0) dxa += Lx;
            if (yi == yj) {
                if (dxa == 1) k -= t;
                if (dxa == Lx - 1) k -= t;
            }
        }
        if (Ly > 1) {
            int dya = (yj - yi) % Ly; if (dya < 0) dya += Ly;
            if (xi == xj) {
                if (dya == 1) k -= t;
                if (dya == Ly - 1) k -= t;
            }
        }
        K[e] = k;
    }
}

int flag_to_status(int f)
{
    if (f & FLAG_ARG) return SLDQMC_ERR_ARG;
    if (f & FLAG_TIMEOUT) return SLDQMC_ERR_TIMEOUT;
    if (f & FLAG_NUMERICAL) return SLDQMC_ERR_NUMERICAL;
    return SLDQMC_OK;
}

int sync_and_flag(sldqmc_ctx *c)
{
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return SLDQMC_ERR_CUDA;
    if (c->twin && cudaStreamSynchronize(c->twin->st) != cudaSuccess) return SLDQMC_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return SLDQMC_ERR_CUDA;
    int f = 0, g = 0;
    if (cudaMemcpy(&f, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SLDQMC_ERR_CUDA;
    if (f) cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->st);
    if (c->twin) {
        if (cudaMemcpy(&g, c->twin->d_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SLDQMC_ERR_CUDA;
        if (g) cudaMemsetAsync(c->twin->d_flag, 0, sizeof(int), c->twin->st);
    }
    return flag_to_status(f | g);
}

template <typename T>
int dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) return SLDQMC_OK;
    if (cudaMalloc((void **)p, sizeof(T) * count) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return SLDQMC_ERR_OOM;
    }
    return SLDQMC_OK;
}

bool host_field_ok(const int8_t *s, long long n)
{
    for (long long e = 0; e < n; ++e)
        if (s[e] != 1 && s[e] != -1) return false;
    return true;
}

// One batch of weight (or Green's function) evaluations on device data.
// Slices are processed in the cyclic order tau0, tau0+1, ... (0-based),
// i.e. the product B_tau0 .. B_1 B_M .. B_{tau0+1}.
int weight_run(sldqmc_ctx *c, const int8_t *d_s, int B, int eta, int tau0, double *d_ld, int *d_sign,
               double *d_G, double scale, int accumulate)
{
    const int N = c->N, M = c->M;
    const long long nn = c->nn;
    const double cu = c->ex_scale[eta < 0][0], cd = c->ex_scale[eta < 0][1];
    double *Ut = c->buf[0], *Yb = c->buf[5], *X1 = c->buf[2], *X2 = c->buf[3];
    launch_init_udv(c, Ut, c->buf[1], B);
    std::vector<int> slices;
    for (int m = 0; m < M; m += c->p.n_wrap) {
        const int nb = std::min(c->p.n_wrap, M - m);
        double *Xt;
        if (c->kinetic == SLDQMC_KINETIC_SEPARABLE) {
            sep_chain_block(c, Ut, d_s, B, cu, cd, (tau0 + m) % M, nb, c->d_Einv + nn, X1);
            Xt = X1;
        } else if (c->p.prec == SLDQMC_FP64) {
            const double *cur = Ut;
            double *outs[2] = {X1, X2};
            int o = 0;
            for (int j = 0; j < nb; ++j) {
                const int slice = (tau0 + m + j) % M;
                GemmF64 g = gemm_desc(N, N, N, cur, N, nn, c->d_E, N, 0, outs[o], N, nn, B);
                g.cu = cu; g.cd = cd;
                if (j == 0) { g.s_k = d_s + (long long)slice * N; g.sSk = (long long)M * N; }
                if (j < nb - 1) { g.s_n = d_s + (long long)((tau0 + m + j + 1) % M) * N; g.sSn = (long long)M * N; }
                gemm_ctx(c, g, false, false);
                cur = outs[o];
                o ^= 1;
            }
            Xt = const_cast<double *>(cur);
        } else {
            slices.assign(nb, 0);
            for (int j = 0; j < nb; ++j) slices[j] = (tau0 + m + j) % M;
            tc_chain_block(c, Ut, d_s, B, cu, cd, slices.data(), nb, X1, X2, Yb);
            Xt = X1;
        }
        stabilize(c, Xt, Ut, Yb, B, m + nb >= M ? 2 : 1);
        std::swap(Ut, Yb);
    }
    finalize(c, Ut, B, d_ld, d_sign, d_G, scale, accumulate);
    return SLDQMC_OK;
}

// A second context with the same parameters, twice the batch capacity and
// its own stream, for the two flavours of the exact log weight.  B_tau(eta =
// -1) for the field s is B_tau(eta = +1) for the field -s (the flavour only
// picks which of the two scale constants goes with s = +1), so the items
// [s_1 .. s_B, -s_1 .. -s_B] at eta = +1 give ld(+1) and ld(-1) of every
// configuration in one batch, and each latency-bound kernel of the
// stabilisation (diagonal-block factors, panel products, pivot tournaments)
// serves both flavours in one launch.  That is the form taken while 2B
// items fit in one wave of CTAs (2B <= SMs); for larger batches those
// kernels already fill the GPU, and the flavours run as two batches on the
// two streams at once, where each fills the other's serial phases.  Created
// on first use when its workspace takes under a third of the free device
// memory; otherwise the flavours run in sequence on the context itself.
sldqmc_ctx *get_twin(sldqmc_ctx *c)
{
    if (c->no_twin) return nullptr;
    if (c->twin) return c->twin;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        c->no_twin = 1;
        return nullptr;
    }
    const double ws_bytes = 2.0 * (12.0 * (double)c->nn * 8.0 * c->cap + 2.0 * c->M * (double)c->N * c->cap);
    if (ws_bytes * 3.0 > (double)free_b) { c->no_twin = 1; return nullptr; }
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->no_twin = 1;
        return nullptr;
    }
    sldqmc_ctx *t = nullptr;
    sldqmc_params p = c->p;
    p.max_batch = 2 * c->cap;
    if (sldqmc_create(&p, (void *)st, &t) != SLDQMC_OK ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        if (t) sldqmc_destroy(t);
        cudaStreamDestroy(st);
        cudaGetLastError();
        c->no_twin = 1;
        return nullptr;
    }
    t->no_twin = 1;
    t->kinetic = c->kinetic;
    if (c->tile_n == 128) tc_set_tile_n(t, 128);
    t->tile_n = c->tile_n;
    c->twin = t;
    return t;
}

// out = [s; -s] for B configurations of V spins each.
__global__ void k_pair_fields(const int8_t *__restrict__ s, int8_t *__restrict__ out, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int8_t v = s[i];
        out[i] = v;
        out[n + i] = (int8_t)(-v);
    }
}

__global__ void k_add_vec(double *a, const double *b, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B) a[i] += b[i];
}

// d_lw[b] = ld[b] + ld[B + b]: the two flavours' 2 log|det| of configuration b.
__global__ void k_add_halves(double *d_lw, const double *ld, int B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B) d_lw[i] = ld[i] + ld[B + i];
}

// log omega = log phi + 2 ld(+1) + 2 ld(-1) into d_lw.
int log_weight_run(sldqmc_ctx *c, const int8_t *d_s, int B, double *d_lw)
{
    sldqmc_ctx *t = (c->prof && c->prof->on) ? nullptr : get_twin(c);
    if (t && 2 * B > t->cap) t = nullptr;  // callers chunk by the context's capacity; never more
    if (!t) {
        int rc = weight_run(c, d_s, B, 1, 0, d_lw, nullptr, nullptr, 2.0, 0);
        if (rc) return rc;
        rc = weight_run(c, d_s, B, -1, 0, d_lw, nullptr, nullptr, 2.0, 1);
        if (rc) return rc;
        launch_log_bare(c, d_s, B, d_lw, 1);
        return SLDQMC_OK;
    }
    cudaStream_t tst = t->st;
    cudaEventRecord(c->ev_fork, c->st);
    cudaStreamWaitEvent(tst, c->ev_fork, 0);
    if (2 * B <= c->num_sms) {
        // one batch [s; -s] at eta = +1 on the twin
        const long long n = (long long)B * c->M * c->N;
        k_pair_fields<<<(int)std::min<long long>(cdiv(n, 256), 4096), 256, 0, tst>>>(d_s, t->d_s_one, n);
        t->launches++;
        int rc = weight_run(t, t->d_s_one, 2 * B, 1, 0, t->d_ld_tmp, nullptr, nullptr, 2.0, 0);
        if (rc) return rc;
        cudaEventRecord(c->ev_join, tst);
        cudaStreamWaitEvent(c->st, c->ev_join, 0);
        k_add_halves<<<cdiv(B, 128), 128, 0, c->st>>>(d_lw, t->d_ld_tmp, B);
    } else {
        // eta = -1 on the twin's stream while eta = +1 runs on the context's
        int rc = weight_run(t, d_s, B, -1, 0, t->d_ld_tmp, nullptr, nullptr, 2.0, 0);
        if (rc) return rc;
        rc = weight_run(c, d_s, B, 1, 0, d_lw, nullptr, nullptr, 2.0, 0);
        if (rc) return rc;
        cudaEventRecord(c->ev_join, tst);
        cudaStreamWaitEvent(c->st, c->ev_join, 0);
        k_add_vec<<<cdiv(B, 128), 128, 0, c->st>>>(d_lw, t->d_ld_tmp, B);
    }
    c->launches++;
    launch_log_bare(c, d_s, B, d_lw, 1);
    return SLDQMC_OK;
}

int ensure_local_buffers(sldqmc_ctx *c)
{
    if (c->d_G[0]) return SLDQMC_OK;
    const size_t n = (size_t)c->cap * c->nn;
    const size_t uv = 2 * (size_t)c->cap * 32 * c->N;
    int rc = dalloc(&c->d_G[0], 6 * n + 2 * uv);
    if (rc) return rc;
    c->d_G[1] = c->d_G[0] + n;
    c->d_U = c->d_G[0] + 6 * n;
    c->d_V = c->d_U + uv;
    return SLDQMC_OK;
}

// The flips of slice tau: one launch of immediate rank-1 updates, or blocks
// of local_rank sites whose pending corrections G -= U V are applied by one
// batched GEMM per flavour after each block.
static void local_flips_slice(sldqmc_ctx *c, double *Gp, double *Gm, int8_t *d_s, int B, int tau, uint32_t sweep,
                              uint64_t seed)
{
    const int N = c->N;
    if (c->local_rank <= 1) {
        launch_local_flips(c, Gp, Gm, d_s, B, tau, sweep, seed, c->d_stats);
        return;
    }
    double *G[2] = {Gp, Gm};
    for (int i0 = 0; i0 < N; i0 += c->local_rank) {
        const int ns = std::min(c->local_rank, N - i0);
        launch_local_flips_delayed(c, Gp, Gm, c->d_U, c->d_V, d_s, B, tau, i0, ns, sweep, seed, c->d_stats);
        for (int f = 0; f < 2; ++f) {
            const long long so = (long long)f * c->cap * 32 * N;
            GemmF64 g = gemm_desc(N, N, 32, c->d_U + so, 32, 32LL * N, c->d_V + so, N, 32LL * N, G[f], N, c->nn, B);
            g.alpha = -1.0;
            g.beta = 1.0;
            gemm_ctx(c, g, false, false);
        }
    }
}

// Greedy colouring of the effective model's interaction graph: sites
// v = tau*N + i in increasing order take the smallest colour not used by an
// already coloured neighbour (v +- o for every offset o, self excluded).
void build_colouring(sldqmc_ctx *c, std::vector<int> &start, std::vector<int> &sites)
{
    const int Lx = c->p.Lx, Ly = c->p.Ly, M = c->M, N = c->N, V = N * M;
    std::vector<int> colour(V, -1);
    std::vector<int> nbr;
    int ncol = 0;
    auto wrap = [](int a, int L) { a %= L; return a < 0 ? a + L : a; };
    std::vector<char> used;
    for (int v = 0; v < V; ++v) {
        const int tau = v / N, i = v % N, x = i % Lx, y = i / Lx;
        used.assign(ncol + 2, 0);
        for (int q = 0; q < c->n_off_total; ++q) {
            const int *o = c->h_offsets + 3 * q;
            for (int sg = -1; sg <= 1; sg += 2) {
                const int w = wrap(tau + sg * o[2], M) * N + wrap(x + sg * o[0], Lx) + Lx * wrap(y + sg * o[1], Ly);
                if (w != v && colour[w] >= 0) used[colour[w]] = 1;
            }
        }
        int col = 0;
        while (used[col]) ++col;
        colour[v] = col;
        ncol = std::max(ncol, col + 1);
    }
    start.assign(ncol + 1, 0);
    for (int v = 0; v < V; ++v) start[colour[v] + 1]++;
    for (int k = 0; k < ncol; ++k) start[k + 1] += start[k];
    sites.assign(V, 0);
    std::vector<int> pos(start.begin(), start.end() - 1);
    for (int v = 0; v < V; ++v) sites[pos[colour[v]]++] = v;
}

// Least squares min |A x - y| for a tall n x p matrix (column-major
// work copy) by modified Gram-Schmidt applied twice (reorthogonalised),
// then back substitution.  Host FP64; p is at most 33.
int lstsq_mgs2(int n, int p, const std::vector<double> &A_rowmajor, const std::vector<double> &y,
               std::vector<double> &x)
{
    std::vector<double> Q((size_t)n * p), R((size_t)p * p, 0.0);
    for (int r = 0; r < n; ++r)
        for (int k = 0; k < p; ++k) Q[(size_t)k * n + r] = A_rowmajor[(size_t)r * p + k];
    for (int k = 0; k < p; ++k) {
        double *qk = &Q[(size_t)k * n];
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < k; ++j) {
                const double *qj = &Q[(size_t)j * n];
                double d = 0.0;
                for (int r = 0; r < n; ++r) d += qj[r] * qk[r];
                R[(size_t)j * p + k] += d;
                for (int r = 0; r < n; ++r) qk[r] -= d * qj[r];
            }
        double nrm = 0.0;
        for (int r = 0; r < n; ++r) nrm += qk[r] * qk[r];
        nrm = sqrt(nrm);
        if (!(nrm > 0.0)) return SLDQMC_ERR_NUMERICAL;
        R[(size_t)k * p + k] = nrm;
        for (int r = 0; r < n; ++r) qk[r] /= nrm;
    }
    std::vector<double> qty(p, 0.0);
    std::vector<double> res(y);
    for (int k = 0; k < p; ++k) {
        const double *qk = &Q[(size_t)k * n];
        double d = 0.0;
        for (int r = 0; r < n; ++r) d += qk[r] * res[r];
        qty[k] = d;
        for (int r = 0; r < n; ++r) res[r] -= d * qk[r];
    }
    x.assign(p, 0.0);
    for (int k = p - 1; k >= 0; --k) {
        double acc = qty[k];
        for (int j = k + 1; j < p; ++j) acc -= R[(size_t)k * p + j] * x[j];
        x[k] = acc / R[(size_t)k * p + k];
    }
    return SLDQMC_OK;
}

// One cumulative update (steps iii + iv) of B chains, stream-ordered: copy,
// effective sweeps, features, exact log weight of the proposal, Eq. 4
// acceptance, commit.
int cumulative_step(sldqmc_ctx *c, int8_t *d_s, double *d_logw, int B, int n_eff, uint64_t seed, uint32_t step,
                    int *d_accepts, double *d_log_r)
{
    const long long V = (long long)c->N * c->M;
    int8_t *sp = c->d_s_tmp;
    int *accepted = c->d_sg_tmp;  // B ints of scratch (2*cap available)
    cudaMemcpyAsync(sp, d_s, (size_t)(V * B), cudaMemcpyDeviceToDevice, c->st);
    launch_eff_sweeps(c, sp, B, n_eff, seed, step, -1, nullptr, nullptr);
    launch_features(c, d_s, B, c->d_feat0);
    launch_features(c, sp, B, c->d_feat1);
    int rc = log_weight_run(c, sp, B, c->d_ld_tmp);
    if (rc) return rc;
    launch_cumulative_accept(c, c->d_ld_tmp, d_logw, c->d_feat0, c->d_feat1, seed, step, B, accepted, d_accepts,
                             d_log_r, nullptr);
    launch_commit(c, d_s, sp, accepted, B);
    return SLDQMC_OK;
}

}  // namespace

namespace sldqmc {

// Entry points for the allocation-free variant in noalloc.cu: the same
// kernels and launch sequence as a context's weight evaluation, on
// caller-provided workspace.
void build_K_into(sldqmc_ctx *c, double *ring)
{
    const sldqmc_params *p = &c->p;
    double *ex_p = ring, *ey_p = ex_p + p->Lx, *ex_m = ey_p + p->Ly, *ey_m = ex_m + p->Lx;
    k_ring<<<cdiv(p->Lx, 128), 128, 0, c->st>>>(p->Lx, p->dtau * p->t, ex_p);
    k_ring<<<cdiv(p->Ly, 128), 128, 0, c->st>>>(p->Ly, p->dtau * p->t, ey_p);
    k_ring<<<cdiv(p->Lx, 128), 128, 0, c->st>>>(p->Lx, -p->dtau * p->t, ex_m);
    k_ring<<<cdiv(p->Ly, 128), 128, 0, c->st>>>(p->Ly, -p->dtau * p->t, ey_m);
    int g = cdiv(c->nn, 256);
    if (g > 4096) g = 4096;
    k_build_K<<<g, 256, 0, c->st>>>(p->Lx, p->Ly, p->t, p->mu, p->dtau, ex_p, ey_p, ex_m, ey_m, c->d_K, c->d_E,
                                    c->d_Einv);
    c->launches += 5;
}

int weight_run_into(sldqmc_ctx *c, const int8_t *d_s, int B, int eta, double *d_ld, int *d_sign)
{
    launch_check_field(c, d_s, (long long)c->N * c->M * B);
    return weight_run(c, d_s, B, eta, 0, d_ld, d_sign, nullptr, 1.0, 0);
}

}  // namespace sldqmc

extern "C" {

const char *sldqmc_strerror(int status)
{
    switch (status) {
    case SLDQMC_OK: return "ok";
    case SLDQMC_ERR_ARG: return "invalid argument";
    case SLDQMC_ERR_OOM: return "device out of memory";
    case SLDQMC_ERR_CUDA: return "CUDA runtime error";
    case SLDQMC_ERR_NUMERICAL: return "numerical failure (non-positive pivot or non-finite value)";
    case SLDQMC_ERR_TIMEOUT: return "device wait timed out";
    case SLDQMC_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
    }
}

long long sldqmc_kernel_launches(const sldqmc_ctx *ctx)
{
    return ctx ? ctx->launches + (ctx->twin ? ctx->twin->launches : 0) : 0;
}

int sldqmc_dims(const sldqmc_ctx *ctx, int *N, int *M)
{
    if (!ctx) return SLDQMC_ERR_ARG;
    if (N) *N = ctx->N;
    if (M) *M = ctx->M;
    return SLDQMC_OK;
}

int sldqmc_sync(sldqmc_ctx *ctx)
{
    if (!ctx) return SLDQMC_ERR_ARG;
    return sync_and_flag(ctx);
}

void sldqmc_destroy(sldqmc_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->st);
    if (c->twin) {
        cudaStream_t tst = c->twin->st;
        sldqmc_destroy(c->twin);
        cudaStreamDestroy(tst);
        cudaEventDestroy(c->ev_fork);
        cudaEventDestroy(c->ev_join);
    }
    tc_release(c);
    oz_release(c);
    if (c->prof) {
        for (cudaEvent_t e : c->prof->pool) cudaEventDestroy(e);
        delete c->prof;
    }
    cudaFree(c->d_flag);
    cudaFree(c->d_K);
    cudaFree(c->buf[0]);
    cudaFree(c->d_D);
    cudaFree(c->d_perm);
    cudaFree(c->d_s_tmp);
    cudaFree(c->d_G[0]);
    cudaFree(c->d_ld_tmp);
    cudaFree(c->d_stats);
    cudaFree(c->d_col_start);
    cudaFree(c->d_col_sites);
    cudaFree(c->d_feat0);
    cudaFree(c->d_step);
    free(c);
}

int sldqmc_create(const sldqmc_params *p, void *stream, sldqmc_ctx **out)
{
    if (!p || !out) return SLDQMC_ERR_ARG;
    *out = nullptr;
    if (p->Lx < 1 || p->Ly < 1 || p->n_wrap < 1 || p->max_batch < 1 || !(p->dtau > 0.0) ||
        !(p->beta > 0.0) || p->prec < 0 || p->prec > 3 || !isfinite(p->t) || !isfinite(p->mu) ||
        !isfinite(p->xi) || !isfinite(p->J_ising) || !(p->h > 0.0))
        return SLDQMC_ERR_ARG;
    const long long N = (long long)p->Lx * p->Ly;
    const long long M = llround(p->beta / p->dtau);
    if (M < 1 || fabs((double)M * p->dtau - p->beta) > 1e-12 * p->beta) return SLDQMC_ERR_ARG;
    if (N > 16384 || M > 100000) return SLDQMC_ERR_UNSUPPORTED;
    // Cholesky-QR of one block needs kappa(X)^2 eps << 1; kappa(X) is
    // bounded by exp(n_wrap dtau (8|t| + 2|xi|)).
    const double logk = (double)std::min<long long>(p->n_wrap, M) * p->dtau * (8.0 * fabs(p->t) + 2.0 * fabs(p->xi));
    if (logk > 16.0) return SLDQMC_ERR_UNSUPPORTED;

    sldqmc_ctx *c = (sldqmc_ctx *)calloc(1, sizeof(sldqmc_ctx));
    if (!c) return SLDQMC_ERR_OOM;
    c->p = *p;
    c->N = (int)N;
    c->M = (int)M;
    c->p.beta = (double)M * p->dtau;
    c->st = (cudaStream_t)stream;
    c->cap = p->max_batch;
    c->nn = N * N;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c->num_sms < 1) {
            cudaGetLastError();
            c->num_sms = 148;
        }
    }
    for (int e = 0; e < 2; ++e) {
        const double eta = e == 0 ? 1.0 : -1.0;
        c->ex_scale[e][0] = exp(eta * p->dtau * p->xi);
        c->ex_scale[e][1] = exp(-eta * p->dtau * p->xi);
    }
    c->dtauJ = p->dtau * p->J_ising;
    c->Ktau = -0.5 * log(tanh(p->dtau * p->h));
    c->prof = new Prof();
    c->local_rank = 1;
    c->tile_n = 64;
    int rc = SLDQMC_OK;
    const size_t nn = (size_t)c->nn, cap = (size_t)c->cap;
    if ((rc = dalloc(&c->d_flag, 1))) goto fail;
    cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->st);
    if ((rc = dalloc(&c->d_K, 3 * nn + 4 * (size_t)(p->Lx + p->Ly)))) goto fail;
    c->d_E = c->d_K + nn;
    c->d_Einv = c->d_E + nn;
    // 9 workspaces; W (index 4) is twice the size for the LU with a
    // right-hand side.
    if ((rc = dalloc(&c->buf[0], 10 * nn * cap))) goto fail;
    {
        double *q = c->buf[0];
        for (int k = 0; k < 9; ++k) {
            c->buf[k] = q;
            q += (k == 4 ? 2 : 1) * nn * cap;
        }
    }
    if ((rc = dalloc(&c->d_D, 2 * N * cap + cap + 4 * cap))) goto fail;
    c->d_Dp = c->d_D + N * cap;
    c->d_logacc = c->d_Dp + N * cap;
    c->d_ld_tmp = nullptr;
    if ((rc = dalloc(&c->d_perm, 2 * N * cap + 2 * cap + 2 * cap + 24 * 32 * cap))) goto fail;
    c->d_piv = c->d_perm + N * cap;
    c->d_sgn = c->d_piv + N * cap;
    c->d_sg_tmp = c->d_sgn + 2 * cap;
    c->d_tslu = c->d_sg_tmp + 2 * cap;
    if ((rc = dalloc(&c->d_s_tmp, 2 * (size_t)M * N * cap))) goto fail;
    c->d_s_one = c->d_s_tmp + (size_t)M * N * cap;
    if ((rc = dalloc(&c->d_ld_tmp, 4 * cap))) goto fail;
    c->d_ld_tmp2 = c->d_ld_tmp + cap;
    if ((rc = dalloc(&c->d_stats, 4 * cap + 8 * cap))) goto fail;
    if (p->prec != SLDQMC_FP64 && (rc = tc_prepare(c))) goto fail;
    if (p->prec != SLDQMC_FP64 && (rc = oz_prepare(c))) goto fail;
    {
        // build K, E, E^{-1}
        double *ex_p = c->d_Einv + nn, *ey_p = ex_p + p->Lx, *ex_m = ey_p + p->Ly, *ey_m = ex_m + p->Lx;
        k_ring<<<cdiv(p->Lx, 128), 128, 0, c->st>>>(p->Lx, p->dtau * p->t, ex_p);
        k_ring<<<cdiv(p->Ly, 128), 128, 0, c->st>>>(p->Ly, p->dtau * p->t, ey_p);
        k_ring<<<cdiv(p->Lx, 128), 128, 0, c->st>>>(p->Lx, -p->dtau * p->t, ex_m);
        k_ring<<<cdiv(p->Ly, 128), 128, 0, c->st>>>(p->Ly, -p->dtau * p->t, ey_m);
        int g = cdiv((long long)nn, 256);
        if (g > 4096) g = 4096;
        k_build_K<<<g, 256, 0, c->st>>>(p->Lx, p->Ly, p->t, p->mu, p->dtau, ex_p, ey_p, ex_m, ey_m, c->d_K,
                                        c->d_E, c->d_Einv);
        c->launches += 5;
    }
    if (p->prec != SLDQMC_FP64) tc_convert_E(c);
    set_eff_smem_limits();
    sep_set_limits();
    {
        int Npad = 1;
        while (Npad < N) Npad <<= 1;
        stab_set_limits(Npad);
    }
    rc = sync_and_flag(c);
    if (rc) goto fail;
    *out = c;
    return SLDQMC_OK;
fail:
    sldqmc_destroy(c);
    return rc;
}

int sldqmc_build_K(sldqmc_ctx *c, double *K, double *expmK, double *exppK)
{
    if (!c) return SLDQMC_ERR_ARG;
    const size_t bytes = sizeof(double) * (size_t)c->nn;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return SLDQMC_ERR_CUDA;
    if (K && cudaMemcpy(K, c->d_K, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return SLDQMC_ERR_CUDA;
    if (expmK && cudaMemcpy(expmK, c->d_E, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return SLDQMC_ERR_CUDA;
    if (exppK && cudaMemcpy(exppK, c->d_Einv, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return SLDQMC_ERR_CUDA;
    return SLDQMC_OK;
}

int sldqmc_weight_batch_dev(sldqmc_ctx *c, const int8_t *d_s, int B, int eta, double *d_ld, int *d_sign)
{
    if (!c || B < 0 || (B > 0 && (!d_s || !d_ld)) || (eta != 1 && eta != -1)) return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    launch_check_field(c, d_s, V * B);
    for (int b0 = 0; b0 < B; b0 += c->cap) {
        const int nb = std::min(c->cap, B - b0);
        int rc = weight_run(c, d_s + V * b0, nb, eta, 0, d_ld + b0, d_sign ? d_sign + b0 : nullptr, nullptr,
                            1.0, 0);
        if (rc) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? SLDQMC_OK : SLDQMC_ERR_CUDA;
}

int sldqmc_log_weight_batch_dev(sldqmc_ctx *c, const int8_t *d_s, int B, double *d_lw)
{
    if (!c || B < 0 || (B > 0 && (!d_s || !d_lw))) return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    launch_check_field(c, d_s, V * B);
    for (int b0 = 0; b0 < B; b0 += c->cap) {
        const int nb = std::min(c->cap, B - b0);
        int rc = log_weight_run(c, d_s + V * b0, nb, d_lw + b0);
        if (rc) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? SLDQMC_OK : SLDQMC_ERR_CUDA;
}

int sldqmc_weight_batch(sldqmc_ctx *c, const int8_t *s, int B, int eta, double *ld, int *sign)
{
    if (!c || B < 0 || (B > 0 && (!s || !ld)) || eta < -1 || eta > 1) return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    if (!host_field_ok(s, V * B)) return SLDQMC_ERR_ARG;
    std::vector<double> hld(B);
    std::vector<int> hsg(B, 1);
    for (int b0 = 0; b0 < B; b0 += c->cap) {
        const int nb = std::min(c->cap, B - b0);
        if (cudaMemcpyAsync(c->d_s_one, s + V * b0, (size_t)(V * nb), cudaMemcpyHostToDevice, c->st) != cudaSuccess)
            return SLDQMC_ERR_CUDA;
        int rc;
        if (eta == 0) {
            rc = weight_run(c, c->d_s_one, nb, 1, 0, c->d_ld_tmp, nullptr, nullptr, 2.0, 0);
            if (!rc) rc = weight_run(c, c->d_s_one, nb, -1, 0, c->d_ld_tmp, nullptr, nullptr, 2.0, 1);
        } else {
            rc = weight_run(c, c->d_s_one, nb, eta, 0, c->d_ld_tmp, c->d_sg_tmp, nullptr, 1.0, 0);
        }
        if (rc) return rc;
        if (cudaMemcpyAsync(hld.data() + b0, c->d_ld_tmp, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->st) !=
            cudaSuccess)
            return SLDQMC_ERR_CUDA;
        if (eta != 0 && cudaMemcpyAsync(hsg.data() + b0, c->d_sg_tmp, sizeof(int) * nb, cudaMemcpyDeviceToHost,
                                        c->st) != cudaSuccess)
            return SLDQMC_ERR_CUDA;
        rc = sync_and_flag(c);
        if (rc) return rc;
    }
    memcpy(ld, hld.data(), sizeof(double) * B);
    if (sign) memcpy(sign, hsg.data(), sizeof(int) * B);
    return SLDQMC_OK;
}

int sldqmc_weight(sldqmc_ctx *c, const int8_t *s, int eta, double *logabsdet, int *sign)
{
    return sldqmc_weight_batch(c, s, 1, eta, logabsdet, sign);
}

int sldqmc_green_batch_dev(sldqmc_ctx *c, const int8_t *d_s, int B, int eta, int tau, double *d_G,
                           double *d_ld, int *d_sign)
{
    if (!c || B < 0 || (eta != 1 && eta != -1) || tau < 0 || tau > c->M || (B > 0 && (!d_s || !d_G)))
        return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    launch_check_field(c, d_s, V * B);
    for (int b0 = 0; b0 < B; b0 += c->cap) {
        const int nb = std::min(c->cap, B - b0);
        int rc = weight_run(c, d_s + V * b0, nb, eta, tau % c->M, d_ld ? d_ld + b0 : c->d_ld_tmp,
                            d_sign ? d_sign + b0 : nullptr, d_G + (long long)b0 * c->nn, 1.0, 0);
        if (rc) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? SLDQMC_OK : SLDQMC_ERR_CUDA;
}

int sldqmc_green(sldqmc_ctx *c, const int8_t *s, int eta, int tau, double *G, double *logabsdet, int *sign)
{
    if (!c || !s || !G || (eta != 1 && eta != -1) || tau < 0 || tau > c->M) return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    if (!host_field_ok(s, V)) return SLDQMC_ERR_ARG;
    double *dG = c->buf[2];  // reuse a workspace slot not used by the finalisation's output copy
    // the chain uses buf[2] as scratch, so copy G out through the d_G staging of the local path
    int rc = ensure_local_buffers(c);
    if (rc) return rc;
    dG = c->d_G[0] + 2 * (size_t)c->cap * c->nn;
    if (cudaMemcpyAsync(c->d_s_one, s, (size_t)V, cudaMemcpyHostToDevice, c->st) != cudaSuccess) return SLDQMC_ERR_CUDA;
    rc = weight_run(c, c->d_s_one, 1, eta, tau % c->M, c->d_ld_tmp, c->d_sg_tmp, dG, 1.0, 0);
    if (rc) return rc;
    double ld;
    int sg;
    if (cudaMemcpyAsync(G, dG, sizeof(double) * c->nn, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaMemcpyAsync(&ld, c->d_ld_tmp, sizeof(double), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaMemcpyAsync(&sg, c->d_sg_tmp, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
        return SLDQMC_ERR_CUDA;
    rc = sync_and_flag(c);
    if (rc) return rc;
    if (logabsdet) *logabsdet = ld;
    if (sign) *sign = sg;
    return SLDQMC_OK;
}

int sldqmc_log_bare_weight(sldqmc_ctx *c, const int8_t *s, double *log_phi)
{
    if (!c || !s || !log_phi) return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    if (!host_field_ok(s, V)) return SLDQMC_ERR_ARG;
    if (cudaMemcpyAsync(c->d_s_one, s, (size_t)V, cudaMemcpyHostToDevice, c->st) != cudaSuccess) return SLDQMC_ERR_CUDA;
    launch_log_bare(c, c->d_s_one, 1, c->d_ld_tmp, 0);
    double v;
    if (cudaMemcpyAsync(&v, c->d_ld_tmp, sizeof(double), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
        return SLDQMC_ERR_CUDA;
    int rc = sync_and_flag(c);
    if (rc) return rc;
    *log_phi = v;
    return SLDQMC_OK;
}

// Fresh Gt_f = E^{-1} G(tau1) E for both flavours into dst[f] (B items).
static int fresh_gt(sldqmc_ctx *c, const int8_t *d_s, int B, int tau1, double *dstp, double *dstm)
{
    const int N = c->N;
    const long long nn = c->nn;
    double *Gt = c->d_G[0] + 2 * (size_t)c->cap * nn;  // G(tau1) staging
    double *T = Gt + (size_t)c->cap * nn;
    double *dst[2] = {dstp, dstm};
    for (int f = 0; f < 2; ++f) {
        int rc = weight_run(c, d_s, B, f == 0 ? 1 : -1, tau1 % c->M, c->d_ld_tmp2, nullptr, Gt, 1.0, 0);
        if (rc) return rc;
        GemmF64 g = gemm_desc(N, N, N, c->d_Einv, N, 0, Gt, N, nn, T, N, nn, B);
        gemm_ctx(c, g, false, false);
        GemmF64 h = gemm_desc(N, N, N, T, N, nn, c->d_E, N, 0, dst[f], N, nn, B);
        gemm_ctx(c, h, false, false);
    }
    return SLDQMC_OK;
}

// Gt <- D_tau E Gt E^{-1} D_tau^{-1} for both flavours, result into dst.
static void wrap_gt(sldqmc_ctx *c, const int8_t *d_s, int B, int tau, double *srcp, double *srcm,
                    double *dstp, double *dstm)
{
    const int N = c->N, M = c->M;
    const long long nn = c->nn;
    double *T = c->d_G[0] + 3 * (size_t)c->cap * nn;
    double *src[2] = {srcp, srcm}, *dst[2] = {dstp, dstm};
    for (int f = 0; f < 2; ++f) {
        const double cu = c->ex_scale[f][0], cd = c->ex_scale[f][1];
        GemmF64 g = gemm_desc(N, N, N, src[f], N, nn, c->d_Einv, N, 0, T, N, nn, B);
        g.s_n = d_s + (long long)tau * N; g.sSn = (long long)M * N;
        g.cu = 1.0 / cu; g.cd = 1.0 / cd;
        gemm_ctx(c, g, false, false);
        GemmF64 h = gemm_desc(N, N, N, c->d_E, N, 0, T, N, nn, dst[f], N, nn, B);
        h.s_m = d_s + (long long)tau * N; h.sSm = (long long)M * N;
        h.cu = cu; h.cd = cd;
        gemm_ctx(c, h, false, false);
    }
}

int sldqmc_local_sweep_batch_dev(sldqmc_ctx *c, int8_t *d_s, int B, uint64_t seed, uint64_t sweep0,
                                 int n_sweeps, sldqmc_stats *stats)
{
    if (!c || B < 1 || B > c->cap || !d_s || n_sweeps < 0) return SLDQMC_ERR_ARG;
    // the rank-1 flip kernel stages a column and a row of both Green's
    // functions and the slice's log-uniforms in shared memory: 5N doubles
    // within the 200 KB opt-in limit (the delayed path keeps its pairs in
    // global memory)
    if (c->N > 5120 && c->local_rank <= 1) return SLDQMC_ERR_UNSUPPORTED;
    int rc = ensure_local_buffers(c);
    if (rc) return rc;
    const long long V = (long long)c->N * c->M;
    launch_check_field(c, d_s, V * B);
    const long long nn = c->nn;
    cudaMemsetAsync(c->d_stats, 0, sizeof(long long) * 4 * B, c->st);
    double *Gp = c->d_G[0], *Gm = c->d_G[1];
    // wrapped copies live in areas 4 and 5 of the local-update buffer
    double *Wp = c->d_G[0] + 4 * (size_t)c->cap * nn, *Wm = Wp + (size_t)c->cap * nn;
    for (int sw = 0; sw < n_sweeps; ++sw) {
        const uint32_t sweep_id = (uint32_t)(sweep0 + (uint64_t)sw);
        for (int tau = 0; tau < c->M; ++tau) {
            if (tau == 0) {
                rc = fresh_gt(c, d_s, B, tau + 1, Gp, Gm);
                if (rc) return rc;
            } else if (tau % c->p.n_wrap == 0) {
                wrap_gt(c, d_s, B, tau, Gp, Gm, Wp, Wm);
                rc = fresh_gt(c, d_s, B, tau + 1, Gp, Gm);
                if (rc) return rc;
                launch_drift(c, Wp, Gp, B, B, c->d_stats);
                launch_drift(c, Wm, Gm, B, B, c->d_stats);
            } else {
                wrap_gt(c, d_s, B, tau, Gp, Gm, Wp, Wm);
                std::swap(Gp, Wp);
                std::swap(Gm, Wm);
            }
            local_flips_slice(c, Gp, Gm, d_s, B, tau, sweep_id, seed);
        }
    }
    if (stats) {
        std::vector<long long> h(4 * (size_t)B);
        if (cudaMemcpyAsync(h.data(), c->d_stats, sizeof(long long) * 4 * B, cudaMemcpyDeviceToHost, c->st) !=
            cudaSuccess)
            return SLDQMC_ERR_CUDA;
        rc = sync_and_flag(c);
        if (rc) return rc;
        for (int b = 0; b < B; ++b) {
            stats[b].accepted = h[4 * b];
            stats[b].proposed = h[4 * b + 1];
            stats[b].margin_events = h[4 * b + 2];
            double d;
            memcpy(&d, &h[4 * b + 3], sizeof(double));
            stats[b].max_drift = d;
        }
    }
    return cudaGetLastError() == cudaSuccess ? SLDQMC_OK : SLDQMC_ERR_CUDA;
}

int sldqmc_local_sweep(sldqmc_ctx *c, int8_t *s, uint64_t seed, uint64_t sweep0, int n_sweeps, sldqmc_stats *stats)
{
    if (!c || !s || n_sweeps < 0) return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    if (!host_field_ok(s, V)) return SLDQMC_ERR_ARG;
    if (cudaMemcpyAsync(c->d_s_one, s, (size_t)V, cudaMemcpyHostToDevice, c->st) != cudaSuccess) return SLDQMC_ERR_CUDA;
    sldqmc_stats st;
    int rc = sldqmc_local_sweep_batch_dev(c, c->d_s_one, 1, seed, sweep0, n_sweeps, &st);
    if (rc) return rc;
    std::vector<int8_t> tmp(V);
    if (cudaMemcpyAsync(tmp.data(), c->d_s_one, (size_t)V, cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
        return SLDQMC_ERR_CUDA;
    rc = sync_and_flag(c);
    if (rc) return rc;
    memcpy(s, tmp.data(), (size_t)V);
    if (stats) *stats = st;
    return SLDQMC_OK;
}

int sldqmc_set_effective_model(sldqmc_ctx *c, int n_class, const int *n_off, const int *offsets,
                               const double *J, double E0)
{
    if (!c || n_class < 1 || n_class > 32 || !n_off || !offsets || !J) return SLDQMC_ERR_ARG;
    int tot = 0;
    for (int k = 0; k < n_class; ++k) {
        if (n_off[k] < 1) return SLDQMC_ERR_ARG;
        tot += n_off[k];
    }
    if (tot > 64) return SLDQMC_ERR_ARG;
    for (int k = 0; k < n_class; ++k)
        if (!isfinite(J[k])) return SLDQMC_ERR_ARG;
    c->n_class = n_class;
    c->n_off_total = tot;
    memset(c->h_n_off, 0, sizeof(c->h_n_off));
    memset(c->h_offsets, 0, sizeof(c->h_offsets));
    memset(c->h_J, 0, sizeof(c->h_J));
    memcpy(c->h_n_off, n_off, sizeof(int) * n_class);
    memcpy(c->h_offsets, offsets, sizeof(int) * 3 * tot);
    memcpy(c->h_J, J, sizeof(double) * n_class);
    c->E0 = E0;
    std::vector<int> start, sites;
    build_colouring(c, start, sites);
    c->n_colors = (int)start.size() - 1;
    cudaFree(c->d_col_start);
    cudaFree(c->d_col_sites);
    c->d_col_start = nullptr;
    c->d_col_sites = nullptr;
    int rc = dalloc(&c->d_col_start, start.size());
    if (!rc) rc = dalloc(&c->d_col_sites, sites.size());
    if (rc) return rc;
    // stream-ordered copies: the context's stream need not synchronise with
    // the legacy default stream
    if (cudaMemcpyAsync(c->d_col_start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice, c->st) !=
            cudaSuccess ||
        cudaMemcpyAsync(c->d_col_sites, sites.data(), sizeof(int) * sites.size(), cudaMemcpyHostToDevice, c->st) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess) {
        cudaStreamSynchronize(c->st);
        return SLDQMC_ERR_CUDA;
    }
    if (!c->d_feat0) {
        rc = dalloc(&c->d_feat0, 2 * 32 * (size_t)c->cap);
        if (rc) return rc;
        c->d_feat1 = c->d_feat0 + 32 * (size_t)c->cap;
    }
    c->have_model = 1;
    return sync_and_flag(c);
}

int sldqmc_features(sldqmc_ctx *c, const int8_t *cfgs, int n_cfg, int64_t *F)
{
    if (!c || !c->have_model || n_cfg < 0 || (n_cfg > 0 && (!cfgs || !F))) return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    if (!host_field_ok(cfgs, V * n_cfg)) return SLDQMC_ERR_ARG;
    for (int b0 = 0; b0 < n_cfg; b0 += c->cap) {
        const int nb = std::min(c->cap, n_cfg - b0);
        if (cudaMemcpyAsync(c->d_s_one, cfgs + V * b0, (size_t)(V * nb), cudaMemcpyHostToDevice, c->st) != cudaSuccess)
            return SLDQMC_ERR_CUDA;
        launch_features(c, c->d_s_one, nb, c->d_feat0);
        if (cudaMemcpyAsync(F + (size_t)b0 * c->n_class, c->d_feat0, sizeof(long long) * nb * c->n_class,
                            cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
            return SLDQMC_ERR_CUDA;
        int rc = sync_and_flag(c);
        if (rc) return rc;
    }
    return SLDQMC_OK;
}

int sldqmc_fit_effective_action(sldqmc_ctx *c, const int8_t *cfgs, const double *logw, int n_cfg, double *J,
                                double *E0, double *r2)
{
    if (!c || !c->have_model || !cfgs || !J || n_cfg < c->n_class + 1) return SLDQMC_ERR_ARG;
    const int nc = c->n_class, p = nc + 1;
    std::vector<int64_t> F((size_t)n_cfg * nc);
    int rc = sldqmc_features(c, cfgs, n_cfg, F.data());
    if (rc) return rc;
    std::vector<double> y(n_cfg);
    if (logw) {
        memcpy(y.data(), logw, sizeof(double) * n_cfg);
    } else {
        const long long V = (long long)c->N * c->M;
        for (int b0 = 0; b0 < n_cfg; b0 += c->cap) {
            const int nb = std::min(c->cap, n_cfg - b0);
            if (cudaMemcpyAsync(c->d_s_one, cfgs + V * b0, (size_t)(V * nb), cudaMemcpyHostToDevice, c->st) !=
                cudaSuccess)
                return SLDQMC_ERR_CUDA;
            rc = log_weight_run(c, c->d_s_one, nb, c->d_ld_tmp);
            if (rc) return rc;
            if (cudaMemcpyAsync(y.data() + b0, c->d_ld_tmp, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->st) !=
                cudaSuccess)
                return SLDQMC_ERR_CUDA;
            rc = sync_and_flag(c);
            if (rc) return rc;
        }
    }
    // centre and scale the feature columns for conditioning, solve, map back
    std::vector<double> mean(nc, 0.0), sc(nc, 0.0);
    for (int r = 0; r < n_cfg; ++r)
        for (int k = 0; k < nc; ++k) mean[k] += (double)F[(size_t)r * nc + k];
    for (int k = 0; k < nc; ++k) mean[k] /= n_cfg;
    for (int r = 0; r < n_cfg; ++r)
        for (int k = 0; k < nc; ++k) {
            double d = (double)F[(size_t)r * nc + k] - mean[k];
            sc[k] += d * d;
        }
    for (int k = 0; k < nc; ++k) sc[k] = sc[k] > 0.0 ? sqrt(sc[k]) : 1.0;
    std::vector<double> A((size_t)n_cfg * p);
    for (int r = 0; r < n_cfg; ++r) {
        A[(size_t)r * p] = 1.0;
        for (int k = 0; k < nc; ++k) A[(size_t)r * p + 1 + k] = ((double)F[(size_t)r * nc + k] - mean[k]) / sc[k];
    }
    std::vector<double> x;
    rc = lstsq_mgs2(n_cfg, p, A, y, x);
    if (rc) return rc;
    std::vector<double> coef(p);
    double a0 = x[0];
    for (int k = 0; k < nc; ++k) {
        coef[1 + k] = x[1 + k] / sc[k];
        a0 -= coef[1 + k] * mean[k];
    }
    coef[0] = a0;
    double ym = 0.0;
    for (int r = 0; r < n_cfg; ++r) ym += y[r];
    ym /= n_cfg;
    double ssr = 0.0, sst = 0.0;
    for (int r = 0; r < n_cfg; ++r) {
        double yh = coef[0];
        for (int k = 0; k < nc; ++k) yh += coef[1 + k] * (double)F[(size_t)r * nc + k];
        ssr += (y[r] - yh) * (y[r] - yh);
        sst += (y[r] - ym) * (y[r] - ym);
    }
    const double beta = c->p.beta;
    for (int k = 0; k < nc; ++k) J[k] = -coef[1 + k] / beta;
    const double e0 = -coef[0] / beta;
    if (E0) *E0 = e0;
    if (r2) *r2 = sst > 0.0 ? 1.0 - ssr / sst : 1.0;
    return sldqmc_set_effective_model(c, nc, c->h_n_off, c->h_offsets, J, e0);
}

int sldqmc_eff_sweeps(sldqmc_ctx *c, int8_t *s, int n_sweeps, uint64_t seed, uint32_t step, int dir,
                      long long *n_accept)
{
    if (!c || !c->have_model || !s || n_sweeps < 0 || (dir != 0 && dir != 1)) return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    if (!host_field_ok(s, V)) return SLDQMC_ERR_ARG;
    if (cudaMemcpyAsync(c->d_s_one, s, (size_t)V, cudaMemcpyHostToDevice, c->st) != cudaSuccess) return SLDQMC_ERR_CUDA;
    long long *cnt = c->d_stats + 4 * (size_t)c->cap;
    cudaMemsetAsync(cnt, 0, sizeof(long long) * 2, c->st);
    launch_eff_sweeps(c, c->d_s_one, 1, n_sweeps, seed, step, dir, cnt, cnt + 1);
    std::vector<int8_t> tmp(V);
    long long h[2];
    if (cudaMemcpyAsync(tmp.data(), c->d_s_one, (size_t)V, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
        return SLDQMC_ERR_CUDA;
    int rc = sync_and_flag(c);
    if (rc) return rc;
    memcpy(s, tmp.data(), (size_t)V);
    if (n_accept) *n_accept = h[0];
    return SLDQMC_OK;
}

int sldqmc_eff_sweeps_batch_dev(sldqmc_ctx *c, int8_t *d_s, int B, int n_sweeps, uint64_t seed, uint32_t step,
                                int dir, long long *d_accepts)
{
    if (!c || !c->have_model || !d_s || B < 1 || n_sweeps < 0 || dir < -1 || dir > 1) return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    launch_check_field(c, d_s, V * B);
    launch_eff_sweeps(c, d_s, B, n_sweeps, seed, step, dir, d_accepts, nullptr);
    return cudaGetLastError() == cudaSuccess ? SLDQMC_OK : SLDQMC_ERR_CUDA;
}

int sldqmc_cumulative_batch_dev(sldqmc_ctx *c, int8_t *d_s, double *d_logw, int B, int n_eff, uint64_t seed,
                                uint32_t step0, int n_steps, int *d_accepts, double *d_log_r)
{
    if (!c || !c->have_model || B < 1 || B > c->cap || !d_s || !d_logw || n_eff < 0 || n_steps < 0)
        return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    launch_check_field(c, d_s, V * B);
    for (int k = 0; k < n_steps; ++k) {
        int rc = cumulative_step(c, d_s, d_logw, B, n_eff, seed, step0 + (uint32_t)k, d_accepts, d_log_r);
        if (rc) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? SLDQMC_OK : SLDQMC_ERR_CUDA;
}

int sldqmc_cumulative_update(sldqmc_ctx *c, int8_t *s, double *logw, int n_eff, uint64_t seed, uint32_t step,
                             int *accepted, double *log_r)
{
    if (!c || !c->have_model || !s || !logw || n_eff < 0) return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    if (!host_field_ok(s, V)) return SLDQMC_ERR_ARG;
    int8_t *ds = c->d_s_one;
    double *dl = c->d_ld_tmp2;
    int *dacc = c->d_sg_tmp + c->cap;
    double *dlr = c->d_ld_tmp2 + 1;
    if (cudaMemcpyAsync(ds, s, (size_t)V, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(dl, logw, sizeof(double), cudaMemcpyHostToDevice, c->st) != cudaSuccess)
        return SLDQMC_ERR_CUDA;
    cudaMemsetAsync(dacc, 0, sizeof(int), c->st);
    int rc = sldqmc_cumulative_batch_dev(c, ds, dl, 1, n_eff, seed, step, 1, dacc, dlr);
    if (rc) return rc;
    std::vector<int8_t> tmp(V);
    double hl[2];
    int ha;
    if (cudaMemcpyAsync(tmp.data(), ds, (size_t)V, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaMemcpyAsync(hl, dl, sizeof(hl), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaMemcpyAsync(&ha, dacc, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
        return SLDQMC_ERR_CUDA;
    rc = sync_and_flag(c);
    if (rc) return rc;
    memcpy(s, tmp.data(), (size_t)V);
    *logw = hl[0];
    if (accepted) *accepted = ha;
    if (log_r) *log_r = hl[1];
    return SLDQMC_OK;
}

int sldqmc_cumulative_batch(sldqmc_ctx *c, int8_t *s, double *logw, int B, int n_eff, uint64_t seed, uint32_t step0,
                            int n_steps, int *accepts)
{
    if (!c || !c->have_model || !s || !logw || B < 1 || B > c->cap || n_eff < 0 || n_steps < 0) return SLDQMC_ERR_ARG;
    const long long V = (long long)c->N * c->M;
    if (!host_field_ok(s, V * B)) return SLDQMC_ERR_ARG;
    int8_t *ds = c->d_s_one;
    double *dl = c->d_ld_tmp2;
    int *dacc = c->d_sg_tmp + c->cap;
    if (cudaMemcpyAsync(ds, s, (size_t)(V * B), cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(dl, logw, sizeof(double) * B, cudaMemcpyHostToDevice, c->st) != cudaSuccess)
        return SLDQMC_ERR_CUDA;
    cudaMemsetAsync(dacc, 0, sizeof(int) * B, c->st);
    int rc = sldqmc_cumulative_batch_dev(c, ds, dl, B, n_eff, seed, step0, n_steps, dacc, nullptr);
    if (rc) return rc;
    std::vector<int> ha(B);
    if (cudaMemcpyAsync(s, ds, (size_t)(V * B), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaMemcpyAsync(logw, dl, sizeof(double) * B, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaMemcpyAsync(ha.data(), dacc, sizeof(int) * B, cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
        return SLDQMC_ERR_CUDA;
    rc = sync_and_flag(c);
    if (rc) return rc;
    if (accepts)
        for (int b = 0; b < B; ++b) accepts[b] += ha[b];
    return SLDQMC_OK;
}

}  // extern "C"

struct sldqmc_graph {
    std::vector<sldqmc_ctx *> ctxs;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaStream_t origin = nullptr;
    bool own_origin = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

void sldqmc_graph_destroy(sldqmc_graph *g)
{
    if (!g) return;
    if (g->origin) cudaStreamSynchronize(g->origin);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    for (cudaEvent_t e : g->events) cudaEventDestroy(e);
    for (cudaStream_t s : g->streams) cudaStreamDestroy(s);
    if (g->own_origin && g->origin) cudaStreamDestroy(g->origin);
    delete g;
}

int sldqmc_graph_create(sldqmc_ctx *const *ctxs, int n, int8_t *const *d_s, double *const *d_logw, const int *B,
                        int n_eff, const uint64_t *seeds, int *const *d_accepts, uint32_t step0, void *stream,
                        sldqmc_graph **out)
{
    if (!ctxs || n < 1 || !d_s || !d_logw || !B || !seeds || !d_accepts || !out || n_eff < 0) return SLDQMC_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        sldqmc_ctx *c = ctxs[i];
        if (!c || !c->have_model || !d_s[i] || !d_logw[i] || !d_accepts[i] || B[i] < 1 || B[i] > c->cap)
            return SLDQMC_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return SLDQMC_ERR_ARG;  // one member per context: members own their workspace
    }
    sldqmc_graph *g = new sldqmc_graph();
    int rc = SLDQMC_OK;
    g->origin = (cudaStream_t)stream;
    if (!g->origin) {
        if (cudaStreamCreateWithFlags(&g->origin, cudaStreamNonBlocking) != cudaSuccess) { delete g; return SLDQMC_ERR_CUDA; }
        g->own_origin = true;
    }
    for (int i = 0; i < n; ++i) {
        sldqmc_ctx *c = ctxs[i];
        g->ctxs.push_back(c);
        if (!c->d_step) {
            rc = dalloc(&c->d_step, 1);
            if (rc) { sldqmc_graph_destroy(g); return rc; }
        }
        if (cudaMemcpyAsync(c->d_step, &step0, sizeof(uint32_t), cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
            cudaStreamSynchronize(c->st) != cudaSuccess) {
            sldqmc_graph_destroy(g);
            return SLDQMC_ERR_CUDA;
        }
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { sldqmc_graph_destroy(g); return SLDQMC_ERR_CUDA; }
        g->streams.push_back(st);
    }
    for (int k = 0; k < n + 1; ++k) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { sldqmc_graph_destroy(g); return SLDQMC_ERR_CUDA; }
        g->events.push_back(e);
    }
    for (int i = 0; i < n; ++i) {
        get_twin(ctxs[i]);  // allocates, so it must exist before the capture starts
        cudaStreamSynchronize(ctxs[i]->st);
    }
    if (cudaStreamBeginCapture(g->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        sldqmc_graph_destroy(g);
        return SLDQMC_ERR_CUDA;
    }
    cudaEventRecord(g->events[0], g->origin);
    for (int i = 0; i < n && !rc; ++i) {
        sldqmc_ctx *c = ctxs[i];
        cudaStream_t saved = c->st;
        const bool prof_on = c->prof && c->prof->on;
        if (prof_on) c->prof->on = false;
        c->st = g->streams[i];
        c->step_dev = c->d_step;
        cudaStreamWaitEvent(c->st, g->events[0], 0);
        launch_check_field(c, d_s[i], (long long)c->N * c->M * B[i]);
        rc = cumulative_step(c, d_s[i], d_logw[i], B[i], n_eff, seeds[i], step0, d_accepts[i], nullptr);
        launch_step_advance(c, c->d_step);
        cudaEventRecord(g->events[i + 1], c->st);
        cudaStreamWaitEvent(g->origin, g->events[i + 1], 0);
        c->st = saved;
        c->step_dev = nullptr;
        if (prof_on) c->prof->on = true;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e1 = cudaStreamEndCapture(g->origin, &graph);
    g->graph = graph;
    if (rc || e1 != cudaSuccess || !graph) {
        cudaGetLastError();
        sldqmc_graph_destroy(g);
        return rc ? rc : SLDQMC_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        sldqmc_graph_destroy(g);
        return SLDQMC_ERR_CUDA;
    }
    *out = g;
    return SLDQMC_OK;
}

int sldqmc_graph_launch(sldqmc_graph *g, int n_steps)
{
    if (!g || n_steps < 0) return SLDQMC_ERR_ARG;
    for (int k = 0; k < n_steps; ++k)
        if (cudaGraphLaunch(g->exec, g->origin) != cudaSuccess) return SLDQMC_ERR_CUDA;
    return SLDQMC_OK;
}

int sldqmc_graph_sync(sldqmc_graph *g)
{
    if (!g) return SLDQMC_ERR_ARG;
    if (cudaStreamSynchronize(g->origin) != cudaSuccess) return SLDQMC_ERR_CUDA;
    int rc = SLDQMC_OK;
    for (sldqmc_ctx *c : g->ctxs) {
        int r = sync_and_flag(c);
        if (r && !rc) rc = r;
    }
    return rc;
}

int sldqmc_gram_batch_dev(sldqmc_ctx *c, const double *d_X, int B, double *d_W)
{
    if (!c || !d_X || !d_W || B < 1 || B > c->cap) return SLDQMC_ERR_ARG;
    const int N = c->N;
    if (c->oz_ws) {
        oz_gram(c, d_X, c->nn, d_W, c->nn, N, B);
    } else {
        GemmF64 g = gemm_desc(N, N, N, d_X, N, c->nn, d_X, N, c->nn, d_W, N, c->nn, B);
        g.c_upper = 1;
        gemm_ctx(c, g, false, true);
    }
    return cudaGetLastError() == cudaSuccess ? SLDQMC_OK : SLDQMC_ERR_CUDA;
}

int sldqmc_wait_selftest(sldqmc_ctx *c, int max_polls)
{
    if (!c || max_polls < 1 || max_polls > (1 << 24)) return SLDQMC_ERR_ARG;
    launch_wait_selftest(c, max_polls);
    return cudaGetLastError() == cudaSuccess ? SLDQMC_OK : SLDQMC_ERR_CUDA;
}

int sldqmc_set_tile_n(sldqmc_ctx *c, int bn)
{
    if (!c) return SLDQMC_ERR_ARG;
    if (c->p.prec == SLDQMC_FP64) return bn == 64 ? SLDQMC_OK : SLDQMC_ERR_UNSUPPORTED;
    int rc = tc_set_tile_n(c, bn);
    if (rc == SLDQMC_OK && c->twin) rc = tc_set_tile_n(c->twin, bn);
    if (rc == SLDQMC_OK) c->tile_n = bn;
    return rc;
}

int sldqmc_set_local_update_rank(sldqmc_ctx *c, int k)
{
    if (!c || k < 1 || k > 32) return SLDQMC_ERR_ARG;
    c->local_rank = k;
    return SLDQMC_OK;
}

int sldqmc_set_kinetic_form(sldqmc_ctx *c, int form)
{
    if (!c || (form != SLDQMC_KINETIC_DENSE && form != SLDQMC_KINETIC_SEPARABLE)) return SLDQMC_ERR_ARG;
    if (form == SLDQMC_KINETIC_SEPARABLE && !sep_supported(c->p.Lx, c->p.Ly)) return SLDQMC_ERR_UNSUPPORTED;
    c->kinetic = form;
    if (c->twin) c->twin->kinetic = form;
    return SLDQMC_OK;
}

int sldqmc_profile_enable(sldqmc_ctx *c, int on)
{
    if (!c || !c->prof) return SLDQMC_ERR_ARG;
    c->prof->on = on != 0;
    return SLDQMC_OK;
}

int sldqmc_profile_read_sites(sldqmc_ctx *c, char *buf, int len)
{
    if (!c || !c->prof || !buf || len < 1) return SLDQMC_ERR_ARG;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return SLDQMC_ERR_CUDA;
    struct Agg { const char *site; int cls; long long n; double ms, flops; };
    std::vector<Agg> agg;
    for (const ProfRec &r : c->prof->recs) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return SLDQMC_ERR_CUDA;
        const char *site = r.site ? r.site : "unnamed";
        size_t k = 0;
        while (k < agg.size() && (strcmp(agg[k].site, site) != 0 || agg[k].cls != r.cls)) ++k;
        if (k == agg.size()) agg.push_back(Agg{site, r.cls, 0, 0.0, 0.0});
        agg[k].n += 1;
        agg[k].ms += t;
        agg[k].flops += r.flops;
    }
    c->prof->recs.clear();
    c->prof->used = 0;
    int off = 0;
    buf[0] = 0;
    for (const Agg &a : agg) {
        const int w = snprintf(buf + off, (size_t)(len - off), "%s %d %lld %.6f %.6e\n", a.site, a.cls, a.n, a.ms,
                               a.flops);
        if (w < 0 || w >= len - off) break;
        off += w;
    }
    return SLDQMC_OK;
}

int sldqmc_profile_read(sldqmc_ctx *c, long long *launches, double *ms, double *flops)
{
    if (!c || !c->prof || !launches || !ms || !flops) return SLDQMC_ERR_ARG;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return SLDQMC_ERR_CUDA;
    for (int k = 0; k < SLDQMC_KC_COUNT; ++k) { launches[k] = 0; ms[k] = 0.0; flops[k] = 0.0; }
    for (const ProfRec &r : c->prof->recs) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return SLDQMC_ERR_CUDA;
        launches[r.cls] += 1;
        ms[r.cls] += t;
        flops[r.cls] += r.flops;
    }
    c->prof->recs.clear();
    c->prof->used = 0;
    return SLDQMC_OK;
}

}  // extern "C"
