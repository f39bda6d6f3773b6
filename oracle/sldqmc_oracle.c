/*
 * sldqmc_oracle.c -- plain, slow, FP64 CPU oracle for self-learning
 * determinantal QMC (Xu, Qi, Liu, Fu, Meng, "Self-Learning Determinantal
 * Quantum Monte Carlo Method", arXiv:1612.03804).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may include,
 * link or call this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg load it (through oracle/oracle.py).  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * Conventions (readings of the paper, each also listed in the design notes):
 *   - N = Lx*Ly sites, site index i = x + Lx*y, periodic in both directions.
 *     A direction of length 1 has no bond; a direction of length 2 carries
 *     its single bond twice (both wrap directions), matching the Fourier
 *     form of the hopping.
 *   - K = -t*A - mu*I (hopping part of H_f, "Results", Eq. 6), and the slice
 *     matrix is B_tau = exp(-dtau*K) * diag(exp(eta*dtau*xi*s_tau)) with
 *     flavour eta = +-1 (the slice matrix of "Basics of DQMC", written with
 *     the sign that makes exp(-beta*K) the free propagator).
 *   - Field s[tau*N + i] in {-1,+1}, tau = 0..M-1 is slice tau+1.
 *   - The weight is det(1 + B_M ... B_1) (Eq. 1); the bilayer of Eq. 6 has
 *     two flavours with eta=+1 and two with eta=-1, so
 *     log omega_F = 2*ld(+1) + 2*ld(-1).
 *
 * All arithmetic is IEEE binary64 with round-to-nearest; compile with
 * -ffp-contract=off so that no fused multiply-add changes a rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_OOM (-2)
#define OR_ERR_SINGULAR (-4)

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 counter-based generator, written from its published      */
/* definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as     */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies, with   */
/* the Weyl key schedule between rounds.                                     */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in [0,1): the top 53 bits of (x1:x0) times 2^-53.  The key is the
 * 64-bit seed split in two words; the counter is (a, b, c, purpose). */
double or_uniform(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t purpose)
{
    uint32_t ctr[4] = {a, b, c, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    uint64_t w = ((uint64_t)o[1] << 32) | (uint64_t)o[0];
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

uint32_t or_random_word(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t purpose)
{
    uint32_t ctr[4] = {a, b, c, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    return o[0];
}

#define OR_PURPOSE_LOCAL 1u
#define OR_PURPOSE_EFF 2u
#define OR_PURPOSE_DIR 3u
#define OR_PURPOSE_ACCEPT 4u

/* ------------------------------------------------------------------------ */
/* Lattice and hopping ("Results", Eq. 6: H_f = -t sum_<ij> c^dag c - mu n). */
/* ------------------------------------------------------------------------ */
static int wrap(int a, int L) { a %= L; return a < 0 ? a + L : a; }

/* K = -t*A - mu*I, row-major N x N. */
void or_build_K(int Lx, int Ly, double t, double mu, double *K)
{
    int N = Lx * Ly;
    memset(K, 0, sizeof(double) * (size_t)N * N);
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            int i = x + Lx * y;
            K[(size_t)i * N + i] -= mu;
            if (Lx > 1) {
                int j1 = wrap(x + 1, Lx) + Lx * y, j2 = wrap(x - 1, Lx) + Lx * y;
                K[(size_t)i * N + j1] -= t;
                K[(size_t)i * N + j2] -= t;
            }
            if (Ly > 1) {
                int j1 = x + Lx * wrap(y + 1, Ly), j2 = x + Lx * wrap(y - 1, Ly);
                K[(size_t)i * N + j1] -= t;
                K[(size_t)i * N + j2] -= t;
            }
        }
}

/* One-dimensional propagator e^{c*A_1} on a ring of length L, by the
 * Fourier sum E1(d) = (1/L) sum_k e^{2c cos k} cos(k d), k = 2 pi n / L.
 * L = 1 has no bond: E1 = [1]. */
static void ring_propagator(int L, double c, double *E1)
{
    if (L == 1) { E1[0] = 1.0; return; }
    for (int d = 0; d < L; ++d) {
        double acc = 0.0;
        for (int n = 0; n < L; ++n) {
            double k = 2.0 * M_PI * (double)n / (double)L;
            acc += exp(2.0 * c * cos(k)) * cos(k * (double)d);
        }
        E1[d] = acc / (double)L;
    }
}

/* E = exp(-sgn*dtau*K) with K = -t A - mu I, i.e. exp(sgn*dtau*mu) *
 * exp(sgn*dtau*t*A_x) (x) exp(sgn*dtau*t*A_y).  sgn=+1 gives E, sgn=-1 its
 * inverse. */
void or_build_E(int Lx, int Ly, double t, double mu, double dtau, double sgn, double *E)
{
    int N = Lx * Ly;
    double *ex = malloc(sizeof(double) * Lx), *ey = malloc(sizeof(double) * Ly);
    ring_propagator(Lx, sgn * dtau * t, ex);
    ring_propagator(Ly, sgn * dtau * t, ey);
    double s = exp(sgn * dtau * mu);
    for (int i = 0; i < N; ++i) {
        int xi = i % Lx, yi = i / Lx;
        for (int j = 0; j < N; ++j) {
            int xj = j % Lx, yj = j / Lx;
            E[(size_t)i * N + j] = s * ex[wrap(xi - xj, Lx)] * ey[wrap(yi - yj, Ly)];
        }
    }
    free(ex);
    free(ey);
}

/* ------------------------------------------------------------------------ */
/* Dense helpers (textbook, unblocked).                                      */
/* ------------------------------------------------------------------------ */
static void matmul(int n, const double *A, const double *B, double *C)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += A[(size_t)i * n + k] * B[(size_t)k * n + j];
            C[(size_t)i * n + j] = acc;
        }
}

/* Householder QR with column pivoting (Businger-Golub): A*P = Q*R.
 * On return A holds R (upper triangle), Q is formed explicitly, perm[k] is
 * the original column at position k, and *nrefl counts the reflectors
 * applied (each has determinant -1).  Column norms are recomputed exactly at
 * every step. */
static int householder_qrcp(int n, double *A, double *Q, int *perm, int *nrefl)
{
    double *vs = calloc((size_t)n * n, sizeof(double));
    double *beta = calloc((size_t)n, sizeof(double));
    if (!vs || !beta) { free(vs); free(beta); return OR_ERR_OOM; }
    for (int j = 0; j < n; ++j) perm[j] = j;
    int cnt = 0;
    for (int k = 0; k < n; ++k) {
        /* pivot: remaining column of largest norm */
        int p = k;
        double best = -1.0;
        for (int j = k; j < n; ++j) {
            double s = 0.0;
            for (int i = k; i < n; ++i) s += A[(size_t)i * n + j] * A[(size_t)i * n + j];
            if (s > best) { best = s; p = j; }
        }
        if (p != k) {
            for (int i = 0; i < n; ++i) {
                double tmp = A[(size_t)i * n + k];
                A[(size_t)i * n + k] = A[(size_t)i * n + p];
                A[(size_t)i * n + p] = tmp;
            }
            int tp = perm[k]; perm[k] = perm[p]; perm[p] = tp;
        }
        /* reflector H = I - beta v v^T mapping A[k:,k] to alpha e_1 */
        double norm = 0.0;
        for (int i = k; i < n; ++i) norm += A[(size_t)i * n + k] * A[(size_t)i * n + k];
        norm = sqrt(norm);
        double *v = vs + (size_t)k * n;
        if (norm == 0.0) { beta[k] = 0.0; continue; }
        double x0 = A[(size_t)k * n + k];
        double alpha = x0 >= 0.0 ? -norm : norm;
        for (int i = k; i < n; ++i) v[i] = A[(size_t)i * n + k];
        v[k] -= alpha;
        double vtv = 0.0;
        for (int i = k; i < n; ++i) vtv += v[i] * v[i];
        beta[k] = 2.0 / vtv;
        cnt++;
        for (int j = k; j < n; ++j) {
            double dot = 0.0;
            for (int i = k; i < n; ++i) dot += v[i] * A[(size_t)i * n + j];
            dot *= beta[k];
            for (int i = k; i < n; ++i) A[(size_t)i * n + j] -= dot * v[i];
        }
        for (int i = k + 1; i < n; ++i) A[(size_t)i * n + k] = 0.0;
        A[(size_t)k * n + k] = alpha;
    }
    /* Q = H_0 H_1 ... H_{n-1} applied to I, accumulated from the right end */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Q[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int k = n - 1; k >= 0; --k) {
        if (beta[k] == 0.0) continue;
        double *v = vs + (size_t)k * n;
        for (int j = 0; j < n; ++j) {
            double dot = 0.0;
            for (int i = k; i < n; ++i) dot += v[i] * Q[(size_t)i * n + j];
            dot *= beta[k];
            for (int i = k; i < n; ++i) Q[(size_t)i * n + j] -= dot * v[i];
        }
    }
    *nrefl = cnt;
    free(vs);
    free(beta);
    return OR_OK;
}

/* LU with partial pivoting, in place.  Returns log|det| and sign. */
static int lu_partial(int n, double *A, int *piv, double *logabs, int *sgn)
{
    int s = 1;
    double lg = 0.0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[(size_t)i * n + k]) > best) { best = fabs(A[(size_t)i * n + k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return OR_ERR_SINGULAR;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double tmp = A[(size_t)k * n + j];
                A[(size_t)k * n + j] = A[(size_t)p * n + j];
                A[(size_t)p * n + j] = tmp;
            }
            s = -s;
        }
        double piv_v = A[(size_t)k * n + k];
        if (piv_v < 0.0) s = -s;
        lg += log(fabs(piv_v));
        for (int i = k + 1; i < n; ++i) {
            double l = A[(size_t)i * n + k] / piv_v;
            A[(size_t)i * n + k] = l;
            for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
        }
    }
    *logabs = lg;
    *sgn = s;
    return OR_OK;
}

/* Solve (LU from lu_partial) X = B for n right-hand sides, B overwritten. */
static void lu_solve(int n, const double *LU, const int *piv, double *B)
{
    for (int k = 0; k < n; ++k)
        if (piv[k] != k)
            for (int j = 0; j < n; ++j) {
                double tmp = B[(size_t)k * n + j];
                B[(size_t)k * n + j] = B[(size_t)piv[k] * n + j];
                B[(size_t)piv[k] * n + j] = tmp;
            }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < i; ++k) {
            double l = LU[(size_t)i * n + k];
            for (int j = 0; j < n; ++j) B[(size_t)i * n + j] -= l * B[(size_t)k * n + j];
        }
    for (int i = n - 1; i >= 0; --i) {
        for (int k = i + 1; k < n; ++k) {
            double u = LU[(size_t)i * n + k];
            for (int j = 0; j < n; ++j) B[(size_t)i * n + j] -= u * B[(size_t)k * n + j];
        }
        double d = LU[(size_t)i * n + i];
        for (int j = 0; j < n; ++j) B[(size_t)i * n + j] /= d;
    }
}

/* ------------------------------------------------------------------------ */
/* Fermion weight det(1 + B_M ... B_1) and G = (1 + B_M ... B_1)^{-1}       */
/* ("Basics of DQMC", Eq. 1), evaluated stably as a running U D V product    */
/* (the scheme of Loh et al. the paper cites) re-factorised by QRCP after    */
/* every n_wrap slices, then finalised with the scale split                  */
/*   1 + U D V = U D_b (D_b^{-1} U^T + D_s V),  D_b = max(D,1), D_s=min(D,1).*/
/* tau0 selects the cyclic start: the product is B_tau0 ... B_1 B_M ...     */
/* B_{tau0+1} (tau0 = 0 or M is the plain chain).                            */
/* ------------------------------------------------------------------------ */
int or_weight(int Lx, int Ly, double t, double mu, double xi, double dtau, int M,
              int n_wrap, int eta, int tau0, const int8_t *s, double *logabsdet, int *sign,
              double *G)
{
    int N = Lx * Ly;
    if (N <= 0 || M <= 0 || n_wrap <= 0 || (eta != 1 && eta != -1) || tau0 < 0 || tau0 > M)
        return OR_ERR_ARG;
    for (int k = 0; k < M * N; ++k)
        if (s[k] != 1 && s[k] != -1) return OR_ERR_ARG;
    size_t nn = (size_t)N * N;
    double *E = malloc(sizeof(double) * nn), *U = malloc(sizeof(double) * nn);
    double *V = malloc(sizeof(double) * nn), *X = malloc(sizeof(double) * nn);
    double *T = malloc(sizeof(double) * nn), *Q = malloc(sizeof(double) * nn);
    double *D = malloc(sizeof(double) * N);
    int *perm = malloc(sizeof(int) * N), *piv = malloc(sizeof(int) * N);
    if (!E || !U || !V || !X || !T || !Q || !D || !perm || !piv) {
        free(E); free(U); free(V); free(X); free(T); free(Q); free(D); free(perm); free(piv);
        return OR_ERR_OOM;
    }
    or_build_E(Lx, Ly, t, mu, dtau, 1.0, E);
    for (size_t k = 0; k < nn; ++k) { U[k] = 0.0; V[k] = 0.0; }
    for (int i = 0; i < N; ++i) { U[(size_t)i * N + i] = 1.0; V[(size_t)i * N + i] = 1.0; D[i] = 1.0; }
    int sgnU = 1; /* sign of det U: parity of the reflectors of the latest QR */
    int rc = OR_OK;

    double c_up = exp((double)eta * dtau * xi), c_dn = exp(-(double)eta * dtau * xi);
    int step = 0;
    /* X accumulates B_k ... B_{k0} U for the current block */
    memcpy(X, U, sizeof(double) * nn);
    for (int m = 0; m < M; ++m) {
        int slice = (tau0 + m) % M; /* 0-based slice index; B_{slice+1} */
        const int8_t *st = s + (size_t)slice * N;
        /* X <- E * diag(d) * X */
        for (int l = 0; l < N; ++l) {
            double d = st[l] > 0 ? c_up : c_dn;
            for (int j = 0; j < N; ++j) X[(size_t)l * N + j] *= d;
        }
        matmul(N, E, X, T);
        memcpy(X, T, sizeof(double) * nn);
        step++;
        if (step == n_wrap || m == M - 1) {
            step = 0;
            /* X diag(D) P = Q R */
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) X[(size_t)i * N + j] *= D[j];
            int nrefl = 0;
            rc = householder_qrcp(N, X, Q, perm, &nrefl);
            if (rc) goto done;
            sgnU = (nrefl & 1) ? -1 : 1;
            memcpy(U, Q, sizeof(double) * nn);
            /* D = |diag R|, V <- D^{-1} R P^T V */
            for (int i = 0; i < N; ++i) D[i] = fabs(X[(size_t)i * N + i]);
            for (int i = 0; i < N; ++i)
                if (D[i] == 0.0) { rc = OR_ERR_SINGULAR; goto done; }
            /* (P^T V)[k,:] = V[perm[k],:] */
            for (int k = 0; k < N; ++k)
                memcpy(T + (size_t)k * N, V + (size_t)perm[k] * N, sizeof(double) * N);
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    double acc = 0.0;
                    for (int k = i; k < N; ++k) acc += X[(size_t)i * N + k] * T[(size_t)k * N + j];
                    V[(size_t)i * N + j] = acc / D[i];
                }
            memcpy(X, U, sizeof(double) * nn);
        }
    }
    /* finalise: M_mid = D_b^{-1} U^T + D_s V */
    {
        double logDb = 0.0;
        for (int i = 0; i < N; ++i) {
            double db = D[i] > 1.0 ? D[i] : 1.0;
            double ds = D[i] > 1.0 ? 1.0 : D[i];
            logDb += log(db);
            for (int j = 0; j < N; ++j)
                T[(size_t)i * N + j] = U[(size_t)j * N + i] / db + ds * V[(size_t)i * N + j];
        }
        double lm;
        int sm;
        rc = lu_partial(N, T, piv, &lm, &sm);
        if (rc) goto done;
        *logabsdet = logDb + lm;
        *sign = sgnU * sm;
        if (G) {
            for (int i = 0; i < N; ++i) {
                double db = D[i] > 1.0 ? D[i] : 1.0;
                for (int j = 0; j < N; ++j) G[(size_t)i * N + j] = U[(size_t)j * N + i] / db;
            }
            lu_solve(N, T, piv, G);
        }
    }
done:
    free(E); free(U); free(V); free(X); free(T); free(Q); free(D); free(perm); free(piv);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Bare Ising weight phi(C) ("Basics of DQMC"; H_s of Eq. 6), read as the   */
/* Suzuki-Trotter map of the transverse-field Ising model:                   */
/*   log phi = dtau*J sum_tau sum_<ij> s s + Kt sum_i sum_tau s_{i,tau}      */
/*             s_{i,tau+1},  Kt = -1/2 ln tanh(dtau*h), periodic in tau,     */
/* dropping the configuration-independent constant.                          */
/* ------------------------------------------------------------------------ */
static double tau_coupling(double dtau, double h) { return -0.5 * log(tanh(dtau * h)); }

double or_log_bare_weight(int Lx, int Ly, int M, double dtau, double J, double h, const int8_t *s)
{
    int N = Lx * Ly;
    long long sp = 0, tm = 0;
    for (int tau = 0; tau < M; ++tau)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x) {
                int i = x + Lx * y;
                int si = s[(size_t)tau * N + i];
                if (Lx > 1) sp += si * s[(size_t)tau * N + wrap(x + 1, Lx) + Lx * y];
                if (Ly > 1) sp += si * s[(size_t)tau * N + x + Lx * wrap(y + 1, Ly)];
                tm += si * s[(size_t)((tau + 1) % M) * N + i];
            }
    return dtau * J * (double)sp + tau_coupling(dtau, h) * (double)tm;
}

/* Change of log phi when s[tau][i] flips sign. */
static double dlog_bare_flip(int Lx, int Ly, int M, double dtau, double J, double h,
                             const int8_t *s, int tau, int i)
{
    int N = Lx * Ly;
    int x = i % Lx, y = i / Lx;
    int si = s[(size_t)tau * N + i];
    int nsp = 0;
    if (Lx > 1) nsp += s[(size_t)tau * N + wrap(x + 1, Lx) + Lx * y] + s[(size_t)tau * N + wrap(x - 1, Lx) + Lx * y];
    if (Ly > 1) nsp += s[(size_t)tau * N + x + Lx * wrap(y + 1, Ly)] + s[(size_t)tau * N + x + Lx * wrap(y - 1, Ly)];
    int ntm = s[(size_t)wrap(tau + 1, M) * N + i] + s[(size_t)wrap(tau - 1, M) * N + i];
    return -2.0 * (double)si * (dtau * J * (double)nsp + tau_coupling(dtau, h) * (double)ntm);
}

/* ------------------------------------------------------------------------ */
/* DQMC local update ("Basics of DQMC"): flip s one by one through the       */
/* space-time lattice, ratio in O(1) from G, Green's function update in      */
/* O(N^2) on acceptance.  Written in the rotated frame                       */
/*   Gt(tau) = E^{-1} G(tau) E = (1 + D_tau B_{tau-1}..B_1 B_M..B_{tau+1} E)^-1,*/
/* where flipping s[tau][i] multiplies D_tau by (1 + Delta e_i e_i^T):       */
/*   R = 1 + Delta (1 - Gt_ii),  Delta = exp(-2 eta dtau xi s) - 1,         */
/*   Gt <- Gt - (Delta/R) Gt[:,i] (e_i^T - Gt[i,:])  (Sherman-Morrison).     */
/* Between slices Gt(tau+1) = D_{tau+1} E Gt(tau) E^{-1} D_{tau+1}^{-1}; at */
/* the start of every n_wrap block Gt is recomputed from the full chain.     */
/* The Metropolis ratio is R(+1)^2 R(-1)^2 * phi'/phi (two flavours each),   */
/* compared in log form: accept iff log u < log r.                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    long long accepted;
    long long proposed;
    long long margin_events; /* |log r - log u| <= 1e-8 */
    double max_drift;        /* max |Gt_wrapped - Gt_fresh| at re-computations */
} or_sweep_stats;

static int fresh_Gt(int Lx, int Ly, double t, double mu, double xi, double dtau, int M, int n_wrap,
                    int eta, int tau1, const int8_t *s, const double *E, const double *Einv,
                    double *Gt, double *tmp)
{
    int N = Lx * Ly;
    double ld;
    int sg;
    /* G(tau1) = (1 + B_tau1 ... B_1 B_M ... B_{tau1+1})^{-1} */
    int rc = or_weight(Lx, Ly, t, mu, xi, dtau, M, n_wrap, eta, tau1, s, &ld, &sg, tmp);
    if (rc) return rc;
    /* Gt = Einv * G * E */
    double *t2 = malloc(sizeof(double) * (size_t)N * N);
    if (!t2) return OR_ERR_OOM;
    matmul(N, Einv, tmp, t2);
    matmul(N, t2, E, Gt);
    free(t2);
    return OR_OK;
}

int or_local_sweep(int Lx, int Ly, double t, double mu, double xi, double dtau, int M, int n_wrap,
                   double J, double h, int8_t *s, uint64_t seed, uint64_t sweep0, int n_sweeps,
                   or_sweep_stats *st)
{
    int N = Lx * Ly;
    if (N <= 0 || M <= 0 || n_wrap <= 0 || n_sweeps < 0) return OR_ERR_ARG;
    size_t nn = (size_t)N * N;
    double *E = malloc(sizeof(double) * nn), *Einv = malloc(sizeof(double) * nn);
    double *Gt[2], *W = malloc(sizeof(double) * nn), *T = malloc(sizeof(double) * nn);
    double *Fr = malloc(sizeof(double) * nn);
    double *col = malloc(sizeof(double) * N), *row = malloc(sizeof(double) * N);
    Gt[0] = malloc(sizeof(double) * nn);
    Gt[1] = malloc(sizeof(double) * nn);
    if (!E || !Einv || !W || !T || !Fr || !col || !row || !Gt[0] || !Gt[1]) return OR_ERR_OOM;
    or_build_E(Lx, Ly, t, mu, dtau, 1.0, E);
    or_build_E(Lx, Ly, t, mu, dtau, -1.0, Einv);
    int rc = OR_OK;
    memset(st, 0, sizeof(*st));
    const int etas[2] = {1, -1};
    for (int sw = 0; sw < n_sweeps; ++sw) {
        uint32_t sweep_id = (uint32_t)(sweep0 + (uint64_t)sw);
        for (int tau = 0; tau < M; ++tau) {
            int tau1 = tau + 1; /* 1-based slice index */
            for (int f = 0; f < 2; ++f) {
                if (tau == 0) {
                    rc = fresh_Gt(Lx, Ly, t, mu, xi, dtau, M, n_wrap, etas[f], tau1, s, E, Einv, Gt[f], T);
                    if (rc) goto done;
                    continue;
                }
                /* wrap: Gt <- D_tau E Gt E^{-1} D_tau^{-1} */
                matmul(N, E, Gt[f], T);
                matmul(N, T, Einv, W);
                double c = (double)etas[f] * dtau * xi;
                for (int i = 0; i < N; ++i)
                    for (int j = 0; j < N; ++j) {
                        double di = exp(c * (double)s[(size_t)tau * N + i]);
                        double dj = exp(c * (double)s[(size_t)tau * N + j]);
                        W[(size_t)i * N + j] = di * W[(size_t)i * N + j] / dj;
                    }
                if (tau % n_wrap == 0) {
                    rc = fresh_Gt(Lx, Ly, t, mu, xi, dtau, M, n_wrap, etas[f], tau1, s, E, Einv, Fr, T);
                    if (rc) goto done;
                    for (size_t k = 0; k < nn; ++k) {
                        double dlt = fabs(W[k] - Fr[k]);
                        if (dlt > st->max_drift) st->max_drift = dlt;
                    }
                    memcpy(Gt[f], Fr, sizeof(double) * nn);
                } else {
                    memcpy(Gt[f], W, sizeof(double) * nn);
                }
            }
            for (int i = 0; i < N; ++i) {
                int sold = s[(size_t)tau * N + i];
                double logr = dlog_bare_flip(Lx, Ly, M, dtau, J, h, s, tau, i);
                double R[2], Dl[2];
                for (int f = 0; f < 2; ++f) {
                    Dl[f] = exp(-2.0 * (double)etas[f] * dtau * xi * (double)sold) - 1.0;
                    R[f] = 1.0 + Dl[f] * (1.0 - Gt[f][(size_t)i * N + i]);
                    logr += 2.0 * log(fabs(R[f]));
                }
                double u = or_uniform(seed, (uint32_t)i, (uint32_t)tau, sweep_id, OR_PURPOSE_LOCAL);
                double lu = log(u);
                st->proposed++;
                if (fabs(logr - lu) <= 1e-8) st->margin_events++;
                if (lu < logr) {
                    st->accepted++;
                    s[(size_t)tau * N + i] = (int8_t)(-sold);
                    for (int f = 0; f < 2; ++f) {
                        double *g = Gt[f];
                        double a = Dl[f] / R[f];
                        for (int k = 0; k < N; ++k) col[k] = g[(size_t)k * N + i];
                        for (int k = 0; k < N; ++k) row[k] = ((k == i) ? 1.0 : 0.0) - g[(size_t)i * N + k];
                        for (int r = 0; r < N; ++r) {
                            double cr = a * col[r];
                            for (int k = 0; k < N; ++k) g[(size_t)r * N + k] -= cr * row[k];
                        }
                    }
                }
            }
        }
    }
done:
    free(E); free(Einv); free(W); free(T); free(Fr); free(col); free(row); free(Gt[0]); free(Gt[1]);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Effective bosonic model (Eq. 2): H_eff = E0 + sum_c J_c f_c(C), where     */
/* class c is a set of space-time offsets o = (dx,dy,dtau) and              */
/* f_c(C) = sum_x sum_{o in c} s_x s_{x+o}   (periodic in space and time).   */
/* Self-pairs (x+o == x after wrapping) contribute the constant 1.           */
/* ------------------------------------------------------------------------ */
static int site_shift(int Lx, int Ly, int M, int x, int y, int tau, const int *o, int sgn)
{
    int N = Lx * Ly;
    int xx = wrap(x + sgn * o[0], Lx), yy = wrap(y + sgn * o[1], Ly), tt = wrap(tau + sgn * o[2], M);
    return tt * N + xx + Lx * yy;
}

/* f[c] for c = 0..n_class-1; offsets[c] is n_off[c] triples. */
void or_features(int Lx, int Ly, int M, int n_class, const int *n_off, const int *offsets,
                 const int8_t *s, long long *f)
{
    int N = Lx * Ly;
    const int *op = offsets;
    for (int c = 0; c < n_class; ++c) {
        long long acc = 0;
        for (int q = 0; q < n_off[c]; ++q, op += 3)
            for (int tau = 0; tau < M; ++tau)
                for (int y = 0; y < Ly; ++y)
                    for (int x = 0; x < Lx; ++x) {
                        int a = tau * N + x + Lx * y;
                        int b = site_shift(Lx, Ly, M, x, y, tau, op, 1);
                        acc += (long long)s[a] * (long long)s[b];
                    }
        f[c] = acc;
    }
}

/* Integer neighbour sum of class c at a site (both directions of each
 * offset, self-pairs excluded). */
static int class_field(int Lx, int Ly, int M, const int *offs, int n, const int8_t *s, int x, int y, int tau)
{
    int N = Lx * Ly;
    int self = tau * N + x + Lx * y;
    int acc = 0;
    for (int q = 0; q < n; ++q) {
        int b1 = site_shift(Lx, Ly, M, x, y, tau, offs + 3 * q, 1);
        int b2 = site_shift(Lx, Ly, M, x, y, tau, offs + 3 * q, -1);
        if (b1 != self) acc += s[b1];
        if (b2 != self) acc += s[b2];
    }
    return acc;
}

/* Greedy colouring of the interaction graph, visiting space-time sites in
 * increasing index tau*N + i and giving each the smallest colour not used by
 * an already coloured neighbour.  Returns the number of colours. */
int or_coloring(int Lx, int Ly, int M, int n_class, const int *n_off, const int *offsets, int *color)
{
    int N = Lx * Ly, V = N * M;
    int tot_off = 0;
    for (int c = 0; c < n_class; ++c) tot_off += n_off[c];
    int ncol = 0;
    char *used = malloc((size_t)(2 * tot_off + 2));
    for (int v = 0; v < V; ++v) color[v] = -1;
    for (int v = 0; v < V; ++v) {
        int tau = v / N, i = v % N, x = i % Lx, y = i / Lx;
        memset(used, 0, (size_t)(2 * tot_off + 2));
        for (int q = 0; q < tot_off; ++q)
            for (int sg = -1; sg <= 1; sg += 2) {
                int b = site_shift(Lx, Ly, M, x, y, tau, offsets + 3 * q, sg);
                if (b != v && color[b] >= 0 && color[b] < 2 * tot_off + 2) used[color[b]] = 1;
            }
        int c = 0;
        while (used[c]) c++;
        color[v] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(used);
    return ncol;
}

/* n_sweeps sweeps of single-spin Metropolis on H_eff (step iii of the
 * method).  A sweep visits the colours in order 0..nc-1 (dir=0) or
 * nc-1..0 (dir=1); within a colour sites do not interact, so their order
 * is immaterial.  Flip of s at x: log acceptance
 *   a = 2 beta s sum_c J_c n_c(x),  accept iff log u < a,
 * with the sum accumulated in class order, one rounding per product and per
 * addition, and a = ((2 beta) * acc) * s. */
int or_eff_sweeps(int Lx, int Ly, int M, double beta, int n_class, const int *n_off,
                  const int *offsets, const double *J, int8_t *s, int n_sweeps, uint64_t seed,
                  uint32_t step, int dir, long long *n_accept, long long *n_margin)
{
    int N = Lx * Ly, V = N * M;
    int *color = malloc(sizeof(int) * V);
    if (!color) return OR_ERR_OOM;
    int nc = or_coloring(Lx, Ly, M, n_class, n_off, offsets, color);
    long long acc_cnt = 0, mg = 0;
    for (int sw = 0; sw < n_sweeps; ++sw)
        for (int cc = 0; cc < nc; ++cc) {
            int col = dir ? (nc - 1 - cc) : cc;
            for (int v = 0; v < V; ++v) {
                if (color[v] != col) continue;
                int tau = v / N, i = v % N, x = i % Lx, y = i / Lx;
                double acc = 0.0;
                const int *op = offsets;
                for (int c = 0; c < n_class; ++c) {
                    int n = class_field(Lx, Ly, M, op, n_off[c], s, x, y, tau);
                    acc = acc + J[c] * (double)n;
                    op += 3 * n_off[c];
                }
                double a = ((2.0 * beta) * acc) * (double)s[v];
                double u = or_uniform(seed, (uint32_t)i, (uint32_t)tau, step,
                                      OR_PURPOSE_EFF | ((uint32_t)sw << 8));
                double lu = log(u);
                if (fabs(a - lu) <= 1e-8) mg++;
                if (lu < a) {
                    s[v] = (int8_t)(-s[v]);
                    acc_cnt++;
                }
            }
        }
    free(color);
    if (n_accept) *n_accept = acc_cnt;
    if (n_margin) *n_margin = mg;
    return OR_OK;
}

/* Full log weight log omega = log phi + 2 ld(+1) + 2 ld(-1) (Eq. 1, bilayer
 * of Eq. 6). */
int or_log_weight_total(int Lx, int Ly, double t, double mu, double xi, double dtau, int M,
                        int n_wrap, double J, double h, const int8_t *s, double *logw)
{
    double lp, lm;
    int sp, sm;
    int rc = or_weight(Lx, Ly, t, mu, xi, dtau, M, n_wrap, 1, 0, s, &lp, &sp, NULL);
    if (rc) return rc;
    rc = or_weight(Lx, Ly, t, mu, xi, dtau, M, n_wrap, -1, 0, s, &lm, &sm, NULL);
    if (rc) return rc;
    *logw = or_log_bare_weight(Lx, Ly, M, dtau, J, h, s) + 2.0 * lp + 2.0 * lm;
    return OR_OK;
}

/* One cumulative update (steps iii and iv; acceptance Eq. 4):
 *   C' = n_eff effective sweeps from C, direction drawn once per step,
 *   log r = [log w(C') - log w(C)] - [log w_eff(C') - log w_eff(C)],
 *   log w_eff = -beta H_eff, so the second bracket is
 *   -beta * sum_c J_c (f_c(C') - f_c(C)) (E0 cancels);
 *   accept iff log u < log r.
 * logw holds log w(C) on entry and log w of the kept configuration on exit. */
int or_cumulative_update(int Lx, int Ly, double t, double mu, double xi, double dtau, int M,
                         int n_wrap, double Jising, double h, int n_class, const int *n_off,
                         const int *offsets, const double *Jeff, int n_eff, int8_t *s,
                         double *logw, uint64_t seed, uint32_t step, int *accepted, double *log_r,
                         long long *eff_accepts, long long *margin_events)
{
    int N = Lx * Ly;
    double beta = dtau * (double)M;
    int8_t *sp = malloc((size_t)N * M);
    long long *f0 = malloc(sizeof(long long) * n_class), *f1 = malloc(sizeof(long long) * n_class);
    if (!sp || !f0 || !f1) return OR_ERR_OOM;
    memcpy(sp, s, (size_t)N * M);
    int dir = (int)(or_random_word(seed, 0, 0, step, OR_PURPOSE_DIR) & 1u);
    long long na = 0, mg = 0;
    int rc = or_eff_sweeps(Lx, Ly, M, beta, n_class, n_off, offsets, Jeff, sp, n_eff, seed, step,
                           dir, &na, &mg);
    if (rc) goto out;
    double lw1;
    rc = or_log_weight_total(Lx, Ly, t, mu, xi, dtau, M, n_wrap, Jising, h, sp, &lw1);
    if (rc) goto out;
    or_features(Lx, Ly, M, n_class, n_off, offsets, s, f0);
    or_features(Lx, Ly, M, n_class, n_off, offsets, sp, f1);
    double acc = 0.0;
    for (int c = 0; c < n_class; ++c) acc = acc + Jeff[c] * (double)(f1[c] - f0[c]);
    double dlweff = -beta * acc;
    double lr = (lw1 - *logw) - dlweff;
    double u = or_uniform(seed, 0, 0, step, OR_PURPOSE_ACCEPT);
    double lu = log(u);
    if (fabs(lr - lu) <= 1e-8) mg++;
    *log_r = lr;
    if (lu < lr) {
        memcpy(s, sp, (size_t)N * M);
        *logw = lw1;
        *accepted = 1;
    } else {
        *accepted = 0;
    }
    if (eff_accepts) *eff_accepts = na;
    if (margin_events) *margin_events = mg;
out:
    free(sp); free(f0); free(f1);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Training (Eq. 3): regress y = ln omega on [1, f_1 .. f_nc] by Householder  */
/* least squares; -beta H_eff = ln omega gives E0 = -a_0/beta, J_c =         */
/* -a_c/beta.  R^2 = 1 - sum (y - yhat)^2 / sum (y - mean y)^2 (the score of */
/* "Results").                                                                */
/* ------------------------------------------------------------------------ */
int or_fit(int n_cfg, int n_class, const double *F /* n_cfg x n_class */, const double *y,
           double beta, double *J, double *E0, double *r2)
{
    int p = n_class + 1;
    if (n_cfg < p) return OR_ERR_ARG;
    double *A = malloc(sizeof(double) * (size_t)n_cfg * p), *b = malloc(sizeof(double) * n_cfg);
    double *coef = calloc((size_t)p, sizeof(double));
    if (!A || !b || !coef) return OR_ERR_OOM;
    for (int r = 0; r < n_cfg; ++r) {
        A[(size_t)r * p] = 1.0;
        for (int c = 0; c < n_class; ++c) A[(size_t)r * p + 1 + c] = F[(size_t)r * n_class + c];
        b[r] = y[r];
    }
    for (int k = 0; k < p; ++k) {
        double norm = 0.0;
        for (int r = k; r < n_cfg; ++r) norm += A[(size_t)r * p + k] * A[(size_t)r * p + k];
        norm = sqrt(norm);
        if (norm == 0.0) { free(A); free(b); free(coef); return OR_ERR_SINGULAR; }
        double x0 = A[(size_t)k * p + k];
        double alpha = x0 >= 0.0 ? -norm : norm;
        double *v = malloc(sizeof(double) * n_cfg);
        for (int r = k; r < n_cfg; ++r) v[r] = A[(size_t)r * p + k];
        v[k] -= alpha;
        double vtv = 0.0;
        for (int r = k; r < n_cfg; ++r) vtv += v[r] * v[r];
        for (int j = k; j < p; ++j) {
            double dot = 0.0;
            for (int r = k; r < n_cfg; ++r) dot += v[r] * A[(size_t)r * p + j];
            dot = 2.0 * dot / vtv;
            for (int r = k; r < n_cfg; ++r) A[(size_t)r * p + j] -= dot * v[r];
        }
        double dot = 0.0;
        for (int r = k; r < n_cfg; ++r) dot += v[r] * b[r];
        dot = 2.0 * dot / vtv;
        for (int r = k; r < n_cfg; ++r) b[r] -= dot * v[r];
        free(v);
    }
    for (int k = p - 1; k >= 0; --k) {
        double acc = b[k];
        for (int j = k + 1; j < p; ++j) acc -= A[(size_t)k * p + j] * coef[j];
        coef[k] = acc / A[(size_t)k * p + k];
    }
    double mean = 0.0;
    for (int r = 0; r < n_cfg; ++r) mean += y[r];
    mean /= (double)n_cfg;
    double ss_res = 0.0, ss_tot = 0.0;
    for (int r = 0; r < n_cfg; ++r) {
        double yh = coef[0];
        for (int c = 0; c < n_class; ++c) yh += coef[1 + c] * F[(size_t)r * n_class + c];
        ss_res += (y[r] - yh) * (y[r] - yh);
        ss_tot += (y[r] - mean) * (y[r] - mean);
    }
    *E0 = -coef[0] / beta;
    for (int c = 0; c < n_class; ++c) J[c] = -coef[1 + c] / beta;
    *r2 = ss_tot > 0.0 ? 1.0 - ss_res / ss_tot : 1.0;
    free(A); free(b); free(coef);
    return OR_OK;
}
