"""ctypes front end of the FP64 CPU oracle (sldqmc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and
by bench.py's CPU-baseline leg; never by the product library.  It shares no
code with the CUDA path.  Each function cites the part of the paper
(Xu, Qi, Liu, Fu, Meng, arXiv:1612.03804) it follows; the C source holds the
arithmetic.

weight_many() and cumulative_chains() only run weight() and
cumulative_update() for many configurations or chains in spawned processes
(so that the tests and the benchmark's CPU baseline use every host core); they
add no arithmetic.

Parity pins: every function here is pinned by tests/test_oracle_pins.py
against closed forms, library routines, brute force or exact enumeration
(free-fermion product formula, uniform-field shift, particle-hole identity,
naive product + numpy slogdet at small beta, cyclic and n_wrap invariance,
brute-force determinant ratios, Philox known-answer vectors, planted-model
regression, exact enumeration chi^2).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sldqmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle with gcc (plain C, -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            d, i, i8p, dp, u64, u32 = (ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32)
            L.or_weight.argtypes = [i, i, d, d, d, d, i, i, i, i, i8p, dp, dp, dp]
            L.or_weight.restype = i
            L.or_build_K.argtypes = [i, i, d, d, dp]
            L.or_build_E.argtypes = [i, i, d, d, d, d, dp]
            L.or_log_bare_weight.argtypes = [i, i, i, d, d, d, i8p]
            L.or_log_bare_weight.restype = d
            L.or_local_sweep.argtypes = [i, i, d, d, d, d, i, i, d, d, i8p, u64, u64, i, dp]
            L.or_local_sweep.restype = i
            L.or_philox4x32_10.argtypes = [dp, dp, dp]
            L.or_uniform.argtypes = [u64, u32, u32, u32, u32]
            L.or_uniform.restype = d
            L.or_random_word.argtypes = [u64, u32, u32, u32, u32]
            L.or_random_word.restype = u32
            L.or_features.argtypes = [i, i, i, i, dp, dp, i8p, dp]
            L.or_coloring.argtypes = [i, i, i, i, dp, dp, dp]
            L.or_coloring.restype = i
            L.or_eff_sweeps.argtypes = [i, i, i, d, i, dp, dp, dp, i8p, i, u64, u32, i, dp, dp]
            L.or_eff_sweeps.restype = i
            L.or_log_weight_total.argtypes = [i, i, d, d, d, d, i, i, d, d, i8p, dp]
            L.or_log_weight_total.restype = i
            L.or_cumulative_update.argtypes = [i, i, d, d, d, d, i, i, d, d, i, dp, dp, dp, i,
                                               i8p, dp, u64, u32, dp, dp, dp, dp]
            L.or_cumulative_update.restype = i
            L.or_fit.argtypes = [i, i, dp, dp, d, dp, dp, dp]
            L.or_fit.restype = i
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what}: oracle status {rc}")


class Model:
    """Parameters of the lattice model (Eq. 6) and its Trotter grid."""

    def __init__(self, Lx, Ly, t=1.0, mu=0.0, xi=1.0, beta=1.0, dtau=0.1, n_wrap=1,
                 J=1.0, h=2.774):
        self.Lx, self.Ly = int(Lx), int(Ly)
        self.N = self.Lx * self.Ly
        self.t, self.mu, self.xi = float(t), float(mu), float(xi)
        self.dtau = float(dtau)
        self.M = int(round(beta / dtau))
        if abs(self.M * self.dtau - beta) > 1e-12 * max(1.0, beta):
            raise ValueError("beta must be a multiple of dtau")
        self.beta = self.M * self.dtau
        self.n_wrap = int(n_wrap)
        self.J, self.h = float(J), float(h)

    def kwargs(self):
        return dict(Lx=self.Lx, Ly=self.Ly, t=self.t, mu=self.mu, xi=self.xi, beta=self.beta,
                    dtau=self.dtau, n_wrap=self.n_wrap, J=self.J, h=self.h)

    def replace(self, **kw):
        d = self.kwargs()
        d.update(kw)
        return Model(**d)


def _field(m, s):
    s = np.ascontiguousarray(s, dtype=np.int8).reshape(m.M, m.N)
    return s


def build_K(m):
    """K = -t A - mu I (hopping part of Eq. 6)."""
    K = np.zeros((m.N, m.N))
    lib().or_build_K(m.Lx, m.Ly, m.t, m.mu, _p(K))
    return K


def build_E(m, sgn=1.0):
    """exp(-sgn*dtau*K) by separable Fourier sums (slice matrix of Eq. 1)."""
    E = np.zeros((m.N, m.N))
    lib().or_build_E(m.Lx, m.Ly, m.t, m.mu, m.dtau, float(sgn), _p(E))
    return E


def weight(m, s, eta, tau0=0, n_wrap=None, want_G=False):
    """(log|det(1+B_tau0..B_1 B_M..B_tau0+1)|, sign[, G]) for flavour eta (Eq. 1)."""
    s = _field(m, s)
    ld = np.zeros(1)
    sg = np.zeros(1, dtype=np.int32)
    G = np.zeros((m.N, m.N)) if want_G else None
    rc = lib().or_weight(m.Lx, m.Ly, m.t, m.mu, m.xi, m.dtau, m.M,
                         m.n_wrap if n_wrap is None else int(n_wrap), int(eta), int(tau0),
                         _p(s), _p(ld), _p(sg), _p(G) if want_G else None)
    _check(rc, "weight")
    if want_G:
        return float(ld[0]), int(sg[0]), G
    return float(ld[0]), int(sg[0])


def _weight_job(job):
    kw, s, eta, tau0, want_G = job
    return weight(Model(**kw), s, eta, tau0=tau0, want_G=want_G)


def weight_many(m, fields, eta, workers=None, tau0=0, want_G=False):
    """weight() of every configuration in `fields`, one oracle call per
    configuration spread over `workers` processes (started with spawn, so a
    pool may be opened after a CUDA context exists in the caller).  The
    arithmetic is that of weight(); only the calls run concurrently."""
    import concurrent.futures as cf
    import multiprocessing as mp
    jobs = [(m.kwargs(), np.ascontiguousarray(f, dtype=np.int8), int(eta), int(tau0), bool(want_G))
            for f in fields]
    workers = max(1, min(len(jobs), workers or len(os.sched_getaffinity(0))))
    if workers == 1:
        return [_weight_job(j) for j in jobs]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_weight_job, jobs))


def _chain_job(job):
    kw, s, logw, classes, J, n_eff, seed, step0, steps = job
    m = Model(**kw)
    mags, acc = [], 0
    for k in range(steps):
        s, logw, a, _, _, _ = cumulative_update(m, s, logw, classes, J, n_eff, seed, step0 + k)
        acc += a
        mags.append(int(np.sum(s.astype(np.int64))))
    return np.array(mags), acc


def cumulative_chains(m, starts, classes, J, n_eff, seeds, step0, steps, workers=None):
    """Independent cumulative-update chains (one per start configuration, each
    with its own seed), run as cumulative_update() calls on `workers` spawned
    processes.  Returns (total magnetisation after every step, shape
    (steps, chains); accepted steps per chain)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    jobs = [(m.kwargs(), np.ascontiguousarray(st, dtype=np.int8), log_weight_total(m, st), classes,
             np.ascontiguousarray(J, dtype=np.float64), int(n_eff), int(sd), int(step0), int(steps))
            for st, sd in zip(starts, seeds)]
    workers = max(1, min(len(jobs), workers or len(os.sched_getaffinity(0))))
    if workers == 1:
        res = [_chain_job(j) for j in jobs]
    else:
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            res = list(ex.map(_chain_job, jobs))
    return np.stack([r[0] for r in res], axis=1), np.array([r[1] for r in res])


def log_bare_weight(m, s):
    """log phi(C): Trotter map of the Ising part H_s of Eq. 6 (constant dropped)."""
    s = _field(m, s)
    return float(lib().or_log_bare_weight(m.Lx, m.Ly, m.M, m.dtau, m.J, m.h, _p(s)))


def log_weight_total(m, s):
    """log omega = log phi + 2 ld(+1) + 2 ld(-1) (Eq. 1 with the bilayer of Eq. 6)."""
    s = _field(m, s)
    out = np.zeros(1)
    _check(lib().or_log_weight_total(m.Lx, m.Ly, m.t, m.mu, m.xi, m.dtau, m.M, m.n_wrap,
                                     m.J, m.h, _p(s), _p(out)), "log_weight_total")
    return float(out[0])


class _SweepStats(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_longlong), ("proposed", ctypes.c_longlong),
                ("margin_events", ctypes.c_longlong), ("max_drift", ctypes.c_double)]


def local_sweep(m, s, seed, sweep0, n_sweeps):
    """DQMC local-update sweeps ("Basics of DQMC"); returns (new s, stats dict)."""
    s = _field(m, s).copy()
    st = _SweepStats()
    rc = lib().or_local_sweep(m.Lx, m.Ly, m.t, m.mu, m.xi, m.dtau, m.M, m.n_wrap, m.J, m.h,
                              _p(s), ctypes.c_uint64(seed), ctypes.c_uint64(sweep0),
                              int(n_sweeps), ctypes.byref(st))
    _check(rc, "local_sweep")
    return s, dict(accepted=st.accepted, proposed=st.proposed,
                   margin_events=st.margin_events, max_drift=st.max_drift)


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def uniform(seed, a, b, c, purpose):
    return float(lib().or_uniform(ctypes.c_uint64(seed), a, b, c, purpose))


def _classes(classes):
    """classes: list of lists of (dx,dy,dtau) offsets."""
    n_off = np.array([len(c) for c in classes], dtype=np.int32)
    offs = np.ascontiguousarray(np.array([o for c in classes for o in c], dtype=np.int32).reshape(-1))
    return n_off, offs


def features(m, s, classes):
    """f_c(C) = sum over pairs of class c of s s (the two-body terms of Eq. 2)."""
    s = _field(m, s)
    n_off, offs = _classes(classes)
    f = np.zeros(len(classes), dtype=np.int64)
    lib().or_features(m.Lx, m.Ly, m.M, len(classes), _p(n_off), _p(offs), _p(s), _p(f))
    return f


def coloring(m, classes):
    n_off, offs = _classes(classes)
    col = np.zeros(m.N * m.M, dtype=np.int32)
    nc = lib().or_coloring(m.Lx, m.Ly, m.M, len(classes), _p(n_off), _p(offs), _p(col))
    return nc, col


def eff_sweeps(m, s, classes, J, n_sweeps, seed, step, direction):
    """Single-spin Metropolis sweeps on H_eff (step iii of the method)."""
    s = _field(m, s).copy()
    n_off, offs = _classes(classes)
    J = np.ascontiguousarray(J, dtype=np.float64)
    na = np.zeros(1, dtype=np.int64)
    mg = np.zeros(1, dtype=np.int64)
    _check(lib().or_eff_sweeps(m.Lx, m.Ly, m.M, m.beta, len(classes), _p(n_off), _p(offs), _p(J),
                               _p(s), int(n_sweeps), ctypes.c_uint64(seed), ctypes.c_uint32(step),
                               int(direction), _p(na), _p(mg)), "eff_sweeps")
    return s, int(na[0]), int(mg[0])


def cumulative_update(m, s, logw, classes, J, n_eff, seed, step):
    """One cumulative update (steps iii+iv, acceptance Eq. 4).

    Returns (s, logw, accepted, log_r, eff_accepts, margin_events)."""
    s = _field(m, s).copy()
    n_off, offs = _classes(classes)
    J = np.ascontiguousarray(J, dtype=np.float64)
    lw = np.array([logw], dtype=np.float64)
    acc = np.zeros(1, dtype=np.int32)
    lr = np.zeros(1)
    na = np.zeros(1, dtype=np.int64)
    mg = np.zeros(1, dtype=np.int64)
    _check(lib().or_cumulative_update(m.Lx, m.Ly, m.t, m.mu, m.xi, m.dtau, m.M, m.n_wrap, m.J,
                                      m.h, len(classes), _p(n_off), _p(offs), _p(J), int(n_eff),
                                      _p(s), _p(lw), ctypes.c_uint64(seed), ctypes.c_uint32(step),
                                      _p(acc), _p(lr), _p(na), _p(mg)), "cumulative_update")
    return s, float(lw[0]), int(acc[0]), float(lr[0]), int(na[0]), int(mg[0])


def fit(F, y, beta):
    """Least-squares training of Eq. 3: returns (J, E0, R^2)."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    n_cfg, n_class = F.shape
    J = np.zeros(n_class)
    E0 = np.zeros(1)
    r2 = np.zeros(1)
    _check(lib().or_fit(n_cfg, n_class, _p(F), _p(y), float(beta), _p(J), _p(E0), _p(r2)), "fit")
    return J, float(E0[0]), float(r2[0])
