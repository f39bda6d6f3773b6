"""Thin ctypes binding of the sldqmc C ABI (include/sldqmc.h).

Argument marshalling only: every step of the computation runs in the CUDA
library's kernels.  Host-array calls take numpy arrays; *_dev calls take
torch CUDA tensors (their data pointers).  Loading fails loudly when the
library has not been built: there is no CPU fallback.
"""
import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsldqmc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sldqmc.h")

OK = 0
ERRORS = {-1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_NUMERICAL", -5: "ERR_TIMEOUT",
          -6: "ERR_UNSUPPORTED"}
FP64, TF32X3, BF16, BF16X3 = 0, 1, 2, 3
PREC = {"fp64": FP64, "3xtf32": TF32X3, "bf16": BF16, "bf16x3": BF16X3}

_lib = None


class SldqmcError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {ERRORS.get(status, status)} ({_lib.sldqmc_strerror(status).decode() if _lib else ''})")


class Params(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("t", ctypes.c_double),
                ("mu", ctypes.c_double), ("xi", ctypes.c_double), ("beta", ctypes.c_double),
                ("dtau", ctypes.c_double), ("n_wrap", ctypes.c_int), ("J_ising", ctypes.c_double),
                ("h", ctypes.c_double), ("prec", ctypes.c_int), ("max_batch", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_longlong), ("proposed", ctypes.c_longlong),
                ("margin_events", ctypes.c_longlong), ("max_drift", ctypes.c_double)]

    def as_dict(self):
        return dict(accepted=self.accepted, proposed=self.proposed,
                    margin_events=self.margin_events, max_drift=self.max_drift)


def declared_functions():
    """Names of the functions include/sldqmc.h declares."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sldqmc_[a-z0-9_]+)\s*\(", src)))


def load(path=None):
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"sldqmc CUDA library not built ({path}); run paper_1612_03804_gb300/build.py")
    L = ctypes.CDLL(path)
    vp, i, d, u64, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32
    sig = {
        "sldqmc_create": ([ctypes.POINTER(Params), vp, ctypes.POINTER(vp)], i),
        "sldqmc_destroy": ([vp], None),
        "sldqmc_strerror": ([i], ctypes.c_char_p),
        "sldqmc_dims": ([vp, vp, vp], i),
        "sldqmc_sync": ([vp], i),
        "sldqmc_build_K": ([vp, vp, vp, vp], i),
        "sldqmc_weight": ([vp, vp, i, vp, vp], i),
        "sldqmc_weight_batch": ([vp, vp, i, i, vp, vp], i),
        "sldqmc_weight_batch_dev": ([vp, vp, i, i, vp, vp], i),
        "sldqmc_green": ([vp, vp, i, i, vp, vp, vp], i),
        "sldqmc_green_batch_dev": ([vp, vp, i, i, i, vp, vp, vp], i),
        "sldqmc_log_bare_weight": ([vp, vp, vp], i),
        "sldqmc_local_sweep": ([vp, vp, u64, u64, i, vp], i),
        "sldqmc_local_sweep_batch_dev": ([vp, vp, i, u64, u64, i, vp], i),
        "sldqmc_set_effective_model": ([vp, i, vp, vp, vp, d], i),
        "sldqmc_features": ([vp, vp, i, vp], i),
        "sldqmc_fit_effective_action": ([vp, vp, vp, i, vp, vp, vp], i),
        "sldqmc_eff_sweeps": ([vp, vp, i, u64, u32, i, vp], i),
        "sldqmc_cumulative_update": ([vp, vp, vp, i, u64, u32, vp, vp], i),
        "sldqmc_cumulative_batch_dev": ([vp, vp, vp, i, i, u64, u32, i, vp, vp], i),
        "sldqmc_log_weight_batch_dev": ([vp, vp, i, vp], i),
        "sldqmc_kernel_launches": ([vp], ctypes.c_longlong),
        "sldqmc_cumulative_batch": ([vp, vp, vp, i, i, u64, u32, i, vp], i),
        "sldqmc_profile_enable": ([vp, i], i),
        "sldqmc_eff_sweeps_batch_dev": ([vp, vp, i, i, u64, u32, i, vp], i),
        "sldqmc_weight_noalloc": ([ctypes.POINTER(Params), vp, vp, i, i, vp, vp], i),
        "sldqmc_graph_create": ([vp, i, vp, vp, vp, i, vp, vp, u32, vp, ctypes.POINTER(vp)], i),
        "sldqmc_graph_launch": ([vp, i], i),
        "sldqmc_graph_sync": ([vp], i),
        "sldqmc_graph_destroy": ([vp], None),
        "sldqmc_wait_selftest": ([vp, i], i),
        "sldqmc_gram_batch_dev": ([vp, vp, i, vp], i),
        "sldqmc_profile_read": ([vp, vp, vp, vp], i),
        "sldqmc_set_kinetic_form": ([vp, i], i),
        "sldqmc_set_local_update_rank": ([vp, i], i),
        "sldqmc_set_tile_n": ([vp, i], i),
        "sldqmc_profile_read_sites": ([vp, ctypes.c_char_p, i], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _tp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _chk(rc, what):
    if rc != OK:
        raise SldqmcError(rc, what)


class Context:
    """One sldqmc context: a lattice model (Eq. 6), its Trotter grid and workspace."""

    def __init__(self, Lx, Ly, t=1.0, mu=0.0, xi=1.0, beta=1.0, dtau=0.1, n_wrap=10, J=1.0, h=2.774,
                 prec="fp64", max_batch=1, stream=None):
        L = load()
        self.params = Params(int(Lx), int(Ly), float(t), float(mu), float(xi), float(beta), float(dtau),
                             int(n_wrap), float(J), float(h), PREC[prec] if isinstance(prec, str) else int(prec),
                             int(max_batch))
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except ImportError:
                stream = 0
        self._stream = stream
        h_ = ctypes.c_void_p()
        _chk(L.sldqmc_create(ctypes.byref(self.params), ctypes.c_void_p(stream), ctypes.byref(h_)), "create")
        self.h = h_
        n = ctypes.c_int()
        m = ctypes.c_int()
        L.sldqmc_dims(self.h, ctypes.byref(n), ctypes.byref(m))
        self.N, self.M = n.value, m.value
        self.V = self.N * self.M
        self.max_batch = int(max_batch)
        self.classes = None

    def close(self):
        if getattr(self, "h", None):
            load().sldqmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ host API
    def _field(self, s, B=None):
        s = np.ascontiguousarray(s, dtype=np.int8)
        if B is None:
            return s.reshape(self.M, self.N)
        return s.reshape(B, self.M, self.N)

    def build_K(self):
        K = np.zeros((self.N, self.N))
        E = np.zeros((self.N, self.N))
        Ei = np.zeros((self.N, self.N))
        _chk(load().sldqmc_build_K(self.h, _p(K), _p(E), _p(Ei)), "build_K")
        return K, E, Ei

    def weight(self, s, eta):
        s = self._field(s)
        ld = np.zeros(1)
        sg = np.zeros(1, dtype=np.int32)
        _chk(load().sldqmc_weight(self.h, _p(s), int(eta), _p(ld), _p(sg)), "weight")
        return float(ld[0]), int(sg[0])

    def weight_batch(self, s, eta):
        s = np.ascontiguousarray(s, dtype=np.int8)
        B = s.shape[0]
        ld = np.zeros(B)
        sg = np.zeros(B, dtype=np.int32)
        _chk(load().sldqmc_weight_batch(self.h, _p(s), B, int(eta), _p(ld), _p(sg)), "weight_batch")
        return ld, sg

    def green(self, s, eta, tau):
        s = self._field(s)
        G = np.zeros((self.N, self.N))
        ld = np.zeros(1)
        sg = np.zeros(1, dtype=np.int32)
        _chk(load().sldqmc_green(self.h, _p(s), int(eta), int(tau), _p(G), _p(ld), _p(sg)), "green")
        return G, float(ld[0]), int(sg[0])

    def log_bare_weight(self, s):
        s = self._field(s)
        out = np.zeros(1)
        _chk(load().sldqmc_log_bare_weight(self.h, _p(s), _p(out)), "log_bare_weight")
        return float(out[0])

    def local_sweep(self, s, seed, sweep0, n_sweeps):
        s = self._field(s).copy()
        st = Stats()
        _chk(load().sldqmc_local_sweep(self.h, _p(s), ctypes.c_uint64(seed), ctypes.c_uint64(sweep0),
                                       int(n_sweeps), ctypes.byref(st)), "local_sweep")
        return s, st.as_dict()

    def set_effective_model(self, classes, J, E0=0.0):
        self.classes = [list(map(tuple, c)) for c in classes]
        n_off = np.array([len(c) for c in classes], dtype=np.int32)
        offs = np.ascontiguousarray(np.array([o for c in classes for o in c], dtype=np.int32).reshape(-1))
        J = np.ascontiguousarray(J, dtype=np.float64)
        _chk(load().sldqmc_set_effective_model(self.h, len(classes), _p(n_off), _p(offs), _p(J), float(E0)),
             "set_effective_model")

    def features(self, cfgs):
        cfgs = np.ascontiguousarray(cfgs, dtype=np.int8)
        n = cfgs.shape[0]
        F = np.zeros((n, len(self.classes)), dtype=np.int64)
        _chk(load().sldqmc_features(self.h, _p(cfgs), n, _p(F)), "features")
        return F

    def fit_effective_action(self, cfgs, logw=None):
        cfgs = np.ascontiguousarray(cfgs, dtype=np.int8)
        n = cfgs.shape[0]
        J = np.zeros(len(self.classes))
        E0 = np.zeros(1)
        r2 = np.zeros(1)
        lw = None if logw is None else np.ascontiguousarray(logw, dtype=np.float64)
        _chk(load().sldqmc_fit_effective_action(self.h, _p(cfgs), _p(lw), n, _p(J), _p(E0), _p(r2)),
             "fit_effective_action")
        return J, float(E0[0]), float(r2[0])

    def eff_sweeps(self, s, n_sweeps, seed, step, direction):
        s = self._field(s).copy()
        na = np.zeros(1, dtype=np.int64)
        _chk(load().sldqmc_eff_sweeps(self.h, _p(s), int(n_sweeps), ctypes.c_uint64(seed),
                                      ctypes.c_uint32(step), int(direction), _p(na)), "eff_sweeps")
        return s, int(na[0])

    def cumulative_update(self, s, logw, n_eff, seed, step):
        s = self._field(s).copy()
        lw = np.array([logw], dtype=np.float64)
        acc = np.zeros(1, dtype=np.int32)
        lr = np.zeros(1)
        _chk(load().sldqmc_cumulative_update(self.h, _p(s), _p(lw), int(n_eff), ctypes.c_uint64(seed),
                                             ctypes.c_uint32(step), _p(acc), _p(lr)), "cumulative_update")
        return s, float(lw[0]), int(acc[0]), float(lr[0])

    # -------------------------------------------------------- device API
    def weight_batch_dev(self, d_s, eta, d_ld, d_sign=None):
        _chk(load().sldqmc_weight_batch_dev(self.h, _tp(d_s), int(d_s.shape[0]), int(eta), _tp(d_ld),
                                            _tp(d_sign)), "weight_batch_dev")

    def green_batch_dev(self, d_s, eta, tau, d_G, d_ld=None, d_sign=None):
        _chk(load().sldqmc_green_batch_dev(self.h, _tp(d_s), int(d_s.shape[0]), int(eta), int(tau), _tp(d_G),
                                           _tp(d_ld), _tp(d_sign)), "green_batch_dev")

    def log_weight_batch_dev(self, d_s, d_lw):
        _chk(load().sldqmc_log_weight_batch_dev(self.h, _tp(d_s), int(d_s.shape[0]), _tp(d_lw)),
             "log_weight_batch_dev")

    def local_sweep_batch_dev(self, d_s, seed, sweep0, n_sweeps, want_stats=True):
        B = int(d_s.shape[0])
        st = (Stats * B)() if want_stats else None
        _chk(load().sldqmc_local_sweep_batch_dev(self.h, _tp(d_s), B, ctypes.c_uint64(seed),
                                                 ctypes.c_uint64(sweep0), int(n_sweeps),
                                                 st if want_stats else None), "local_sweep_batch_dev")
        return [x.as_dict() for x in st] if want_stats else None

    def eff_sweeps_batch_dev(self, d_s, n_sweeps, seed, step, direction=-1, d_accepts=None):
        _chk(load().sldqmc_eff_sweeps_batch_dev(self.h, _tp(d_s), int(d_s.shape[0]), int(n_sweeps),
                                                ctypes.c_uint64(seed), ctypes.c_uint32(step), int(direction),
                                                _tp(d_accepts)), "eff_sweeps_batch_dev")

    def cumulative_batch_dev(self, d_s, d_logw, n_eff, seed, step0, n_steps, d_accepts, d_log_r=None):
        _chk(load().sldqmc_cumulative_batch_dev(self.h, _tp(d_s), _tp(d_logw), int(d_s.shape[0]), int(n_eff),
                                                ctypes.c_uint64(seed), ctypes.c_uint32(step0), int(n_steps),
                                                _tp(d_accepts), _tp(d_log_r)), "cumulative_batch_dev")

    def cumulative_batch(self, s, logw, n_eff, seed, step0, n_steps, accepts):
        """Host buffers (numpy, updated in place): s (B,M,N) int8, logw (B,), accepts (B,) int32."""
        _chk(load().sldqmc_cumulative_batch(self.h, _p(s), _p(logw), int(s.shape[0]), int(n_eff),
                                            ctypes.c_uint64(seed), ctypes.c_uint32(step0), int(n_steps),
                                            _p(accepts)), "cumulative_batch")

    KERNEL_CLASSES = ("gemm_f64", "gemm_tc", "panel_f64", "eff_sweep", "local_flips", "other", "gemm_oz", "sep")
    KINETIC = {"dense": 0, "separable": 1}

    def set_tile_n(self, bn):
        """Tensor-core slice-product tile width: 64 (eight accumulators) or 128 (four)."""
        _chk(load().sldqmc_set_tile_n(self.h, int(bn)), "set_tile_n")

    def set_local_update_rank(self, k):
        """1: immediate rank-1 local updates; 2..32: delayed updates in blocks of k sites."""
        _chk(load().sldqmc_set_local_update_rank(self.h, int(k)), "set_local_update_rank")

    def set_kinetic_form(self, form):
        """'dense' (default) or 'separable' exp(-dtau K) in the slice products."""
        _chk(load().sldqmc_set_kinetic_form(self.h, self.KINETIC[form] if isinstance(form, str) else int(form)),
             "set_kinetic_form")

    def profile(self, on):
        _chk(load().sldqmc_profile_enable(self.h, int(bool(on))), "profile_enable")

    def profile_read(self):
        n = len(self.KERNEL_CLASSES)
        la = np.zeros(n, dtype=np.int64)
        ms = np.zeros(n)
        fl = np.zeros(n)
        _chk(load().sldqmc_profile_read(self.h, _p(la), _p(ms), _p(fl)), "profile_read")
        return {k: dict(launches=int(la[i]), ms=float(ms[i]), flops=float(fl[i]))
                for i, k in enumerate(self.KERNEL_CLASSES)}

    def profile_read_sites(self):
        """Per launch site: {site: dict(cls, launches, ms, flops)} (clears the record)."""
        buf = ctypes.create_string_buffer(1 << 16)
        _chk(load().sldqmc_profile_read_sites(self.h, buf, len(buf)), "profile_read_sites")
        out = {}
        for line in buf.value.decode().splitlines():
            site, cls, n, ms, fl = line.split()
            out[site] = dict(cls=self.KERNEL_CLASSES[int(cls)], launches=int(n), ms=float(ms), flops=float(fl))
        return out

    def gram_batch_dev(self, d_X, d_W):
        """W_b = X_b X_b^T (upper triangle) for (B, N, N) float64 device tensors."""
        _chk(load().sldqmc_gram_batch_dev(self.h, _tp(d_X), int(d_X.shape[0]), _tp(d_W)), "gram_batch_dev")

    def wait_selftest(self, max_polls):
        _chk(load().sldqmc_wait_selftest(self.h, int(max_polls)), "wait_selftest")

    def sync(self):
        _chk(load().sldqmc_sync(self.h), "sync")

    def kernel_launches(self):
        return int(load().sldqmc_kernel_launches(self.h))


class Graph:
    """Uneven chain groups in one CUDA graph (sldqmc_graph_*): one cumulative
    update of every member per replay, branches on separate streams."""

    def __init__(self, members, n_eff, step0=0, stream=None):
        """members: list of (Context, d_s, d_logw, d_accepts, seed) with torch CUDA tensors."""
        L = load()
        n = len(members)
        self._keep = members
        P = ctypes.c_void_p * n
        ctxs = P(*[m[0].h for m in members])
        ds = P(*[m[1].data_ptr() for m in members])
        dl = P(*[m[2].data_ptr() for m in members])
        da = P(*[m[3].data_ptr() for m in members])
        Bs = (ctypes.c_int * n)(*[int(m[1].shape[0]) for m in members])
        seeds = (ctypes.c_uint64 * n)(*[int(m[4]) for m in members])
        h = ctypes.c_void_p()
        _chk(L.sldqmc_graph_create(ctxs, n, ds, dl, Bs, int(n_eff), seeds, da, ctypes.c_uint32(step0),
                                   ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)), "graph_create")
        self.h = h

    def launch(self, n_steps=1):
        _chk(load().sldqmc_graph_launch(self.h, int(n_steps)), "graph_launch")

    def sync(self):
        _chk(load().sldqmc_graph_sync(self.h), "graph_sync")

    def close(self):
        if getattr(self, "h", None):
            load().sldqmc_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
