"""B300-native DIAM sampler (dimension-independent adaptive Metropolis, arXiv 1506.05741).

Thin ctypes binding over ``libdiam.so`` (the C ABI declared in ``include/diam.h``). Every step of the
sampler runs in the library's CUDA kernels; this module only marshals arguments. There is no CPU
fallback: if the library cannot be built or loaded, importing the binding's entry points raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

FP64, FP32, BF16 = 0, 1, 2   # FP32: the BF16 mode with the factor quantised to TF32
PROP_DIAM, PROP_RW = 0, 1
T_DIAG, T_DENSE, T_TANH, T_BANANA, T_REF, T_CALLBACK, T_TWIST = 0, 1, 2, 3, 4, 5, 6
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
          4: "covariance not positive definite", 5: "device wait timed out", 6: "target callback failed",
          7: "context in error state"}

_lib = None
_lock = threading.Lock()

LOGPI_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p)
INTERVAL_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_int64)


class DiamTarget(C.Structure):
    _fields_ = [("kind", C.c_int32), ("d_y", C.c_int32), ("lam", C.c_void_p), ("G", C.c_void_p),
                ("A", C.c_void_p), ("y", C.c_void_p), ("sigma", C.c_double), ("ban_a", C.c_double),
                ("ban_b", C.c_double), ("ban_c", C.c_double), ("fn", LOGPI_FN), ("user", C.c_void_p)]


class DiamConfig(C.Structure):
    _fields_ = [("d", C.c_int32), ("P", C.c_int32), ("n_lag", C.c_int32), ("M", C.c_int32),
                ("beta0", C.c_double), ("infl", C.c_double), ("adapt_beta", C.c_int32), ("xref_mode", C.c_int32),
                ("acc_lo", C.c_double), ("acc_hi", C.c_double), ("beta_factor", C.c_double),
                ("beta_min", C.c_double), ("beta_max", C.c_double), ("eps_jitter", C.c_double),
                ("min_samples_refresh", C.c_int64), ("burnin", C.c_int64), ("refresh_delay", C.c_int32),
                ("prec", C.c_int32), ("seed", C.c_uint64), ("problem_id", C.c_uint32), ("trace_steps", C.c_int32),
                ("keep_block_sums", C.c_int32), ("profile", C.c_int32), ("graphs", C.c_int32),
                ("proposal", C.c_int32), ("carry_map", C.c_int32), ("eps_jitter_min", C.c_double),
                ("reserved", C.c_int32 * 2)]


class DiamDaConfig(C.Structure):
    _fields_ = [("h1", C.c_int32), ("h2", C.c_int32), ("retrain_every", C.c_int32), ("ring", C.c_int32),
                ("train_steps", C.c_int32), ("batch", C.c_int32), ("first_train_min", C.c_int32),
                ("screen_from_start", C.c_int32), ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("adam_eps", C.c_double), ("rmse_bound", C.c_double), ("seed", C.c_uint64)]


class DiamDaStats(C.Structure):
    _fields_ = [("trainings", C.c_int64), ("stage1_tested", C.c_int64), ("stage1_passed", C.c_int64),
                ("exact_evals", C.c_int64), ("ring_filled", C.c_int64), ("last_rmse", C.c_double),
                ("active", C.c_int32), ("pad", C.c_int32)]


class DiamStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("n", C.c_int64), ("accepted", C.c_int64), ("refreshes", C.c_int64),
                ("notspd", C.c_int64), ("nonfinite", C.c_int64), ("beta", C.c_double),
                ("chol_attempts", C.c_int64)]


EXPORTS = ["diam_config_default", "diam_init", "diam_run_batch", "diam_flush", "diam_sync_moments", "diam_get_moments",
           "diam_export_moments", "diam_get_state", "diam_get_factor", "diam_get_trace", "diam_get_block_sums", "diam_get_psrf",
           "diam_save", "diam_load", "diam_get_profile", "diam_destroy", "diam_last_error", "diam_status_string"]
PHASES = ["noise", "xi_gemm", "propose", "target", "accept", "fold", "refresh", "rewhiten", "screen", "train", "step",
          "syrk"]


def kernel_launches() -> int:
    """CUDA kernel launches made by libdiam.so in this process so far."""
    return int(lib().diam_kernel_launches())


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libdiam.so (building it with nvcc if it is missing or older than its sources)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            l = C.CDLL(path)
            P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
            sig = {
                "diam_config_default": (C.c_int, [P, I32, I32]),
                "diam_init": (C.c_int, [P, P, P, P, P, P, P]),
                "diam_run_batch": (C.c_int, [P, I64]),
                "diam_flush": (C.c_int, [P]),
                "diam_get_psrf": (C.c_int, [P, I64, I64, P]),
                "diam_sync_moments": (C.c_int, [P, P, P, I64]),
                "diam_get_moments": (C.c_int, [P, P, P, P]),
                "diam_export_moments": (C.c_int, [P, P, P, P]),
                "diam_export_increment": (C.c_int, [P, P, P, P]),
                "diam_set_interval_hook": (C.c_int, [P, INTERVAL_FN, P]),
                "diam_get_state": (C.c_int, [P, P, P, P]),
                "diam_get_factor": (C.c_int, [P, P, P, P, P]),
                "diam_get_trace": (C.c_int, [P, P, P, P, P, P, I64]),
                "diam_get_block_sums": (C.c_int, [P, P, P, P]),
                "diam_save": (C.c_int, [P, P, P]),
                "diam_load": (C.c_int, [P, P, C.c_size_t]),
                "diam_get_profile": (C.c_int, [P, P, P, I32]),
                "diam_destroy": (None, [P]),
                "diam_last_error": (C.c_char_p, [P]),
                "diam_status_string": (C.c_char_p, [C.c_int]),
                "diam_kernel_launches": (C.c_uint64, []),
                "diam_multi_init": (C.c_int, [I32, P, P, P, P, P]),
                "diam_multi_run": (C.c_int, [P, I64]),
                "diam_multi_context": (P, [P, I32]),
                "diam_multi_destroy": (None, [P]),
                "diam_da_config_default": (C.c_int, [P]),
                "diam_da_enable": (C.c_int, [P, P, P, P, P, P, P, P]),
                "diam_da_train": (C.c_int, [P, P]),
                "diam_da_get_stats": (C.c_int, [P, P]),
                "diam_da_grad": (C.c_int, [P, I32, P, P, P, P, P, P, P, P, P]),
                "diam_da_get_weights": (C.c_int, [P, P, P, P, P, P, P]),
                "diam_da_adam_step": (C.c_int, [P, P, P, P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(l, name)
                f.restype = res
                f.argtypes = args
            _lib = l
    return _lib


class DiamError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# First jitter of the refresh rule in BF16 mode (relative diagonal loading): its C_n comes from the FP32-accumulated
# tensor-core fold, whose noise along near-null directions early in a run is 1e-5 to 1e-4 of the diagonal, so
# smaller loadings fail and only cost retries. A config value (eps_jitter_min), read by the library and the
# oracle alike; default_config applies it to BF16 configurations unless the caller gives eps_jitter_min.
BF16_JITTER_MIN = 1e-4


def default_config(d: int, P: int, **kw) -> dict:
    cs = DiamConfig()
    rc = lib().diam_config_default(C.byref(cs), d, P)
    if rc:
        raise DiamError(rc, "diam_config_default")
    cfg = {k: getattr(cs, k) for k, _ in DiamConfig._fields_ if k != "reserved"}
    for k, v in kw.items():
        if k not in cfg:
            raise KeyError(k)
        cfg[k] = v
    if cfg["prec"] in (BF16, FP32) and "eps_jitter_min" not in kw:
        cfg["eps_jitter_min"] = BF16_JITTER_MIN
    return cfg


def _stream_handle(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover
        pass
    return None


def da_default_config(**kw) -> dict:
    cs = DiamDaConfig()
    lib().diam_da_config_default(C.byref(cs))
    cfg = {k: getattr(cs, k) for k, _ in DiamDaConfig._fields_ if k != "reserved"}
    for k, v in kw.items():
        if k not in cfg:
            raise KeyError(k)
        cfg[k] = v
    return cfg


def _target_struct(target, keep):
    def arr(a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, np.float64)
        keep.append(a)
        return a
    ts = DiamTarget()
    ts.kind = int(target.kind)
    ts.d_y = int(getattr(target, "d_y", 0) or 0)
    ts.lam = _p(arr(getattr(target, "lam", None)))
    ts.G = _p(arr(getattr(target, "G", None)))
    ts.A = _p(arr(getattr(target, "A", None)))
    ts.y = _p(arr(getattr(target, "y", None)))
    ts.sigma = float(getattr(target, "sigma", 0.0) or 0.0)
    ts.ban_a = float(getattr(target, "ban_a", 100.0))
    ts.ban_b = float(getattr(target, "ban_b", 0.1))
    ts.ban_c = float(getattr(target, "ban_c", 10.0))
    return ts


class _View:
    """A problem of a MultiSampler seen through the single-sampler getters (not owning its context)."""

    def __init__(self, l, h, d, P):
        self._l, self._h, self.d, self.P = l, h, d, P

    def close(self):
        pass

    __del__ = close


class MultiSampler:
    """Many independent DIAM problems (uneven d, own targets) run together on one GPU (diam_multi_*)."""

    def __init__(self, cfgs, targets, x0s=None, C0s=None):
        self._l = lib()
        n = len(cfgs)
        keep = []
        carr = (DiamConfig * n)()
        tarr = (DiamTarget * n)()
        for j, (cfg, tg) in enumerate(zip(cfgs, targets)):
            for k, v in cfg.items():
                setattr(carr[j], k, v)
            tarr[j] = _target_struct(tg, keep)

        def ptrs(lst):
            if lst is None:
                return None
            out = (C.c_void_p * n)()
            for j, a in enumerate(lst):
                if a is not None:
                    a = np.ascontiguousarray(a, np.float64)
                    keep.append(a)
                    out[j] = a.ctypes.data
            return out

        h = C.c_void_p()
        rc = self._l.diam_multi_init(n, carr, tarr, ptrs(x0s), ptrs(C0s), C.byref(h))
        if rc:
            raise DiamError(rc, "diam_multi_init")
        self._h = h
        self.n = n
        self.views = []
        for j, cfg in enumerate(cfgs):
            v = Sampler.__new__(Sampler)
            v._l, v._h, v.d, v.P, v.cfg = self._l, C.c_void_p(self._l.diam_multi_context(h, j)), cfg["d"], cfg["P"], cfg
            v._owned = False
            self.views.append(v)

    def run(self, n_steps: int):
        rc = self._l.diam_multi_run(self._h, int(n_steps))
        if rc:
            why = []
            for j, v in enumerate(self.views):
                msg = self._l.diam_last_error(v._h)
                if msg:
                    why.append(f"problem {j} (d={v.d}): {msg.decode(errors='replace')}")
            raise DiamError(rc, "diam_multi_run" + ("; " + "; ".join(why) if why else ""))

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            for v in self.views:
                v._h = None
            self._l.diam_multi_destroy(h)
            self._h = None

    __del__ = close


class Sampler:
    """P concurrent DIAM chains on one GPU (one context of libdiam.so)."""

    def __init__(self, cfg: dict, target, x0=None, C0=None, xref0=None, stream=None):
        self._l = lib()
        self.cfg = dict(cfg)
        d, P = self.cfg["d"], self.cfg["P"]
        self.d, self.P = d, P
        cs = DiamConfig()
        for k, v in self.cfg.items():
            setattr(cs, k, v)
        self._keep = []

        def arr(a, shape=None):
            if a is None:
                return None
            a = np.ascontiguousarray(a, np.float64)
            if shape is not None:
                a = np.ascontiguousarray(np.broadcast_to(a, shape))
            self._keep.append(a)
            return a

        ts = DiamTarget()
        ts.kind = int(target.kind)
        ts.d_y = int(getattr(target, "d_y", 0) or 0)
        ts.lam = _p(arr(getattr(target, "lam", None)))
        ts.G = _p(arr(getattr(target, "G", None)))
        ts.A = _p(arr(getattr(target, "A", None)))
        ts.y = _p(arr(getattr(target, "y", None)))
        ts.sigma = float(getattr(target, "sigma", 0.0) or 0.0)
        ts.ban_a = float(getattr(target, "ban_a", 100.0))
        ts.ban_b = float(getattr(target, "ban_b", 0.1))
        ts.ban_c = float(getattr(target, "ban_c", 10.0))
        fn = getattr(target, "fn", None)
        if fn is not None:
            self._cb = LOGPI_FN(fn)
            ts.fn = self._cb
        h = C.c_void_p()
        x0a = arr(x0, (P, d)) if x0 is not None else None
        rc = self._l.diam_init(C.byref(cs), C.byref(ts), _p(x0a), _p(arr(C0)), _p(arr(xref0)),
                               C.c_void_p(_stream_handle(stream)), C.byref(h))
        if rc:
            raise DiamError(rc, "diam_init")
        self._h = h
        self._keep.clear()

    def _check(self, rc, what):
        if rc:
            raise DiamError(rc, f"{what}: {self._l.diam_last_error(self._h).decode()}")

    def close(self):
        h = getattr(self, "_h", None)
        if h and getattr(self, "_owned", True):
            self._l.diam_destroy(h)
        self._h = None

    __del__ = close

    def run(self, n_steps: int):
        self._hook_exc = None
        rc = self._l.diam_run_batch(self._h, int(n_steps))
        if rc and getattr(self, "_hook_exc", None) is not None:
            exc, self._hook_exc = self._hook_exc, None
            raise exc
        self._check(rc, "diam_run_batch")

    def set_interval_hook(self, fn):
        """fn(interval) runs at the end of every interval, after the fold and before the beta rule and the refresh
        (diam_set_interval_hook); an exception in fn stops run() and is raised from it. None removes the hook."""
        if fn is None:
            self._hook = None
            self._check(self._l.diam_set_interval_hook(self._h, INTERVAL_FN(), None), "diam_set_interval_hook")
            return

        def tramp(user, ctx, k):
            try:
                fn(int(k))
                return 0
            except BaseException as e:   # re-raised by run()
                self._hook_exc = e
                return 6

        self._hook = INTERVAL_FN(tramp)
        self._check(self._l.diam_set_interval_hook(self._h, self._hook, None), "diam_set_interval_hook")

    def export_increment(self):
        """Moments (mean, M2, n) of the samples folded since the last sync_moments (diam_export_increment)."""
        m = np.zeros(self.d)
        M2 = np.zeros((self.d, self.d))
        n = C.c_int64()
        self._check(self._l.diam_export_increment(self._h, _p(m), _p(M2), C.byref(n)), "diam_export_increment")
        return m, M2, n.value

    def flush(self):
        """Wait for a refresh still running beside the chains (refresh_delay >= 1) and apply its outcome."""
        self._check(self._l.diam_flush(self._h), "diam_flush")

    def moments(self):
        m = np.zeros(self.d)
        cov = np.zeros((self.d, self.d))
        n = C.c_int64()
        self._check(self._l.diam_get_moments(self._h, _p(m), _p(cov), C.byref(n)), "diam_get_moments")
        return m, cov, n.value

    def export_moments(self):
        m = np.zeros(self.d)
        M2 = np.zeros((self.d, self.d))
        n = C.c_int64()
        self._check(self._l.diam_export_moments(self._h, _p(m), _p(M2), C.byref(n)), "diam_export_moments")
        return m, M2, n.value

    def sync_moments(self, ext_mean=None, ext_M2=None, ext_n=0):
        em = None if ext_mean is None else np.ascontiguousarray(ext_mean, np.float64)
        eM = None if ext_M2 is None else np.ascontiguousarray(ext_M2, np.float64)
        self._check(self._l.diam_sync_moments(self._h, _p(em), _p(eM), int(ext_n)), "diam_sync_moments")

    def state(self):
        x = np.zeros((self.P, self.d))
        lp = np.zeros(self.P)
        st = DiamStats()
        self._check(self._l.diam_get_state(self._h, _p(x), _p(lp), C.byref(st)), "diam_get_state")
        return x, lp, {k: getattr(st, k) for k, _ in DiamStats._fields_}

    def log_pi(self):
        """log pi of every chain's current state (P doubles, copied to the host)."""
        lp = np.zeros(self.P)
        self._check(self._l.diam_get_state(self._h, None, _p(lp), None), "diam_get_state")
        return lp

    def stats(self):
        st = DiamStats()
        self._check(self._l.diam_get_state(self._h, None, None, C.byref(st)), "diam_get_state")
        return {k: getattr(st, k) for k, _ in DiamStats._fields_}

    def factor(self):
        L = np.zeros((self.d, self.d))
        Lq = np.zeros((self.d, self.d))
        xr = np.zeros(self.d)
        b = C.c_double()
        self._check(self._l.diam_get_factor(self._h, _p(L), _p(Lq), _p(xr), C.byref(b)), "diam_get_factor")
        return L, Lq, xr, b.value

    def trace(self, n_steps: int):
        T = int(n_steps)
        arrs = [np.zeros((T, self.P)) for _ in range(4)]
        acc = np.zeros((T, self.P), np.int8)
        self._check(self._l.diam_get_trace(self._h, *[_p(a) for a in arrs], _p(acc), T), "diam_get_trace")
        return dict(lp_prop=arrs[0], q_prop=arrs[1], q_cur=arrs[2], loga=arrs[3], acc=acc.astype(bool))

    def block_sums(self, n_blocks: int):
        xs = np.zeros((n_blocks, self.P, self.d))
        ls = np.zeros((n_blocks, self.P))
        nb = C.c_int64(n_blocks)
        self._check(self._l.diam_get_block_sums(self._h, _p(xs), _p(ls), C.byref(nb)), "diam_get_block_sums")
        return xs[: nb.value], ls[: nb.value]

    def psrf(self, first_block: int, n_blocks: int) -> np.ndarray:
        """sqrt(R_i) of Sec. 2.4.2 for every coordinate over the given completed intervals (keep_block_sums)."""
        out = np.zeros(self.d)
        self._check(self._l.diam_get_psrf(self._h, int(first_block), int(n_blocks), _p(out)), "diam_get_psrf")
        return out

    def profile(self, reset: bool = True) -> dict:
        """Per-phase timed launch counts and device milliseconds (needs cfg['profile'] = 1)."""
        counts = np.zeros(len(PHASES), np.int64)
        ms = np.zeros(len(PHASES))
        self._check(self._l.diam_get_profile(self._h, _p(counts), _p(ms), int(reset)), "diam_get_profile")
        return {ph: (int(counts[i]), float(ms[i])) for i, ph in enumerate(PHASES)}

    # ---- delayed acceptance (two-stage MH with an MLP surrogate)
    def da_enable(self, cfg: dict, weights: dict):
        cs = DiamDaConfig()
        for k, v in cfg.items():
            setattr(cs, k, v)
        self._da_h = (cfg["h1"], cfg["h2"])
        w = {k: np.ascontiguousarray(weights[k], np.float64) for k in ("W1", "b1", "W2", "b2", "w3", "b3")}
        self._check(self._l.diam_da_enable(self._h, C.byref(cs), *[_p(w[k]) for k in ("W1", "b1", "W2", "b2", "w3", "b3")]),
                    "diam_da_enable")

    def da_train(self) -> float:
        r = C.c_double()
        self._check(self._l.diam_da_train(self._h, C.byref(r)), "diam_da_train")
        return r.value

    def da_stats(self) -> dict:
        s = DiamDaStats()
        self._check(self._l.diam_da_get_stats(self._h, C.byref(s)), "diam_da_get_stats")
        return {k: getattr(s, k) for k, _ in DiamDaStats._fields_ if k != "pad"}

    def da_grad(self, U, t):
        h1, h2 = self._da_h
        U = np.ascontiguousarray(U, np.float64)
        t = np.ascontiguousarray(t, np.float64)
        B = U.shape[0]
        out = {"W1": np.zeros((h1, self.d)), "b1": np.zeros(h1), "W2": np.zeros((h2, h1)), "b2": np.zeros(h2),
               "w3": np.zeros(h2), "b3": np.zeros(1)}
        loss = C.c_double()
        self._check(self._l.diam_da_grad(self._h, B, _p(U), _p(t), C.byref(loss),
                                         *[_p(out[k]) for k in ("W1", "b1", "W2", "b2", "w3", "b3")]), "diam_da_grad")
        return loss.value, out

    def da_adam_step(self, grads: dict):
        """One Adam update of the network with the given gradients (diam_da_adam_step)."""
        g = {k: np.ascontiguousarray(grads[k], np.float64) for k in ("W1", "b1", "W2", "b2", "w3", "b3")}
        self._check(self._l.diam_da_adam_step(self._h, *[_p(g[k]) for k in ("W1", "b1", "W2", "b2", "w3", "b3")]),
                    "diam_da_adam_step")

    def da_weights(self) -> dict:
        h1, h2 = self._da_h
        out = {"W1": np.zeros((h1, self.d)), "b1": np.zeros(h1), "W2": np.zeros((h2, h1)), "b2": np.zeros(h2),
               "w3": np.zeros(h2), "b3": np.zeros(1)}
        self._check(self._l.diam_da_get_weights(self._h, *[_p(out[k]) for k in ("W1", "b1", "W2", "b2", "w3", "b3")]),
                    "diam_da_get_weights")
        return out

    def save(self) -> bytes:
        n = C.c_size_t()
        self._check(self._l.diam_save(self._h, None, C.byref(n)), "diam_save")
        buf = (C.c_char * n.value)()
        self._check(self._l.diam_save(self._h, buf, C.byref(n)), "diam_save")
        return bytes(buf)

    def load(self, blob: bytes):
        buf = (C.c_char * len(blob)).from_buffer_copy(blob)
        self._check(self._l.diam_load(self._h, buf, len(blob)), "diam_load")
