"""Plain FP64 CPU oracle for the DIAM hot path (arXiv 1506.05741).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package. The sampling library never imports it, and it imports nothing of the sampling library.

The arithmetic lives in ``diam_oracle.c`` (plain C, FP64, textbook definitions, each routine citing the
paper passage it follows), ``mlp.py`` (FP64 numpy surrogate network) and ``stats.py`` (batch-means ESS, PSRF).
This module only loads the C library (compiling it with gcc the first time) and marshals arguments.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "diam_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

# prec codes shared with the C side of the oracle
FP64, FP32, BF16 = 0, 1, 2   # FP32: the mixed mode with the factor quantised to TF32 instead of BF16
# target kinds
T_DIAG, T_DENSE, T_TANH, T_BANANA, T_REF, T_TWIST = 0, 1, 2, 3, 4, 6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off keeps every fused multiply-add explicit)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class OrcTarget(C.Structure):
    _fields_ = [("kind", C.c_int32), ("d", C.c_int32), ("d_y", C.c_int32), ("pad_", C.c_int32),
                ("lam", C.c_void_p), ("G", C.c_void_p), ("A", C.c_void_p), ("y", C.c_void_p),
                ("sigma", C.c_double), ("ban_a", C.c_double), ("ban_b", C.c_double), ("ban_c", C.c_double)]


class OrcConfig(C.Structure):
    _fields_ = [("d", C.c_int32), ("P", C.c_int32), ("n_lag", C.c_int32), ("M", C.c_int32),
                ("beta0", C.c_double), ("infl", C.c_double),
                ("adapt_beta", C.c_int32), ("xref_mode", C.c_int32),
                ("acc_lo", C.c_double), ("acc_hi", C.c_double), ("beta_factor", C.c_double),
                ("beta_min", C.c_double), ("beta_max", C.c_double),
                ("eps_jitter", C.c_double), ("min_samples_refresh", C.c_int64),
                ("refresh_delay", C.c_int32), ("prec", C.c_int32),
                ("seed", C.c_uint64), ("problem_id", C.c_uint32), ("threads", C.c_int32),
                ("trace_steps", C.c_int64), ("record_traj", C.c_int32), ("chain0", C.c_uint32),
                ("burnin", C.c_int64), ("proposal", C.c_int32), ("pad2_", C.c_int32), ("eps_jitter_min", C.c_double),
                ("moments_mode", C.c_int32), ("pad3_", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = C.CDLL(build())
            P, D, I64, U32, U64, I32 = C.c_void_p, C.c_double, C.c_int64, C.c_uint32, C.c_uint64, C.c_int32
            sig = {
                "orc_philox4x32_10": (None, [P, P, P]),
                "orc_key": (None, [U64, U32, P]),
                "orc_ln_u24": (C.c_float, [U32]),
                "orc_cossin_u24": (None, [U32, P, P]),
                "orc_boxmuller": (None, [U32, U32, P, P]),
                "orc_normals": (None, [U64, U32, I64, U32, I32, P]),
                "orc_uniform": (D, [U64, U32, U32, I64, U32]),
                "orc_round_bf16": (D, [D]),
                "orc_round_tf32": (D, [D]),
                "orc_round_f32": (D, [D]),
                "orc_cholesky": (I32, [I32, P, P]),
                "orc_forward_sub": (None, [I32, P, P, P]),
                "orc_target_logpi": (D, [P, P]),
                "orc_new": (P, [P, P, P, P, P]),
                "orc_free": (None, [P]),
                "orc_run": (I32, [P, I64, I32]),
                "orc_steps": (I64, [P]),
                "orc_beta": (D, [P]),
                "orc_counts": (None, [P, P]),
                "orc_get_state": (None, [P, P, P]),
                "orc_get_factor": (None, [P, P, P, P]),
                "orc_get_moments": (None, [P, P, P]),
                "orc_get_trace": (None, [P, P, P, P, P, P]),
                "orc_get_traj": (None, [P, P]),
                "orc_get_block_beta": (None, [P, P, I64]),
                "orc_get_chain_factor": (None, [P, I32, P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(l, name)
                f.restype = res
                f.argtypes = args
            _lib = l
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- random numbers (S1 of the hot path)
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def key(seed, problem_id=0):
    out = np.zeros(2, np.uint32)
    lib().orc_key(seed, problem_id, _ptr(out))
    return out


def ln_u24(a):
    return lib().orc_ln_u24(int(a))


def cossin_u24(b):
    c, s = C.c_float(), C.c_float()
    lib().orc_cossin_u24(int(b), C.byref(c), C.byref(s))
    return c.value, s.value


def boxmuller(a, b):
    n0, n1 = C.c_float(), C.c_float()
    lib().orc_boxmuller(int(a), int(b), C.byref(n0), C.byref(n1))
    return n0.value, n1.value


def normals(seed, problem_id, t, p, d):
    """W (FP32) for chain p at step t: the Gaussian draw of Algorithm 1."""
    w = np.zeros(d, np.float32)
    lib().orc_normals(seed, problem_id, t, p, d, _ptr(w))
    return w


def uniform(seed, problem_id, tag, t, p):
    return lib().orc_uniform(seed, problem_id, tag, t, p)


def round_bf16(v):
    f = np.vectorize(lambda z: lib().orc_round_bf16(float(z)), otypes=[np.float64])
    return f(np.asarray(v, np.float64))


def round_tf32(v):
    f = np.vectorize(lambda z: lib().orc_round_tf32(float(z)), otypes=[np.float64])
    return f(np.asarray(v, np.float64))


# ---------------------------------------------------------------- linear algebra
def cholesky(Cm):
    Cm = np.ascontiguousarray(Cm, np.float64)
    n = Cm.shape[0]
    L = np.zeros_like(Cm)
    rc = lib().orc_cholesky(n, _ptr(Cm), _ptr(L))
    return L if rc == 0 else None


def forward_sub(L, b):
    L = np.ascontiguousarray(L, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    y = np.zeros_like(b)
    lib().orc_forward_sub(L.shape[0], _ptr(L), _ptr(b), _ptr(y))
    return y


# ---------------------------------------------------------------- targets
class Target:
    """log pi of a synthetic target (eq. (bayes)); arrays are FP64, row-major."""

    def __init__(self, kind, d, d_y=0, lam=None, G=None, A=None, y=None, sigma=0.0,
                 ban_a=100.0, ban_b=0.1, ban_c=10.0):
        self.kind, self.d, self.d_y = kind, d, d_y
        self.lam = None if lam is None else np.ascontiguousarray(lam, np.float64)
        self.G = None if G is None else np.ascontiguousarray(G, np.float64)
        self.A = None if A is None else np.ascontiguousarray(A, np.float64)
        self.y = None if y is None else np.ascontiguousarray(y, np.float64)
        self.sigma, self.ban_a, self.ban_b, self.ban_c = sigma, ban_a, ban_b, ban_c

    def struct(self):
        return OrcTarget(self.kind, self.d, self.d_y, 0, _ptr(self.lam), _ptr(self.G), _ptr(self.A),
                         _ptr(self.y), self.sigma, self.ban_a, self.ban_b, self.ban_c)

    def logpi(self, x):
        x = np.ascontiguousarray(x, np.float64)
        st = self.struct()
        return lib().orc_target_logpi(C.byref(st), _ptr(x))


def default_config(**kw):
    c = dict(d=0, P=1, n_lag=100, M=10, beta0=0.3, infl=1.0, adapt_beta=1, xref_mode=1,
             acc_lo=0.3, acc_hi=0.5, beta_factor=1.1, beta_min=1e-4, beta_max=0.999,
             eps_jitter=1e-10, min_samples_refresh=-1, refresh_delay=0, prec=FP64,
             seed=0, problem_id=0, threads=1, trace_steps=0, record_traj=0, burnin=0, chain0=0, proposal=0,
             eps_jitter_min=0.0, moments_mode=0)
    c.update(kw)
    if c["min_samples_refresh"] < 0:
        c["min_samples_refresh"] = c["d"] + 1
    return c


class Sampler:
    """The DIAM sampler of Algorithm 1 over P concurrent chains sharing one pooled factor."""

    def __init__(self, cfg: dict, target: Target, x0=None, C0=None, xref0=None):
        self.cfg = dict(cfg)
        self.target = target
        self._cs = OrcConfig(**{k: self.cfg[k] for k, _ in OrcConfig._fields_ if k not in ("pad_", "pad2_", "pad3_")})
        self._ts = target.struct()
        d, P = self.cfg["d"], self.cfg["P"]
        self._x0 = None if x0 is None else np.ascontiguousarray(np.broadcast_to(x0, (P, d)), np.float64)
        self._C0 = None if C0 is None else np.ascontiguousarray(C0, np.float64)
        self._xr = None if xref0 is None else np.ascontiguousarray(xref0, np.float64)
        h = lib().orc_new(C.byref(self._cs), C.byref(self._ts), _ptr(self._x0), _ptr(self._C0), _ptr(self._xr))
        if not h:
            raise ValueError("oracle: initial covariance is not positive definite")
        self._h = C.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_free(h)
            self._h = None

    def run(self, n_steps, record=False):
        # the trajectory exists only if every run from the start recorded it
        self._recorded = bool(record) and (self.steps == 0 or getattr(self, "_recorded", False))
        if lib().orc_run(self._h, int(n_steps), int(bool(record))) != 0:
            raise MemoryError("oracle trajectory record too large")

    @property
    def steps(self):
        return lib().orc_steps(self._h)

    @property
    def beta(self):
        return lib().orc_beta(self._h)

    def counts(self):
        out = np.zeros(5, np.int64)
        lib().orc_counts(self._h, _ptr(out))
        return dict(n=int(out[0]), accepted=int(out[1]), refreshes=int(out[2]), notspd=int(out[3]),
                    chol_attempts=int(out[4]))

    def state(self):
        d, P = self.cfg["d"], self.cfg["P"]
        x = np.zeros((P, d)); lp = np.zeros(P)
        lib().orc_get_state(self._h, _ptr(x), _ptr(lp))
        return x, lp

    def factor(self):
        d = self.cfg["d"]
        L = np.zeros((d, d)); Lq = np.zeros((d, d)); xr = np.zeros(d)
        lib().orc_get_factor(self._h, _ptr(L), _ptr(Lq), _ptr(xr))
        return L, Lq, xr

    def moments(self):
        d = self.cfg["d"]
        m = np.zeros(d); Cm = np.zeros((d, d))
        lib().orc_get_moments(self._h, _ptr(m), _ptr(Cm))
        return m, Cm

    def trace(self):
        P = self.cfg["P"]
        T = min(self.steps, self.cfg["trace_steps"])
        arrs = [np.zeros((T, P)) for _ in range(4)]
        acc = np.zeros((T, P), np.int8)
        lib().orc_get_trace(self._h, *[_ptr(a) for a in arrs], _ptr(acc))
        return dict(lp_prop=arrs[0], q_prop=arrs[1], q_cur=arrs[2], loga=arrs[3], acc=acc.astype(bool))

    def trajectory(self):
        if not getattr(self, "_recorded", False):
            raise RuntimeError("no trajectory: run(..., record=True) from the first step")
        d, P = self.cfg["d"], self.cfg["P"]
        out = np.zeros((self.steps, P, d))
        lib().orc_get_traj(self._h, _ptr(out))
        return out

    def chain_factor(self, p):
        """Per-chain factors (Sec. 2.4.1): chain p's factor, its quantised form, x_ref and beta."""
        d = self.cfg["d"]
        L = np.zeros((d, d)); Lq = np.zeros((d, d)); xr = np.zeros(d); b = C.c_double()
        lib().orc_get_chain_factor(self._h, int(p), _ptr(L), _ptr(Lq), _ptr(xr), C.byref(b))
        return L, Lq, xr, b.value

    def block_betas(self):
        n = self.steps // self.cfg["n_lag"]
        out = np.zeros(n)
        lib().orc_get_block_beta(self._h, _ptr(out), n)
        return out
