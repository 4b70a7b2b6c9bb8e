"""ctypes binding of ``libpanda_gb300.so`` (the C ABI of ``include/panda.h``).

Argument marshalling only: every step of the iteration runs in the library's
CUDA kernels.  The functions keep the C names; :class:`PandaContext` wraps a
context handle.  Importing this module loads the library and raises when it
is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libpanda_gb300.so")

PANDA_OK = 0
PANDA_NOT_CONVERGED = 1
ERRORS = {-1: "PANDA_EINVAL", -2: "PANDA_ENOMEM", -3: "PANDA_ECUDA", -4: "PANDA_ENONFINITE",
          -5: "PANDA_EASYM", -6: "PANDA_EDEGENERATE", -7: "PANDA_ETIMEOUT", -8: "PANDA_EUNSUPPORTED"}
PANDA_FP32, PANDA_BF16X3, PANDA_BF16X2, PANDA_FP8MIX = 0, 1, 2, 3
PANDA_DIAG_D1, PANDA_DIAG_D0_LITERAL, PANDA_DIAG_D2_SIM = 0, 1, 2


class PandaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class panda_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("diag", ctypes.c_int), ("normalize", ctypes.c_int),
                ("t0", ctypes.c_int), ("graph_iters", ctypes.c_int)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1507_07039_gb300.build.build() "
                          "(the CUDA library is required; there is no fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, f, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_longlong
    pvp, pi, pd = ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    popts = ctypes.POINTER(panda_opts)
    sig = {
        "panda_default_opts": (None, [popts]),
        "panda_create": (i, [pvp, i, i, vp, vp, vp, popts]),
        "panda_create_device": (i, [pvp, i, i, vp, vp, vp, popts, vp]),
        "panda_step": (i, [vp, f, pd]),
        "panda_run": (i, [vp, f, d, i, pi, pd]),
        "panda_get": (i, [vp, vp, vp, vp]),
        "panda_get_device": (i, [vp, vp, vp, vp]),
        "panda_get_state": (i, [vp, vp, vp, vp, pi]),
        "panda_set_state": (i, [vp, vp, vp, vp, i]),
        "panda_checkpoint_bytes": (ll, [vp]),
        "panda_save": (i, [vp, vp, ll]),
        "panda_load": (i, [vp, vp, ll]),
        "panda_get_history": (i, [vp, pd, i, pi]),
        "panda_info": (i, [vp, pi, pi, pi, pi]),
        "panda_device_bytes": (ll, [vp]),
        "panda_device_bytes_peak": (ll, [vp]),
        "panda_stream": (vp, [vp]),
        "panda_set_profiling": (i, [vp, i]),
        "panda_kernel_count": (i, [vp]),
        "panda_kernel_stats": (i, [vp, i, ctypes.c_char_p, i, pd, ctypes.POINTER(ll)]),
        "panda_last_error": (ctypes.c_char_p, [vp]),
        "panda_precision_supported": (i, [i]),
        "panda_step_static": (i, [i, i, vp, vp, vp, f, i, i, pd, vp]),
        "panda_selftest_tc_gemm": (i, [i, i, i, vp, vp, vp, i]),
        "panda_selftest_timeout": (i, []),
        "panda_measure_ffma_peak": (i, [pd]),
        "panda_create_from_expression": (i, [pvp, i, i, i, vp, vp, vp, popts]),
        "panda_batch_create": (i, [pvp, i, pi, pi, pvp, pvp, pvp, popts]),
        "panda_batch_run": (i, [vp, f, d, i, pi, pd]),
        "panda_batch_get": (i, [vp, i, vp, vp, vp]),
        "panda_batch_size": (i, [vp]),
        "panda_batch_context": (vp, [vp, i]),
        "panda_batch_last_error": (ctypes.c_char_p, [vp]),
        "panda_batch_schedule": (i, [vp, pi, pi, ctypes.POINTER(ctypes.c_float), i,
                                     ctypes.POINTER(ctypes.c_float), i, pi]),
        "panda_batch_schedule_name": (ctypes.c_char_p, [i, i]),
        "panda_phase1_plan": (i, [i, i, i, i, i, pi, i, pi]),
        "panda_phase1_layout": (i, [vp, pi, pi, pi]),
        "panda_batch_destroy": (None, [vp]),
        "panda_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _last_error(ctx) -> str:
    m = lib.panda_last_error(ctx)
    return m.decode() if m else ""


def _check(rc: int, ctx=None) -> int:
    if rc < 0:
        raise PandaError(rc, _last_error(ctx))
    return rc


def _host_f32(a, shape) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    return a


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def default_opts(**kw) -> panda_opts:
    o = panda_opts()
    lib.panda_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


# ---- the C functions, same names -------------------------------------------------

def panda_create(T, G, W0, P0, C0, opts: panda_opts | None = None):
    """Host numpy inputs; returns a context handle (c_void_p)."""
    W0, P0, C0 = _host_f32(W0, (T, G)), _host_f32(P0, (T, T)), _host_f32(C0, (G, G))
    h = ctypes.c_void_p()
    _check(lib.panda_create(ctypes.byref(h), T, G, _ptr(W0), _ptr(P0), _ptr(C0),
                            ctypes.byref(opts) if opts is not None else None))
    return h


def panda_create_from_expression(W0, P0, X, opts: panda_opts | None = None):
    """C0 from the expression matrix X (G x N) on the GPU (Pearson, Sec. II-A);
    P0 may be None (identity).  Host numpy inputs; returns a context handle."""
    T, G = np.shape(W0)
    N = np.shape(X)[1]
    W0, X = _host_f32(W0, (T, G)), _host_f32(X, (G, N))
    P0 = None if P0 is None else _host_f32(P0, (T, T))
    h = ctypes.c_void_p()
    _check(lib.panda_create_from_expression(ctypes.byref(h), T, G, N, _ptr(W0), None if P0 is None else _ptr(P0),
                                            _ptr(X), ctypes.byref(opts) if opts is not None else None))
    return h


def panda_create_device(T, G, dW0, dP0, dC0, opts: panda_opts | None = None, stream=None):
    """Device inputs given as torch CUDA tensors (float32, contiguous) or raw pointers."""
    def ptr(x):
        return ctypes.c_void_p(x if isinstance(x, int) else x.data_ptr())
    h = ctypes.c_void_p()
    _check(lib.panda_create_device(ctypes.byref(h), T, G, ptr(dW0), ptr(dP0), ptr(dC0),
                                   ctypes.byref(opts) if opts is not None else None,
                                   ctypes.c_void_p(stream or 0)))
    return h


def panda_step(ctx, alpha: float) -> float:
    h = ctypes.c_double(0.0)
    _check(lib.panda_step(ctx, float(alpha), ctypes.byref(h)), ctx)
    return h.value


def panda_run(ctx, alpha: float, tol: float, max_iter: int):
    """Returns (converged, iterations, last h)."""
    n, h = ctypes.c_int(0), ctypes.c_double(0.0)
    rc = _check(lib.panda_run(ctx, float(alpha), float(tol), int(max_iter), ctypes.byref(n),
                              ctypes.byref(h)), ctx)
    return rc == PANDA_OK, n.value, h.value


def panda_get(ctx, T, G, want=(True, True, True)):
    W = np.empty((T, G), np.float32) if want[0] else None
    P = np.empty((T, T), np.float32) if want[1] else None
    C = np.empty((G, G), np.float32) if want[2] else None
    _check(lib.panda_get(ctx, *(None if x is None else _ptr(x) for x in (W, P, C))), ctx)
    return W, P, C


def panda_get_into(ctx, W=None, P=None, C=None):
    """panda_get into caller-allocated C-contiguous float32 host arrays."""
    for x in (W, P, C):
        if x is not None and (x.dtype != np.float32 or not x.flags.c_contiguous):
            raise ValueError("outputs must be C-contiguous float32 arrays")
    _check(lib.panda_get(ctx, *(None if x is None else _ptr(x) for x in (W, P, C))), ctx)


def panda_precision_supported(prec: int) -> bool:
    return bool(lib.panda_precision_supported(int(prec)))


def tensor_path_available() -> bool:
    return panda_precision_supported(PANDA_BF16X3)


def panda_get_device(ctx, dW=None, dP=None, dC=None):
    def ptr(x):
        return None if x is None else ctypes.c_void_p(x if isinstance(x, int) else x.data_ptr())
    _check(lib.panda_get_device(ctx, ptr(dW), ptr(dP), ptr(dC)), ctx)


def panda_get_state(ctx, T, G):
    W, P, C = (np.empty(s, np.float32) for s in ((T, G), (T, T), (G, G)))
    t = ctypes.c_int(0)
    _check(lib.panda_get_state(ctx, _ptr(W), _ptr(P), _ptr(C), ctypes.byref(t)), ctx)
    return W, P, C, t.value


def panda_set_state(ctx, W, P, C, t):
    T, G = np.shape(W)
    W, P, C = _host_f32(W, (T, G)), _host_f32(P, (T, T)), _host_f32(C, (G, G))
    _check(lib.panda_set_state(ctx, _ptr(W), _ptr(P), _ptr(C), int(t)), ctx)


def panda_set_state_device(ctx, dW, dP, dC, t):
    """panda_set_state from device buffers (torch CUDA tensors or raw pointers
    of this device)."""
    def ptr(x):
        return ctypes.c_void_p(x if isinstance(x, int) else x.data_ptr())
    _check(lib.panda_set_state(ctx, ptr(dW), ptr(dP), ptr(dC), int(t)), ctx)


def panda_save(ctx) -> bytes:
    n = lib.panda_checkpoint_bytes(ctx)
    buf = ctypes.create_string_buffer(n)
    _check(lib.panda_save(ctx, buf, n), ctx)
    return buf.raw


def panda_load(ctx, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib.panda_load(ctx, buf, len(blob)), ctx)


def panda_get_history(ctx) -> np.ndarray:
    n = ctypes.c_int(0)
    _check(lib.panda_get_history(ctx, None, 0, ctypes.byref(n)), ctx)
    k = min(n.value, 1 << 16)
    h = np.zeros(max(k, 1))
    _check(lib.panda_get_history(ctx, h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), k,
                                 ctypes.byref(n)), ctx)
    return h[:k]


def panda_info(ctx):
    T, G, p, t = (ctypes.c_int() for _ in range(4))
    _check(lib.panda_info(ctx, ctypes.byref(T), ctypes.byref(G), ctypes.byref(p), ctypes.byref(t)), ctx)
    return T.value, G.value, p.value, t.value


def panda_device_bytes(ctx) -> int:
    return int(lib.panda_device_bytes(ctx))


def panda_device_bytes_peak(ctx) -> int:
    return int(lib.panda_device_bytes_peak(ctx))


def panda_stream(ctx) -> int:
    return int(lib.panda_stream(ctx) or 0)


def panda_set_profiling(ctx, on: bool):
    _check(lib.panda_set_profiling(ctx, int(bool(on))), ctx)


def panda_kernel_count(ctx) -> int:
    return int(lib.panda_kernel_count(ctx))


def panda_kernel_stats(ctx, i: int):
    """(name, summed device ms, launches that did work) of kernel i."""
    name = ctypes.create_string_buffer(64)
    ms, n = ctypes.c_double(0.0), ctypes.c_longlong(0)
    _check(lib.panda_kernel_stats(ctx, int(i), name, 64, ctypes.byref(ms), ctypes.byref(n)), ctx)
    return name.value.decode(), ms.value, n.value


def panda_selftest_tc_gemm(A, B, terms: int = 3) -> np.ndarray:
    """D = A . B^T on the tensor-core pipeline (A: M x K, B: N x K, host)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    M, K = A.shape
    N = B.shape[0]
    assert B.shape[1] == K
    D = np.empty((M, N), np.float32)
    _check(lib.panda_selftest_tc_gemm(M, N, K, _ptr(A), _ptr(B), _ptr(D), int(terms)))
    return D


def panda_measure_ffma_peak() -> float:
    """FP32 FFMA throughput of the current device in TFLOP/s (measured)."""
    t = ctypes.c_double(0.0)
    _check(lib.panda_measure_ffma_peak(ctypes.byref(t)))
    return t.value


def panda_phase1_plan(T: int, G: int, prec: int, pairs: int, all_resident: bool = True):
    """How phase 1 of a T x G network is spread over `pairs` CTA pairs (host
    only): (number of cut tiles, int array of pieces with columns pair, mt,
    nt, c0, c1, cut)."""
    n = ctypes.c_int(0)
    _check(lib.panda_phase1_plan(int(T), int(G), int(prec), int(pairs), int(bool(all_resident)), None, 0,
                                 ctypes.byref(n)))
    out = np.zeros((n.value, 6), np.int32)
    cuts = _check(lib.panda_phase1_plan(int(T), int(G), int(prec), int(pairs), int(bool(all_resident)),
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n.value, ctypes.byref(n)))
    return cuts, out


def panda_phase1_layout(ctx) -> dict:
    """The phase-1 launch of a tensor-core context: CTA pairs, resident
    two-CTA clusters, cut tiles."""
    p, k, n = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(lib.panda_phase1_layout(ctx, ctypes.byref(p), ctypes.byref(k), ctypes.byref(n)), ctx)
    return {"pairs": p.value, "clusters": k.value, "cuts": n.value}


def panda_selftest_timeout() -> int:
    """Return code of the planted-timeout self-test (PANDA_ETIMEOUT = -7 expected)."""
    return int(lib.panda_selftest_timeout())


PANDA_STATIC_MAX_NODES = 512


def panda_step_static(T, G, dW, dP, dC, alpha: float, t: int, diag: int = PANDA_DIAG_D1, stream=None) -> float:
    """One iteration in place on caller-owned device networks (torch CUDA
    tensors or raw pointers) with no device allocation; returns h."""
    def ptr(x):
        return ctypes.c_void_p(x if isinstance(x, int) else x.data_ptr())
    h = ctypes.c_double(0.0)
    _check(lib.panda_step_static(int(T), int(G), ptr(dW), ptr(dP), ptr(dC), float(alpha), int(t),
                                 int(diag), ctypes.byref(h), ctypes.c_void_p(stream or 0)))
    return h.value


def panda_last_error(ctx=None) -> str:
    return _last_error(ctx)


def panda_destroy(ctx):
    lib.panda_destroy(ctx)


class PandaContext:
    """Owns one library context; a thin convenience over the C functions."""

    def __init__(self, W0, P0, C0, prec=PANDA_FP32, diag=PANDA_DIAG_D1, normalize=True, t0=0,
                 graph_iters=8, device=False, stream=None):
        if device:
            T, G = int(W0.shape[0]), int(W0.shape[1])
        else:
            T, G = np.shape(W0)
        self.T, self.G = T, G
        opts = default_opts(prec=prec, diag=diag, normalize=int(bool(normalize)), t0=t0,
                            graph_iters=graph_iters)
        if device:
            self.h = panda_create_device(T, G, W0, P0, C0, opts, stream)
        else:
            self.h = panda_create(T, G, W0, P0, C0, opts)

    @classmethod
    def from_expression(cls, W0, P0, X, prec=PANDA_FP32, diag=PANDA_DIAG_D1, normalize=True, t0=0,
                        graph_iters=8):
        """A context whose C0 is the Pearson correlation of X's rows, computed on the GPU."""
        self = cls.__new__(cls)
        self.T, self.G = np.shape(W0)
        opts = default_opts(prec=prec, diag=diag, normalize=int(bool(normalize)), t0=t0,
                            graph_iters=graph_iters)
        self.h = panda_create_from_expression(W0, P0, X, opts)
        return self

    def step(self, alpha=0.1) -> float:
        return panda_step(self.h, alpha)

    def run(self, alpha=0.1, tol=1e-3, max_iter=200):
        return panda_run(self.h, alpha, tol, max_iter)

    def get(self, want=(True, True, True)):
        return panda_get(self.h, self.T, self.G, want)

    def history(self):
        return panda_get_history(self.h)

    def info(self):
        return panda_info(self.h)

    @property
    def device_bytes(self):
        return panda_device_bytes(self.h)

    @property
    def device_bytes_peak(self):
        return panda_device_bytes_peak(self.h)

    @property
    def stream(self):
        return panda_stream(self.h)

    def close(self):
        if self.h:
            panda_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- sets of networks --------------------------------------------------------------

def panda_batch_create(nets, opts: panda_opts | None = None):
    """nets: sequence of (W0, P0, C0) host arrays; returns a batch handle."""
    n = len(nets)
    host = [(_host_f32(W, np.shape(W)), _host_f32(P, np.shape(P)), _host_f32(C, np.shape(C))) for W, P, C in nets]
    T = (ctypes.c_int * n)(*[h[0].shape[0] for h in host])
    G = (ctypes.c_int * n)(*[h[0].shape[1] for h in host])
    ptrs = [(ctypes.c_void_p * n)(*[h[q].ctypes.data for h in host]) for q in range(3)]
    b = ctypes.c_void_p()
    _check(lib.panda_batch_create(ctypes.byref(b), n, T, G, ptrs[0], ptrs[1], ptrs[2],
                                  ctypes.byref(opts) if opts is not None else None))
    return b


def panda_batch_run(b, alpha: float, tol: float, max_iter: int):
    """Returns (all converged, iterations per network, last h per network)."""
    n = lib.panda_batch_size(b)
    iters = (ctypes.c_int * n)()
    hl = (ctypes.c_double * n)()
    rc = lib.panda_batch_run(b, float(alpha), float(tol), int(max_iter), iters, hl)
    if rc < 0:
        m = lib.panda_batch_last_error(b)
        raise PandaError(rc, m.decode() if m else "")
    return rc == PANDA_OK, list(iters), list(hl)


def panda_batch_get(b, k: int, T: int, G: int):
    W, P, C = (np.empty(s, np.float32) for s in ((T, G), (T, T), (G, G)))
    rc = lib.panda_batch_get(b, int(k), _ptr(W), _ptr(P), _ptr(C))
    if rc < 0:
        m = lib.panda_batch_last_error(b)
        raise PandaError(rc, m.decode() if m else "")
    return W, P, C


class PandaBatch:
    """A set of independent networks iterated together (see panda_batch_run)."""

    def __init__(self, nets, prec=PANDA_FP32, diag=PANDA_DIAG_D1, normalize=True, graph_iters=8):
        self.shapes = [np.shape(W) for W, _, _ in nets]
        opts = default_opts(prec=prec, diag=diag, normalize=int(bool(normalize)), graph_iters=graph_iters)
        self.h = panda_batch_create(nets, opts)

    def __len__(self):
        return len(self.shapes)

    def run(self, alpha=0.1, tol=1e-3, max_iter=200):
        return panda_batch_run(self.h, alpha, tol, max_iter)

    def get(self, k):
        T, G = self.shapes[k]
        return panda_batch_get(self.h, k, T, G)

    def context(self, k):
        """Network k's context handle (owned by the batch)."""
        return ctypes.c_void_p(lib.panda_batch_context(self.h, int(k)))

    def schedule(self):
        """The schedule autotuning of a tensor-core batch: dict with the
        phase-1 and phase-2 candidates in use (p1, p2), their descriptions,
        the median trial times in ms of every candidate (p1_ms, p2_ms) and
        whether the trials are over; None for an FP32 batch."""
        p1, p2, done = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        m1, m2 = (ctypes.c_float * 16)(), (ctypes.c_float * 16)()
        n = lib.panda_batch_schedule(self.h, ctypes.byref(p1), ctypes.byref(p2), m1, 16, m2, 16,
                                     ctypes.byref(done))
        if n < 0:
            raise PandaError(n, "panda_batch_schedule")
        if n == 0:
            return None
        names = {ph: [] for ph in (1, 2)}
        for ph in (1, 2):
            while (nm := lib.panda_batch_schedule_name(ph, len(names[ph]))) is not None:
                names[ph].append(nm.decode())
        return {"p1": p1.value, "p2": p2.value, "p1_names": names[1], "p2_names": names[2],
                "p1_ms": [m1[q] for q in range(len(names[1]))], "p2_ms": [m2[q] for q in range(len(names[2]))],
                "done": bool(done.value)}

    def close(self):
        if self.h:
            lib.panda_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

