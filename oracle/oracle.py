"""Python access to the FP64 PANDA oracle (``panda_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow statement of the
paper's element-wise equations (Eqs. 1-8) that the CUDA library is checked
against.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this module; the product path never does.

The shared library is compiled with gcc on first use (or by :func:`build`)
into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "panda_oracle.c")
_HDR = os.path.join(_HERE, "panda_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")

DIAG_D1, DIAG_D0, DIAG_D2 = 0, 1, 2

_lock = threading.Lock()
_lib = None

# -ffp-contract=off: a product and a sum are rounded separately on x86 and on
# aarch64 alike, so every machine computes the same FP64 bits.
CFLAGS = ["-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11"]


def compile_library(src: str = _SRC, out: str = _LIB, extra: list[str] | None = None) -> str:
    """Compile ``src`` into the shared library ``out`` with gcc."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, *(extra or []), "-I", _HERE, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Build ``oracle/_build/liboracle.so`` if it is missing or stale."""
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        compile_library()
    return _LIB


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
    pd, pi = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    sig = {
        "oracle_tanimoto": (d, [pd, l, pd, l, l]),
        "oracle_zscore": (i, [pd, l]),
        "oracle_normalize": (i, [i, i, pd, pd, pd]),
        "oracle_pearson": (i, [i, i, pd, pd]),
        "oracle_responsibility": (d, [i, i, pd, pd, i, i]),
        "oracle_availability": (d, [i, i, pd, pd, i, i]),
        "oracle_w_entry": (d, [i, i, pd, pd, pd, d, i, i]),
        "oracle_w_row": (None, [i, i, pd, pd, pd, d, i, pd]),
        "oracle_w_col": (None, [i, i, pd, pd, pd, d, i, pd]),
        "oracle_w_rows": (i, [i, i, pd, pd, pd, d, i, pi, pd]),
        "oracle_eq5_entry": (d, [d, d, pd, l, pd, l, l]),
        "oracle_diag_value": (d, [pd, i, i, d, d, d, i, i]),
        "oracle_p_rows": (i, [i, i, pd, pd, d, i, pi, pd, pd]),
        "oracle_c_rows": (i, [i, i, pd, pd, d, i, pi, pd, pd]),
        "oracle_step": (i, [i, i, pd, pd, pd, d, i, i, pd, pd, pd, pd]),
        "oracle_run": (i, [i, i, pd, pd, pd, d, d, i, i, i, pi, pd]),
        "oracle_set_threads": (None, [i]),
        "oracle_get_threads": (i, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (building first if needed) the oracle library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """Thin numpy wrapper over one loaded oracle library (the default one, or a
    separately compiled variant such as a planted-mistake build)."""

    def __init__(self, lib: ctypes.CDLL | None = None):
        self.lib = lib if lib is not None else load()

    # threads -------------------------------------------------------------
    def set_threads(self, n: int) -> None:
        self.lib.oracle_set_threads(int(n))

    def threads(self) -> int:
        return int(self.lib.oracle_get_threads())

    # Eq. 1 -----------------------------------------------------------------
    def tanimoto(self, x, y) -> float:
        x, y = _f64(x), _f64(y)
        assert x.shape == y.shape and x.ndim == 1
        return float(self.lib.oracle_tanimoto(_p(x), 1, _p(y), 1, x.size))

    # normalisation -----------------------------------------------------------
    def zscore(self, a) -> np.ndarray:
        a = _f64(a).copy()
        rc = self.lib.oracle_zscore(_p(a), a.size)
        if rc:
            raise ValueError(f"oracle_zscore failed ({rc})")
        return a

    def pearson(self, X):
        """Sec. II-A: the G x G Pearson correlation of the rows of X (G x N)."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        G, N = X.shape
        C = np.empty((G, G), np.float64)
        rc = self.lib.oracle_pearson(G, N, _p(X), _p(C))
        if rc:
            raise ValueError(f"oracle_pearson failed ({rc})")
        return C

    def normalize(self, W, P, C):
        W, P, C = _f64(W).copy(), _f64(P).copy(), _f64(C).copy()
        T, G = W.shape
        rc = self.lib.oracle_normalize(T, G, _p(W), _p(P), _p(C))
        if rc:
            raise ValueError(f"oracle_normalize failed ({rc})")
        return W, P, C

    # single entries ------------------------------------------------------------
    def responsibility(self, W, P, i, j) -> float:
        W, P = _f64(W), _f64(P)
        T, G = W.shape
        return float(self.lib.oracle_responsibility(T, G, _p(W), _p(P), int(i), int(j)))

    def availability(self, W, C, i, j) -> float:
        W, C = _f64(W), _f64(C)
        T, G = W.shape
        return float(self.lib.oracle_availability(T, G, _p(W), _p(C), int(i), int(j)))

    def w_entry(self, W, P, C, alpha, i, j) -> float:
        W, P, C = _f64(W), _f64(P), _f64(C)
        T, G = W.shape
        return float(self.lib.oracle_w_entry(T, G, _p(W), _p(P), _p(C), float(alpha), int(i), int(j)))

    def w_col(self, W, P, C, alpha, j) -> np.ndarray:
        W, P, C = _f64(W), _f64(P), _f64(C)
        T, G = W.shape
        out = np.empty(T)
        self.lib.oracle_w_col(T, G, _p(W), _p(P), _p(C), float(alpha), int(j), _p(out))
        return out

    def w_rows(self, W, P, C, alpha, rows) -> np.ndarray:
        W, P, C = _f64(W), _f64(P), _f64(C)
        T, G = W.shape
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        out = np.empty((rows.size, G))
        rc = self.lib.oracle_w_rows(T, G, _p(W), _p(P), _p(C), float(alpha), rows.size,
                                    rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(out))
        if rc:
            raise ValueError(f"oracle_w_rows failed ({rc})")
        return out

    def eq5_entry(self, old, alpha, x, y) -> float:
        """Eq. 5 for one off-diagonal entry."""
        x, y = _f64(x), _f64(y)
        return float(self.lib.oracle_eq5_entry(float(old), float(alpha), _p(x), 1, _p(y), 1, x.size))

    def diag_value(self, row, i, mult, old, alpha, t, diag=DIAG_D1) -> float:
        """Eq. 6 for one diagonal entry from row i of the updated network."""
        row = _f64(row)
        return float(self.lib.oracle_diag_value(_p(row), row.size, int(i), float(mult), float(old),
                                                float(alpha), int(t), int(diag)))

    def p_rows(self, Wn, P, alpha, rows, want_sim=False):
        Wn, P = _f64(Wn), _f64(P)
        T, G = Wn.shape
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        out = np.empty((rows.size, T))
        sim = np.empty((rows.size, T)) if want_sim else None
        rc = self.lib.oracle_p_rows(T, G, _p(Wn), _p(P), float(alpha), rows.size,
                                    rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(out),
                                    _p(sim) if want_sim else None)
        if rc:
            raise ValueError(f"oracle_p_rows failed ({rc})")
        return (out, sim) if want_sim else out

    def c_rows(self, Wn, C, alpha, rows, want_sim=False):
        Wn, C = _f64(Wn), _f64(C)
        T, G = Wn.shape
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        out = np.empty((rows.size, G))
        sim = np.empty((rows.size, G)) if want_sim else None
        rc = self.lib.oracle_c_rows(T, G, _p(Wn), _p(C), float(alpha), rows.size,
                                    rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(out),
                                    _p(sim) if want_sim else None)
        if rc:
            raise ValueError(f"oracle_c_rows failed ({rc})")
        return (out, sim) if want_sim else out

    # whole iterations -------------------------------------------------------------
    def step(self, W, P, C, alpha, t=1, diag=DIAG_D1):
        """One iteration (Eqs. 2-7); returns (W', P', C', h)."""
        W, P, C = _f64(W), _f64(P), _f64(C)
        T, G = W.shape
        Wn, Pn, Cn = np.empty_like(W), np.empty_like(P), np.empty_like(C)
        h = ctypes.c_double(0.0)
        rc = self.lib.oracle_step(T, G, _p(W), _p(P), _p(C), float(alpha), int(t), int(diag),
                                  _p(Wn), _p(Pn), _p(Cn), ctypes.byref(h))
        if rc:
            raise ValueError(f"oracle_step failed ({rc})")
        return Wn, Pn, Cn, h.value

    def run(self, W, P, C, alpha=0.1, tol=1e-3, max_iter=200, t0=0, diag=DIAG_D1):
        """Iterate from (W, P, C); returns (W, P, C, iters, h_history, converged)."""
        W, P, C = _f64(W).copy(), _f64(P).copy(), _f64(C).copy()
        T, G = W.shape
        iters = ctypes.c_int(0)
        hist = np.zeros(max(int(max_iter), 1))
        rc = self.lib.oracle_run(T, G, _p(W), _p(P), _p(C), float(alpha), float(tol),
                                 int(max_iter), int(t0), int(diag), ctypes.byref(iters), _p(hist))
        if rc < 0:
            raise ValueError(f"oracle_run failed ({rc})")
        n = iters.value
        return W, P, C, n, hist[:n].copy(), rc == 0
