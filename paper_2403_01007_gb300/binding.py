"""Thin ctypes binding of the C ABI declared in include/sccsd.h.

Argument marshalling only: arrays are passed as raw pointers (NumPy arrays
for host memory, CUDA torch tensors for device memory), every computation
happens in the compiled library. Importing fails loudly when the library
has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsccsd.so")

FP64, BF16X3, BF16 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "bf16x3": BF16X3, "bf16": BF16}

_dp = ctypes.c_void_p


def _declare(lib):
    lib.sccsd_init.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, _dp, _dp, ctypes.c_int, _dp]
    lib.sccsd_residual.argtypes = [_dp, _dp, ctypes.c_double, _dp, _dp, _dp, _dp]
    lib.sccsd_jacobian_right.argtypes = [_dp, ctypes.c_int, _dp, _dp, _dp]
    lib.sccsd_jacobian_left.argtypes = [_dp, ctypes.c_int, _dp, _dp]
    lib.sccsd_densities.argtypes = [_dp, ctypes.c_double, _dp, ctypes.c_double, _dp, _dp, _dp]
    lib.sccsd_gemm_tn.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong,
                                  ctypes.c_longlong, ctypes.c_double, _dp, _dp, _dp, _dp]
    lib.sccsd_gemm_tn.restype = ctypes.c_int
    lib.sccsd_profile.argtypes = [_dp, ctypes.c_int]
    lib.sccsd_profile.restype = ctypes.c_int
    lib.sccsd_profile_read.argtypes = [_dp, _dp, _dp, _dp, _dp]
    lib.sccsd_profile_read.restype = ctypes.c_int
    lib.sccsd_gemm_tn_noalloc.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong,
                                          ctypes.c_double, _dp, _dp, _dp, _dp]
    lib.sccsd_gemm_tn_noalloc.restype = ctypes.c_int
    lib.sccsd_gemm_tn_noalloc_capacity.argtypes = []
    lib.sccsd_gemm_tn_noalloc_capacity.restype = ctypes.c_longlong
    lib.sccsd_set_precision.argtypes = [_dp, ctypes.c_int]
    lib.sccsd_set_precision.restype = ctypes.c_int
    lib.sccsd_set_autotune.argtypes = [_dp, ctypes.c_int]
    lib.sccsd_set_autotune.restype = ctypes.c_int
    lib.sccsd_autotune_export.argtypes = [ctypes.c_char_p, ctypes.c_longlong,
                                          ctypes.POINTER(ctypes.c_longlong)]
    lib.sccsd_autotune_export.restype = ctypes.c_int
    lib.sccsd_autotune_import.argtypes = [ctypes.c_char_p]
    lib.sccsd_autotune_import.restype = ctypes.c_int
    lib.sccsd_autotune_clear.argtypes = []
    lib.sccsd_autotune_clear.restype = None
    lib.sccsd_autotune_entries.argtypes = []
    lib.sccsd_autotune_entries.restype = ctypes.c_longlong
    lib.sccsd_solve_ground.argtypes = [_dp, _dp, ctypes.c_double, _dp, _dp, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
    lib.sccsd_solve_ground.restype = ctypes.c_int
    lib.sccsd_normalize_left.argtypes = [_dp, ctypes.c_int, _dp, _dp]
    lib.sccsd_normalize_left.restype = ctypes.c_int
    lib.sccsd_solve_states.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
    lib.sccsd_solve_states.restype = ctypes.c_int
    lib.sccsd_overlap.argtypes = [_dp, ctypes.c_double, _dp, ctypes.c_double, _dp, _dp]
    lib.sccsd_overlap_states.argtypes = [_dp, ctypes.c_double, _dp, ctypes.c_double, _dp, _dp]
    lib.sccsd_overlap_states.restype = ctypes.c_int
    lib.sccsd_set_projection.argtypes = [_dp, ctypes.c_int]
    lib.sccsd_set_projection.restype = ctypes.c_int
    lib.sccsd_overlap.restype = ctypes.c_int
    lib.sccsd_solve_scc.argtypes = [_dp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    lib.sccsd_solve_scc.restype = ctypes.c_int
    lib.sccsd_overlaps.argtypes = [_dp, ctypes.c_int, _dp, _dp, ctypes.c_int, _dp]
    lib.sccsd_overlaps.restype = ctypes.c_int
    lib.sccsd_residual_states.argtypes = [_dp, _dp, ctypes.c_int, _dp, _dp, _dp, _dp]
    lib.sccsd_residual_states.restype = ctypes.c_int
    lib.sccsd_solve_ground_states.argtypes = [_dp, _dp, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                              ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
    lib.sccsd_solve_ground_states.restype = ctypes.c_int
    lib.sccsd_solve_scc_states.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp,
                                           _dp, _dp, _dp]
    lib.sccsd_solve_scc_states.restype = ctypes.c_int
    # The MLP entry points live in their own translation unit (mlp.cu), which
    # the host test double links without; every entry point the library
    # exports gets its signature (the export test checks that the product
    # library has every declared symbol). Undeclared pointer arguments would be
    # passed as C ints.
    _int = ctypes.c_int
    learned = {
        "sccsd_mlp_create": ([ctypes.POINTER(ctypes.c_void_p), _int, _int, _int, _int,
                              ctypes.c_ulonglong, _dp], _int),
        "sccsd_mlp_destroy": ([_dp], None),
        "sccsd_mlp_last_error": ([_dp], ctypes.c_char_p),
        "sccsd_mlp_num_params": ([_dp], ctypes.c_longlong),
        "sccsd_mlp_get_params": ([_dp, _dp], _int),
        "sccsd_mlp_set_params": ([_dp, _dp], _int),
        "sccsd_mlp_forward": ([_dp, _dp, ctypes.c_longlong, _dp], _int),
        "sccsd_mlp_gradient": ([_dp, _dp, _dp, ctypes.c_longlong, _dp, _dp], _int),
        "sccsd_mlp_train_step": ([_dp, _dp, _dp, ctypes.c_longlong, ctypes.c_float, _dp], _int),
        "sccsd_learned_features": ([_dp, _dp, _dp], _int),
        "sccsd_learned_targets": ([_dp, _dp, ctypes.c_double, _dp], _int),
        "sccsd_learned_guess": ([_dp, _dp, _dp, _dp], _int),
        "sccsd_set_preconditioner": ([_dp, _dp], _int),
    }
    for name, (args, res) in learned.items():
        if hasattr(lib, name):
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
    lib.sccsd_solve_multipliers.argtypes = [_dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp]
    lib.sccsd_solve_multipliers.restype = ctypes.c_int
    lib.sccsd_multiplier_residual.argtypes = [_dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, _dp, _dp]
    lib.sccsd_multiplier_residual.restype = ctypes.c_int
    lib.sccsd_integral_derivative.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp]
    lib.sccsd_integral_derivative.restype = ctypes.c_int
    lib.sccsd_input_derivative.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp]
    lib.sccsd_input_derivative.restype = ctypes.c_int
    lib.sccsd_state_amplitudes.argtypes = [_dp, _dp]
    lib.sccsd_state_amplitudes.restype = ctypes.c_int
    lib.sccsd_capture_transform.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                            ctypes.POINTER(ctypes.c_void_p)]
    lib.sccsd_capture_transform.restype = ctypes.c_int
    lib.sccsd_graph_join.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_void_p)]
    lib.sccsd_graph_join.restype = ctypes.c_int
    lib.sccsd_graph_launch.argtypes = [_dp, _dp]
    lib.sccsd_graph_launch.restype = ctypes.c_int
    lib.sccsd_graph_destroy.argtypes = [_dp]
    lib.sccsd_graph_destroy.restype = None
    lib.sccsd_graph_exec_destroy.argtypes = [_dp]
    lib.sccsd_graph_exec_destroy.restype = None
    lib.sccsd_dim.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.sccsd_dim.restype = ctypes.c_longlong
    lib.sccsd_last_error.argtypes = [_dp]
    lib.sccsd_last_error.restype = ctypes.c_char_p
    lib.sccsd_strerror.argtypes = [ctypes.c_int]
    lib.sccsd_strerror.restype = ctypes.c_char_p
    lib.sccsd_destroy.argtypes = [_dp]
    lib.sccsd_destroy.restype = None
    for f in ("sccsd_init", "sccsd_residual", "sccsd_jacobian_right",
              "sccsd_jacobian_left", "sccsd_densities"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


_LIB = None


def load(path: str | None = None):
    """Load the compiled library (raises if it is missing)."""
    global _LIB
    if path is None and _LIB is not None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"compiled SCCSD library not found at {p}; run the build first")
    lib = _declare(ctypes.CDLL(p))
    if path is None:
        _LIB = lib
    return lib


class SccsdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sccsd error {code}: {msg}")
        self.code = code


def _ptr(x):
    """Pointer of a float64 array: NumPy (host) or torch tensor (host/device)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise TypeError("arrays must be C-contiguous float64")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def autotune_export(lib=None) -> str:
    """The process-wide table of tuned launch shapes as text."""
    lib = lib or load()
    n = ctypes.c_longlong()
    lib.sccsd_autotune_export(None, 0, ctypes.byref(n))
    for _ in range(8):          # the table may grow between the two calls
        buf = ctypes.create_string_buffer(n.value)
        rc = lib.sccsd_autotune_export(buf, n.value, ctypes.byref(n))
        if rc == 0:
            return buf.value.decode()
    raise SccsdError(rc, "autotune export")


def autotune_import(text: str, lib=None):
    """Merge a table written by autotune_export (all or nothing)."""
    lib = lib or load()
    rc = lib.sccsd_autotune_import(text.encode())
    if rc != 0:
        raise SccsdError(rc, "malformed or invalid autotune table")


def autotune_clear(lib=None):
    (lib or load()).sccsd_autotune_clear()


def autotune_entries(lib=None) -> int:
    return int((lib or load()).sccsd_autotune_entries())


def dim(o: int, v: int) -> int:
    ov = o * v
    return ov + ov * (ov + 1) // 2


def gemm_tn(A, B, C, alpha=1.0, precision="fp64", lib=None):
    """C = alpha * A @ B.T on device tensors through the library's kernels."""
    lib = lib or load()
    M, K = A.shape
    N = B.shape[0]
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    rc = lib.sccsd_gemm_tn(prec, M, N, K, float(alpha), _ptr(A), _ptr(B), _ptr(C), None)
    if rc != 0:
        raise SccsdError(rc, lib.sccsd_strerror(rc).decode())
    return C


def gemm_tn_noalloc(A, B, C, alpha=1.0, stream=None, lib=None):
    """FP64 C = alpha * A @ B.T on device tensors without any device allocation.
    The work is enqueued on `stream` (a torch.cuda.Stream, default the legacy
    default stream) and the call returns without waiting for it."""
    lib = lib or load()
    M, K = A.shape
    N = B.shape[0]
    sp = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    rc = lib.sccsd_gemm_tn_noalloc(M, N, K, float(alpha), _ptr(A), _ptr(B), _ptr(C), sp)
    if rc != 0:
        raise SccsdError(rc, lib.sccsd_strerror(rc).decode())
    return C


def _fptr(x):
    """Pointer of a float32 array (NumPy or torch)."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float32 or not x.flags.c_contiguous:
            raise TypeError("arrays must be C-contiguous float32")
        return x.ctypes.data
    import torch
    if x.dtype != torch.float32 or not x.is_contiguous():
        raise TypeError("tensors must be contiguous float32")
    return x.data_ptr()


class GraphBatch:
    """One executable CUDA graph joining captured per-instance graphs."""

    def __init__(self, graphs, lib=None):
        self.lib = lib or load()
        arr = (ctypes.c_void_p * len(graphs))(*[g.value for g in graphs])
        e = ctypes.c_void_p()
        rc = self.lib.sccsd_graph_join(arr, len(graphs), ctypes.byref(e))
        if rc != 0:
            raise SccsdError(rc, "graph join failed")
        self.exec = e
        self.graphs = graphs

    def launch(self, stream=None):
        rc = self.lib.sccsd_graph_launch(self.exec, None if stream is None else ctypes.c_void_p(stream))
        if rc != 0:
            raise SccsdError(rc, "graph launch failed")

    def close(self):
        if getattr(self, "exec", None):
            self.lib.sccsd_graph_exec_destroy(self.exec)
            for g in self.graphs:
                self.lib.sccsd_graph_destroy(g)
            self.exec = None


class Mlp:
    """Per-amplitude network of the learned guess (BF16 weights, FP32 accumulation)."""

    def __init__(self, n_in=10, hidden=256, layers=3, n_out=2, seed=1, lib=None):
        self.lib = lib or load()
        h = ctypes.c_void_p()
        rc = self.lib.sccsd_mlp_create(ctypes.byref(h), n_in, hidden, layers, n_out, seed, None)
        if rc != 0:
            raise SccsdError(rc, "mlp create failed")
        self.h = h
        self.n_in, self.n_out = n_in, n_out

    def _check(self, rc):
        if rc != 0:
            raise SccsdError(rc, self.lib.sccsd_mlp_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.sccsd_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self):
        return self.lib.sccsd_mlp_num_params(self.h)

    def get_params(self):
        p = np.empty(self.num_params(), dtype=np.float32)
        self._check(self.lib.sccsd_mlp_get_params(self.h, p.ctypes.data))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self.lib.sccsd_mlp_set_params(self.h, p.ctypes.data))

    def forward(self, X, Y):
        self._check(self.lib.sccsd_mlp_forward(self.h, _fptr(X), X.shape[0], _fptr(Y)))
        return Y

    def gradient(self, X, T):
        g = np.empty(self.num_params(), dtype=np.float32)
        loss = ctypes.c_float()
        self._check(self.lib.sccsd_mlp_gradient(self.h, _fptr(X), _fptr(T), X.shape[0],
                                                g.ctypes.data, ctypes.addressof(loss)))
        return g, loss.value

    def train_step(self, X, T, lr):
        loss = ctypes.c_float()
        self._check(self.lib.sccsd_mlp_train_step(self.h, _fptr(X), _fptr(T), X.shape[0],
                                                  float(lr), ctypes.addressof(loss)))
        return loss.value


class Context:
    """One system: orbital energies eps[n] and Cholesky vectors L[J][n][n]."""

    def __init__(self, o, v, J, eps, L, precision="fp64", stream=None, lib=None):
        self.lib = lib or load()
        self.o, self.v, self.J = o, v, J
        self.n = o + v
        self.dim = dim(o, v)
        h = ctypes.c_void_p()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        s = None if stream is None else ctypes.c_void_p(stream)
        rc = self.lib.sccsd_init(ctypes.byref(h), o, v, J, _ptr(eps), _ptr(L), prec, s)
        if rc != 0:
            raise SccsdError(rc, self.lib.sccsd_strerror(rc).decode())
        self.h = h
        self._keep = (eps, L)

    def _check(self, rc):
        if rc != 0:
            raise SccsdError(rc, self.lib.sccsd_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.sccsd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def residual(self, t, omega=None, scc=None):
        """Return (e_corr, omega); scc = (zeta, Ra, Rb) or None."""
        if omega is None:
            omega = np.empty(self.dim)
        e = ctypes.c_double()
        zeta, Ra, Rb = (0.0, None, None) if scc is None else scc
        self._check(self.lib.sccsd_residual(self.h, _ptr(t), float(zeta), _ptr(Ra), _ptr(Rb),
                                            _ptr(omega), ctypes.addressof(e)))
        return e.value, omega

    def jacobian_right(self, R, sigma=None, with_eta=False):
        nvec = 1 if R.ndim == 1 else R.shape[0]
        if sigma is None:
            sigma = np.empty_like(R) if isinstance(R, np.ndarray) else R.new_empty(R.shape)
        eta = np.empty(nvec) if with_eta else None
        self._check(self.lib.sccsd_jacobian_right(self.h, nvec, _ptr(R), _ptr(sigma), _ptr(eta)))
        return (sigma, eta) if with_eta else sigma

    def jacobian_left(self, L, sigma=None):
        nvec = 1 if L.ndim == 1 else L.shape[0]
        if sigma is None:
            sigma = np.empty_like(L) if isinstance(L, np.ndarray) else L.new_empty(L.shape)
        self._check(self.lib.sccsd_jacobian_left(self.h, nvec, _ptr(L), _ptr(sigma)))
        return sigma

    def set_precision(self, precision):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._check(self.lib.sccsd_set_precision(self.h, prec))

    def set_autotune(self, enable=True):
        """Time the launch shapes of each new tensor-core contraction shape of
        this context and record the fastest in the process-wide table."""
        self._check(self.lib.sccsd_set_autotune(self.h, 1 if enable else 0))

    def solve_ground(self, t0=None, tol=1e-10, maxit=200, refine_tol=1e-4, scc=None, t_out=None):
        """Converge the ground state; returns (e_corr, t, iterations)."""
        if t_out is None:
            t_out = np.empty(self.dim)
        e = ctypes.c_double()
        it = ctypes.c_int()
        zeta, Ra, Rb = (0.0, None, None) if scc is None else scc
        self._check(self.lib.sccsd_solve_ground(self.h, _ptr(t0), float(zeta), _ptr(Ra), _ptr(Rb),
                                                float(tol), int(maxit), float(refine_tol),
                                                _ptr(t_out), ctypes.addressof(e),
                                                ctypes.addressof(it)))
        return e.value, t_out, it.value

    def solve_states(self, nroots, side="right", tol=1e-8, maxit=200, refine_tol=1e-4, vecs=True):
        """Lowest EOM roots; returns (omega[nroots], vecs[nroots][dim] or None, iterations)."""
        w = np.empty(nroots)
        V = np.empty((nroots, self.dim)) if vecs else None
        it = ctypes.c_int()
        sd = 0 if side in ("right", 0) else 1
        self._check(self.lib.sccsd_solve_states(self.h, int(nroots), sd, float(tol), int(maxit),
                                                float(refine_tol), w.ctypes.data, _ptr(V),
                                                ctypes.addressof(it)))
        return w, V, it.value

    def normalize_left(self, R, L):
        """L_k scaled in place so that L_k . R_k = 1 (the library's kernels do
        the arithmetic); R and L are [nvec][dim] host arrays or device tensors."""
        def c(x):
            if hasattr(x, "data_ptr"):
                return x
            return np.ascontiguousarray(x, dtype=np.float64)
        R = c(R)
        L = c(L)
        nvec = int(L.shape[0]) if L.ndim == 2 else 1
        self._check(self.lib.sccsd_normalize_left(self.h, nvec, _ptr(R), _ptr(L)))
        return L

    def overlap(self, ra0, Ra, rb0, Rb):
        """SCC orthogonality O_ab at the fixed state (natural projection)."""
        out = ctypes.c_double()
        self._check(self.lib.sccsd_overlap(self.h, float(ra0), _ptr(Ra), float(rb0), _ptr(Rb),
                                           ctypes.addressof(out)))
        return out.value

    def overlap_states(self, ra0, Ra, rb0, Rb):
        """SCC orthogonality O_ab with the state projection over K = {a, b}."""
        out = ctypes.c_double()
        self._check(self.lib.sccsd_overlap_states(self.h, float(ra0), _ptr(Ra), float(rb0),
                                                  _ptr(Rb), ctypes.addressof(out)))
        return out.value

    def overlaps(self, r0, R, projection="natural"):
        """O_kl of every pair k < l of the states (r0[k], R[k]) at the fixed
        state, natural or state projection over all of them; {(k, l): O_kl}."""
        p = {"natural": 0, "state": 1}.get(projection, projection)
        r0 = np.ascontiguousarray(r0, dtype=np.float64)
        R = R if hasattr(R, "data_ptr") else np.ascontiguousarray(R, dtype=np.float64)
        n = int(R.shape[0])
        out = np.empty(n * (n - 1) // 2)
        self._check(self.lib.sccsd_overlaps(self.h, n, r0.ctypes.data, _ptr(R), int(p),
                                            out.ctypes.data))
        pairs = [(k, l) for k in range(n) for l in range(k + 1, n)]
        return dict(zip(pairs, out.tolist()))

    def set_projection(self, projection):
        """0 / "natural": SCCSD(E); 1 / "state": SCCSD(K), for sccsd_solve_scc."""
        p = {"natural": 0, "state": 1}.get(projection, projection)
        self._check(self.lib.sccsd_set_projection(self.h, int(p)))

    def solve_scc(self, tol=1e-10, maxit=40, ground_tol=1e-11, eom_tol=1e-9):
        """Self-consistent SCCSD for the two lowest states; returns a dict."""
        z, e = ctypes.c_double(), ctypes.c_double()
        w, r0 = np.empty(2), np.empty(2)
        Ra, Rb = np.empty(self.dim), np.empty(self.dim)
        it = ctypes.c_int()
        self._check(self.lib.sccsd_solve_scc(self.h, float(tol), int(maxit), float(ground_tol),
                                             float(eom_tol), ctypes.addressof(z),
                                             ctypes.addressof(e), w.ctypes.data, r0.ctypes.data,
                                             Ra.ctypes.data, Rb.ctypes.data,
                                             ctypes.addressof(it)))
        return {"zeta": z.value, "e_corr": e.value, "omega": w, "r0": r0, "Ra": Ra, "Rb": Rb,
                "iterations": it.value}

    def residual_states(self, t, zeta, R, omega=None):
        """(e_corr, omega) with the X3 terms of several constrained states:
        zeta[n(n-1)/2] in the pair order (0,1), (0,2), ..., (1,2), ...; R[n][dim]."""
        if omega is None:
            omega = np.empty(self.dim)
        z = np.ascontiguousarray(zeta, dtype=np.float64)
        R = R if hasattr(R, "data_ptr") else np.ascontiguousarray(R, dtype=np.float64)
        e = ctypes.c_double()
        self._check(self.lib.sccsd_residual_states(self.h, _ptr(t), int(R.shape[0]), _ptr(z),
                                                   _ptr(R), _ptr(omega), ctypes.addressof(e)))
        return e.value, omega

    def solve_ground_states(self, zeta, R, t0=None, tol=1e-10, maxit=200, refine_tol=1e-4):
        """Ground state with the X3 terms of several states; (e_corr, t, iterations)."""
        t_out = np.empty(self.dim)
        z = np.ascontiguousarray(zeta, dtype=np.float64)
        R = R if hasattr(R, "data_ptr") else np.ascontiguousarray(R, dtype=np.float64)
        e, it = ctypes.c_double(), ctypes.c_int()
        self._check(self.lib.sccsd_solve_ground_states(
            self.h, _ptr(t0), int(R.shape[0]), _ptr(z), _ptr(R), float(tol), int(maxit),
            float(refine_tol), _ptr(t_out), ctypes.addressof(e), ctypes.addressof(it)))
        return e.value, t_out, it.value

    def solve_scc_states(self, nstates, tol=1e-10, maxit=60, ground_tol=1e-11, eom_tol=1e-9):
        """Self-consistent SCCSD for the nstates lowest states (one zeta per
        pair, Broyden; the projection of set_projection); returns a dict."""
        npair = nstates * (nstates - 1) // 2
        z, O = np.empty(npair), np.empty(npair)
        w, r0 = np.empty(nstates), np.empty(nstates)
        R = np.empty((nstates, self.dim))
        e, it = ctypes.c_double(), ctypes.c_int()
        self._check(self.lib.sccsd_solve_scc_states(
            self.h, int(nstates), float(tol), int(maxit), float(ground_tol), float(eom_tol),
            z.ctypes.data, O.ctypes.data, ctypes.addressof(e), w.ctypes.data, r0.ctypes.data,
            R.ctypes.data, ctypes.addressof(it)))
        pairs = [(k, l) for k in range(nstates) for l in range(k + 1, nstates)]
        return {"zeta": dict(zip(pairs, z.tolist())), "O": dict(zip(pairs, O.tolist())),
                "e_corr": e.value, "omega": w, "r0": r0, "R": R, "iterations": it.value}

    def learned_features(self, X):
        """Features [o^2 v^2][10] (device float32) at the MP2 amplitudes; returns scales."""
        sc = np.empty(3)
        self._check(self.lib.sccsd_learned_features(self.h, _fptr(X), sc.ctypes.data))
        return sc

    def learned_targets(self, t, s_t, Y):
        self._check(self.lib.sccsd_learned_targets(self.h, _ptr(t), float(s_t), _fptr(Y)))
        return Y

    def learned_guess(self, net):
        t0, D = np.empty(self.dim), np.empty(self.dim)
        self._check(self.lib.sccsd_learned_guess(self.h, net.h, t0.ctypes.data, D.ctypes.data))
        return t0, D

    def set_preconditioner(self, D=None):
        self._check(self.lib.sccsd_set_preconditioner(self.h, _ptr(D)))

    def integral_derivative(self, D1, Gamma, h1, L1):
        """sum D1 h1 + sum Gamma L1: a gradient or coupling along a perturbation
        (h1, L1) of the integrals, from the effective densities."""
        def c(x):   # NumPy arrays made contiguous; tensors (host or device) as given
            if x is None or hasattr(x, "data_ptr"):
                return x
            return np.ascontiguousarray(x, dtype=np.float64)
        out = ctypes.c_double()
        self._check(self.lib.sccsd_integral_derivative(
            self.h, _ptr(c(D1)), _ptr(c(Gamma)), _ptr(c(h1)), _ptr(c(L1)),
            ctypes.addressof(out)))
        return out.value

    def input_derivative(self, D1, Gamma, deps, dL):
        """A gradient or coupling along a perturbation (deps, dL) of eps and L,
        the inputs of the context (h follows them)."""
        def c(x):
            if x is None or hasattr(x, "data_ptr"):
                return x
            return np.ascontiguousarray(x, dtype=np.float64)
        out = ctypes.c_double()
        self._check(self.lib.sccsd_input_derivative(
            self.h, _ptr(c(D1)), _ptr(c(Gamma)), _ptr(c(deps)), _ptr(c(dL)),
            ctypes.addressof(out)))
        return out.value

    def state_amplitudes(self):
        t = np.empty(self.dim)
        self._check(self.lib.sccsd_state_amplitudes(self.h, _ptr(t)))
        return t

    def scc_state(self, tol=1e-10, maxit=40, ground_tol=1e-11, eom_tol=1e-9, left_tol=1e-9,
                  left_maxit=200):
        """Converged SCCSD for the two lowest states plus their left vectors
        (L_k . R_k = 1): the state dict taken by solve_multipliers."""
        r = self.solve_scc(tol=tol, maxit=maxit, ground_tol=ground_tol, eom_tol=eom_tol)
        t = self.state_amplitudes()
        wl, VL, _ = self.solve_states(2, side="left", tol=left_tol, maxit=left_maxit)
        VL = self.normalize_left(np.stack([r["Ra"], r["Rb"]]), VL)
        return {"t": t, "Ra": r["Ra"], "Rb": r["Rb"], "La": VL[0], "Lb": VL[1], "zeta": r["zeta"],
                "r0a": float(r["r0"][0]), "r0b": float(r["r0"][1]),
                "omega_a": float(r["omega"][0]), "omega_b": float(r["omega"][1]),
                "omega_left": wl, "e_corr": r["e_corr"]}

    @staticmethod
    def _mult_args(state, target):
        vecs = np.ascontiguousarray(np.concatenate(
            [np.asarray(state[k], dtype=np.float64).reshape(-1) for k in ("t", "Ra", "Rb", "La", "Lb")]))
        scal = np.array([state["zeta"], state["r0a"], state["r0b"], state["omega_a"],
                         state["omega_b"]], dtype=np.float64)
        if target[0] == "gradient":
            return vecs, scal, 0, 0, int(target[1])
        return vecs, scal, 1, int(target[1]), int(target[2])

    def multiplier_residual(self, state, target, u):
        vecs, scal, kind, m, n = self._mult_args(state, target)
        u = np.ascontiguousarray(u, dtype=np.float64)
        r = np.empty(3 * self.dim + 1)
        self._check(self.lib.sccsd_multiplier_residual(self.h, _ptr(vecs), _ptr(scal), kind, m, n,
                                                       _ptr(u), _ptr(r)))
        return r

    def solve_multipliers(self, state, target, tol=1e-9, maxit=400, refine_tol=1e-6,
                          densities=True):
        """Multipliers of the SCCSD Lagrangian for target ("gradient", n) or
        ("coupling", m, n) at the converged state (dict with t, Ra, Rb, La, Lb
        packed vectors and zeta, r0a, r0b, omega_a, omega_b)."""
        dim = self.dim
        vecs, scal, kind, m, n = self._mult_args(state, target)
        zbar = np.empty(dim)
        K = np.empty((2, dim))
        sc = np.empty(5)
        D1 = np.empty((self.n, self.n)) if densities else None
        G = np.empty((self.J, self.n, self.n)) if densities else None
        it = ctypes.c_int()
        self._check(self.lib.sccsd_solve_multipliers(
            self.h, _ptr(vecs), _ptr(scal), kind, m, n, float(tol), int(maxit), float(refine_tol),
            _ptr(zbar), _ptr(K), _ptr(sc), _ptr(D1), _ptr(G), ctypes.addressof(it)))
        return {"zbar": zbar, "K": K, "gbar": sc[0], "lb0": sc[1:3], "Ebar": sc[3:5],
                "D1": D1, "Gamma": G, "iterations": it.value}

    def capture_transform(self, V, W, side="right"):
        """CUDA graph (handle) of W = A V (right) or A^T V (left), device tensors."""
        g = ctypes.c_void_p()
        nvec = 1 if V.ndim == 1 else V.shape[0]
        sd = {"right": 0, "left": 1}[side]
        self._check(self.lib.sccsd_capture_transform(self.h, sd, nvec, _ptr(V), _ptr(W),
                                                     ctypes.byref(g)))
        return g

    def profile(self, enable=True):
        self._check(self.lib.sccsd_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """(ladder_ms, ladder_calls, ladder_flops, kernel_launches) since the reset."""
        ms, fl = ctypes.c_double(), ctypes.c_double()
        calls, launches = ctypes.c_longlong(), ctypes.c_longlong()
        self._check(self.lib.sccsd_profile_read(self.h, ctypes.addressof(ms), ctypes.addressof(calls),
                                                ctypes.addressof(fl), ctypes.addressof(launches)))
        return ms.value, calls.value, fl.value, launches.value

    def densities(self, l0, L, r0, R, gamma=True):
        n = self.n
        D1 = np.empty((n, n))
        G = np.empty((self.J, n, n)) if gamma else None
        self._check(self.lib.sccsd_densities(self.h, float(l0), _ptr(L), float(r0), _ptr(R),
                                             _ptr(D1), _ptr(G)))
        return D1, G
