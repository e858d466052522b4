"""ctypes binding of ``libthcsox.so`` (argument marshalling only).

Every function here has the name of the C entry point it wraps and only turns
tensors into pointers and sizes; all arithmetic runs in the library's CUDA
kernels.  Tensors may be CUDA tensors or host (CPU / numpy) float64 arrays;
host buffers are staged by the library itself.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libthcsox.so")

SOX_OK, SOX_ERR_INVALID_ARG, SOX_ERR_SHAPE, SOX_ERR_UNSUPPORTED, SOX_ERR_OOM, SOX_ERR_CUDA, SOX_ERR_TIMEOUT = range(7)
PRECISIONS = {"fp64": 0, "f16x2": 1}
SOX_REAL64, SOX_COMPLEX128 = 0, 1

_ERRNAMES = {1: "SOX_ERR_INVALID_ARG", 2: "SOX_ERR_SHAPE", 3: "SOX_ERR_UNSUPPORTED", 4: "SOX_ERR_OOM",
             5: "SOX_ERR_CUDA", 6: "SOX_ERR_TIMEOUT"}


class SoxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class sox_problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("N", ctypes.c_int), ("n_tau", ctypes.c_int),
                ("n_spin", ctypes.c_int), ("nk", ctypes.c_int * 3), ("dtype", ctypes.c_int),
                ("beta", ctypes.c_double)]


class sox_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("device", ctypes.c_int), ("spin_limit", ctypes.c_longlong),
                ("workspace_limit", ctypes.c_longlong), ("no_autotune", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "sox_version": ([], _I),
    "sox_create": ([ctypes.POINTER(_P), ctypes.POINTER(sox_options)], _I),
    "sox_destroy": ([_P], _I),
    "sox_last_error": ([_P], ctypes.c_char_p),
    "sox_reserve": ([_P, ctypes.POINTER(sox_problem)], _I),
    "sox_check_device": ([_P], _I),
    "sox_set_v_range": ([_P, _I, _I], _I),
    "sox_set_kernel_variant": ([_P, _I], _I),
    "sox_profile_enable": ([_P, _I], _I),
    "sox_profile_read": ([_P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)], _I),
    "sox_tau_grid": ([_I, ctypes.c_double, _P, _P], _I),
    "thc_project_G": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P, _P], _I),
    "sox_sigma": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P], _I),
    "sox_sigma_general": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P, _P], _I),
    "sosex_static_sigma": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _I, _P, _P], _I),
    "sox_pi0": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P], _I),
    "sox_w_static": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P], _I),
    "phi_sox": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P, _P, _P], _I),
    "phi_sox_backward": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P, _P, _P, _P, _P], _I),
    "phi_sox_grad_G": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P], _I),
    "sosex_dynamic_sigma": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P, _P, _I, _P, _P], _I),
    "sox_w_dynamic": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _I, _P, _P], _I),
    "sox_sigma_batch": ([_P, _I, ctypes.POINTER(sox_problem), ctypes.POINTER(_P), ctypes.POINTER(_P),
                         ctypes.POINTER(_P), ctypes.POINTER(_P), _P], _I),
    "phi_sox_batch": ([_P, _I, ctypes.POINTER(sox_problem)] + [ctypes.POINTER(_P)] * 6 + [_P], _I),
    "sox_sigma_fp64_noalloc": ([ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P], _I),
    "g3w2_static_sigma": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P], _I),
    "sosex2_static_sigma": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P, _P], _I),
    "sox_sigma_batch_plan": ([_P, _I, ctypes.POINTER(sox_problem), ctypes.POINTER(_P), ctypes.POINTER(_P),
                              ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)], _I),
    "sox_plan_launch": ([_P, _P], _I),
    "sox_plan_check_device": ([_P], _I),
    "sox_plan_last_error": ([_P], ctypes.c_char_p),
    "sox_plan_destroy": ([_P], _I),
    "sox_dyson": ([_P, ctypes.POINTER(sox_problem), _I, _P, ctypes.c_double, _P, _P, _P, _P], _I),
    "sox_green_tails": ([_P, ctypes.POINTER(sox_problem), ctypes.c_double, _P, _P, _P, _P], _I),
    "sox_iw_to_tau": ([_P, ctypes.POINTER(sox_problem), _I, _P, _P, _P, _I, _P, _P, _P], _I),
    "sox_tau_to_iw": ([_P, ctypes.POINTER(sox_problem), _I, _P, _P, _P, _P], _I),
    "sox_find_mu": ([_P, ctypes.POINTER(sox_problem), _I, _P, ctypes.c_double, _P, _P, _P, ctypes.c_double,
                     ctypes.c_double, ctypes.c_double, _I, ctypes.POINTER(ctypes.c_double)], _I),
    "sox_density_matrix": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P], _I),
    "sox_sigma_hf": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P, _P, _P], _I),
    "sox_gm_energies": ([_P, ctypes.POINTER(sox_problem), _P, _P, _P, _P, _P, _P, _P, _P], _I),
    "sox_mix_green": ([_P, ctypes.c_longlong, ctypes.c_double, _P, _P, ctypes.POINTER(ctypes.c_double), _P], _I),
}
EXPORTED = tuple(_SIGS)

_lib = None


def lib() -> ctypes.CDLL:
    """Load libthcsox.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(handle, name)
            fn.argtypes = args
            fn.restype = res
        _lib = handle
    return _lib


def _ptr(t):
    """Raw pointer of a contiguous float64 or complex128 tensor/array (None -> NULL).

    complex128 data are passed as interleaved (re, im) doubles, the library's
    SOX_COMPLEX128 layout."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if t.dtype not in (np.float64, np.complex128) or not t.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays must be C-contiguous float64 or complex128")
        return t.ctypes.data
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"unsupported tensor type {type(t)}")
    if t.dtype not in (torch.float64, torch.complex128) or not t.is_contiguous():
        raise ValueError("tensors must be contiguous float64 or complex128")
    return t.data_ptr()


def _len(t) -> int:
    """Length of a 1-D array or tensor."""
    return int(t.shape[0])


def _stream(stream):
    if stream is None:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def problem(n, N, n_tau, n_spin=1, beta=100.0, nk=(1, 1, 1), dtype=SOX_REAL64) -> sox_problem:
    p = sox_problem()
    p.n, p.N, p.n_tau, p.n_spin = int(n), int(N), int(n_tau), int(n_spin)
    p.nk[0], p.nk[1], p.nk[2] = (int(x) for x in nk)
    p.dtype = int(dtype)
    p.beta = float(beta)
    return p


class Handle:
    """Owns a ``sox_handle`` (device workspace, precision choice)."""

    def __init__(self, precision: str = "fp64", device: int = 0, spin_limit: int = 0, workspace_limit: int = 0,
                 autotune: bool = True):
        o = sox_options(PRECISIONS[precision], int(device), int(spin_limit), int(workspace_limit),
                        0 if autotune else 1)
        h = _P()
        rc = lib().sox_create(ctypes.byref(h), ctypes.byref(o))
        if rc != SOX_OK:
            raise SoxError(rc, "sox_create failed")
        self._h = h
        self.precision = precision

    @property
    def ptr(self):
        if self._h is None:
            raise RuntimeError("handle closed")
        return self._h

    def check(self, rc: int):
        if rc != SOX_OK:
            raise SoxError(rc, lib().sox_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().sox_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def sox_version() -> int:
    return lib().sox_version()


def sox_tau_grid(n_tau: int, beta: float):
    tau = np.zeros(n_tau)
    w = np.zeros(n_tau)
    rc = lib().sox_tau_grid(int(n_tau), float(beta), tau.ctypes.data, w.ctypes.data)
    if rc != SOX_OK:
        raise SoxError(rc, "sox_tau_grid: bad arguments")
    return tau, w


def sox_check_device(h: Handle):
    h.check(lib().sox_check_device(h.ptr))


def sox_set_v_range(h: Handle, v0: int = 0, v1: int = 0):
    """Restrict the handle's later builds to the terms with v in [v0, v1) (0, 0: all)."""
    h.check(lib().sox_set_v_range(h.ptr, int(v0), int(v1)))


KERNEL_VARIANTS = {"auto": 0, "resident": 1, "streamed": 2, "pair": 3}


def sox_set_kernel_variant(h: Handle, variant: str = "auto"):
    """Force the split path's fused B/C/D kernel variant ("resident", "streamed", "pair")
    or return to timing them on the first call per shape ("auto")."""
    h.check(lib().sox_set_kernel_variant(h.ptr, KERNEL_VARIANTS[variant]))


def sox_profile_enable(h: Handle, enable: bool = True):
    h.check(lib().sox_profile_enable(h.ptr, int(bool(enable))))


def sox_profile_read(h: Handle, kernel: str | None = None):
    """(launches, ms) of a hot kernel, or (total kernel launches, 0.0) for kernel=None."""
    n = ctypes.c_longlong(0)
    ms = ctypes.c_double(0.0)
    h.check(lib().sox_profile_read(h.ptr, kernel.encode() if kernel else None, ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def sox_reserve(h: Handle, p: sox_problem):
    h.check(lib().sox_reserve(h.ptr, ctypes.byref(p)))


def thc_project_G(h: Handle, p: sox_problem, G, X, G_Rq=None, G_wP=None, G_PQ=None, stream=None):
    h.check(lib().thc_project_G(h.ptr, ctypes.byref(p), _ptr(G), _ptr(X), _ptr(G_Rq), _ptr(G_wP),
                                _ptr(G_PQ), _stream(stream)))


def sox_sigma(h: Handle, p: sox_problem, G, X, V, Sigma, stream=None):
    h.check(lib().sox_sigma(h.ptr, ctypes.byref(p), _ptr(G), _ptr(X), _ptr(V), _ptr(Sigma),
                            _stream(stream)))


def sox_sigma_general(h: Handle, p: sox_problem, G, X, U1, U2, Sigma, stream=None):
    h.check(lib().sox_sigma_general(h.ptr, ctypes.byref(p), _ptr(G), _ptr(X), _ptr(U1), _ptr(U2),
                                    _ptr(Sigma), _stream(stream)))


def sosex_static_sigma(h: Handle, p: sox_problem, G, X, V, W0, Sigma, slot: int = 1, stream=None):
    h.check(lib().sosex_static_sigma(h.ptr, ctypes.byref(p), _ptr(G), _ptr(X), _ptr(V), _ptr(W0),
                                     int(slot), _ptr(Sigma), _stream(stream)))


def g3w2_static_sigma(h: Handle, p: sox_problem, G, X, W0, Sigma, stream=None):
    h.check(lib().g3w2_static_sigma(h.ptr, ctypes.byref(p), _ptr(G), _ptr(X), _ptr(W0), _ptr(Sigma),
                                    _stream(stream)))


def sosex2_static_sigma(h: Handle, p: sox_problem, G, X, V, W0, Sigma, stream=None):
    h.check(lib().sosex2_static_sigma(h.ptr, ctypes.byref(p), _ptr(G), _ptr(X), _ptr(V), _ptr(W0), _ptr(Sigma),
                                      _stream(stream)))


def sox_pi0(h: Handle, p: sox_problem, G, X, w, Pi0, stream=None):
    h.check(lib().sox_pi0(h.ptr, ctypes.byref(p), _ptr(G), _ptr(X), _ptr(w), _ptr(Pi0), _stream(stream)))


def sox_w_static(h: Handle, p: sox_problem, V, Pi, W0, stream=None):
    h.check(lib().sox_w_static(h.ptr, ctypes.byref(p), _ptr(V), _ptr(Pi), _ptr(W0), _stream(stream)))


def phi_sox(h: Handle, p: sox_problem, G, X, V, w, phi, Sigma=None, stream=None):
    h.check(lib().phi_sox(h.ptr, ctypes.byref(p), _ptr(G), _ptr(X), _ptr(V), _ptr(w), _ptr(phi),
                          _ptr(Sigma), _stream(stream)))


def phi_sox_backward(h: Handle, p: sox_problem, G, X, V, w, dphi, dG=None, dX=None, dV=None,
                     stream=None):
    h.check(lib().phi_sox_backward(h.ptr, ctypes.byref(p), _ptr(G), _ptr(X), _ptr(V), _ptr(w),
                                   _ptr(dphi), _ptr(dG), _ptr(dX), _ptr(dV), _stream(stream)))


def phi_sox_grad_G(h: Handle, p: sox_problem, Sigma, w, dphi, dG, stream=None):
    h.check(lib().phi_sox_grad_G(h.ptr, ctypes.byref(p), _ptr(Sigma), _ptr(w), _ptr(dphi), _ptr(dG),
                                 _stream(stream)))


def sosex_dynamic_sigma(h: Handle, p: sox_problem, G, X, V, Wd, T_fwd, T_inv, n_omega, Sigma,
                        stream=None):
    h.check(lib().sosex_dynamic_sigma(h.ptr, ctypes.byref(p), _ptr(G), _ptr(X), _ptr(V), _ptr(Wd),
                                      _ptr(T_fwd), _ptr(T_inv), int(n_omega), _ptr(Sigma),
                                      _stream(stream)))


def sox_w_dynamic(h: Handle, p: sox_problem, G, X, V, T_fwd, n_omega, Wd, stream=None):
    h.check(lib().sox_w_dynamic(h.ptr, ctypes.byref(p), _ptr(G), _ptr(X), _ptr(V), _ptr(T_fwd), int(n_omega),
                                _ptr(Wd), _stream(stream)))


def sox_sigma_batch(h: Handle, probs, G, X, V, Sigma, stream=None):
    count = len(probs)
    arr = (sox_problem * count)(*probs)
    mk = lambda ts: (_P * count)(*[_ptr(t) for t in ts])  # noqa: E731
    h.check(lib().sox_sigma_batch(h.ptr, count, arr, mk(G), mk(X), mk(V), mk(Sigma), _stream(stream)))


def phi_sox_batch(h: Handle, probs, G, X, V, w, phi, Sigma, stream=None):
    """phi_sox for a batch of molecules: lists of per-instance tensors (w [n_tau], phi
    [n_spin], Sigma as for phi_sox); one persistent fused launch per tau chunk on a
    split-precision handle."""
    count = len(probs)
    arr = (sox_problem * count)(*probs)
    mk = lambda ts: (_P * count)(*[_ptr(t) for t in ts])  # noqa: E731
    h.check(lib().phi_sox_batch(h.ptr, count, arr, mk(G), mk(X), mk(V), mk(w), mk(phi), mk(Sigma), _stream(stream)))


class SigmaBatchPlan:
    """``sox_sigma_batch_plan``: the sox_sigma sequence of a batch of molecules recorded
    once into a CUDA graph.  The tensors (device memory) must outlive the plan; each
    ``launch`` recomputes every Sigma from the current G, X, V."""

    def __init__(self, h: Handle, probs, G, X, V, Sigma):
        count = len(probs)
        arr = (sox_problem * count)(*probs)
        mk = lambda ts: (_P * count)(*[_ptr(t) for t in ts])  # noqa: E731
        self._keep = (list(G), list(X), list(V), list(Sigma))
        p = _P()
        h.check(lib().sox_sigma_batch_plan(h.ptr, count, arr, mk(G), mk(X), mk(V), mk(Sigma), ctypes.byref(p)))
        self._p = p

    def _check(self, rc, what):
        if rc != SOX_OK:
            msg = lib().sox_plan_last_error(self._p)
            raise SoxError(rc, f"{what}: " + (msg.decode() if msg else ""))

    def launch(self, stream=None):
        self._check(lib().sox_plan_launch(self._p, _stream(stream)), "sox_plan_launch")

    def check_device(self):
        self._check(lib().sox_plan_check_device(self._p), "sox_plan_check_device")

    def close(self):
        if self._p:
            lib().sox_plan_destroy(self._p)
            self._p = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sox_sigma_fp64_noalloc(p: sox_problem, G, X, V, Sigma, stream=None):
    """Bare SOX on the FP64 path with the library's fixed scratch array (no handle,
    no device allocation).  Device tensors only; raises SoxError on failure."""
    rc = lib().sox_sigma_fp64_noalloc(ctypes.byref(p), _ptr(G), _ptr(X), _ptr(V), _ptr(Sigma), _stream(stream))
    if rc != SOX_OK:
        raise SoxError(rc, "sox_sigma_fp64_noalloc failed (see include/thc_sox.h for the status meanings)")


# ---------------------------------------------------------------------------
# The self-consistent loop's device steps (Sec. II A); argument marshalling only.
# ---------------------------------------------------------------------------
def sox_dyson(h: Handle, p: sox_problem, omegas, mu: float, F, Sigma_iw, G_iw, stream=None):
    h.check(lib().sox_dyson(h.ptr, ctypes.byref(p), _len(omegas), _ptr(omegas), float(mu), _ptr(F), _ptr(Sigma_iw),
                            _ptr(G_iw), _stream(stream)))


def sox_green_tails(h: Handle, p: sox_problem, mu: float, F, Sigma_tau, tails, stream=None):
    h.check(lib().sox_green_tails(h.ptr, ctypes.byref(p), float(mu), _ptr(F), _ptr(Sigma_tau), _ptr(tails),
                                  _stream(stream)))


def sox_iw_to_tau(h: Handle, p: sox_problem, omegas, G_iw, tails, tau, G_tau, stream=None):
    h.check(lib().sox_iw_to_tau(h.ptr, ctypes.byref(p), _len(omegas), _ptr(omegas), _ptr(G_iw), _ptr(tails),
                                _len(tau), _ptr(tau), _ptr(G_tau), _stream(stream)))


def sox_tau_to_iw(h: Handle, p: sox_problem, T_w, F_tau, F_iw, stream=None):
    n_w = int(T_w.shape[0])
    h.check(lib().sox_tau_to_iw(h.ptr, ctypes.byref(p), n_w, _ptr(T_w), _ptr(F_tau), _ptr(F_iw), _stream(stream)))


def sox_find_mu(h: Handle, p: sox_problem, omegas, target: float, F, Sigma_iw=None, Sigma_tau=None,
                lo: float = -50.0, hi: float = 50.0, tol: float = 1e-13, max_iter: int = 200) -> float:
    mu = ctypes.c_double(0.0)
    h.check(lib().sox_find_mu(h.ptr, ctypes.byref(p), _len(omegas), _ptr(omegas), float(target), _ptr(F),
                              _ptr(Sigma_iw), _ptr(Sigma_tau), float(lo), float(hi), float(tol), int(max_iter),
                              ctypes.byref(mu)))
    return mu.value


def sox_density_matrix(h: Handle, p: sox_problem, G_tau, gamma, stream=None):
    h.check(lib().sox_density_matrix(h.ptr, ctypes.byref(p), _ptr(G_tau), _ptr(gamma), _stream(stream)))


def sox_sigma_hf(h: Handle, p: sox_problem, X, V, gamma, Sigma_hf, H0=None, F=None, stream=None):
    h.check(lib().sox_sigma_hf(h.ptr, ctypes.byref(p), _ptr(X), _ptr(V), _ptr(gamma), _ptr(H0), _ptr(Sigma_hf),
                               _ptr(F), _stream(stream)))


def sox_gm_energies(h: Handle, p: sox_problem, H0, Sigma_hf, gamma, Sigma_tau, G_tau, w, E, stream=None):
    h.check(lib().sox_gm_energies(h.ptr, ctypes.byref(p), _ptr(H0), _ptr(Sigma_hf), _ptr(gamma), _ptr(Sigma_tau),
                                  _ptr(G_tau), _ptr(w), _ptr(E), _stream(stream)))


def sox_mix_green(h: Handle, G, G_new, a: float, stream=None) -> float:
    change = ctypes.c_double(0.0)
    h.check(lib().sox_mix_green(h.ptr, int(G.numel()), float(a), _ptr(G), _ptr(G_new), ctypes.byref(change),
                                _stream(stream)))
    return change.value

