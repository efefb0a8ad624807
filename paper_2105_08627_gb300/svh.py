"""Thin ctypes binding of the C ABI in ``include/svh.h`` (argument marshalling only).

Every computation runs in ``lib/libsvh.so``; this module converts NumPy arrays
and torch tensors to pointers and raises :class:`SVHError` on a non-zero
status. Importing it does not need a GPU; creating a :class:`Handle` does.
If the library has not been built, :func:`lib` raises instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libsvh.so")

SVH_OK = 0
SVH_ERR_ARG = 1
SVH_ERR_CUDA = 2
SVH_ERR_OOM = 3
SVH_ERR_NOT_CONVERGED = 4
SVH_ERR_TIMEOUT = 5
SVH_ERR_SINGULAR = 6
SVH_ERR_STATE = 7
SVH_FP32 = 0
SVH_FP64 = 1
SVH_KERNELS_RESIDENT = 0
SVH_KERNELS_TUCKER_REBUILD = 1
KERNELS = ("G00", "Sx", "Sy", "Sz", "Qx", "Qy", "Qz")


class SVHError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"svh error {code}: {msg}")
        self.code = code


class svh_port(C.Structure):
    _fields_ = [("n_plus", C.c_int32), ("plus", C.POINTER(C.c_int32)),
                ("n_minus", C.c_int32), ("minus", C.POINTER(C.c_int32))]


class svh_options(C.Structure):
    _fields_ = [("restart", C.c_int32), ("max_iterations", C.c_int32), ("max_refinements", C.c_int32),
                ("inner_precision", C.c_int32), ("rre", C.c_double), ("amg_tol", C.c_double),
                ("amg_on_device", C.c_int32)]


class svh_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("refinements", C.c_int32), ("amg_levels", C.c_int32),
                ("amg_avg_iterations", C.c_double), ("final_rre", C.c_double), ("setup_seconds", C.c_double),
                ("solve_seconds", C.c_double)]


class svh_grid_info(C.Structure):
    _fields_ = [("Kx", C.c_int32), ("Ky", C.c_int32), ("Kz", C.c_int32),
                ("Px", C.c_int32), ("Py", C.c_int32), ("Pz", C.c_int32),
                ("Hx", C.c_int32), ("Hy", C.c_int32), ("Hz", C.c_int32),
                ("K", C.c_int64), ("M", C.c_int64), ("N", C.c_int64),
                ("nports", C.c_int32), ("n_fixed_nodes", C.c_int32),
                ("n_active_planes", C.c_int32), ("n_active_rows", C.c_int32),
                ("dx", C.c_double)]


_P = C.c_void_p
_DP = C.POINTER(C.c_double)
_FP = C.POINTER(C.c_float)
_I32P = C.POINTER(C.c_int32)
_I64P = C.POINTER(C.c_int64)
_U8P = C.POINTER(C.c_uint8)

# name -> (restype, argtypes); every symbol declared in include/svh.h
SIGNATURES = {
    "svh_create": (C.c_int, [C.POINTER(_P), C.c_int, _P]),
    "svh_destroy": (C.c_int, [_P]),
    "svh_last_error": (C.c_char_p, [_P]),
    "svh_set_stream": (C.c_int, [_P, _P]),
    "svh_setup_grid": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, _U8P, _DP, _DP,
                                 C.POINTER(svh_port), C.c_int]),
    "svh_set_fft_sizes": (C.c_int, [_P, C.c_int, C.c_int, C.c_int]),
    "svh_get_grid_info": (C.c_int, [_P, C.POINTER(svh_grid_info)]),
    "svh_get_nodes": (C.c_int, [_P, _I32P]),
    "svh_generate_toeplitz": (C.c_int, [_P]),
    "svh_load_toeplitz": (C.c_int, [_P, _DP]),
    "svh_get_toeplitz": (C.c_int, [_P, _DP]),
    "svh_get_spectra": (C.c_int, [_P, _DP]),
    "svh_get_spectra32": (C.c_int, [_P, _FP]),
    "svh_load_tucker": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _DP, _DP, _DP, _DP]),
    "svh_tucker_compress": (C.c_int, [_P, C.c_double, _I32P]),
    "svh_tucker_compress_on": (C.c_int, [_P, C.c_double, _I32P, C.c_int]),
    "svh_get_tucker": (C.c_int, [_P, C.c_int, _I32P, _DP, _DP, _DP, _DP]),
    "svh_set_kernel_mode": (C.c_int, [_P, C.c_int]),
    "svh_rebuild_spectra": (C.c_int, [_P]),
    "svh_matvec": (C.c_int, [_P, C.c_double, C.c_int, _P, _P, C.c_int]),
    "svh_matvec_host": (C.c_int, [_P, C.c_double, C.c_int, _P, _P, C.c_int]),
    "svh_matvec_omegas": (C.c_int, [_P, _DP, C.c_int, _P, _P, C.c_int]),
    "svh_default_options": (None, [C.POINTER(svh_options)]),
    "svh_solve": (C.c_int, [_P, _DP, C.c_int, C.POINTER(svh_options), _DP, _DP, C.POINTER(svh_stats)]),
    "svh_get_solution": (C.c_int, [_P, C.c_int, _DP]),
    "svh_precond_apply": (C.c_int, [_P, C.c_double, C.c_int, _DP, _DP]),
    "svh_set_materials": (C.c_int, [_P, _DP, _DP]),
    "svh_get_materials": (C.c_int, [_P, _DP, _DP]),
    "svh_grad_inductance": (C.c_int, [_P, C.c_int, C.c_int, _DP, _DP]),
    "svh_matvec_noalloc": (C.c_int, [_P, C.c_double, C.c_int, _P, _P, C.c_int]),
    "svh_batch_create": (C.c_int, [C.POINTER(_P), C.c_int]),
    "svh_batch_destroy": (C.c_int, [_P]),
    "svh_batch_last_error": (C.c_char_p, [_P]),
    "svh_batch_add": (C.c_int, [_P, _P]),
    "svh_batch_size": (C.c_int, [_P]),
    "svh_batch_matvec": (C.c_int, [_P, _I32P, C.POINTER(_DP), C.POINTER(_P), C.POINTER(_P), C.c_int]),
    "svh_batch_sync": (C.c_int, [_P]),
    "svh_batch_set_wait": (C.c_int, [_P, C.c_double, C.c_int, C.c_int]),
    "svh_batch_set_mode": (C.c_int, [_P, C.c_int]),
    "svh_batch_get_mode": (C.c_int, [_P]),
    "svh_batch_autotune": (C.c_int, [_P, _I32P, C.POINTER(_DP), C.POINTER(_P), C.POINTER(_P), C.c_int, _DP]),
    "svh_batch_stream": (_P, [_P]),
    "svh_batch_solve": (C.c_int, [_P, _DP, C.c_int, C.POINTER(svh_options), C.POINTER(_DP), C.POINTER(_DP),
                                  C.c_int, C.POINTER(svh_stats)]),
    "svh_profile_begin": (C.c_int, [_P, C.c_int]),
    "svh_autotune": (C.c_int, [_P, C.c_int, _I32P, _DP]),
    "svh_get_device_status": (C.c_int, [_P, _I32P, C.c_int]),
    "svh_set_pass_variant": (C.c_int, [_P, C.c_int, C.c_int]),
    "svh_get_pass_variants": (C.c_int, [_P, _I32P, _I32P]),
    "svh_profile_end": (C.c_int, [_P, _DP, _I32P]),
    "svh_host_face_nodes": (C.c_int, [C.c_int, C.c_int, C.c_int, _U8P, _I64P, _I64P, _I32P]),
    "svh_host_spectra": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _DP, _DP]),
    "svh_host_amg_solve": (C.c_int, [C.c_int, _I32P, _I32P, _DP, _DP, _DP, C.c_double, C.c_int, _I32P, _I32P]),
    "svh_device_amg_solve": (C.c_int, [C.c_int, _I32P, _I32P, _DP, _DP, _DP, C.c_int, C.c_double, C.c_int, _I32P,
                                        _I32P]),
    "svh_toeplitz_store_write": (C.c_int, [C.c_char_p, C.c_int, C.c_int, C.c_int, _DP, C.c_double]),
    "svh_toeplitz_store_read": (C.c_int, [C.c_char_p, C.c_int, C.c_int, C.c_int, _DP, _I32P]),
    "svh_load_toeplitz_store": (C.c_int, [_P, C.c_char_p]),
    "svh_host_tucker_svd": (C.c_int, [_DP, C.c_int, C.c_int, C.c_int, C.c_double, _I32P, _DP, _DP, _DP, _DP]),
}

_lib = None


def lib():
    """Load lib/libsvh.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not found: build it with "
                               "`python -m paper_2105_08627_gb300.build` (no fallback exists)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_DP)


def _fp(a):
    return a.ctypes.data_as(_FP)


def _i32p(a):
    return a.ctypes.data_as(_I32P)


def _check_host(rc, what):
    if rc != SVH_OK:
        raise SVHError(rc, what)


# ---------------------------------------------------------------- host utilities
def host_face_nodes(occ):
    occ = np.ascontiguousarray(occ, np.uint8)
    Kz, Ky, Kx = occ.shape
    K = C.c_int64()
    M = C.c_int64()
    _check_host(lib().svh_host_face_nodes(Kx, Ky, Kz, occ.ctypes.data_as(_U8P), C.byref(K), C.byref(M), None),
                "svh_host_face_nodes")
    node = np.empty(K.value * 6, np.int32)
    _check_host(lib().svh_host_face_nodes(Kx, Ky, Kz, occ.ctypes.data_as(_U8P), C.byref(K), C.byref(M),
                                          _i32p(node)), "svh_host_face_nodes")
    return node.reshape(K.value, 6), M.value


def host_spectra(T, P):
    T = np.ascontiguousarray(T, np.float64)
    _, Kz, Ky, Kx = T.shape
    Px, Py, Pz = P
    S = np.empty((7, Pz // 2 + 1, Py // 2 + 1, Px // 2 + 1))
    _check_host(lib().svh_host_spectra(Kx, Ky, Kz, Px, Py, Pz, _dp(T), _dp(S)), "svh_host_spectra")
    return S


def host_amg_solve(S, b, tol=1e-8, maxit=500):
    """x = S^-1 b by the library's AMG-preconditioned CG (S: scipy CSR, SPD) -> (x, iters, levels)."""
    S = S.tocsr()
    rp = np.ascontiguousarray(S.indptr, np.int32)
    ci = np.ascontiguousarray(S.indices, np.int32)
    v = np.ascontiguousarray(S.data, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros_like(b)
    it = C.c_int32()
    lv = C.c_int32()
    _check_host(lib().svh_host_amg_solve(S.shape[0], _i32p(rp), _i32p(ci), _dp(v), _dp(b), _dp(x), tol, maxit,
                                         C.byref(it), C.byref(lv)), "svh_host_amg_solve")
    return x, it.value, lv.value


def device_amg_solve(S, b, tol=1e-8, maxit=500):
    """x = S^-1 b by the device AMG-CG (S: scipy CSR, SPD; b: complex [nrhs, n] or [n];
    real and imaginary parts are separate systems) -> (x, mean iterations, levels)."""
    S = S.tocsr()
    rp = np.ascontiguousarray(S.indptr, np.int32)
    ci = np.ascontiguousarray(S.indices, np.int32)
    v = np.ascontiguousarray(S.data, np.float64)
    b = np.asarray(b, np.complex128)
    shape = b.shape
    b2 = np.ascontiguousarray(b.reshape(-1, S.shape[0]))
    x = np.zeros_like(b2)
    it = C.c_int32()
    lv = C.c_int32()
    _check_host(lib().svh_device_amg_solve(S.shape[0], _i32p(rp), _i32p(ci), _dp(v), _dp(b2.view(np.float64)),
                                           _dp(x.view(np.float64)), b2.shape[0], tol, maxit, C.byref(it),
                                           C.byref(lv)), "svh_device_amg_solve")
    return x.reshape(shape), it.value, lv.value


def toeplitz_store_write(path, K, tol, T=None):
    """Algorithm 2, install stage: store the Tucker data of the unit Toeplitz tensors of a
    K = (Kx, Ky, Kz) domain (T[7, Kz, Ky, Kx] given, or None: computed on the current device)."""
    Kx, Ky, Kz = (int(v) for v in K)
    Tp = None
    if T is not None:
        T = np.ascontiguousarray(T, np.float64)
        if T.shape != (7, Kz, Ky, Kx):
            raise ValueError("T must have shape (7, Kz, Ky, Kx)")
        Tp = _dp(T)
    _check_host(lib().svh_toeplitz_store_write(os.fsencode(path), Kx, Ky, Kz, Tp, tol), "svh_toeplitz_store_write")


def toeplitz_store_read(path, K):
    """Algorithm 2, set-up stage: the leading K block of the stored tensors -> (T[7, Kz, Ky, Kx], ranks[7, 3])."""
    Kx, Ky, Kz = (int(v) for v in K)
    T = np.empty((7, Kz, Ky, Kx))
    r = np.zeros(21, np.int32)
    _check_host(lib().svh_toeplitz_store_read(os.fsencode(path), Kx, Ky, Kz, _dp(T), _i32p(r)),
                "svh_toeplitz_store_read")
    return T, r.reshape(7, 3)


def host_tucker_svd(O, tol):
    """Algorithm 1 on O[D3, D2, D1] (mode 1 = last axis) -> (core[d3,d2,d1], [F1, F2, F3])."""
    O = np.ascontiguousarray(O, np.float64)
    D3, D2, D1 = O.shape
    d = np.zeros(3, np.int32)
    core = np.empty(O.size)
    F = [np.empty(D * D) for D in (D1, D2, D3)]
    _check_host(lib().svh_host_tucker_svd(_dp(O), D1, D2, D3, tol, _i32p(d), _dp(core), _dp(F[0]), _dp(F[1]),
                                          _dp(F[2])), "svh_host_tucker_svd")
    d1, d2, d3 = (int(v) for v in d)
    return (core[:d1 * d2 * d3].reshape(d3, d2, d1).copy(),
            [F[0][:D1 * d1].reshape(D1, d1).copy(), F[1][:D2 * d2].reshape(D2, d2).copy(),
             F[2][:D3 * d3].reshape(D3, d3).copy()])


# ---------------------------------------------------------------- handle
class Handle:
    """One library handle bound to a CUDA device and stream."""

    def __init__(self, device=0, stream=None):
        self._h = _P()
        self.device = int(device)
        rc = lib().svh_create(C.byref(self._h), int(device), _P(stream or 0))
        if rc != SVH_OK:
            raise SVHError(rc, "svh_create failed (no CUDA device?)")

    def _ck(self, rc, what=""):
        if rc != SVH_OK:
            msg = lib().svh_last_error(self._h)
            raise SVHError(rc, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if self._h:
            lib().svh_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._ck(lib().svh_set_stream(self._h, _P(stream or 0)), "svh_set_stream")

    # -------------------------------------------------------- grid
    def setup_grid(self, Kx, Ky, Kz, dx, occ, lam, sigma0, ports=()):
        occ = np.ascontiguousarray(occ, np.uint8).ravel()
        lam = np.ascontiguousarray(lam, np.float64).ravel()
        sigma0 = np.ascontiguousarray(sigma0, np.float64).ravel()
        keep = []
        arr = (svh_port * max(1, len(ports)))()
        for i, p in enumerate(ports):
            plus = np.ascontiguousarray(p.plus if hasattr(p, "plus") else p[0], np.int32)
            minus = np.ascontiguousarray(p.minus if hasattr(p, "minus") else p[1], np.int32)
            keep += [plus, minus]
            arr[i] = svh_port(plus.size, _i32p(plus), minus.size, _i32p(minus))
        self._ck(lib().svh_setup_grid(self._h, Kx, Ky, Kz, dx, occ.ctypes.data_as(_U8P), _dp(lam), _dp(sigma0),
                                      arr, len(ports)), "svh_setup_grid")

    def setup_structure(self, s):
        """Set up from an object with Kx, Ky, Kz, dx, occ, lam, sigma0, ports (e.g. svh_synth.Structure)."""
        self.setup_grid(s.Kx, s.Ky, s.Kz, s.dx, s.occ, s.lam, s.sigma0, s.ports)

    def set_fft_sizes(self, Px, Py, Pz):
        self._ck(lib().svh_set_fft_sizes(self._h, Px, Py, Pz), "svh_set_fft_sizes")

    def info(self):
        gi = svh_grid_info()
        self._ck(lib().svh_get_grid_info(self._h, C.byref(gi)), "svh_get_grid_info")
        return {f: getattr(gi, f) for f, _ in svh_grid_info._fields_}

    def nodes(self):
        K = self.info()["K"]
        out = np.empty(K * 6, np.int32)
        self._ck(lib().svh_get_nodes(self._h, _i32p(out)), "svh_get_nodes")
        return out.reshape(K, 6)

    # -------------------------------------------------------- kernels
    def load_toeplitz_store(self, path):
        """Kernels from an Algorithm 2 store (cropped to this grid)."""
        self._ck(lib().svh_load_toeplitz_store(self._h, os.fsencode(path)), "svh_load_toeplitz_store")

    def generate_toeplitz(self):
        self._ck(lib().svh_generate_toeplitz(self._h), "svh_generate_toeplitz")

    def load_toeplitz(self, T):
        i = self.info()
        T = np.ascontiguousarray(T, np.float64)
        if T.shape != (7, i["Kz"], i["Ky"], i["Kx"]):
            raise ValueError(f"Toeplitz kernels must have shape (7, Kz, Ky, Kx), got {T.shape}")
        self._ck(lib().svh_load_toeplitz(self._h, _dp(T)), "svh_load_toeplitz")

    def toeplitz(self):
        i = self.info()
        T = np.empty((7, i["Kz"], i["Ky"], i["Kx"]))
        self._ck(lib().svh_get_toeplitz(self._h, _dp(T)), "svh_get_toeplitz")
        return T

    def spectra(self):
        i = self.info()
        S = np.empty((7, i["Hz"], i["Hy"], i["Hx"]))
        self._ck(lib().svh_get_spectra(self._h, _dp(S)), "svh_get_spectra")
        return S

    def spectra32(self):
        """The FP32 octant spectra on the device (what FP32 products read)."""
        i = self.info()
        S = np.empty((7, i["Hz"], i["Hy"], i["Hx"]), np.float32)
        self._ck(lib().svh_get_spectra32(self._h, _fp(S)), "svh_get_spectra32")
        return S

    def load_tucker(self, u, core, Fs):
        core = np.ascontiguousarray(core, np.float64)
        d3, d2, d1 = core.shape
        F1, F2, F3 = (np.ascontiguousarray(f, np.float64) for f in Fs)
        self._ck(lib().svh_load_tucker(self._h, u, d1, d2, d3, _dp(core), _dp(F1), _dp(F2), _dp(F3)),
                 "svh_load_tucker")

    def tucker_compress(self, tol, device=True):
        """Algorithm 1 on the current spectra (device by default, host cores with device=False)."""
        r = np.zeros(21, np.int32)
        self._ck(lib().svh_tucker_compress_on(self._h, tol, _i32p(r), int(bool(device))), "svh_tucker_compress")
        return r.reshape(7, 3)

    def get_tucker(self, u):
        i = self.info()
        d = np.zeros(3, np.int32)
        self._ck(lib().svh_get_tucker(self._h, u, _i32p(d), None, None, None, None), "svh_get_tucker")
        d1, d2, d3 = (int(v) for v in d)
        core = np.empty((d3, d2, d1))
        F1, F2, F3 = np.empty((i["Hx"], d1)), np.empty((i["Hy"], d2)), np.empty((i["Hz"], d3))
        self._ck(lib().svh_get_tucker(self._h, u, _i32p(d), _dp(core), _dp(F1), _dp(F2), _dp(F3)),
                 "svh_get_tucker")
        return core, [F1, F2, F3]

    def set_kernel_mode(self, mode):
        self._ck(lib().svh_set_kernel_mode(self._h, mode), "svh_set_kernel_mode")

    def rebuild_spectra(self):
        self._ck(lib().svh_rebuild_spectra(self._h), "svh_rebuild_spectra")

    # -------------------------------------------------------- operator
    def matvec_ptr(self, omega, nb, x_ptr, y_ptr, precision):
        self._ck(lib().svh_matvec(self._h, float(omega), int(nb), _P(x_ptr), _P(y_ptr), int(precision)),
                 "svh_matvec")

    def matvec(self, omega, x, y=None):
        """y = Kop x for torch tensors on the handle's device (complex64 -> FP32, complex128 -> FP64).

        x has shape (N,) or (nb, N); y (allocated when None) has the same shape."""
        import torch
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous CUDA tensor")
        prec = {torch.complex64: SVH_FP32, torch.complex128: SVH_FP64}.get(x.dtype)
        if prec is None:
            raise ValueError("x must be complex64 or complex128")
        N = self.info()["N"]
        nb = 1 if x.dim() == 1 else x.shape[0]
        if x.numel() != nb * N:
            raise ValueError(f"x must hold nb*N = {nb}*{N} values")
        if y is None:
            y = torch.empty_like(x)
        self.matvec_ptr(omega, nb, x.data_ptr(), y.data_ptr(), prec)
        return y

    def matvec_noalloc_ptr(self, omega, nb, x_ptr, y_ptr, precision):
        """svh_matvec_noalloc: the product on the library's fixed 64 MiB device scratch (no allocation)."""
        self._ck(lib().svh_matvec_noalloc(self._h, float(omega), int(nb), _P(x_ptr), _P(y_ptr), int(precision)),
                 "svh_matvec_noalloc")

    def solve(self, freqs, **opts):
        """Port impedances at the given frequencies (Hz) -> dict(Z[f,p,q], L = Im Z / omega, R, stats).

        opts override svh_options fields (restart, max_iterations, max_refinements,
        inner_precision, rre, amg_tol, amg_on_device). Raises SVHError on failure; a solve that
        stops above rre raises with code SVH_ERR_NOT_CONVERGED unless
        allow_unconverged=True."""
        allow = opts.pop("allow_unconverged", False)
        o = svh_options()
        lib().svh_default_options(C.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        freqs = np.atleast_1d(np.asarray(freqs, np.float64))
        om = np.ascontiguousarray(2 * np.pi * freqs)
        npt = self.info()["nports"]
        Z = np.zeros((freqs.size, npt, npt, 2))
        L = np.zeros((freqs.size, npt, npt))
        st = svh_stats()
        rc = lib().svh_solve(self._h, _dp(om), om.size, C.byref(o), _dp(Z), _dp(L), C.byref(st))
        if rc != SVH_OK and not (allow and rc == SVH_ERR_NOT_CONVERGED):
            self._ck(rc, "svh_solve")
        Zc = Z[..., 0] + 1j * Z[..., 1]
        stats = {f: getattr(st, f) for f, _ in svh_stats._fields_}
        stats["status"] = rc
        return {"Z": Zc, "L": L, "R": Z[..., 0].copy(), "stats": stats}

    def set_materials(self, lam_vox, sigma0_vox):
        lam = np.ascontiguousarray(lam_vox, np.float64)
        sig = np.ascontiguousarray(sigma0_vox, np.float64)
        self._ck(lib().svh_set_materials(self._h, _dp(lam), _dp(sig)), "svh_set_materials")

    def materials(self):
        K = self.info()["K"]
        lam, sig = np.empty(K), np.empty(K)
        self._ck(lib().svh_get_materials(self._h, _dp(lam), _dp(sig)), "svh_get_materials")
        return lam, sig

    def grad_inductance(self, i, j):
        """(dL_ij/dlambda[K], dL_ij/dsigma0[K]) at the last solved frequency (adjoint)."""
        K = self.info()["K"]
        gl, gs = np.empty(K), np.empty(K)
        self._ck(lib().svh_grad_inductance(self._h, i, j, _dp(gl), _dp(gs)), "svh_grad_inductance")
        return gl, gs

    def solution(self, port):
        N = self.info()["N"]
        x = np.empty(2 * N)
        self._ck(lib().svh_get_solution(self._h, port, _dp(x)), "svh_get_solution")
        return x[0::2] + 1j * x[1::2]

    def precond_apply(self, omega, v):
        v = np.ascontiguousarray(np.atleast_2d(v), np.complex128)
        out = np.empty_like(v)
        self._ck(lib().svh_precond_apply(self._h, float(omega), v.shape[0], v.ctypes.data_as(_DP),
                                         out.ctypes.data_as(_DP)), "svh_precond_apply")
        return out

    PASSES = ("tucker_rebuild", "x_fwd", "y_fwd", "z_pass", "y_inv", "x_inv_epilogue", "node_rows")

    FFT_PASSES = ("x_fwd", "y_fwd", "z_pass", "y_inv", "x_inv_epilogue", "path", "streams")

    def autotune(self, nb, timings=True):
        """Time every FP32 tile variant of the five FFT passes for nb items, then the
        fused y/z/y path against the separate passes, then the stream schedules, and
        keep the fastest -> (variants[7], ms per launch[7]); variants[5]: 0 separate passes,
        1 fused; variants[6]: 0 restore + node rows overlapped, 1 node rows only, 2 one stream,
        3 node rows beside the x forward pass only.
        timings=False asks for no timings (ms is None), so that an equal grid tuned earlier in
        the process is taken from the cache without timing anything."""
        v = np.zeros(7, np.int32)
        ms = np.zeros(7) if timings else None
        self._ck(lib().svh_autotune(self._h, int(nb), _i32p(v), _dp(ms) if timings else None), "svh_autotune")
        return v, ms

    def device_status(self, clear=True):
        """Status word set by kernels whose bounded waits expired (0: none)."""
        st = C.c_int32()
        self._ck(lib().svh_get_device_status(self._h, C.byref(st), int(clear)), "svh_get_device_status")
        return st.value

    def set_pass_variant(self, p, v):
        self._ck(lib().svh_set_pass_variant(self._h, int(p), int(v)), "svh_set_pass_variant")

    def pass_variants(self):
        """-> (number of variants per FFT pass (0: generic kernel), current choice);
        entry 5 is the path (2 choices when the fused y/z/y kernel applies), entry 6 the
        stream schedule (4 choices)."""
        n = np.zeros(7, np.int32)
        c = np.zeros(7, np.int32)
        self._ck(lib().svh_get_pass_variants(self._h, _i32p(n), _i32p(c)), "svh_get_pass_variants")
        return n, c

    def profile_begin(self, max_calls):
        self._ck(lib().svh_profile_begin(self._h, int(max_calls)), "svh_profile_begin")

    def profile_end(self):
        """-> (dict pass -> summed ms, number of calls recorded)."""
        ms = np.zeros(len(self.PASSES))
        n = C.c_int32()
        self._ck(lib().svh_profile_end(self._h, _dp(ms), C.byref(n)), "svh_profile_end")
        return dict(zip(self.PASSES, ms.tolist())), n.value

    def matvec_omegas(self, omegas, x, y=None):
        """Batched product with one angular frequency per item (x: (nb, N) CUDA tensor)."""
        import torch
        prec = {torch.complex64: SVH_FP32, torch.complex128: SVH_FP64}[x.dtype]
        om = np.ascontiguousarray(omegas, np.float64)
        if y is None:
            y = torch.empty_like(x)
        self._ck(lib().svh_matvec_omegas(self._h, _dp(om), om.size, _P(x.data_ptr()), _P(y.data_ptr()), prec),
                 "svh_matvec_omegas")
        return y

    def matvec_host(self, omega, x):
        """Host-memory product (copies in, applies, copies out); x complex64 or complex128 NumPy."""
        x = np.ascontiguousarray(x)
        prec = {np.complex64: SVH_FP32, np.complex128: SVH_FP64}.get(x.dtype.type)
        if prec is None:
            raise ValueError("x must be complex64 or complex128")
        N = self.info()["N"]
        nb = x.size // N
        y = np.empty_like(x)
        self._ck(lib().svh_matvec_host(self._h, float(omega), nb, x.ctypes.data_as(_P), y.ctypes.data_as(_P), prec),
                 "svh_matvec_host")
        return y


class Batch:
    """Several structures (handles) applied or solved together (see svh_batch_* in include/svh.h)."""

    def __init__(self, device=0):
        self._b = _P()
        rc = lib().svh_batch_create(C.byref(self._b), int(device))
        if rc != SVH_OK:
            raise SVHError(rc, "svh_batch_create failed")
        self.handles = []

    def _ck(self, rc, what):
        if rc != SVH_OK:
            msg = lib().svh_batch_last_error(self._b)
            raise SVHError(rc, f"{what}: {msg.decode() if msg else ''}")

    def add(self, handle):
        self._ck(lib().svh_batch_add(self._b, handle._h), "svh_batch_add")
        self.handles.append(handle)

    def _args(self, omegas, xs, ys):
        nbs = np.array([1 if x.dim() == 1 else x.shape[0] for x in xs], np.int32)
        oms = [np.ascontiguousarray(np.broadcast_to(np.asarray(o, np.float64), (int(n),)))
               for o, n in zip(omegas, nbs)]
        self._keep = (nbs, oms)
        op = (_DP * len(oms))(*[_dp(o) for o in oms])
        xp = (_P * len(xs))(*[x.data_ptr() for x in xs])
        yp = (_P * len(ys))(*[y.data_ptr() for y in ys])
        return nbs, op, xp, yp

    def matvec(self, omegas, xs, ys, precision=SVH_FP32):
        """Every structure's product in one graph launch (mode 0: the persistent queue; mode 1:
        the structures' own launch sequences): xs[i], ys[i] are contiguous CUDA tensors of shape
        (nb_i, N_i) (or (N_i,)); omegas[i] holds nb_i angular frequencies (or one for all)."""
        nbs, op, xp, yp = self._args(omegas, xs, ys)
        self._ck(lib().svh_batch_matvec(self._b, _i32p(nbs), op, xp, yp, precision), "svh_batch_matvec")

    def set_mode(self, mode):
        self._ck(lib().svh_batch_set_mode(self._b, int(mode)), "svh_batch_set_mode")

    @property
    def mode(self):
        return lib().svh_batch_get_mode(self._b)

    def autotune(self, omegas, xs, ys, precision=SVH_FP32):
        """Times both modes on these arguments, keeps the faster -> ms per launch [mode 0, mode 1]."""
        nbs, op, xp, yp = self._args(omegas, xs, ys)
        ms = np.zeros(2)
        self._ck(lib().svh_batch_autotune(self._b, _i32p(nbs), op, xp, yp, precision, _dp(ms)),
                 "svh_batch_autotune")
        return ms

    def set_wait(self, limit_ms, hold_item=-1, hold_phase=-1):
        """Bound of each wait of the batch queue; (hold_item, hold_phase) names a pass whose
        completion is never counted (diagnostics: the launch then ends with SVH_ERR_TIMEOUT)."""
        self._ck(lib().svh_batch_set_wait(self._b, float(limit_ms), int(hold_item), int(hold_phase)),
                 "svh_batch_set_wait")

    def sync(self):
        self._ck(lib().svh_batch_sync(self._b), "svh_batch_sync")

    @property
    def stream(self):
        return lib().svh_batch_stream(self._b)

    def solve(self, freqs, n_workers=4, **opts):
        o = svh_options()
        lib().svh_default_options(C.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        freqs = np.atleast_1d(np.asarray(freqs, np.float64))
        om = np.ascontiguousarray(2 * np.pi * freqs)
        outs = [np.zeros((freqs.size, h.info()["nports"], h.info()["nports"], 2)) for h in self.handles]
        Ls = [np.zeros(z.shape[:3]) for z in outs]
        ptrs = (_DP * len(outs))(*[_dp(z) for z in outs])
        lptrs = (_DP * len(Ls))(*[_dp(l) for l in Ls])
        st = svh_stats()
        self._ck(lib().svh_batch_solve(self._b, _dp(om), om.size, C.byref(o), ptrs, lptrs, int(n_workers),
                                       C.byref(st)), "svh_batch_solve")
        Zs = [z[..., 0] + 1j * z[..., 1] for z in outs]
        return {"Z": Zs, "L": Ls, "stats": {f: getattr(st, f) for f, _ in svh_stats._fields_}}

    def close(self):
        if self._b:
            lib().svh_batch_destroy(self._b)
            self._b = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
