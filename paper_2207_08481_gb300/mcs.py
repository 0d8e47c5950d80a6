"""ctypes binding of libmcs (argument marshalling only; every step runs in the library).

Device vectors are torch CUDA tensors (float64, contiguous, on the handle's device); the
handle's stream is torch's current stream at set-up unless one is given.  The library must
have been built (``paper_2207_08481_gb300.build.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmcs.so")

MCS_OK = 0
MCS_ERR_INVALID_ARG = -1
MCS_ERR_OOM = -2
MCS_ERR_CUDA = -3
MCS_ERR_NOT_CONVERGED = -4
MCS_ERR_BREAKDOWN = -5
MCS_ERR_TIMEOUT = -6
MCS_ERR_UNSUPPORTED = -7
MCS_FP64 = 0
MCS_MIXED = 1

EXPORTED = ["mcs_version", "mcs_last_error", "mcs_default_options", "mcs_setup_structured", "mcs_setup_mesh",
            "mcs_sizes", "mcs_export_mesh", "mcs_export_dofmap", "mcs_export_pattern", "mcs_condense",
            "mcs_condense_batch",
            "mcs_copy_element_matrices", "mcs_copy_schur", "mcs_load_points", "mcs_load_vector",
            "mcs_mass_velocity", "mcs_apply", "mcs_residual", "mcs_recover_stress", "mcs_precond", "mcs_solve", "mcs_solve_host", "mcs_profile",
            "mcs_profile_read", "mcs_launch_count", "mcs_condense_noalloc", "mcs_destroy"]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("smooth_steps", ctypes.c_int), ("gmg_levels", ctypes.c_int),
                ("gmg_smooth", ctypes.c_int), ("rtol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("max_refine", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("residual_dd", ctypes.c_int), ("asp", ctypes.c_int), ("lo_stab", ctypes.c_int),
                ("outflow", ctypes.c_int), ("etol", ctypes.c_double), ("tune", ctypes.c_int),
                ("tune_cache", ctypes.c_char_p), ("facet_push", ctypes.c_int)]


class Sizes(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("ndof", "n_dd", "n_oo", "n_hat", "n_pres", "off_o", "off_h", "off_p",
                                               "ne", "nint", "nfacets", "nvertices", "np1")] + \
               [(n, ctypes.c_int32) for n in ("dim", "k", "nF", "n_bub", "nhF", "n_p", "n_A", "n_c", "mF",
                                               "ncolours", "gmg_levels", "nq_load")] + \
               [("bytes_resident", ctypes.c_int64)] + \
               [(n, ctypes.c_int32) for n in ("facet_batch", "facet_threads", "apply_batch", "push_warps")]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int), ("status", ctypes.c_int),
                ("rel_res_precond", ctypes.c_double), ("rel_res_true", ctypes.c_double),
                ("err_est", ctypes.c_double)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class McsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libmcs error {code}: {msg}")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmcs is not built ({LIB_PATH} missing); run paper_2207_08481_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32p = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)
        L.mcs_last_error.restype = ctypes.c_char_p
        L.mcs_setup_structured.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.POINTER(Options), vp, ctypes.POINTER(vp)]
        L.mcs_setup_mesh.argtypes = [ctypes.c_int, i64, vp, i64, vp, ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(Options), vp, ctypes.POINTER(vp)]
        L.mcs_sizes.argtypes = [vp, ctypes.POINTER(Sizes)]
        L.mcs_export_mesh.argtypes = [vp, vp, vp, vp, vp]
        L.mcs_export_dofmap.argtypes = [vp, vp]
        L.mcs_export_pattern.argtypes = [vp, vp, vp]
        L.mcs_condense.argtypes = [vp]
        L.mcs_copy_element_matrices.argtypes = [vp, i64, i64, vp]
        L.mcs_copy_schur.argtypes = [vp, i64, i64, vp, vp]
        L.mcs_load_points.argtypes = [vp, vp]
        L.mcs_load_vector.argtypes = [vp, vp, vp]
        L.mcs_mass_velocity.argtypes = [vp, vp, vp]
        L.mcs_apply.argtypes = [vp, vp, vp]
        L.mcs_residual.argtypes = [vp, vp, vp, vp]
        L.mcs_recover_stress.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp]
        L.mcs_precond.argtypes = [vp, vp, vp]
        L.mcs_solve.argtypes = [vp, vp, vp, ctypes.POINTER(SolveInfo)]
        L.mcs_solve_host.argtypes = [vp, vp, vp, ctypes.POINTER(SolveInfo)]
        L.mcs_destroy.argtypes = [vp]
        L.mcs_profile.argtypes = [vp, ctypes.c_int]
        L.mcs_profile_read.argtypes = [vp, ctypes.POINTER(KernelStat), ctypes.c_int]
        L.mcs_condense_noalloc.argtypes = [vp, i64, i64, vp]
        L.mcs_launch_count.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        L.mcs_condense_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
        L.mcs_default_options.argtypes = [ctypes.POINTER(Options)]
        del i32p
        _lib = L
    return _lib


def _check(rc):
    if rc != MCS_OK:
        raise McsError(rc, lib().mcs_last_error().decode())
    return rc


def condense_batch(handles) -> None:
    """Condenses several handles (same precision, any mesh and k) in one persistent launch."""
    arr = (ctypes.c_void_p * len(handles))(*[h._h.value for h in handles])
    _check(lib().mcs_condense_batch(arr, len(handles)))


def launch_count() -> int:
    """Kernels launched by the library in this process (graph nodes counted per graph launch)."""
    n = ctypes.c_uint64(0)
    _check(lib().mcs_launch_count(ctypes.byref(n)))
    return int(n.value)


def default_options(**kw) -> Options:
    o = Options()
    lib().mcs_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v.encode() if isinstance(v, str) else v)
    return o


def _dptr(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


class Handle:
    """One set-up problem (mesh, k, nu) with its resident operators."""

    def __init__(self, ptr, stream=None):
        self._h = ptr
        self.stream = stream
        s = Sizes()
        _check(lib().mcs_sizes(self._h, ctypes.byref(s)))
        self.sizes = s

    @classmethod
    def structured(cls, dim, N, k, nu, stream=None, **opts):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        o = default_options(**opts)
        h = ctypes.c_void_p()
        _check(lib().mcs_setup_structured(dim, N, k, float(nu), ctypes.byref(o), ctypes.c_void_p(st.cuda_stream),
                                          ctypes.byref(h)))
        return cls(h, st)

    @classmethod
    def from_mesh(cls, dim, coords, elems, k, nu, stream=None, **opts):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        c = np.ascontiguousarray(coords, dtype=np.float64)
        e = np.ascontiguousarray(elems, dtype=np.int32)
        o = default_options(**opts)
        h = ctypes.c_void_p()
        _check(lib().mcs_setup_mesh(dim, c.shape[0], _hptr(c), e.shape[0], _hptr(e), k, float(nu), ctypes.byref(o),
                                    ctypes.c_void_p(st.cuda_stream), ctypes.byref(h)))
        return cls(h, st)

    def close(self):
        if self._h:
            _check(lib().mcs_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- exports
    def export_mesh(self):
        s = self.sizes
        facets = np.zeros((s.nfacets, s.dim), np.int32)
        ef = np.zeros((s.ne, s.dim + 1), np.int32)
        sg = np.zeros((s.ne, s.dim + 1), np.int8)
        col = np.zeros(s.nint, np.int32)
        _check(lib().mcs_export_mesh(self._h, _hptr(facets), _hptr(ef), _hptr(sg), _hptr(col)))
        return facets, ef, sg, col

    def export_dofmap(self):
        s = self.sizes
        out = np.zeros((s.ne, s.n_A + s.n_p), np.int64)
        _check(lib().mcs_export_dofmap(self._h, _hptr(out)))
        return out

    def export_pattern(self):
        s = self.sizes
        rp = np.zeros(s.ndof + 1, np.int64)
        _check(lib().mcs_export_pattern(self._h, _hptr(rp), None))
        col = np.zeros(int(rp[-1]), np.int32)
        _check(lib().mcs_export_pattern(self._h, _hptr(rp), _hptr(col)))
        return rp, col

    # ---------------------------------------------------------------- compute
    def condense(self):
        _check(lib().mcs_condense(self._h))
        # the launch shapes in use can change at the first condensation (tune = 1)
        s = Sizes()
        _check(lib().mcs_sizes(self._h, ctypes.byref(s)))
        self.sizes = s

    def element_matrices(self, T0, count):
        nA = self.sizes.n_A
        out = np.zeros((count, nA * (nA + 1) // 2))
        _check(lib().mcs_copy_element_matrices(self._h, T0, count, _hptr(out)))
        return out

    def schur(self, T0, count):
        s = self.sizes
        Ad = np.zeros((count, s.n_c, s.n_c))
        G = np.zeros((count, s.n_bub, s.n_c))
        _check(lib().mcs_copy_schur(self._h, T0, count, _hptr(Ad), _hptr(G)))
        return Ad, G

    def load_points(self, xq):
        _check(lib().mcs_load_points(self._h, _dptr(xq)))

    def load_vector(self, fq, F):
        _check(lib().mcs_load_vector(self._h, _dptr(fq), _dptr(F)))

    def mass_velocity(self, c, F):
        _check(lib().mcs_mass_velocity(self._h, _dptr(c), _dptr(F)))

    def apply(self, x, y):
        _check(lib().mcs_apply(self._h, _dptr(x), _dptr(y)))

    def residual(self, F, x, r):
        _check(lib().mcs_residual(self._h, _dptr(F), _dptr(x), _dptr(r)))

    def recover_stress(self, x, xhat, sigma, omega=None):
        """sigma_h, omega_h of every element at the reference points xhat [nq, dim] (host) into the device
        tensors sigma, omega [ne, nq, dim, dim] (omega optional)."""
        xh = np.ascontiguousarray(xhat, dtype=np.float64)
        _check(lib().mcs_recover_stress(self._h, _dptr(x), xh.shape[0], _hptr(xh), _dptr(sigma),
                                        _dptr(omega) if omega is not None else None))

    def precond(self, r, z):
        _check(lib().mcs_precond(self._h, _dptr(r), _dptr(z)))

    def solve(self, F, x, check=True):
        info = SolveInfo()
        rc = lib().mcs_solve(self._h, _dptr(F), _dptr(x), ctypes.byref(info))
        if check and rc not in (MCS_OK,):
            raise McsError(rc, lib().mcs_last_error().decode())
        return info

    def profile(self, enable: bool):
        _check(lib().mcs_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        buf = (KernelStat * 16)()
        n = lib().mcs_profile_read(self._h, buf, 16)
        if n < 0:
            _check(n)
        return {buf[i].name.decode(): dict(launches=buf[i].launches, ms=buf[i].total_ms, bytes=buf[i].bytes,
                                             flops=buf[i].flops) for i in range(n)}

    def condense_noalloc(self, T0, count, AT_out):
        """A_T of elements T0 .. T0+count-1 into the device tensor AT_out [count, n_A, n_A] (no allocation).
        The kernel writes count * n_A^2 doubles: a shorter, non-float64 or other-device tensor is refused
        here, before the library sees the pointer."""
        import torch
        nA = int(self.sizes.n_A)
        if AT_out.dtype != torch.float64:
            raise ValueError("AT_out must be float64")
        if AT_out.numel() < int(count) * nA * nA:
            raise ValueError(f"AT_out holds {AT_out.numel()} doubles, {int(count) * nA * nA} are written")
        if AT_out.device != torch.device("cuda", torch.cuda.current_device()):
            raise ValueError("AT_out must be on the current CUDA device (the handle's device)")
        _check(lib().mcs_condense_noalloc(self._h, T0, count, _dptr(AT_out)))

    def solve_host(self, F: np.ndarray, x: np.ndarray, check=True):
        info = SolveInfo()
        rc = lib().mcs_solve_host(self._h, _hptr(F), _hptr(x), ctypes.byref(info))
        if check and rc not in (MCS_OK,):
            raise McsError(rc, lib().mcs_last_error().decode())
        return info
