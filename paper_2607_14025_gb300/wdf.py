"""ctypes binding of libwdf.so (include/wdf.h): argument marshalling only.

Every computation happens in the library's CUDA kernels. Arrays may be torch tensors on the
context's GPU (passed as device pointers) or numpy arrays (host memory, copied by the library).
Complex half-sphere vectors are complex128 arrays of shape (n, npw_h). There is no CPU fallback:
if the shared library is missing or does not load, every call raises.
"""

from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libwdf.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "wdf.h")

WDF_OK, WDF_EINVAL, WDF_ENOMEM, WDF_ECUDA, WDF_ENOCONV, WDF_ETIMEOUT, WDF_ENAN, WDF_ESTATE = range(8)
WDF_MEM_HOST, WDF_MEM_DEVICE = 0, 1
WDF_FP64, WDF_MIXED, WDF_MIXED_DF = 0, 1, 2
WDF_PRECOND_NONE, WDF_PRECOND_TPA, WDF_PRECOND_LEARNED = 0, 1, 2
MODEL_NPARAM, MODEL_FLOATS = 4610, 4618


class WdfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"wdf error {code}: {msg}")
        self.code = code


class NotConverged(WdfError):
    """An iteration hit its limit; ``result`` holds what the call produced."""

    def __init__(self, code, msg, result=None):
        super().__init__(code, msg)
        self.result = result


class _System(ctypes.Structure):
    _fields_ = [
        ("cell", ctypes.c_double * 9),
        ("n", ctypes.c_int * 3),
        ("npw_h", ctypes.c_int),
        ("miller", ctypes.c_void_p),
        ("vloc_r", ctypes.c_void_p),
        ("nproj", ctypes.c_int),
        ("beta", ctypes.c_void_p),
        ("dij", ctypes.c_void_p),
        ("nocc", ctypes.c_int),
        ("psi", ctypes.c_void_p),
        ("eps", ctypes.c_void_p),
        ("mem", ctypes.c_int),
    ]


class _Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("precond", ctypes.c_int),
        ("cg_tol", ctypes.c_double),
        ("cg_maxiter", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("max_batch", ctypes.c_int),
        ("gs_tol", ctypes.c_double),
        ("gs_maxiter", ctypes.c_int),
        ("gs_extra", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("device", ctypes.c_int),
        ("warm_start", ctypes.c_int),
        ("residual_update", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("nsolve", ctypes.c_int64),
        ("cg_iters", ctypes.c_int64),
        ("cg_iters_max", ctypes.c_int32),
        ("refinements", ctypes.c_int32),
        ("max_residual", ctypes.c_double),
        ("napply", ctypes.c_int64),
        ("davidson_iters", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("ms", ctypes.c_double),
        ("fallbacks", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TrainOpts(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("lr", ctypes.c_double), ("npert", ctypes.c_int), ("seed", ctypes.c_uint64)]


class TrainStats(ctypes.Structure):
    _fields_ = [
        ("nsamples", ctypes.c_int64),
        ("steps", ctypes.c_int32),
        ("loss_first", ctypes.c_double),
        ("loss_last", ctypes.c_double),
        ("ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


# out = A in for wdf_davidson: (user, nvec, in, out) -> status
OPERATOR_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)


class _DeviceArray:
    """A view of library-owned device memory for torch.as_tensor (no copy)."""

    def __init__(self, ptr: int, shape, device: int):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (ptr, False), "version": 2}
        self.device = device


def load(path: str = LIB_PATH):
    """Load libwdf.so (once). Raises if it is missing: the library has no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2607_14025_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "wdf_default_options": (None, [P]),
        "wdf_setup_hamiltonian": (I, [ctypes.POINTER(P), P, P]),
        "wdf_destroy": (None, [P]),
        "wdf_get_orbitals": (I, [P, P, P, I]),
        "wdf_apply_hamiltonian": (I, [P, I, P, P, I]),
        "wdf_sternheimer": (I, [P, I, P, P, P, I, P]),
        "wdf_apply_sternheimer_operator": (I, [P, I, P, P, P, I]),
        "wdf_set_residual_update": (I, [P, I]),
        "wdf_apply_chi0": (I, [P, I, P, P, P, I, P]),
        "wdf_pdep_davidson": (I, [P, I, I, I, D, I, P, P, P, I, P]),
        "wdf_apply_hamiltonian_noalloc": (I, [P, I, P, P]),
        "wdf_apply_chi0_multi": (I, [I, P, P, P, P, I, P]),
        "wdf_apply_wp": (I, [P, I, P, P, I, P, P, I]),
        "wdf_davidson": (I, [P, OPERATOR_FN, P, I, I, I, D, I, I, P, P, P, I, P]),
        "wdf_half_sphere": (I, [P, D, P, P]),
        "wdf_get_gvectors": (I, [P, P]),
        "wdf_reset_error": (I, [P]),
        "wdf_pdep_davidson_seeded": (I, [P, I, I, I, D, ctypes.c_uint64, P, P, I, P]),
        "wdf_default_train_opts": (None, [P]),
        "wdf_model_create": (I, [I, ctypes.c_uint64, ctypes.POINTER(P)]),
        "wdf_model_free": (None, [P]),
        "wdf_model_set_weights": (I, [P, P]),
        "wdf_model_get_weights": (I, [P, P]),
        "wdf_model_add_solves": (I, [P, P, I, P, I, P]),
        "wdf_model_num_samples": (ctypes.c_int64, [P]),
        "wdf_model_set_samples": (I, [P, ctypes.c_int64, P, P, P]),
        "wdf_model_get_samples": (I, [P, ctypes.c_int64, ctypes.c_int64, P, P, P]),
        "wdf_model_loss_grad": (I, [P, P, P]),
        "wdf_model_train": (I, [P, P, P]),
        "wdf_model_predict": (I, [P, ctypes.c_int64, P, P]),
        "wdf_set_model": (I, [P, P]),
        "wdf_train_preconditioner": (I, [P, I, P, ctypes.POINTER(P), P]),
        "wdf_profile_kernel": (I, [P, ctypes.c_char_p]),
        "wdf_profile_read": (I, [P, P, P]),
        "wdf_profile_units": (I, [P, P]),
        "wdf_plane_variant": (I, [P, I, ctypes.POINTER(I)]),
        "wdf_launch_count": (ctypes.c_int64, []),
        "wdf_device_bytes": (ctypes.c_int64, []),
        "wdf_alloc_count": (ctypes.c_int64, []),
        "wdf_set_device_limit": (None, [ctypes.c_int64]),
        "wdf_set_wait_limit": (I, [P, ctypes.c_int64]),
        "wdf_strerror": (ctypes.c_char_p, [I]),
        "wdf_last_error": (ctypes.c_char_p, [P]),
        "wdf_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_functions(path: str = HEADER):
    """Names of the functions declared in include/wdf.h."""
    text = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|int64_t|const char \*)\s*\*?\s*(wdf_\w+)\s*\(", text, flags=re.M)))


def launch_count() -> int:
    """Kernel launches made by the library in this process."""
    return int(load().wdf_launch_count())


def device_bytes() -> int:
    """Device memory held by the library's buffers in this process (wdf_device_bytes)."""
    return int(load().wdf_device_bytes())


def alloc_count() -> int:
    """cudaMalloc calls the library has made in this process (wdf_alloc_count)."""
    return int(load().wdf_alloc_count())


def set_device_limit(nbytes: int) -> None:
    """Cap the device memory the library may hold (0: no cap); growth past it is WDF_ENOMEM."""
    load().wdf_set_device_limit(int(nbytes))


# ------------------------------------------------------------------------------------------------
# array marshalling


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr_in(x, dtype, keep: list):
    """(pointer, mem) of an input array; numpy inputs are made contiguous with the given dtype."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch

        want = {np.complex128: torch.complex128, np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if x.dtype != want:
            raise TypeError(f"expected a tensor of {want}, got {x.dtype}")
        if x.is_cuda:
            t = x.contiguous()
            keep.append(t)
            return t.data_ptr(), WDF_MEM_DEVICE
        x = x.numpy()
    a = np.ascontiguousarray(x, dtype=dtype)
    keep.append(a)
    return a.ctypes.data, WDF_MEM_HOST


class Context:
    """One model system on one GPU (wraps wdf_setup_hamiltonian / wdf_destroy).

    ``system`` needs the attributes cell (3x3), grid (n1, n2, n3), miller (npw_h x 3),
    vloc_r (n3, n2, n1), beta (nproj x npw_h complex), dij (nproj) and nocc. When ``psi`` and
    ``eps`` are None the library computes the occupied ground state itself.
    """

    def __init__(self, system, psi=None, eps=None, precision: str = "mixed", precond: str = "tpa", cg_tol: float = 1e-8,
                 cg_maxiter: int = 1000, inner_tol: float = 1e-5, alpha: float = 0.0, max_batch: int = 0,
                 gs_tol: float = 1e-10, gs_maxiter: int = 300, gs_extra: int = 8, stream: Optional[int] = None,
                 device: int = 0, data_on_device: bool = False, warm_start: bool = False, residual_update: bool = False):
        self._lib = load()
        self._ctx = ctypes.c_void_p()
        opt = _Options()
        self._lib.wdf_default_options(ctypes.byref(opt))
        opt.precision = {"fp64": WDF_FP64, "mixed": WDF_MIXED, "mixed_df": WDF_MIXED_DF}[precision]
        opt.precond = {"none": WDF_PRECOND_NONE, "tpa": WDF_PRECOND_TPA}[precond]
        opt.cg_tol, opt.cg_maxiter, opt.inner_tol, opt.alpha = cg_tol, cg_maxiter, inner_tol, alpha
        opt.max_batch, opt.gs_tol, opt.gs_maxiter, opt.gs_extra = max_batch, gs_tol, gs_maxiter, gs_extra
        opt.stream = stream
        opt.device = device
        opt.warm_start = 1 if warm_start else 0
        opt.residual_update = 1 if residual_update else 0
        keep: list = []
        s = _System()
        s.cell[:] = [float(v) for v in np.asarray(system.cell, dtype=np.float64).reshape(9)]
        s.n[:] = [int(v) for v in system.grid]
        miller = np.ascontiguousarray(system.miller, dtype=np.int32)
        keep.append(miller)
        s.npw_h = miller.shape[0]
        s.miller = miller.ctypes.data
        dij = np.ascontiguousarray(system.dij, dtype=np.float64)
        keep.append(dij)
        s.nproj = int(np.asarray(system.beta).shape[0]) if not _is_torch(system.beta) else int(system.beta.shape[0])
        s.dij = dij.ctypes.data if s.nproj else None
        s.nocc = int(system.nocc)
        vp, m1 = _ptr_in(system.vloc_r, np.float64, keep)
        bp, m2 = _ptr_in(system.beta, np.complex128, keep) if s.nproj else (None, m1)
        pp, m3 = _ptr_in(psi, np.complex128, keep)
        if m3 is not None and len({m1, m2, m3}) != 1 or (m2 != m1):
            raise ValueError("vloc_r, beta and psi must all be host arrays or all device tensors")
        s.vloc_r, s.beta, s.psi = vp, bp, pp
        s.mem = m1
        e = None
        if eps is not None:
            e = np.ascontiguousarray(eps, dtype=np.float64)
            keep.append(e)
            s.eps = e.ctypes.data
        self.npw_h = s.npw_h
        self.nocc = s.nocc
        self.device = device
        rc = self._lib.wdf_setup_hamiltonian(ctypes.byref(self._ctx), ctypes.byref(s), ctypes.byref(opt))
        self.setup_status = rc
        if rc not in (WDF_OK, WDF_ENOCONV):
            raise WdfError(rc, self._lib.wdf_last_error(None).decode())
        if rc == WDF_ENOCONV:
            self.setup_message = self._lib.wdf_last_error(self._ctx).decode()

    # -- helpers ----------------------------------------------------------------------------------
    def _check(self, rc, result=None):
        if rc == WDF_OK:
            return
        msg = self._lib.wdf_last_error(self._ctx).decode()
        if rc == WDF_ENOCONV:
            raise NotConverged(rc, msg, result)
        raise WdfError(rc, msg)

    def _out_like(self, x, n):
        if x is not None and _is_torch(x) and x.is_cuda:
            import torch

            t = torch.empty((n, self.npw_h), dtype=torch.complex128, device=x.device)
            return t, t.data_ptr()
        a = np.empty((n, self.npw_h), dtype=np.complex128)
        return a, a.ctypes.data

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._lib.wdf_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- entry points ---------------------------------------------------------------------------
    def orbitals(self, device_tensor=None):
        """(eps[nocc], psi[nocc, npw_h]) of the occupied ground state."""
        eps = np.empty(self.nocc)
        out, ptr = self._out_like(device_tensor, self.nocc)
        mem = WDF_MEM_DEVICE if device_tensor is not None and _is_torch(device_tensor) and device_tensor.is_cuda else WDF_MEM_HOST
        self._check(self._lib.wdf_get_orbitals(self._ctx, eps.ctypes.data, ptr, mem))
        return eps, out

    def apply_hamiltonian(self, x):
        keep: list = []
        x2 = x if (_is_torch(x) and x.is_cuda) else np.atleast_2d(x)
        p, mem = _ptr_in(x2, np.complex128, keep)
        n = x2.shape[0]
        out, op = self._out_like(x2, n)
        self._check(self._lib.wdf_apply_hamiltonian(self._ctx, n, p, op, mem))
        return out

    def apply_hamiltonian_noalloc(self, x, out):
        """H x into ``out`` without any device allocation by the library.

        For callers that cannot allocate GPU memory (a process whose device memory belongs to
        another allocator, or a service with a fixed memory budget): x and out are complex128
        CUDA tensors of shape (nvec, npw_h) on the context's GPU that the caller owns; ``out``
        may be ``x`` itself. The library's temporaries live in a fixed 64 MiB device array. The
        first call on a device must come before any stream capture.
        """
        import torch

        for name, t in (("x", x), ("out", out)):
            if not (_is_torch(t) and t.is_cuda):
                raise TypeError(f"apply_hamiltonian_noalloc takes CUDA tensors; {name} is not one")
            if t.dtype != torch.complex128 or t.ndim != 2 or t.shape[1] != self.npw_h:
                raise ValueError(f"{name} must be complex128 of shape (nvec, {self.npw_h}), got {t.dtype} {tuple(t.shape)}")
            if t.device.index != self.device:
                raise ValueError(f"{name} is on cuda:{t.device.index}, the context on cuda:{self.device}")
            if not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
        if out.shape != x.shape:
            raise ValueError("out must have the shape of x")
        self._check(self._lib.wdf_apply_hamiltonian_noalloc(self._ctx, x.shape[0], x.data_ptr(), out.data_ptr()))
        return out

    def set_wait_limit(self, polls: int):
        """Polls of the software device waits before they give up (wdf_set_wait_limit; 0: default)."""
        self._check(self._lib.wdf_set_wait_limit(self._ctx, int(polls)))

    def set_residual_update(self, on: bool):
        """Switch the bounded residual updates of the FP32 inner forms (wdf_options.residual_update)."""
        self._check(self._lib.wdf_set_residual_update(self._ctx, 1 if on else 0))

    def apply_sternheimer_operator(self, vidx, x):
        """(H - eps_v + alpha P) x, vector k with v = vidx[k], in the residuals' precision."""
        keep: list = []
        v = np.ascontiguousarray(vidx, dtype=np.int32)
        x2 = x if (_is_torch(x) and x.is_cuda) else np.atleast_2d(x)
        p, mem = _ptr_in(x2, np.complex128, keep)
        n = x2.shape[0]
        if v.shape[0] != n:
            raise ValueError("one orbital index per vector")
        out, op = self._out_like(x2, n)
        self._check(self._lib.wdf_apply_sternheimer_operator(self._ctx, n, v.ctypes.data, p, op, mem))
        return out

    def sternheimer(self, vidx, rhs):
        keep: list = []
        v = np.ascontiguousarray(vidx, dtype=np.int32)
        p, mem = _ptr_in(rhs, np.complex128, keep)
        n = v.shape[0]
        out, op = self._out_like(rhs, n)
        st = Stats()
        rc = self._lib.wdf_sternheimer(self._ctx, n, v.ctypes.data, p, op, mem, ctypes.byref(st))
        self._check(rc, (out, st))
        return out, st

    def apply_chi0(self, phi, want_drho: bool = False):
        """chi0bar phi; returns (out, drho or None, Stats)."""
        keep: list = []
        p, mem = _ptr_in(phi, np.complex128, keep)
        n = phi.shape[0]
        out, op = self._out_like(phi, n)
        drho, dp = self._out_like(phi, n) if want_drho else (None, None)
        st = Stats()
        rc = self._lib.wdf_apply_chi0(self._ctx, n, p, op, dp, mem, ctypes.byref(st))
        self._check(rc, (out, drho, st))
        return out, drho, st

    def profile_kernel(self, kernel):
        """Start timing one kernel class (see include/wdf.h), or stop with None."""
        self._check(self._lib.wdf_profile_kernel(self._ctx, kernel.encode() if kernel else None))

    def profile_read(self):
        """(launches, total ms) of the timed kernel class."""
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        self._check(self._lib.wdf_profile_read(self._ctx, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def plane_variant(self, bits: int = 32) -> int:
        """V_loc plane kernel chosen at setup for the given arithmetic (32, 64 or 48 = double-float)."""
        v = ctypes.c_int()
        self._check(self._lib.wdf_plane_variant(self._ctx, int(bits), ctypes.byref(v)))
        return v.value

    def profile_units(self) -> int:
        """Work units of the timed launches: thread blocks, or (pair, z plane) units for plane_vloc."""
        b = ctypes.c_int64()
        self._check(self._lib.wdf_profile_units(self._ctx, ctypes.byref(b)))
        return b.value

    def pdep(self, neig: int, guess, nbasis_max: int = 0, maxiter: int = 100, tol: float = 1e-10):
        """Lowest neig eigenpairs of chi0bar: (lambda[neig], phibar[neig, npw_h], Stats)."""
        keep: list = []
        p, mem = _ptr_in(guess, np.complex128, keep)
        lam = np.empty(neig)
        vec, vp = self._out_like(guess, neig)
        st = Stats()
        rc = self._lib.wdf_pdep_davidson(self._ctx, neig, nbasis_max, maxiter, tol, guess.shape[0], p, lam.ctypes.data, vp, mem,
                                         ctypes.byref(st))
        self._check(rc, (lam, vec, st))
        return lam, vec, st

    def apply_wp(self, lam, phibar, x):
        """W_p x from PDEP eigenpairs (wdf_apply_wp; Eq. 5 without Xi)."""
        keep: list = []
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        pp, mem = _ptr_in(phibar, np.complex128, keep)
        xp, mem2 = _ptr_in(x, np.complex128, keep)
        if mem != mem2:
            raise ValueError("phibar and x must both be host arrays or both device tensors")
        out, op = self._out_like(x, x.shape[0])
        self._check(self._lib.wdf_apply_wp(self._ctx, lam.shape[0], lam.ctypes.data, pp, x.shape[0], xp, op, mem))
        return out

    def davidson(self, apply, neig: int, guess, nbasis_max: int = 0, maxiter: int = 100, tol: float = 1e-10,
                 zero_g0: bool = True):
        """Lowest neig eigenpairs of a caller's operator by the library's Davidson (wdf_davidson).

        ``apply(x, out)`` gets two complex128 CUDA tensors of shape (nvec, npw_h) that view the
        library's buffers and must write A x into ``out`` (synchronised) before returning.
        Returns (lambda[neig], vectors[neig, npw_h], Stats).
        """
        import torch

        npw = self.npw_h
        dev = self.device

        def trampoline(user, nvec, pin, pout):
            try:
                x = torch.view_as_complex(torch.as_tensor(_DeviceArray(pin, (nvec, npw, 2), dev), device=f"cuda:{dev}"))
                out = torch.view_as_complex(torch.as_tensor(_DeviceArray(pout, (nvec, npw, 2), dev), device=f"cuda:{dev}"))
                apply(x, out)
                torch.cuda.synchronize(dev)
                return 0
            except Exception:  # noqa: BLE001 - reported to the library as a failed callback
                import traceback

                traceback.print_exc()
                return 1

        fn = OPERATOR_FN(trampoline)
        keep: list = []
        p, mem = _ptr_in(guess, np.complex128, keep)
        lam = np.empty(neig)
        vec, vp = self._out_like(guess, neig)
        st = Stats()
        rc = self._lib.wdf_davidson(self._ctx, fn, None, neig, nbasis_max, maxiter, tol, 1 if zero_g0 else 0, guess.shape[0], p,
                                    lam.ctypes.data, vp, mem, ctypes.byref(st))
        self._check(rc, (lam, vec, st))
        return lam, vec, st

    def gvectors(self) -> np.ndarray:
        """The context's Miller triples (npw_h, 3)."""
        m = np.empty((self.npw_h, 3), dtype=np.int32)
        self._check(self._lib.wdf_get_gvectors(self._ctx, m.ctypes.data))
        return m

    def reset_error(self):
        """Clear a recoverable failure (see wdf_reset_error)."""
        self._check(self._lib.wdf_reset_error(self._ctx))

    def pdep_seeded(self, neig: int, seed: int = 0, nbasis_max: int = 0, maxiter: int = 100, tol: float = 1e-10):
        """PDEP from a start block the library draws from splitmix64(seed)."""
        lam = np.empty(neig)
        vec = np.empty((neig, self.npw_h), dtype=np.complex128)
        st = Stats()
        rc = self._lib.wdf_pdep_davidson_seeded(self._ctx, neig, nbasis_max, maxiter, tol, seed, lam.ctypes.data, vec.ctypes.data,
                                                WDF_MEM_HOST, ctypes.byref(st))
        self._check(rc, (lam, vec, st))
        return lam, vec, st

    def set_model(self, model: Optional["Model"]):
        """Use a trained model as preconditioner (WDF_PRECOND_LEARNED); None: back to TPA."""
        self._check(self._lib.wdf_set_model(self._ctx, model._m if model is not None else None))


def _check_global(lib, rc, obj=None):
    if rc != WDF_OK:
        raise WdfError(rc, lib.wdf_last_error(None).decode())


class Model:
    """A learned-preconditioner model on one GPU (wdf_model_*; layout in include/wdf.h)."""

    def __init__(self, device: int = 0, seed: int = 0, _handle=None):
        self._lib = load()
        self._m = ctypes.c_void_p()
        if _handle is not None:
            self._m = _handle
        else:
            _check_global(self._lib, self._lib.wdf_model_create(device, seed, ctypes.byref(self._m)))

    def close(self):
        if getattr(self, "_m", None) and self._m.value:
            self._lib.wdf_model_free(self._m)
            self._m = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        _check_global(self._lib, rc)

    @property
    def weights(self) -> np.ndarray:
        w = np.empty(MODEL_FLOATS, dtype=np.float32)
        self._check(self._lib.wdf_model_get_weights(self._m, w.ctypes.data))
        return w

    @weights.setter
    def weights(self, w):
        a = np.ascontiguousarray(w, dtype=np.float32).reshape(MODEL_FLOATS)
        self._check(self._lib.wdf_model_set_weights(self._m, a.ctypes.data))

    def add_solves(self, ctx: Context, phi):
        """Append the samples of TPA solves of chi0bar phi on ctx; returns the Stats."""
        keep: list = []
        p, mem = _ptr_in(phi, np.complex128, keep)
        st = Stats()
        rc = self._lib.wdf_model_add_solves(self._m, ctx._ctx, int(phi.shape[0]), p, mem, ctypes.byref(st))
        if rc not in (WDF_OK, WDF_ENOCONV):
            self._check(rc)
        return st

    @property
    def num_samples(self) -> int:
        return int(self._lib.wdf_model_num_samples(self._m))

    def set_samples(self, feat, tgt, wt):
        f = np.ascontiguousarray(feat, dtype=np.float32).reshape(-1, 4)
        t = np.ascontiguousarray(tgt, dtype=np.float32).reshape(-1, 2)
        w = np.ascontiguousarray(wt, dtype=np.float32).reshape(-1, 2)
        if not (f.shape[0] == t.shape[0] == w.shape[0]):
            raise ValueError("features, targets and weights must have one row per sample")
        self._check(self._lib.wdf_model_set_samples(self._m, f.shape[0], f.ctypes.data, t.ctypes.data, w.ctypes.data))

    def samples(self, first: int = 0, count: Optional[int] = None):
        """(features[n, 4], targets[n, 2], weights[n, 2]) as float32 arrays."""
        n = self.num_samples - first if count is None else count
        f = np.empty((n, 4), dtype=np.float32)
        t = np.empty((n, 2), dtype=np.float32)
        w = np.empty((n, 2), dtype=np.float32)
        self._check(self._lib.wdf_model_get_samples(self._m, first, n, f.ctypes.data, t.ctypes.data, w.ctypes.data))
        return f, t, w

    def loss_grad(self):
        g = np.empty(MODEL_NPARAM)
        loss = ctypes.c_double()
        self._check(self._lib.wdf_model_loss_grad(self._m, ctypes.byref(loss), g.ctypes.data))
        return loss.value, g

    def train(self, steps: int = 600, lr: float = 3e-3) -> TrainStats:
        o = TrainOpts()
        self._lib.wdf_default_train_opts(ctypes.byref(o))
        o.steps, o.lr = steps, lr
        st = TrainStats()
        self._check(self._lib.wdf_model_train(self._m, ctypes.byref(o), ctypes.byref(st)))
        return st

    def predict(self, feat) -> np.ndarray:
        f = np.ascontiguousarray(feat, dtype=np.float32).reshape(-1, 4)
        out = np.empty((f.shape[0], 2), dtype=np.float32)
        self._check(self._lib.wdf_model_predict(self._m, f.shape[0], f.ctypes.data, out.ctypes.data))
        return out


def train_preconditioner(contexts, npert: int = 8, steps: int = 600, lr: float = 3e-3, seed: int = 0):
    """wdf_train_preconditioner over a list of contexts: returns (Model, TrainStats)."""
    lib = load()
    arr = (ctypes.c_void_p * len(contexts))(*[c._ctx.value for c in contexts])
    o = TrainOpts()
    lib.wdf_default_train_opts(ctypes.byref(o))
    o.steps, o.lr, o.npert, o.seed = steps, lr, npert, seed
    h = ctypes.c_void_p()
    st = TrainStats()
    _check_global(lib, lib.wdf_train_preconditioner(arr, len(contexts), ctypes.byref(o), ctypes.byref(h), ctypes.byref(st)))
    return Model(_handle=h), st


def apply_chi0_multi(contexts, phis):
    """chi0bar for several systems at once (wdf_apply_chi0_multi): returns (outs, stats).

    ``phis[k]`` are host arrays (npert_k, npw_h of context k); the systems run concurrently.
    """
    lib = load()
    n = len(contexts)
    keep = [np.ascontiguousarray(p, dtype=np.complex128) for p in phis]
    outs = [np.empty_like(p) for p in keep]
    ctxa = (ctypes.c_void_p * n)(*[c._ctx.value for c in contexts])
    npa = (ctypes.c_int * n)(*[p.shape[0] for p in keep])
    pa = (ctypes.c_void_p * n)(*[p.ctypes.data for p in keep])
    oa = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
    st = (Stats * n)()
    rc = lib.wdf_apply_chi0_multi(n, ctxa, npa, pa, oa, WDF_MEM_HOST, st)
    if rc == WDF_ENOCONV:
        raise NotConverged(rc, lib.wdf_last_error(None).decode(), (outs, list(st)))
    _check_global(lib, rc)
    return outs, list(st)


def half_sphere(cell, ecut: float) -> np.ndarray:
    """wdf_half_sphere: the canonical Gamma half sphere (npw_h, 3) for a cell and cutoff."""
    lib = load()
    c = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    n = ctypes.c_int(0)
    _check_global(lib, lib.wdf_half_sphere(c.ctypes.data, ecut, None, ctypes.byref(n)))
    m = np.empty((n.value, 3), dtype=np.int32)
    _check_global(lib, lib.wdf_half_sphere(c.ctypes.data, ecut, m.ctypes.data, ctypes.byref(n)))
    return m
