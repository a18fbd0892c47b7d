"""Thin Python binding of the C ABI in include/multipole.h (libmultipole.so).

Argument marshalling only: every step of the solve runs in the CUDA library.
PyTorch supplies device memory and streams.  Importing works without a GPU;
using a mesh needs the compiled library and a CUDA device, and fails loudly
otherwise (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmultipole.so")

MP_OK = 0
STATUS_NAMES = {
    0: "MP_OK", 1: "MP_ERR_INVALID_ARG", 2: "MP_ERR_RANGE", 3: "MP_ERR_CUDA", 4: "MP_ERR_OOM",
    5: "MP_ERR_NOT_READY", 6: "MP_ERR_NONFINITE", 7: "MP_ERR_TIMEOUT", 8: "MP_ERR_UNSUPPORTED",
}
PRECISIONS = {"fp64": 0, "bf16x3": 1, "bf16x6": 2}

_lib = None


class MultipoleError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {self.name}: {detail}")


class MeshInfo(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int), ("n_theta", ctypes.c_int), ("n_phi", ctypes.c_int),
                ("l_max", ctypes.c_int), ("n_moments", ctypes.c_int), ("precision", ctypes.c_int),
                ("effective_precision", ctypes.c_int), ("r_ref", ctypes.c_double), ("G", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("tuned_candidates", ctypes.c_int),
                ("theta_tensor_cores", ctypes.c_int)]


def load_library(path: str = LIB_PATH):
    """Load libmultipole.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    sigs = {
        "mp_mesh_create": [dp, i, dp, i, dp, i, i, d, i, vp, ctypes.POINTER(vp)],
        "mp_mesh_destroy": [vp],
        "mp_mesh_set_stream": [vp, vp],
        "mp_mesh_get_info": [vp, ctypes.POINTER(MeshInfo)],
        "mp_set_density": [vp, vp],
        "mp_set_phi_output": [vp, vp],
        "mp_solve": [vp],
        "mp_get_phi": [vp, vp],
        "mp_get_moments": [vp, vp, vp, vp],
        "mp_solve_host": [vp, vp, vp],
        "mp_solve_host_async": [vp, vp, vp],
        "mp_mesh_synchronize": [vp],
        "mp_set_wait_budget": [vp, ctypes.c_longlong],
        "mp_set_theta_engine": [vp, i],
        "mp_mesh_create_slab": [dp, i, i, i, dp, i, dp, i, i, d, i, vp, ctypes.POINTER(vp)],
        "mp_slab_moments": [vp, vp],
        "mp_slab_potential": [vp, vp],
        "mp_profile_enable": [vp, i],
        "mp_profile_read": [vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(i), dp, i, ctypes.POINTER(i)],
        "mp_batch_create": [ctypes.POINTER(vp), i, ctypes.POINTER(vp)],
        "mp_batch_solve": [vp],
        "mp_batch_destroy": [vp],
        "mp_autotune": [vp, ctypes.c_char_p],
        "mp_last_error_detail": [ctypes.c_char_p, i],
        "mp_probe_rates": [dp, dp],
        "mp_moments_noalloc": [vp, vp, vp],
        "mp_gravity_sources": [vp, vp, vp, vp, vp, vp, vp],
        "mp_coarsen": [vp, vp, ctypes.c_int, ctypes.c_longlong],
        "mp_coarsening_factors": [vp, vp, vp],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.mp_status_string.argtypes = [i]
    lib.mp_status_string.restype = ctypes.c_char_p
    lib.mp_version.argtypes = []
    lib.mp_version.restype = ctypes.c_int
    _lib = lib
    return lib


def _detail(lib) -> str:
    buf = ctypes.create_string_buffer(512)
    lib.mp_last_error_detail(buf, 512)
    return buf.value.decode(errors="replace")


def _check(status: int, where: str):
    if status != MP_OK:
        lib = load_library()
        raise MultipoleError(status, where, _detail(lib))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _tensor_ptr(t, n: int, name: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return t.data_ptr()


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Mesh:
    """A spherical mesh with its device tables (mp_mesh_create)."""

    def __init__(self, r_edges, theta_edges, phi_edges, l_max: int, G: float = 1.0,
                 precision: str = "fp64", stream=None, slab=None):
        """slab=(i0, i1): shells [i0, i1) of the mesh with these radial edges
        (mp_mesh_create_slab); the mesh's arrays then cover only those shells."""
        lib = load_library()
        self._lib = lib
        r_all = np.ascontiguousarray(r_edges, dtype=np.float64)
        self.r = r_all if slab is None else np.ascontiguousarray(r_all[slab[0]:slab[1] + 1])
        self.theta = np.ascontiguousarray(theta_edges, dtype=np.float64)
        self.phi = np.ascontiguousarray(phi_edges, dtype=np.float64)
        self.shape = (self.r.size - 1, self.theta.size - 1, self.phi.size - 1)
        self.l_max = int(l_max)
        self.precision = precision
        self.slab = slab
        self._stream = stream
        handle = ctypes.c_void_p()
        if slab is None:
            st = lib.mp_mesh_create(_dptr(self.r), self.shape[0], _dptr(self.theta), self.shape[1],
                                    _dptr(self.phi), self.shape[2], self.l_max, float(G),
                                    PRECISIONS[precision], ctypes.c_void_p(_stream_handle(stream)),
                                    ctypes.byref(handle))
            _check(st, "mp_mesh_create")
        else:
            st = lib.mp_mesh_create_slab(_dptr(r_all), r_all.size - 1, int(slab[0]), int(slab[1]), _dptr(self.theta),
                                         self.shape[1], _dptr(self.phi), self.shape[2], self.l_max, float(G),
                                         PRECISIONS[precision], ctypes.c_void_p(_stream_handle(stream)),
                                         ctypes.byref(handle))
            _check(st, "mp_mesh_create_slab")
        self._h = handle
        self._rho = None
        self._phi = None

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.mp_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def cells(self) -> int:
        n_r, n_t, n_p = self.shape
        return n_r * n_t * n_p

    @property
    def n_moments(self) -> int:
        return (self.l_max + 1) ** 2

    def info(self) -> dict:
        inf = MeshInfo()
        _check(self._lib.mp_mesh_get_info(self._h, ctypes.byref(inf)), "mp_mesh_get_info")
        return {f: getattr(inf, f) for f, _ in MeshInfo._fields_}

    def set_stream(self, stream):
        _check(self._lib.mp_mesh_set_stream(self._h, ctypes.c_void_p(_stream_handle(stream))), "mp_mesh_set_stream")

    # -- bindings and solve
    def set_density(self, rho):
        _check(self._lib.mp_set_density(self._h, ctypes.c_void_p(_tensor_ptr(rho, self.cells, "rho"))),
               "mp_set_density")
        self._rho = rho

    def set_phi_output(self, phi):
        ptr = None if phi is None else _tensor_ptr(phi, self.cells, "phi")
        _check(self._lib.mp_set_phi_output(self._h, ctypes.c_void_p(ptr)), "mp_set_phi_output")
        self._phi = phi

    def solve(self):
        _check(self._lib.mp_solve(self._h), "mp_solve")

    def get_phi(self, out):
        _check(self._lib.mp_get_phi(self._h, ctypes.c_void_p(_tensor_ptr(out, self.cells, "out"))), "mp_get_phi")
        return out

    def get_moments(self, ang=None, mr=None, mi=None):
        n_r, K = self.shape[0], self.n_moments
        p = [None if t is None else ctypes.c_void_p(_tensor_ptr(t, s, nm))
             for t, s, nm in ((ang, n_r * K, "ang"), (mr, (n_r + 1) * K, "mr"), (mi, (n_r + 1) * K, "mi"))]
        _check(self._lib.mp_get_moments(self._h, *p), "mp_get_moments")

    def gravity_sources(self, phi=None, rho=None, v=None, grad=None, S=None, E=None):
        """Gravitational source terms (mp_gravity_sources): grad / S [3 * cells] and E
        [cells] CUDA float64 tensors (any may be None); phi / rho None: the last solve's
        potential / the bound density; v [3 * cells] contravariant velocity."""
        n = self.cells
        args = [None if t is None else ctypes.c_void_p(_tensor_ptr(t, size, name))
                for t, size, name in ((phi, n, "phi"), (rho, n, "rho"), (v, 3 * n, "v"),
                                      (grad, 3 * n, "grad"), (S, 3 * n, "S"), (E, n, "E"))]
        _check(self._lib.mp_gravity_sources(self._h, *args), "mp_gravity_sources")

    def coarsen(self, fields, n_fields: int = 1, field_stride: int | None = None):
        """Coarsening-block averaging in place (mp_coarsen) of n_fields float64 fields of
        cells values each, the f-th at offset f * field_stride in the CUDA tensor."""
        stride = self.cells if field_stride is None else int(field_stride)
        need = (n_fields - 1) * stride + self.cells if n_fields > 0 else 0
        import torch
        if not isinstance(fields, torch.Tensor) or not fields.is_cuda or fields.dtype != torch.float64:
            raise TypeError("fields must be a CUDA float64 tensor")
        if not fields.is_contiguous() or fields.numel() < need:
            raise ValueError(f"fields must be contiguous with at least {need} elements")
        _check(self._lib.mp_coarsen(self._h, ctypes.c_void_p(fields.data_ptr()), int(n_fields), stride), "mp_coarsen")

    def coarsening_factors(self):
        """(c_theta [n_r], c_phi [n_r][n_theta]) block sizes of the coarsening."""
        n_r, n_t = self.shape[0], self.shape[1]
        ct = np.zeros(n_r, dtype=np.int32)
        cp = np.zeros((n_r, n_t), dtype=np.int32)
        _check(self._lib.mp_coarsening_factors(self._h, ctypes.c_void_p(ct.ctypes.data),
                                               ctypes.c_void_p(cp.ctypes.data)), "mp_coarsening_factors")
        return ct, cp

    def moments_noalloc(self, rho, out):
        """Angular moments of rho into out [n_r * K_L] without device allocation
        (mp_moments_noalloc; for callers that cannot allocate at the point of use, such as
        loops with a fixed memory budget or plug-ins whose host owns every allocation)."""
        _check(self._lib.mp_moments_noalloc(self._h, ctypes.c_void_p(_tensor_ptr(rho, self.cells, "rho")),
                                            ctypes.c_void_p(_tensor_ptr(out, self.shape[0] * self.n_moments,
                                                                        "out"))),
               "mp_moments_noalloc")

    def synchronize(self):
        _check(self._lib.mp_mesh_synchronize(self._h), "mp_mesh_synchronize")

    def slab_moments(self, totals):
        """Moments of the bound density and this slab's radial totals into totals
        ([2 * K_L] CUDA float64: sums of W^R A and of W^I A over its shells)."""
        _check(self._lib.mp_slab_moments(self._h, ctypes.c_void_p(_tensor_ptr(totals, 2 * self.n_moments, "totals"))),
               "mp_slab_moments")

    def slab_potential(self, outer):
        """Potential of this slab given the other slabs' sums outer ([2 * K_L] CUDA float64)."""
        _check(self._lib.mp_slab_potential(self._h, ctypes.c_void_p(_tensor_ptr(outer, 2 * self.n_moments, "outer"))),
               "mp_slab_potential")

    def set_theta_engine(self, engine: str):
        """Engine of the theta stages on the split path: "auto", "tensor" (tcgen05 for the
        orders m >= 1) or "cuda" (every order on CUDA cores)."""
        code = {"auto": 0, "tensor": 1, "cuda": 2}[engine]
        _check(self._lib.mp_set_theta_engine(self._h, code), "mp_set_theta_engine")

    def set_wait_budget(self, cycles: int):
        """Budget of the device-side pipeline waits in SM clock cycles (0: the default)."""
        _check(self._lib.mp_set_wait_budget(self._h, int(cycles)), "mp_set_wait_budget")

    def solve_host(self, rho_host: np.ndarray, phi_host: np.ndarray):
        """End-to-end solve from host arrays (float64, rho layout; pinned is fastest)."""
        for a, nm in ((rho_host, "rho_host"), (phi_host, "phi_host")):
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != self.cells:
                raise ValueError(f"{nm} must be a contiguous float64 array of {self.cells} values")
        _check(self._lib.mp_solve_host(self._h, ctypes.c_void_p(rho_host.ctypes.data),
                                       ctypes.c_void_p(phi_host.ctypes.data)), "mp_solve_host")

    def solve_host_ptr(self, rho_ptr: int, phi_ptr: int):
        """End-to-end solve from host addresses (e.g. pinned torch tensors)."""
        _check(self._lib.mp_solve_host(self._h, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(phi_ptr)),
               "mp_solve_host")

    def solve_host_ptr_async(self, rho_ptr: int, phi_ptr: int):
        """Enqueue an end-to-end solve from pinned host addresses without waiting
        (mp_solve_host_async): consecutive calls overlap one download with the next
        upload.  The buffers stay in use until synchronize()."""
        _check(self._lib.mp_solve_host_async(self._h, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(phi_ptr)),
               "mp_solve_host_async")

    # -- per-kernel timing
    def profile(self, enable: bool = True):
        _check(self._lib.mp_profile_enable(self._h, int(enable)), "mp_profile_enable")

    def profile_read(self) -> dict:
        cap = 32
        names = (ctypes.c_char_p * cap)()
        launches = (ctypes.c_int * cap)()
        ms = (ctypes.c_double * cap)()
        n = ctypes.c_int(0)
        _check(self._lib.mp_profile_read(self._h, names, launches, ms, cap, ctypes.byref(n)), "mp_profile_read")
        return {names[k].decode(): {"launches": launches[k], "total_ms": ms[k]} for k in range(min(cap, n.value))}

    def autotune(self, cache_path: str | None = None):
        _check(self._lib.mp_autotune(self._h, cache_path.encode() if cache_path else None), "mp_autotune")


class Batch:
    """Several meshes solved together as one captured CUDA graph (mp_batch_*)."""

    def __init__(self, meshes):
        lib = load_library()
        self._lib = lib
        self.meshes = list(meshes)
        arr = (ctypes.c_void_p * len(self.meshes))(*[m._h.value for m in self.meshes])
        h = ctypes.c_void_p()
        _check(lib.mp_batch_create(arr, len(self.meshes), ctypes.byref(h)), "mp_batch_create")
        self._h = h

    def solve(self):
        _check(self._lib.mp_batch_solve(self._h), "mp_batch_solve")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_rates() -> dict:
    """Measured float64 FMA rate (TFLOP/s) and float64->float32 conversion rate of the current device."""
    lib = load_library()
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib.mp_probe_rates(ctypes.byref(a), ctypes.byref(b)), "mp_probe_rates")
    return {"fp64_tflops": a.value, "cvt_f64_f32_per_s": b.value}


def status_string(code: int) -> str:
    return load_library().mp_status_string(code).decode()


def version() -> int:
    return load_library().mp_version()
