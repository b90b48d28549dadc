"""GB300 matrix-free shifted boundary method (SBM) operator.

Thin Python binding of the C ABI in ``include/sbm.h`` (``libsbm.so``, built
in-tree by ``paper_2507_17053_gb300._build.build()``).  The functions here
only marshal arguments: every step of the operator runs in the library's CUDA
kernels.  PyTorch tensors are accepted for device and host buffers; streams
are ``torch.cuda.Stream`` objects (default: the current stream).

There is no CPU fallback: if the library cannot be loaded, every entry point
raises.
"""
from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsbm.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "sbm.h")

SBM_OK = 0
STATUS = {
    0: "SBM_OK", 1: "SBM_ERR_ARG", 2: "SBM_ERR_OOM", 3: "SBM_ERR_CUDA",
    4: "SBM_ERR_EMPTY_DOMAIN", 5: "SBM_ERR_NOT_CONVERGED", 6: "SBM_ERR_TIMEOUT",
    7: "SBM_ERR_STATE", 8: "SBM_ERR_UNSUPPORTED", 9: "SBM_ERR_GEOMETRY",
}
GEOM_KIND = {"ball": 0, "ellipsoid": 1, "torus": 2, "box": 3, "balls": 4}
EXTENSION = {"exact": 0, "taylor1": 1}
ACTIVITY = {"centre": 0, "volume": 1}


class SbmError(RuntimeError):
    def __init__(self, status: int, func: str, detail: str):
        super().__init__(f"{func}: {STATUS.get(status, status)} ({detail})")
        self.status = status


class sbm_desc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("degree", ctypes.c_int),
        ("cells_per_side", ctypes.c_int),
        ("dg", ctypes.c_int),
        ("geom_kind", ctypes.c_int),
        ("geom", ctypes.c_double * 16),
        ("pen_shift", ctypes.c_double),
        ("pen_interior", ctypes.c_double),
        ("extension", ctypes.c_int),
        ("nballs", ctypes.c_int),
        ("balls", ctypes.c_void_p),
        ("activity", ctypes.c_int),
        ("vf_threshold", ctypes.c_double),
    ]


_c_i64p = ctypes.POINTER(ctypes.c_int64)
_SIGS = {
    "sbm_create": (ctypes.c_int, [ctypes.POINTER(sbm_desc), ctypes.POINTER(ctypes.c_void_p)]),
    "sbm_create_gpu": (ctypes.c_int, [ctypes.POINTER(sbm_desc), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "sbm_setup_face_data": (ctypes.c_int, [ctypes.c_void_p]),
    "sbm_destroy": (None, [ctypes.c_void_p]),
    "sbm_sizes": (ctypes.c_int, [ctypes.c_void_p, _c_i64p, _c_i64p, _c_i64p, _c_i64p]),
    "sbm_export_geometry": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "sbm_apply_f64": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "sbm_apply_f64_host": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "sbm_apply_f64_noalloc": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "sbm_diagonal": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "sbm_apply_f32": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p]),
    "sbm_cg": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                        ctypes.POINTER(ctypes.c_int),
                                                        ctypes.POINTER(ctypes.c_double),
                                                        ctypes.c_void_p]),
    "sbm_gmres": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_double, ctypes.c_int,
                                                           ctypes.c_int,
                                                           ctypes.POINTER(ctypes.c_int),
                                                           ctypes.POINTER(ctypes.c_double),
                                                           ctypes.c_void_p]),
    "sbm_bicgstab": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_double, ctypes.c_int,
                                                              ctypes.POINTER(ctypes.c_int),
                                                              ctypes.POINTER(ctypes.c_double),
                                                              ctypes.c_void_p]),
    "sbm_bicgstab_f32": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_double, ctypes.c_int,
                                                                  ctypes.c_int,
                                                                  ctypes.POINTER(ctypes.c_int),
                                                                  ctypes.POINTER(ctypes.c_double),
                                                                  ctypes.c_void_p]),
    "sbm_solve_ir": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_double, ctypes.c_int,
                                                              ctypes.c_int, ctypes.c_double,
                                                              ctypes.c_int, ctypes.c_int,
                                                              ctypes.c_int,
                                                              ctypes.POINTER(ctypes.c_int),
                                                              ctypes.POINTER(ctypes.c_int),
                                                              ctypes.POINTER(ctypes.c_double),
                                                              ctypes.c_void_p]),
    "sbm_bicgstab_mixed": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_double, ctypes.c_int,
                                                                    ctypes.c_int,
                                                                    ctypes.POINTER(ctypes.c_int),
                                                                    ctypes.POINTER(ctypes.c_int),
                                                                    ctypes.POINTER(ctypes.c_double),
                                                                    ctypes.c_void_p]),
    "sbm_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "sbm_rhs_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "sbm_interpolate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "sbm_batch_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "sbm_batch_apply_f32": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "sbm_batch_apply_f64": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "sbm_batch_tile_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]),
    "sbm_batch_set_tile_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "sbm_batch_destroy": (None, [ctypes.c_void_p]),
    "sbm_batch_knobs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "sbm_batch_device_status": (ctypes.c_int, [ctypes.c_void_p]),
    "sbm_batch_set_knobs": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 5),
    "sbm_batch_selftest_timeout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sbm_batch_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                       ctypes.c_void_p]),
    "sbm_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "sbm_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _c_i64p]),
    "sbm_device_status": (ctypes.c_int, [ctypes.c_void_p]),
    "sbm_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]),
    "sbm_set_tile_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "sbm_set_ordered_stores": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "sbm_ordered_stores": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
    "sbm_selftest_timeout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sbm_peak_probe": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.c_void_p]),
    "sbm_fill_random": (ctypes.c_int, [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_int, ctypes.c_void_p]),
    "sbm_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sbm_last_error_detail": (ctypes.c_char_p, []),
}

_lib = None


def header_functions() -> list[str]:
    """Names of every function declared in include/sbm.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sbm_[a-z0-9_]+)\s*\(", text)))


def lib() -> ctypes.CDLL:
    """Load libsbm.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not built; run paper_2507_17053_gb300._build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, func: str):
    if status != SBM_OK:
        detail = lib().sbm_last_error_detail().decode()
        raise SbmError(status, func, detail)


def _ptr(t) -> int:
    """Raw data pointer of a tensor/ndarray (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data            # numpy


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_desc(dim, degree, cells, kind, geom, dg=False, pen_shift=10.0,
              pen_interior=1.0, extension="exact", activity="centre",
              vf_threshold=0.5) -> sbm_desc:
    d = sbm_desc()
    d.dim, d.degree, d.cells_per_side, d.dg = dim, degree, cells, int(bool(dg))
    d.geom_kind = GEOM_KIND[kind] if isinstance(kind, str) else int(kind)
    g = list(geom)
    if d.geom_kind == GEOM_KIND["balls"]:
        # the balls travel in a separate host array (kept alive with the desc)
        arr = (ctypes.c_double * len(g))(*[float(v) for v in g])
        d._balls_ref = arr
        d.nballs = len(g) // (dim + 1)
        d.balls = ctypes.cast(arr, ctypes.c_void_p)
        g = []
    if len(g) > 16:
        raise ValueError("at most 16 geometry parameters")
    for i, v in enumerate(g):
        d.geom[i] = float(v)
    d.pen_shift, d.pen_interior = float(pen_shift), float(pen_interior)
    d.extension = EXTENSION[extension] if isinstance(extension, str) else int(extension)
    d.activity = ACTIVITY[activity] if isinstance(activity, str) else int(activity)
    d.vf_threshold = float(vf_threshold)
    return d


# ---- entry points with the C names ------------------------------------------

def sbm_create(desc: sbm_desc) -> int:
    h = ctypes.c_void_p()
    _check(lib().sbm_create(ctypes.byref(desc), ctypes.byref(h)), "sbm_create")
    return h.value


def sbm_create_gpu(desc: sbm_desc, device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().sbm_create_gpu(ctypes.byref(desc), int(device), ctypes.byref(h)),
           "sbm_create_gpu")
    return h.value


def sbm_setup_face_data(handle: int) -> None:
    _check(lib().sbm_setup_face_data(handle), "sbm_setup_face_data")


def sbm_destroy(handle: int) -> None:
    lib().sbm_destroy(handle)


def sbm_sizes(handle: int) -> dict:
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().sbm_sizes(handle, *[ctypes.byref(x) for x in v]), "sbm_sizes")
    return dict(n_dofs=v[0].value, n_cells=v[1].value, n_sfaces=v[2].value, n_ifaces=v[3].value)


def sbm_export_geometry(handle: int, cells=None, sfaces=None, face_x=None) -> None:
    _check(lib().sbm_export_geometry(handle, _ptr(cells), _ptr(sfaces), _ptr(face_x)),
           "sbm_export_geometry")


def sbm_apply_f64(handle: int, x, y, stream=None) -> None:
    _check(lib().sbm_apply_f64(handle, _ptr(x), _ptr(y), _stream(stream)), "sbm_apply_f64")


def sbm_apply_f64_host(handle: int, x_host, y_host, stream=None) -> None:
    _check(lib().sbm_apply_f64_host(handle, _ptr(x_host), _ptr(y_host), _stream(stream)),
           "sbm_apply_f64_host")


def sbm_apply_f64_noalloc(handle: int, x, y, stream=None) -> None:
    _check(lib().sbm_apply_f64_noalloc(handle, _ptr(x), _ptr(y), _stream(stream)),
           "sbm_apply_f64_noalloc")


def sbm_diagonal(handle: int, diag, stream=None) -> None:
    _check(lib().sbm_diagonal(handle, _ptr(diag), _stream(stream)), "sbm_diagonal")


FACE_MODE = {"fp32": 0, "tf32": 1, "bf16": 2}
PRECOND = {"none": 0, "jacobi": 1}
INNER = {"gmres": 0, "bicgstab": 1, "bicgstab_mixed": 2}
BATCH_SOLVE = {"fp64": 0, "mixed": 1}


def sbm_apply_f32(handle: int, x, y, face_mode=0, stream=None) -> None:
    _check(lib().sbm_apply_f32(handle, _ptr(x), _ptr(y), int(face_mode), _stream(stream)),
           "sbm_apply_f32")


def _solve_call(name, status, it, rr, raise_not_converged):
    if status == 5 and not raise_not_converged:
        return it.value, rr.value, False
    _check(status, name)
    return it.value, rr.value, True


def sbm_cg(handle: int, b, x, rtol=1e-10, maxit=10000, precond=0, stream=None,
           raise_not_converged=False):
    it, rr = ctypes.c_int(), ctypes.c_double()
    st = lib().sbm_cg(handle, _ptr(b), _ptr(x), rtol, maxit, int(precond), ctypes.byref(it),
                      ctypes.byref(rr), _stream(stream))
    return _solve_call("sbm_cg", st, it, rr, raise_not_converged)


def sbm_gmres(handle: int, b, x, rtol=1e-10, maxit=10000, restart=100, stream=None,
              raise_not_converged=False):
    it, rr = ctypes.c_int(), ctypes.c_double()
    st = lib().sbm_gmres(handle, _ptr(b), _ptr(x), rtol, maxit, restart, ctypes.byref(it),
                         ctypes.byref(rr), _stream(stream))
    return _solve_call("sbm_gmres", st, it, rr, raise_not_converged)


def sbm_bicgstab(handle: int, b, x, rtol=1e-10, maxit=10000, stream=None,
                 raise_not_converged=False):
    it, rr = ctypes.c_int(), ctypes.c_double()
    st = lib().sbm_bicgstab(handle, _ptr(b), _ptr(x), rtol, maxit, ctypes.byref(it),
                            ctypes.byref(rr), _stream(stream))
    return _solve_call("sbm_bicgstab", st, it, rr, raise_not_converged)


def sbm_bicgstab_f32(handle: int, b, x, rtol=1e-5, maxit=10000, face_mode=0, stream=None,
                     raise_not_converged=False):
    it, rr = ctypes.c_int(), ctypes.c_double()
    st = lib().sbm_bicgstab_f32(handle, _ptr(b), _ptr(x), rtol, maxit, int(face_mode),
                                ctypes.byref(it), ctypes.byref(rr), _stream(stream))
    return _solve_call("sbm_bicgstab_f32", st, it, rr, raise_not_converged)


def sbm_bicgstab_mixed(handle: int, b, x, rtol=1e-10, maxit=20000, face_mode=0, stream=None,
                       raise_not_converged=False):
    """Returns (iterations, true relative residual, converged, reliable updates)."""
    it, rep, rr = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    st = lib().sbm_bicgstab_mixed(handle, _ptr(b), _ptr(x), rtol, maxit, int(face_mode),
                                  ctypes.byref(it), ctypes.byref(rep), ctypes.byref(rr),
                                  _stream(stream))
    return _solve_call("sbm_bicgstab_mixed", st, it, rr, raise_not_converged) + (rep.value,)


def sbm_solve_ir(handle: int, b, x, rtol=1e-10, max_outer=30, restart=100, inner_rtol=1e-4,
                 inner_maxit=2000, face_mode=0, inner_solver=0, stream=None,
                 raise_not_converged=False):
    it, outer, rr = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    st = lib().sbm_solve_ir(handle, _ptr(b), _ptr(x), rtol, max_outer, restart, inner_rtol,
                            inner_maxit, int(face_mode), int(inner_solver), ctypes.byref(it),
                            ctypes.byref(outer), ctypes.byref(rr), _stream(stream))
    res = _solve_call("sbm_solve_ir", st, it, rr, raise_not_converged)
    return res + (outer.value,)


def sbm_rhs(handle: int, manufactured: int, b_host) -> None:
    _check(lib().sbm_rhs(handle, int(manufactured), _ptr(b_host)), "sbm_rhs")


def sbm_interpolate(handle: int, manufactured: int, u_host) -> None:
    _check(lib().sbm_interpolate(handle, int(manufactured), _ptr(u_host)), "sbm_interpolate")


def sbm_device_status(handle: int) -> None:
    _check(lib().sbm_device_status(handle), "sbm_device_status")


def sbm_autotune(handle: int) -> tuple[int, int]:
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().sbm_autotune(handle, ctypes.byref(a), ctypes.byref(b)), "sbm_autotune")
    return a.value, b.value


def sbm_set_tile_shape(handle: int, shape64=-1, shape32=-1) -> None:
    _check(lib().sbm_set_tile_shape(handle, int(shape64), int(shape32)), "sbm_set_tile_shape")


def sbm_set_ordered_stores(handle: int, ordered64=-1, ordered32=-1) -> None:
    _check(lib().sbm_set_ordered_stores(handle, int(ordered64), int(ordered32)),
           "sbm_set_ordered_stores")


def sbm_ordered_stores(handle: int) -> tuple[int, int]:
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().sbm_ordered_stores(handle, ctypes.byref(a), ctypes.byref(b)),
           "sbm_ordered_stores")
    return a.value, b.value


def sbm_selftest_timeout(handle: int, stream=None) -> None:
    _check(lib().sbm_selftest_timeout(handle, _stream(stream)), "sbm_selftest_timeout")


def sbm_profile_enable(handle: int, on: bool) -> None:
    _check(lib().sbm_profile_enable(handle, int(bool(on))), "sbm_profile_enable")


def sbm_peak_probe(precision: int = 64, stream=None) -> float:
    """Measured FMA rate of the current GPU: G FMA thread-operations/s."""
    v = ctypes.c_double()
    _check(lib().sbm_peak_probe(precision, ctypes.byref(v), _stream(stream)), "sbm_peak_probe")
    return v.value


DIST = {"uniform": 0, "normal": 1}


def sbm_fill_random(n: int, seed: int, dist="uniform", offset: int = 0):
    """The library's seeded input generator: a numpy float64 array of n
    values (U(-1,1) or N(0,1)) from stream ``seed`` starting at ``offset``."""
    import numpy as np
    out = np.empty(n, dtype=np.float64)
    _check(lib().sbm_fill_random(n, seed & 0xFFFFFFFFFFFFFFFF, offset, DIST.get(dist, -1),
                                 out.ctypes.data), "sbm_fill_random")
    return out


def sbm_profile_read(handle: int) -> tuple[list, int]:
    """([face_ms, cell_ms, assembly_ms] summed since the last read, kernel launches)."""
    ms, n = (ctypes.c_double * 3)(), ctypes.c_int64()
    _check(lib().sbm_profile_read(handle, ms, ctypes.byref(n)), "sbm_profile_read")
    return list(ms), n.value


class Batch:
    """Owning wrapper around an sbm_batch (the problems must outlive it)."""

    def __init__(self, problems, nrhs, autotune=True, tensor_cores=False):
        self.problems = list(problems)
        self.nrhs = nrhs
        arr = (ctypes.c_void_p * len(self.problems))(*[p.handle for p in self.problems])
        h = ctypes.c_void_p()
        flags = (1 if autotune else 0) | (2 if tensor_cores else 0)
        _check(lib().sbm_batch_create(arr, len(self.problems), nrhs, flags, ctypes.byref(h)),
               "sbm_batch_create")
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            lib().sbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, xs, ys, stream=None):
        """ys[k] = A_k xs[k] (tensors of nrhs * n_dofs_k, float32 or float64)."""
        import torch
        n = len(self.problems)
        xa = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        ya = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
        for p, x, y in zip(self.problems, xs, ys):
            if x.numel() != p.n_dofs * self.nrhs or y.numel() != x.numel() or x.dtype != y.dtype:
                raise ValueError("batch vector has the wrong size or dtype")
        if xs[0].dtype == torch.float32:
            _check(lib().sbm_batch_apply_f32(self.handle, xa, ya, _stream(stream)),
                   "sbm_batch_apply_f32")
        else:
            _check(lib().sbm_batch_apply_f64(self.handle, xa, ya, _stream(stream)),
                   "sbm_batch_apply_f64")
        return ys

    def solve(self, bs, xs, mode="mixed", rtol=1e-10, maxit=None, inner_rtol=1e-2,
              inner_maxit=300, stream=None, check=True):
        """Solve A_k xs[k] = bs[k] for every problem and right-hand side
        (float64 tensors of nrhs * n_dofs_k).  Returns (status, iters,
        relres, outer): per-system BiCGStab iterations and true relative
        residuals, indexed k * nrhs + r; raises SbmError on failure unless
        check is False (then status may be SBM_ERR_NOT_CONVERGED)."""
        import numpy as np
        import torch
        n = len(self.problems)
        for p, b, x in zip(self.problems, bs, xs):
            if (b.numel() != p.n_dofs * self.nrhs or x.numel() != b.numel()
                    or b.dtype != torch.float64 or x.dtype != torch.float64):
                raise ValueError("batch vector has the wrong size or dtype")
        if maxit is None:
            maxit = 20000 if mode == "fp64" else 50
        ba = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
        xa = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        nsys = n * self.nrhs
        iters = np.zeros(nsys, dtype=np.int32)
        relres = np.zeros(nsys, dtype=np.float64)
        outer = ctypes.c_int()
        st = lib().sbm_batch_solve(self.handle, ba, xa, BATCH_SOLVE[mode], rtol, maxit,
                                   inner_rtol, inner_maxit, iters.ctypes.data,
                                   relres.ctypes.data, ctypes.byref(outer), _stream(stream))
        if check:
            _check(st, "sbm_batch_solve")
        return st, iters, relres, outer.value

    def tile_shape(self, k):
        v = ctypes.c_int()
        _check(lib().sbm_batch_tile_shape(self.handle, k, ctypes.byref(v)), "sbm_batch_tile_shape")
        return v.value

    def set_tile_shape(self, k, variant):
        _check(lib().sbm_batch_set_tile_shape(self.handle, k, variant), "sbm_batch_set_tile_shape")

    def knobs(self, precision, degree):
        """The autotuner's choice for one degree: dict with tile_shape,
        face_batch, tensor_cores and ms (the timed options, index shape +
        2 face_batch + 4 tensor_cores for tile shapes 0 and 1, 8 +
        face_batch for tile shape 3; None where not timed)."""
        v, f, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_float * 10)()
        _check(lib().sbm_batch_knobs(self.handle, precision, degree, ctypes.byref(v),
                                     ctypes.byref(f), ctypes.byref(t), ms), "sbm_batch_knobs")
        return {"tile_shape": v.value, "face_batch": f.value, "tensor_cores": t.value,
                "ms": [float(m) if m >= 0 else None for m in ms]}

    def set_knobs(self, precision, degree, tile_shape=0, face_batch=0, tensor_cores=0):
        _check(lib().sbm_batch_set_knobs(self.handle, precision, degree, tile_shape, face_batch,
                                         tensor_cores), "sbm_batch_set_knobs")

    def device_status(self):
        """Raises SbmError if a bounded wait of an earlier batched apply expired."""
        _check(lib().sbm_batch_device_status(self.handle), "sbm_batch_device_status")

    def selftest_timeout(self, stream=None):
        _check(lib().sbm_batch_selftest_timeout(self.handle, _stream(stream)),
               "sbm_batch_selftest_timeout")


def _current_device() -> int:
    import torch
    return torch.cuda.current_device()


class Problem:
    """Owning wrapper around an sbm_problem handle."""

    def __init__(self, dim, degree, cells, kind, geom, dg=False, pen_shift=10.0,
                 pen_interior=1.0, device=True, extension="exact", activity="centre",
                 vf_threshold=0.5, gpu_setup=False):
        self.desc = make_desc(dim, degree, cells, kind, geom, dg, pen_shift, pen_interior,
                              extension, activity, vf_threshold)
        self.dim, self.degree, self.dg = dim, degree, bool(dg)
        # gpu_setup: the geometry stage on the current CUDA device (same result)
        self.handle = (sbm_create_gpu(self.desc, _current_device()) if gpu_setup
                       else sbm_create(self.desc))
        if device:
            sbm_setup_face_data(self.handle)
        s = sbm_sizes(self.handle)
        self.n_dofs, self.n_cells = s["n_dofs"], s["n_cells"]
        self.n_sfaces, self.n_ifaces = s["n_sfaces"], s["n_ifaces"]

    @classmethod
    def from_workload(cls, w, device=True, gpu_setup=False):
        return cls(w.dim, w.degree, w.cells, w.kind, w.geom, dg=w.dg, pen_shift=w.pen_shift,
                   pen_interior=w.pen_interior, device=device, gpu_setup=gpu_setup,
                   extension=getattr(w, "extension", "exact"),
                   activity=getattr(w, "activity", "centre"),
                   vf_threshold=getattr(w, "vf_threshold", 0.5))

    def close(self):
        if getattr(self, "handle", None):
            sbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def geometry(self):
        import numpy as np
        n = self.degree + 1
        Q = n ** (self.dim - 1)
        cells = np.zeros((self.n_cells, self.dim), dtype=np.int32)
        sfaces = np.zeros((self.n_sfaces, 3), dtype=np.int32)
        fx = np.zeros((self.n_sfaces, Q, self.dim), dtype=np.float64)
        sbm_export_geometry(self.handle, cells, sfaces, fx)
        return cells, sfaces, fx

    def apply_f64(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        _expect(x, torch.float64, self.n_dofs)
        _expect(y, torch.float64, self.n_dofs)
        sbm_apply_f64(self.handle, x, y, stream)
        return y

    def rhs(self, manufactured=0):
        import numpy as np
        b = np.zeros(self.n_dofs)
        sbm_rhs(self.handle, manufactured, b)
        return b

    def rhs_device(self, manufactured=0, out=None, stream=None):
        """The right-hand side as a device float64 tensor (sbm_rhs_device)."""
        import torch
        if out is None:
            out = torch.empty(self.n_dofs, dtype=torch.float64, device="cuda")
        _expect(out, torch.float64, self.n_dofs)
        _check(lib().sbm_rhs_device(self.handle, manufactured, _ptr(out), _stream(stream)),
               "sbm_rhs_device")
        return out

    def interpolate(self, manufactured=0):
        import numpy as np
        u = np.zeros(self.n_dofs)
        sbm_interpolate(self.handle, manufactured, u)
        return u

    def diagonal(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.n_dofs, dtype=torch.float64, device="cuda")
        _expect(out, torch.float64, self.n_dofs)
        sbm_diagonal(self.handle, out, stream)
        return out

    def apply_f32(self, x, y=None, face_mode=0, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        _expect(x, torch.float32, self.n_dofs)
        _expect(y, torch.float32, self.n_dofs)
        sbm_apply_f32(self.handle, x, y, FACE_MODE.get(face_mode, face_mode), stream)
        return y

    def apply_f64_host(self, x_host, y_host=None, stream=None):
        import numpy as np
        if y_host is None:
            y_host = np.empty(self.n_dofs, dtype=np.float64)
        sbm_apply_f64_host(self.handle, x_host, y_host, stream)
        return y_host


def _expect(t, dtype, n):
    if t.dtype != dtype or t.numel() != n or not t.is_contiguous() or not t.is_cuda:
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor of {n} elements")
