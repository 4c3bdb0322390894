"""ctypes binding of the C ABI in ``include/fea.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls.  Device arrays
are torch CUDA tensors (PyTorch supplies device memory and streams); all the
arithmetic runs in the CUDA library ``_build/libfea.so``.  If that library is
missing the import of any call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libfea.so")

FEA_TET4, FEA_HEX8, FEA_HEX27, FEA_PEN6, FEA_PYR5 = 0, 1, 2, 3, 4
FEA_F64_PLAIN, FEA_F32_FUSED = 0, 1
FEA_TERM_MASS, FEA_TERM_CONV, FEA_TERM_DIFF, FEA_TERM_REAC, FEA_TERM_SUPG, FEA_TERM_ALL = 1, 2, 4, 8, 16, 31
FEA_SCATTER_AUTO, FEA_SCATTER_ATOMIC, FEA_SCATTER_ROWOWNED, FEA_SCATTER_GATHER = 0, 1, 2, 3
FEA_CONTRACT_AUTO, FEA_CONTRACT_CUDA, FEA_CONTRACT_TC_BF16X3, FEA_CONTRACT_TC_TF32X3 = 0, 1, 2, 3
FEA_MAP_AUTO, FEA_MAP_TYPE_KERNEL, FEA_MAP_WARP_PER_ELEMENT, FEA_MAP_TWO_THREADS_PER_ITEM = 0, 1, 2, 3
STATUS = {0: "FEA_OK", 1: "FEA_ERR_ARG", 2: "FEA_ERR_RANGE", 3: "FEA_ERR_DUP_NODE", 4: "FEA_ERR_INVERTED",
          5: "FEA_ERR_TOO_LARGE", 6: "FEA_ERR_OOM", 7: "FEA_ERR_CUDA", 8: "FEA_ERR_TIMEOUT", 9: "FEA_ERR_STATE"}
NEN = {FEA_TET4: 4, FEA_HEX8: 8, FEA_HEX27: 27, FEA_PEN6: 6, FEA_PYR5: 5}

# Every symbol include/fea.h declares (checked by the tests).
EXPORTS = ["fea_default_opts", "fea_mesh_create", "fea_mesh_create_mixed", "fea_mesh_destroy", "fea_mesh_set_stream", "fea_sync",
           "fea_pattern_build", "fea_pattern_get", "fea_pattern_destroy", "fea_assemble", "fea_residual",
           "fea_explicit_step",
           "fea_assemble_host",
           "fea_pack_plan", "fea_csr_rowptr_noalloc", "fea_update_fields", "fea_graph_capture_steps",
           "fea_graph_launch", "fea_graph_destroy", "fea_spmv", "fea_pcg", "fea_tuned_strategy", "fea_tuned_config",
           "fea_tune_candidates", "fea_cancel_rows", "fea_last_error",
           "fea_kernel_launches", "fea_version"]


class FeaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class fea_assemble_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("terms", C.c_int32), ("scatter", C.c_int32), ("accumulate", C.c_int32),
                ("kappa_threshold", C.c_double), ("event_begin", C.c_void_p), ("event_end", C.c_void_p),
                ("eq_groups", C.c_int32), ("cancel_check", C.c_int32), ("host_parts", C.c_int32),
                ("contraction", C.c_int32), ("mapping", C.c_int32), ("elems_per_cta", C.c_int32),
                ("reserved", C.c_int32 * 2)]


class fea_tuning(C.Structure):
    _fields_ = [("scatter", C.c_int32), ("eq_groups", C.c_int32), ("mapping", C.c_int32),
                ("elems_per_cta", C.c_int32), ("contraction", C.c_int32), ("from_cache", C.c_int32),
                ("ms", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib(path: str = LIB_PATH):
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise FileNotFoundError(f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; "
                                    f"g.build()')")
        L = C.CDLL(path)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        L.fea_default_opts.argtypes = [C.POINTER(fea_assemble_opts)]
        L.fea_mesh_create.argtypes = [vp, i64, vp, i64, C.c_int, vp, C.POINTER(vp)]
        L.fea_mesh_create_mixed.argtypes = [vp, i64, i32, vp, vp, vp, vp, C.POINTER(vp)]
        L.fea_mesh_destroy.argtypes = [vp]
        L.fea_mesh_set_stream.argtypes = [vp, vp]
        L.fea_sync.argtypes = [vp]
        L.fea_pattern_build.argtypes = [vp, C.POINTER(vp)]
        L.fea_pattern_get.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(i64)]
        L.fea_pattern_destroy.argtypes = [vp]
        L.fea_assemble.argtypes = [vp, vp, vp, vp, vp, vp, dbl, i32, C.POINTER(fea_assemble_opts), vp, vp]
        L.fea_assemble_host.argtypes = [vp, vp, vp, vp, vp, vp, dbl, i32, C.POINTER(fea_assemble_opts), vp, vp]
        L.fea_residual.argtypes = [vp, vp, vp, vp, vp, vp, vp, dbl, i32, C.POINTER(fea_assemble_opts), vp]
        L.fea_explicit_step.argtypes = [vp, vp, vp, vp, vp, vp, dbl, i32, i32, C.POINTER(fea_assemble_opts)]
        L.fea_pack_plan.argtypes = [vp, i32, i32, vp, vp]
        L.fea_csr_rowptr_noalloc.argtypes = [vp, i64, vp, vp]
        L.fea_update_fields.argtypes = [vp, vp, i32, vp]
        L.fea_graph_capture_steps.argtypes = [vp, vp, vp, vp, vp, vp, dbl, i32, C.POINTER(fea_assemble_opts), vp, vp,
                                              vp, i32, C.POINTER(vp)]
        L.fea_graph_launch.argtypes = [vp]
        L.fea_tuned_strategy.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32)]
        L.fea_tuned_config.argtypes = [vp, i32, i32, C.POINTER(fea_tuning)]
        L.fea_tune_candidates.argtypes = [vp, i32, i32, vp, i32, C.POINTER(i32)]
        L.fea_spmv.argtypes = [vp, vp, vp, vp, i32, i32, vp]
        L.fea_pcg.argtypes = [vp, vp, vp, vp, i32, i32, dbl, vp, vp, vp]
        L.fea_cancel_rows.argtypes = [vp, i32, C.POINTER(i64)]
        L.fea_graph_destroy.argtypes = [vp]
        L.fea_last_error.restype = C.c_char_p
        L.fea_version.restype = C.c_int32
        L.fea_kernel_launches.restype = C.c_int64
        for name in EXPORTS:
            if name not in ("fea_last_error", "fea_version", "fea_kernel_launches"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(code: int):
    if code != 0:
        raise FeaError(code, lib().fea_last_error().decode())


def _ptr(x) -> int | None:
    """Address of a torch tensor or numpy array (None passes NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def fea_default_opts(**kw) -> fea_assemble_opts:
    o = fea_assemble_opts()
    _check(lib().fea_default_opts(C.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def fea_mesh_create(coords, conn, elem_type: int, stream=None) -> C.c_void_p:
    """coords [N][3] float64 and conn [E][nen] int32, numpy (host) or torch CUDA tensors."""
    if isinstance(coords, np.ndarray):
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        conn = np.ascontiguousarray(conn, dtype=np.int32)
    else:
        assert coords.dtype.__str__() == "torch.float64" and conn.dtype.__str__() == "torch.int32"
        assert coords.is_contiguous() and conn.is_contiguous()
    out = C.c_void_p()
    _check(lib().fea_mesh_create(_ptr(coords), coords.shape[0], _ptr(conn), conn.shape[0], int(elem_type),
                                 _stream_ptr(stream), C.byref(out)))
    return out


def fea_mesh_create_mixed(coords, blocks, stream=None) -> C.c_void_p:
    """coords [N][3] float64 and blocks [(elem_type, conn [E_b][nen_b] int32), ...] (numpy or
    torch CUDA tensors); elements are numbered block by block."""
    if isinstance(coords, np.ndarray):
        coords = np.ascontiguousarray(coords, dtype=np.float64)
    conns = [np.ascontiguousarray(c, dtype=np.int32) if isinstance(c, np.ndarray) else c for _, c in blocks]
    nb = len(blocks)
    types = (C.c_int * nb)(*[int(t) for t, _ in blocks])
    ptrs = (C.c_void_p * nb)(*[_ptr(c) for c in conns])
    counts = (C.c_int64 * nb)(*[int(c.shape[0]) for c in conns])
    out = C.c_void_p()
    _check(lib().fea_mesh_create_mixed(_ptr(coords), coords.shape[0], nb, types, ptrs, counts, _stream_ptr(stream),
                                       C.byref(out)))
    return out


def fea_mesh_destroy(mesh):
    _check(lib().fea_mesh_destroy(mesh))


def fea_mesh_set_stream(mesh, stream):
    _check(lib().fea_mesh_set_stream(mesh, _stream_ptr(stream)))


def fea_sync(mesh):
    _check(lib().fea_sync(mesh))


def fea_pattern_build(mesh) -> C.c_void_p:
    out = C.c_void_p()
    _check(lib().fea_pattern_build(mesh, C.byref(out)))
    return out


def fea_pattern_get(pattern):
    """(rowptr, colind, pos, nnz): borrowed device addresses and the nnz."""
    r, c, p, n = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_int64()
    _check(lib().fea_pattern_get(pattern, C.byref(r), C.byref(c), C.byref(p), C.byref(n)))
    return r.value, c.value, p.value, n.value


def fea_pattern_destroy(pattern):
    _check(lib().fea_pattern_destroy(pattern))


def fea_assemble(mesh, pattern, velocity, diffusivity, reaction, phi_old, dt: float, n_eq: int, opts, values, rhs):
    """All arrays are torch CUDA tensors of the precision's dtype; enqueued on the mesh's stream."""
    _check(lib().fea_assemble(mesh, pattern, _ptr(velocity), _ptr(diffusivity), _ptr(reaction), _ptr(phi_old),
                              float(dt), int(n_eq), C.byref(opts) if opts is not None else None, _ptr(values),
                              _ptr(rhs)))


def fea_residual(mesh, pattern, velocity, diffusivity, reaction, phi_old, phi, dt: float, n_eq: int, opts, r):
    """Matrix-free residual r = b - A phi (torch CUDA tensors of the precision's dtype)."""
    _check(lib().fea_residual(mesh, pattern, _ptr(velocity), _ptr(diffusivity), _ptr(reaction), _ptr(phi_old),
                              _ptr(phi), float(dt), int(n_eq), C.byref(opts) if opts is not None else None, _ptr(r)))


def fea_explicit_step(mesh, pattern, velocity, diffusivity, reaction, phi, dt: float, n_eq: int, stages: int = 3,
                      opts=None):
    """One explicit step (forward Euler or SSP-RK3) of M_L dphi/dt = -A phi, phi advanced in place
    (device tensors of the precision in opts)."""
    _check(lib().fea_explicit_step(mesh, pattern, _ptr(velocity), _ptr(diffusivity), _ptr(reaction), _ptr(phi),
                                   float(dt), int(n_eq), int(stages), C.byref(opts) if opts is not None else None))


def fea_assemble_host(mesh, pattern, velocity, diffusivity, reaction, phi_old, dt: float, n_eq: int, opts, values,
                      rhs):
    """Host-array variant (numpy or pinned torch CPU tensors); waits for completion."""
    _check(lib().fea_assemble_host(mesh, pattern, _ptr(velocity), _ptr(diffusivity), _ptr(reaction), _ptr(phi_old),
                                   float(dt), int(n_eq), C.byref(opts) if opts is not None else None, _ptr(values),
                                   _ptr(rhs)))


def fea_pack_plan(count_by_type, vector_size: int):
    counts = np.ascontiguousarray(count_by_type, dtype=np.int64)
    packs = np.zeros_like(counts)
    pads = np.zeros_like(counts)
    _check(lib().fea_pack_plan(counts.ctypes.data, counts.size, int(vector_size), packs.ctypes.data,
                               pads.ctypes.data))
    return packs, pads


def fea_csr_rowptr_noalloc(counts, n: int, rowptr, stream=None):
    """rowptr[n+1] (int64 CUDA tensor) from counts[n] (int32 CUDA tensor) without device allocation."""
    _check(lib().fea_csr_rowptr_noalloc(_ptr(counts), int(n), _ptr(rowptr), _stream_ptr(stream)))


def fea_update_fields(mesh, phi, n_eq: int, params):
    """phi [n_eq][N] float32 CUDA tensor, updated in place; params [n_eq][5] float32 CUDA tensor."""
    _check(lib().fea_update_fields(mesh, _ptr(phi), int(n_eq), _ptr(params)))


def fea_graph_capture_steps(mesh, pattern, velocity, diffusivity, reaction, phi_old, dt: float, n_eq: int, opts,
                            values, rhs, params, n_steps: int) -> C.c_void_p:
    """Records n_steps (assemble, update) steps in one CUDA graph; params [n_steps][n_eq][5] float32."""
    out = C.c_void_p()
    _check(lib().fea_graph_capture_steps(mesh, pattern, _ptr(velocity), _ptr(diffusivity), _ptr(reaction),
                                         _ptr(phi_old), float(dt), int(n_eq),
                                         C.byref(opts) if opts is not None else None, _ptr(values), _ptr(rhs),
                                         _ptr(params), int(n_steps), C.byref(out)))
    return out


def fea_graph_launch(graph):
    _check(lib().fea_graph_launch(graph))


def fea_graph_destroy(graph):
    _check(lib().fea_graph_destroy(graph))


def fea_spmv(pattern, values, x, y, n_eq: int, accumulate: int = 0, stream=None):
    """y[q] = A_q x[q] for all equations (float32 CUDA tensors [n_eq][nnz], [n_eq][N])."""
    _check(lib().fea_spmv(pattern, _ptr(values), _ptr(x), _ptr(y), int(n_eq), int(accumulate), _stream_ptr(stream)))


def fea_pcg(pattern, values, b, x, n_eq: int, max_iter: int, rtol: float, stream=None):
    """Solves A_q x_q = b_q in place (float32 CUDA tensors); returns (iterations, relative residuals)
    per equation as numpy arrays."""
    iters = np.zeros(int(n_eq), dtype=np.int32)
    rel = np.zeros(int(n_eq), dtype=np.float64)
    _check(lib().fea_pcg(pattern, _ptr(values), _ptr(b), _ptr(x), int(n_eq), int(max_iter), float(rtol),
                         iters.ctypes.data, rel.ctypes.data, _stream_ptr(stream)))
    return iters, rel


def fea_tuned_strategy(pattern, n_eq: int):
    """(scatter, eq_groups) chosen by FEA_SCATTER_AUTO for this pattern and equation count."""
    s, g = C.c_int32(), C.c_int32()
    _check(lib().fea_tuned_strategy(pattern, int(n_eq), C.byref(s), C.byref(g)))
    return s.value, g.value


def fea_tuned_config(pattern, n_eq: int, terms: int = FEA_TERM_ALL) -> dict:
    """Every dimension FEA_SCATTER_AUTO chose for this pattern, equation count and term mask."""
    t = fea_tuning()
    _check(lib().fea_tuned_config(pattern, int(n_eq), int(terms), C.byref(t)))
    return t.as_dict()


def fea_tune_candidates(pattern, n_eq: int, terms: int = FEA_TERM_ALL) -> list:
    """The configurations FEA_SCATTER_AUTO may time, as dicts of fea_tuning fields."""
    n = C.c_int32()
    _check(lib().fea_tune_candidates(pattern, int(n_eq), int(terms), None, 0, C.byref(n)))
    arr = (fea_tuning * max(1, n.value))()
    _check(lib().fea_tune_candidates(pattern, int(n_eq), int(terms), arr, n.value, C.byref(n)))
    return [arr[i].as_dict() for i in range(n.value)]


def fea_cancel_rows(pattern, n_eq: int) -> int:
    """Number of rows the cancellation check flagged for this pattern and equation count."""
    n = C.c_int64()
    _check(lib().fea_cancel_rows(pattern, int(n_eq), C.byref(n)))
    return n.value


def fea_last_error() -> str:
    return lib().fea_last_error().decode()


def fea_kernel_launches() -> int:
    return lib().fea_kernel_launches()


def fea_version() -> int:
    return lib().fea_version()


# ------------------------------------------------------------------ device-array views

class _DevView:
    """Exposes a borrowed device buffer through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def pattern_tensors(pattern, n_node: int, n_elem: int, nen: int):
    """Copies of the pattern arrays as torch CUDA tensors: rowptr, colind, pos."""
    import torch
    r, c, p, nnz = fea_pattern_get(pattern)
    rowptr = torch.as_tensor(_DevView(r, (n_node + 1,), "<i8"), device="cuda").clone()
    colind = torch.as_tensor(_DevView(c, (max(nnz, 1),), "<i4"), device="cuda")[:nnz].clone()
    pos = torch.as_tensor(_DevView(p, (max(n_elem, 1), nen, nen), "<i4"), device="cuda")[:n_elem].clone()
    return rowptr, colind, pos
