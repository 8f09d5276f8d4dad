"""Python binding of libsgweno.so, the GB300 sparse-grid fifth-order WENO library.

Thin ctypes marshalling over the C ABI declared in include/sgweno.h; every function has
the C name.  All computation runs in the library's CUDA kernels: there is no CPU path, and
loading fails loudly if the library has not been built (``paper_2007_10196_gb300.build``).
PyTorch is optional plumbing: pass ``torch.cuda.current_stream().cuda_stream`` as
``cuda_stream`` and call :func:`use_torch_allocator` to route device memory through
PyTorch's caching allocator.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsgweno.so")
MAX_DIM = 6

# status codes
SG_OK, SG_ERR_ARG, SG_ERR_STATE, SG_ERR_NOMEM, SG_ERR_CUDA = 0, 1, 2, 3, 4
SG_ERR_NONFINITE, SG_ERR_TIMEOUT, SG_ERR_UNSUPPORTED = 5, 6, 7
SG_PDE_ADVECTION, SG_PDE_BURGERS, SG_PDE_VLASOV, SG_PDE_VLASOV_BOLTZMANN = 0, 1, 2, 3
SG_BC_PERIODIC, SG_BC_ZERO = 0, 1
SG_F64, SG_F32 = 0, 1
SG_PLAIN, SG_BATCHED = 0, 1
SG_WENO5, SG_LINEAR5 = 0, 1
SG_PROLONG_WENO5, SG_PROLONG_LAGRANGE5 = 0, 1
SG_DT_POW53, SG_DT_CFL = 0, 1
SG_STAGE_AUTO, SG_STAGE_TILED, SG_STAGE_SWEEP, SG_STAGE_SWEEP2 = 0, 1, 2, 3
SG_IC_SINE, SG_IC_LANDAU, SG_IC_RELAX = 0, 1, 2
SG_REDUCE_MASS, SG_REDUCE_ENERGY, SG_REDUCE_MIN, SG_REDUCE_MAX = 0, 1, 2, 3
SG_REDUCE_L1_EXACT, SG_REDUCE_LINF_EXACT, SG_REDUCE_FIELD_ENERGY = 4, 5, 6
SG_REDUCE_ENTROPY_H2, SG_REDUCE_ENTROPY_LOG = 7, 8
SG_WHICH_COMBINED, SG_WHICH_ALL_GRIDS = -1, -2

EXPORTED = [
    "sg_params_init", "sg_create", "sg_init", "sg_init_grid", "sg_init_grids", "sg_step",
    "sg_prolong_combine", "sg_read", "sg_reduce", "sg_num_grids", "sg_grid_info", "sg_time",
    "sg_batch_create", "sg_destroy", "sg_last_error", "sg_set_allocator", "sg_launch_count",
    "sg_set_profiling", "sg_profile", "sg_step_grid_noalloc", "sg_stage_config", "sg_read_points",
]
SG_NOALLOC_MAX_POINTS = 1048576
SG_PROF_STAGE = 0


class SgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("sg status %d: %s" % (status, message))
        self.status = status


class sg_params(C.Structure):
    _fields_ = [
        ("struct_size", C.c_size_t),
        ("lo", C.c_double * MAX_DIM), ("hi", C.c_double * MAX_DIM),
        ("bc", C.c_int * MAX_DIM), ("adv_speed", C.c_double * MAX_DIM),
        ("precision", C.c_int), ("exec", C.c_int), ("scheme", C.c_int), ("prolong", C.c_int),
        ("eps", C.c_double), ("dt_rule", C.c_int), ("dt_coef", C.c_double), ("cfl", C.c_double),
        ("cuda_stream", C.c_void_p), ("graph_steps", C.c_int), ("tile_points", C.c_int),
        ("combine_budget_gb", C.c_double), ("stage_kernel", C.c_int),
        ("theta", C.c_double), ("tau", C.c_double),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)

_lib = None


def build(force: bool = False) -> str:
    """Compiles libsgweno.so in-tree if any source is newer (paper_2007_10196_gb300/build.py)."""
    import importlib
    return importlib.import_module(__name__ + ".build").build(force=force)


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsgweno.so is not built (%s); run paper_2007_10196_gb300.build()" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    H = C.c_void_p
    st = C.c_int
    sig = {
        "sg_params_init": (st, [C.POINTER(sg_params)]),
        "sg_create": (st, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(sg_params), C.POINTER(H)]),
        "sg_init": (st, [H, C.c_int, C.POINTER(C.c_double), C.c_int]),
        "sg_init_grid": (st, [H, C.c_int, C.c_void_p, C.c_size_t]),
        "sg_init_grids": (st, [H, C.c_void_p, C.c_size_t]),
        "sg_step": (st, [H, C.c_double, C.c_long, C.POINTER(C.c_double)]),
        "sg_prolong_combine": (st, [H]),
        "sg_read": (st, [H, C.c_int, C.c_void_p, C.c_size_t]),
        "sg_reduce": (st, [H, C.c_int, C.c_int, C.POINTER(C.c_double)]),
        "sg_num_grids": (st, [H, C.POINTER(C.c_int)]),
        "sg_grid_info": (st, [H, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_long), C.POINTER(C.c_double)]),
        "sg_time": (st, [H, C.POINTER(C.c_double), C.POINTER(C.c_long)]),
        "sg_batch_create": (st, [C.POINTER(H), C.c_int, C.POINTER(H)]),
        "sg_destroy": (st, [H]),
        "sg_last_error": (C.c_char_p, []),
        "sg_set_allocator": (st, [ALLOC_FN, FREE_FN, C.c_void_p]),
        "sg_launch_count": (st, [H, C.POINTER(C.c_long)]),
        "sg_step_grid_noalloc": (st, [C.c_int, C.POINTER(C.c_long), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double), C.c_int,
                                      C.c_double, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
        "sg_set_profiling": (st, [H, C.c_int]),
        "sg_profile": (st, [H, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_long)]),
        "sg_stage_config": (st, [H, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "sg_read_points": (st, [H, C.c_int, C.POINTER(C.c_longlong), C.c_size_t, C.c_void_p, C.c_size_t]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != SG_OK:
        raise SgError(status, lib().sg_last_error().decode())


def sg_last_error() -> str:
    return lib().sg_last_error().decode()


def sg_params_init(**overrides) -> sg_params:
    p = sg_params()
    _check(lib().sg_params_init(C.byref(p)))
    for k, v in overrides.items():
        if k in ("lo", "hi", "adv_speed", "bc"):
            arr = getattr(p, k)
            vals = list(np.broadcast_to(np.asarray(v), (MAX_DIM,))) if np.ndim(v) == 0 else list(v)
            for i, x in enumerate(vals[:MAX_DIM]):
                arr[i] = int(x) if k == "bc" else float(x)
        else:
            setattr(p, k, v)
    return p


def sg_create(dim: int, root_cells: int, level: int, pde: int, params: sg_params | None = None):
    h = C.c_void_p()
    _check(lib().sg_create(dim, root_cells, level, pde, C.byref(params) if params is not None else None,
                           C.byref(h)))
    _PREC[h.value] = params.precision if params is not None else SG_F64
    return h


def sg_init(h, ic_kind: int, ic_params):
    arr = (C.c_double * len(ic_params))(*[float(x) for x in ic_params])
    _check(lib().sg_init(h, ic_kind, arr, len(ic_params)))


def _host_buffer(values, dtype):
    a = np.ascontiguousarray(values, dtype=dtype)
    return a, a.ctypes.data, a.nbytes


def _dtype(h) -> np.dtype:
    return np.dtype(np.float64) if _precision(h) == SG_F64 else np.dtype(np.float32)


_PREC = {}


def _precision(h) -> int:
    return _PREC.get(h.value, SG_F64)


def sg_init_grid(h, grid: int, values):
    """values: host array (numpy, or a CPU tensor's .numpy(); pinned memory works) of grid `grid`."""
    a, ptr, n = _host_buffer(values, _dtype(h))
    _check(lib().sg_init_grid(h, grid, ptr, n))


def sg_init_grids(h, values):
    a, ptr, n = _host_buffer(values, _dtype(h))
    _check(lib().sg_init_grids(h, ptr, n))


def sg_step(h, t_end: float, max_steps: int = (1 << 62)) -> float:
    t = C.c_double()
    _check(lib().sg_step(h, float(t_end), int(min(max_steps, (1 << 62))), C.byref(t)))
    return t.value


def sg_prolong_combine(h):
    _check(lib().sg_prolong_combine(h))


def sg_num_grids(h) -> int:
    n = C.c_int()
    _check(lib().sg_num_grids(h, C.byref(n)))
    return n.value


def sg_grid_info(h, g: int, dim: int):
    lev = (C.c_int * MAX_DIM)()
    shp = (C.c_long * MAX_DIM)()
    co = C.c_double()
    _check(lib().sg_grid_info(h, g, lev, shp, C.byref(co)))
    return tuple(lev[:dim]), tuple(shp[:dim]), co.value


def sg_read(h, which: int, out=None, count: int | None = None):
    """Copies grid `which` (or the combined solution, which = -1; all grids, -2) into `out`
    (a host numpy array, allocated if None, of `count` elements)."""
    dt = np.dtype(np.float64) if which == SG_WHICH_COMBINED else _dtype(h)
    if out is None:
        if count is None:
            raise ValueError("count is required when out is None")
        out = np.empty(count, dtype=dt)
    _check(lib().sg_read(h, which, out.ctypes.data, out.nbytes))
    return out


def sg_read_points(h, which: int, idx):
    """Values at flat indices `idx` of the combined solution (which = -1, doubles), of grid
    `which` or of all grids (-2), gathered on the device."""
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    dt = np.dtype(np.float64) if which == SG_WHICH_COMBINED else _dtype(h)
    out = np.empty(ix.size, dtype=dt)
    _check(lib().sg_read_points(h, which, ix.ctypes.data_as(C.POINTER(C.c_longlong)), ix.size,
                                out.ctypes.data, out.nbytes))
    return out


def sg_reduce(h, which: int, kind: int) -> float:
    r = C.c_double()
    _check(lib().sg_reduce(h, which, kind, C.byref(r)))
    return r.value


def sg_time(h):
    t, n = C.c_double(), C.c_long()
    _check(lib().sg_time(h, C.byref(t), C.byref(n)))
    return t.value, n.value


def sg_batch_create(handles):
    arr = (C.c_void_p * len(handles))(*[x.value for x in handles])
    b = C.c_void_p()
    _check(lib().sg_batch_create(arr, len(handles), C.byref(b)))
    return b


def sg_destroy(h):
    if h is not None and h.value:
        _PREC.pop(h.value, None)
        _check(lib().sg_destroy(h))


def sg_launch_count(h) -> int:
    n = C.c_long()
    _check(lib().sg_launch_count(h, C.byref(n)))
    return n.value


def sg_step_grid_noalloc(shape, lo, hi, pde, u_in_ptr: int, u_out_ptr: int, dt: float,
                         adv_speed=None, scheme: int = SG_WENO5, eps: float = 1e-3, stream: int = 0):
    """One RK3 step of one periodic FP64 grid in caller device memory (pointers as ints, e.g.
    a CUDA tensor's data_ptr()) without any device allocation; see include/sgweno.h."""
    dim = len(shape)
    shp = (C.c_long * dim)(*[int(x) for x in shape])
    lo_ = (C.c_double * dim)(*np.broadcast_to(np.asarray(lo, float), (dim,)))
    hi_ = (C.c_double * dim)(*np.broadcast_to(np.asarray(hi, float), (dim,)))
    adv = None if adv_speed is None else (C.c_double * dim)(*[float(a) for a in adv_speed])
    _check(lib().sg_step_grid_noalloc(dim, shp, lo_, hi_, pde, adv, scheme, float(eps), C.c_void_p(u_in_ptr),
                                      C.c_void_p(u_out_ptr), float(dt), C.c_void_p(stream)))


def sg_set_profiling(h, on: bool = True):
    _check(lib().sg_set_profiling(h, int(bool(on))))


def sg_profile(h, kind: int = SG_PROF_STAGE):
    """(milliseconds, launches) of the stage kernel since profiling was switched on."""
    ms, n = C.c_double(), C.c_long()
    _check(lib().sg_profile(h, kind, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def sg_stage_config(h):
    """(kernel, tile_points, tune_ms): the stage-kernel configuration the handle steps with."""
    k, tp, ms = C.c_int(), C.c_int(), C.c_double()
    _check(lib().sg_stage_config(h, C.byref(k), C.byref(tp), C.byref(ms)))
    return k.value, tp.value, ms.value


_alloc_refs = None


def sg_set_allocator(alloc_fn=None, free_fn=None, ctx=None):
    global _alloc_refs
    if alloc_fn is None:
        _check(lib().sg_set_allocator(ALLOC_FN(), FREE_FN(), None))
        _alloc_refs = None
        return
    a, f = ALLOC_FN(alloc_fn), FREE_FN(free_fn)
    _check(lib().sg_set_allocator(a, f, ctx))
    _alloc_refs = (a, f)


def use_torch_allocator(device: int = 0):
    """Route the library's device allocations through PyTorch's caching allocator."""
    import torch

    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device)
        except Exception:  # the library reports SG_ERR_NOMEM
            return None

    def _free(ptr, nbytes, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    sg_set_allocator(_alloc, _free)


def create(dim, root_cells, level, pde, **params):
    """sg_create with keyword parameters (fields of sg_params)."""
    p = sg_params_init(**params)
    return sg_create(dim, root_cells, level, pde, p)


def grid_shapes(h, dim):
    return [sg_grid_info(h, g, dim)[1] for g in range(sg_num_grids(h))]
