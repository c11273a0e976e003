"""ctypes binding of libad.so (include/ad.h).  Argument marshalling only.

Every function here has the name of the C entry point it calls and raises
``ADError`` when the call returns a status other than AD_OK.  Arrays may be
numpy arrays (host memory) or torch tensors (host or CUDA); they are passed
as raw pointers.  There is no fallback: if libad.so cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libad.so")

AD_OK = 0
STATUS = {0: "AD_OK", 1: "AD_ERR_INVALID_ARG", 2: "AD_ERR_NOT_SYMMETRIC", 3: "AD_ERR_SELF_LOOP",
          4: "AD_ERR_DUPLICATE_EDGE", 5: "AD_ERR_BAD_WEIGHT", 6: "AD_ERR_OOM", 7: "AD_ERR_CUDA",
          8: "AD_ERR_TIMEOUT", 9: "AD_ERR_STATE", 10: "AD_ERR_BAD_CSR"}
AD_MODE_LOCAL, AD_MODE_GLOBAL = 0, 1
AD_SCOPE_PER_NODE, AD_SCOPE_WHOLE_GRAPH = 0, 1
AD_STORAGE_FP32, AD_STORAGE_BF16, AD_STORAGE_FP16, AD_STORAGE_Q16 = 0, 1, 2, 3
AD_CREATE_SKIP_VALIDATION = 0x1
AD_DIST_NORMALIZE = 0x1
AD_DIST_KEEP_STATE = 0x2
AD_DIST_PERSISTENT = 0x4
AD_DIST_SQRT_CHECKPOINTS = 0x8

MODES = {"local": AD_MODE_LOCAL, "global": AD_MODE_GLOBAL}
SCOPES = {"per_node": AD_SCOPE_PER_NODE, "whole_graph": AD_SCOPE_WHOLE_GRAPH}
STORAGES = {"fp32": AD_STORAGE_FP32, "bf16": AD_STORAGE_BF16, "fp16": AD_STORAGE_FP16, "q16": AD_STORAGE_Q16}


class ADError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class ad_ml_params(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int32), ("k", ctypes.c_int32), ("omega", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("Q", ctypes.c_double), ("coarsest_n", ctypes.c_int64),
                ("max_levels", ctypes.c_int32), ("mode", ctypes.c_int), ("storage", ctypes.c_int)]


_VP = ctypes.c_void_p
_I32, _I64, _U32, _U64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PD = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "ad_version": (ctypes.c_char_p, []),
    "ad_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ad_last_error": (ctypes.c_char_p, []),
    "ad_set_allocator": (ctypes.c_int, [_VP, _VP, _VP]),
    "ad_kernel_launch_count": (_U64, []),
    "ad_selftest_barrier_timeout": (ctypes.c_int, [_VP, _U32, _PI32]),
    "ad_graph_set_profiling": (ctypes.c_int, [_VP, _I32]),
    "ad_graph_phase_time": (ctypes.c_int, [_VP, ctypes.c_char_p, _PD, _PI64, _I32]),
    "ad_graph_create": (ctypes.c_int, [_I64, _VP, _VP, _VP, _I32, _VP, ctypes.POINTER(_VP)]),
    "ad_graph_create_batched": (ctypes.c_int, [_I32, _VP, _I64, _VP, _VP, _VP, _I32, _VP, ctypes.POINTER(_VP)]),
    "ad_graph_destroy": (ctypes.c_int, [_VP]),
    "ad_graph_info": (ctypes.c_int, [_VP, _PI64, _PI64, _PI64, _PI64, _PI32]),
    "ad_graph_edge_offsets": (ctypes.c_int, [_VP, _VP]),
    "ad_graph_export": (ctypes.c_int, [_VP, _VP, _VP, _VP, _PI32]),
    "ad_graph_set_edge_weights": (ctypes.c_int, [_VP, _VP]),
    "ad_algebraic_distance": (ctypes.c_int, [_VP, _I32, _I32, _D, _U64, _U32, ctypes.c_int, _I32, _VP]),
    "ad_algebraic_distance_backward": (ctypes.c_int, [_VP, _VP, _VP]),
    "ad_sparsify": (ctypes.c_int, [_VP, _D, ctypes.c_int, ctypes.c_int, _VP, _PI64, _PD]),
    "ad_sparsify_scores": (ctypes.c_int, [_VP, _VP, _D, ctypes.c_int, ctypes.c_int, _VP, _PI64, _PD]),
    "ad_sparsify_local_global": (ctypes.c_int, [_VP, _D, _VP, _VP, _VP, _VP]),
    "ad_select_per_node": (ctypes.c_int, [_VP, _VP, _D, ctypes.c_int, _VP, _PI64]),
    "ad_sparsify_binned": (ctypes.c_int, [_VP, _VP, _D, _U64, _VP, _PI64, _PD]),
    "ad_binned_ranks": (ctypes.c_int, [_VP, _VP, _U64, _VP, _VP]),
    "ad_graph_autotune": (ctypes.c_int, [_VP, _I32, ctypes.c_int, _PI32, _PI32, _PI32]),
    "ad_sparsify_local_degree": (ctypes.c_int, [_VP, _D, _VP, _PI64, _PD]),
    "ad_select_whole_graph_noalloc": (ctypes.c_int, [_VP, _I64, _D, ctypes.c_int, _VP, _PI64, _VP]),
    "ad_ml_build": (ctypes.c_int, [_VP, ctypes.POINTER(ad_ml_params), ctypes.POINTER(_VP)]),
    "ad_ml_levels": (ctypes.c_int, [_VP, _PI32]),
    "ad_ml_level_size": (ctypes.c_int, [_VP, _I32, _PI64, _PI64]),
    "ad_ml_sparsify": (ctypes.c_int, [_VP, _VP, _I32, _D, _VP, _PI64, _PD]),
    "ad_ml_segment_ratios": (ctypes.c_int, [_I32, _I32, _I32, _D, _VP]),
    "ad_ml_destroy": (ctypes.c_int, [_VP]),
    "ad_multilevel": (ctypes.c_int, [_VP, ctypes.POINTER(ad_ml_params), _VP, _I32, _D, _VP, _PI32]),
    "ad_ml_level_export": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _PI32, _VP, _VP, _VP]),
    "ad_ml_set_trace": (ctypes.c_int, [_VP, _I32]),
    "ad_ml_level_trace": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP]),
    "ad_coarsen": (ctypes.c_int, [_VP, _VP, _D, _VP, _PI64, ctypes.POINTER(_VP), _VP]),
}

_lock = threading.Lock()
_lib = None
_alloc_hooks = None   # keeps the ctypes callbacks alive


def exported_symbols():
    return list(_SIGS)


def load(path: str = LIB_PATH):
    """Load libad.so once; raise if it is missing (there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"{path} is missing: build it with `python -m paper_1601_05527_gb300.build`")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(status: int):
    if status != AD_OK:
        msg = load().ad_last_error()
        raise ADError(status, msg.decode() if msg else "")


class _Arr:
    """Pointer to a numpy array or torch tensor, keeping a contiguous copy alive."""

    def __init__(self, x, dtype):
        self.keep = None
        if x is None:
            self.ptr = None
            return
        try:
            import torch
            if isinstance(x, torch.Tensor):
                tdt = {np.int64: torch.int64, np.int32: torch.int32, np.float32: torch.float32,
                       np.uint8: torch.uint8, np.float64: torch.float64,
                       np.uint32: getattr(torch, "uint32", torch.int32)}[dtype]
                if x.dtype != tdt:
                    raise TypeError(f"expected {tdt}, got {x.dtype}")
                if not x.is_contiguous():
                    x = x.contiguous()
                self.keep = x
                self.ptr = x.data_ptr()
                return
        except ImportError:
            pass
        a = np.ascontiguousarray(x, dtype=dtype)
        self.keep = a
        self.ptr = a.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def ad_selftest_barrier_timeout(polls=1000, stream=None) -> int:
    """Status recorded by a grid barrier that cannot complete (AD_ERR_TIMEOUT = 8 when the limit works)."""
    st = ctypes.c_int32()
    _check(load().ad_selftest_barrier_timeout(_stream_ptr(stream), int(polls), ctypes.byref(st)))
    return st.value


# --------------------------------------------------------------------------- allocator
def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    global _alloc_hooks
    import torch
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass

    hooks = (ALLOC(_alloc), FREE(_free))
    _check(load().ad_set_allocator(ctypes.cast(hooks[0], ctypes.c_void_p), ctypes.cast(hooks[1], ctypes.c_void_p),
                                   None))
    _alloc_hooks = hooks


def use_default_allocator():
    global _alloc_hooks
    _check(load().ad_set_allocator(None, None, None))
    _alloc_hooks = None


# --------------------------------------------------------------------------- library
def ad_version() -> str:
    return load().ad_version().decode()


def ad_status_string(s: int) -> str:
    return load().ad_status_string(s).decode()


def ad_last_error() -> str:
    return load().ad_last_error().decode()


def ad_kernel_launch_count() -> int:
    return int(load().ad_kernel_launch_count())


def ad_graph_set_profiling(g, enable: bool):
    _check(load().ad_graph_set_profiling(g, int(bool(enable))))


def ad_graph_phase_time(g, phase: str, reset: bool = False):
    ms = ctypes.c_double(0)
    cnt = ctypes.c_int64(0)
    _check(load().ad_graph_phase_time(g, phase.encode(), ctypes.byref(ms), ctypes.byref(cnt), int(reset)))
    return ms.value, cnt.value


# --------------------------------------------------------------------------- graphs
def ad_graph_create(n, row_ptr, col, weight=None, flags=0, stream=None):
    rp, ci, w = _Arr(row_ptr, np.int64), _Arr(col, np.int32), _Arr(weight, np.float32)
    out = ctypes.c_void_p()
    _check(load().ad_graph_create(int(n), rp.ptr, ci.ptr, w.ptr, int(flags), _stream_ptr(stream), ctypes.byref(out)))
    return out


def ad_graph_create_batched(vertex_offset, n, row_ptr, col, weight=None, flags=0, stream=None):
    vo = np.ascontiguousarray(vertex_offset, dtype=np.int64)
    rp, ci, w = _Arr(row_ptr, np.int64), _Arr(col, np.int32), _Arr(weight, np.float32)
    out = ctypes.c_void_p()
    _check(load().ad_graph_create_batched(len(vo) - 1, vo.ctypes.data, int(n), rp.ptr, ci.ptr, w.ptr, int(flags),
                                          _stream_ptr(stream), ctypes.byref(out)))
    return out


def ad_graph_destroy(g):
    if g is not None:
        _check(load().ad_graph_destroy(g))


def ad_graph_info(g):
    n, m, nnz, na = (ctypes.c_int64() for _ in range(4))
    G = ctypes.c_int32()
    _check(load().ad_graph_info(g, ctypes.byref(n), ctypes.byref(m), ctypes.byref(nnz), ctypes.byref(na),
                                ctypes.byref(G)))
    return {"n": n.value, "m": m.value, "nnz": nnz.value, "n_active": na.value, "n_graphs": G.value}


def ad_graph_edge_offsets(g):
    G = ad_graph_info(g)["n_graphs"]
    out = np.zeros(G + 1, dtype=np.int64)
    _check(load().ad_graph_edge_offsets(g, out.ctypes.data))
    return out


def ad_graph_export(g):
    """(row_ptr int64[n+1], col int32[nnz], weight float32[nnz] or None) of a handle."""
    info = ad_graph_info(g)
    rp = np.zeros(info["n"] + 1, np.int64)
    col = np.zeros(info["nnz"], np.int32)
    w = np.zeros(info["nnz"], np.float32)
    hw = ctypes.c_int32()
    _check(load().ad_graph_export(g, rp.ctypes.data, col.ctypes.data, w.ctypes.data, ctypes.byref(hw)))
    return rp, col, (w if hw.value else None)


def ad_graph_set_edge_weights(g, w_edge):
    a = _Arr(w_edge, np.float32)
    _check(load().ad_graph_set_edge_weights(g, a.ptr))


# --------------------------------------------------------------------------- Alg. 1
def ad_algebraic_distance(g, R, k, omega, seed, stream_id=0, storage="fp32", flags=0, rho_out=None):
    """rho_out: numpy float32[m] / torch float32 tensor[m] (host or CUDA) or None."""
    out = _Arr(rho_out, np.float32) if rho_out is not None else None
    _check(load().ad_algebraic_distance(g, int(R), int(k), float(omega), int(seed) & (2**64 - 1), int(stream_id),
                                        STORAGES.get(storage, storage), int(flags), out.ptr if out else None))
    return rho_out


def ad_algebraic_distance_backward(g, rho_bar, w_bar):
    a, b = _Arr(rho_bar, np.float32), _Arr(w_bar, np.float32)
    _check(load().ad_algebraic_distance_backward(g, a.ptr, b.ptr))
    return w_bar


# --------------------------------------------------------------------------- Alg. 2
def ad_sparsify(g, fraction, mode, scope, keep_out):
    k = _Arr(keep_out, np.uint8)
    nk = ctypes.c_int64()
    e = ctypes.c_double()
    _check(load().ad_sparsify(g, float(fraction), MODES.get(mode, mode), SCOPES.get(scope, scope), k.ptr,
                              ctypes.byref(nk), ctypes.byref(e)))
    return nk.value, e.value


def ad_sparsify_local_global(g, fraction, keep_local, keep_global):
    """Both per-node selections (local, global) of Alg. 2 in one call;
    returns ((kept_local, kept_global), (e_local, e_global))."""
    kl, kg = _Arr(keep_local, np.uint8), _Arr(keep_global, np.uint8)
    nk = (ctypes.c_int64 * 2)()
    e = (ctypes.c_double * 2)()
    _check(load().ad_sparsify_local_global(g, float(fraction), kl.ptr, kg.ptr, ctypes.cast(nk, _VP),
                                           ctypes.cast(e, _VP)))
    return (nk[0], nk[1]), (e[0], e[1])


def ad_sparsify_scores(g, score, fraction, mode, scope, keep_out):
    s, k = _Arr(score, np.float32), _Arr(keep_out, np.uint8)
    nk = ctypes.c_int64()
    e = ctypes.c_double()
    _check(load().ad_sparsify_scores(g, s.ptr, float(fraction), MODES.get(mode, mode), SCOPES.get(scope, scope),
                                     k.ptr, ctypes.byref(nk), ctypes.byref(e)))
    return nk.value, e.value


def ad_select_per_node(g, score, e, mode, keep_out):
    s, k = _Arr(score, np.float32), _Arr(keep_out, np.uint8)
    nk = ctypes.c_int64()
    _check(load().ad_select_per_node(g, s.ptr, float(e), MODES.get(mode, mode), k.ptr, ctypes.byref(nk)))
    return nk.value


def ad_graph_autotune(g, R, storage="fp32"):
    """Choose the sweep's launch shape for (R, storage) by timing; returns
    (lanes_per_row, chunks_per_lane, ctas_per_sm) (0: as many as fit)."""
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().ad_graph_autotune(g, int(R), STORAGES.get(storage, storage), ctypes.byref(a), ctypes.byref(b),
                                    ctypes.byref(c)))
    return a.value, b.value, c.value


def ad_sparsify_binned(g, score, fraction, seed, keep_out):
    """SparsifyB (Alg. 3) to a target fraction; score None = the handle's distances.
    Returns (n_kept, e_used)."""
    s, k = _Arr(score, np.float32), _Arr(keep_out, np.uint8)
    nk, eu = ctypes.c_int64(), ctypes.c_double()
    _check(load().ad_sparsify_binned(g, s.ptr, float(fraction), int(seed) & (2**64 - 1), k.ptr, ctypes.byref(nk),
                                     ctypes.byref(eu)))
    return nk.value, eu.value


def ad_binned_ranks(g, score, seed, rank_out, bin_out=None):
    """Per-entry SparsifyB (Alg. 3) selection rank and bin, uint32 in CSR order;
    score None = the handle's distances."""
    s, r, b = _Arr(score, np.float32), _Arr(rank_out, np.uint32), _Arr(bin_out, np.uint32)
    _check(load().ad_binned_ranks(g, s.ptr, int(seed) & (2**64 - 1), r.ptr, b.ptr))


def ad_sparsify_local_degree(g, fraction, keep_out):
    """Local Degree (the paper's comparison method) to a target fraction: (n_kept, e_used)."""
    k = _Arr(keep_out, np.uint8)
    nk, eu = ctypes.c_int64(), ctypes.c_double()
    _check(load().ad_sparsify_local_degree(g, float(fraction), k.ptr, ctypes.byref(nk), ctypes.byref(eu)))
    return nk.value, eu.value


def ad_select_whole_graph_noalloc(score, m, fraction, mode, keep_out, stream=None):
    """Whole-graph ranking with no device allocation (device score/keep arrays)."""
    s, k = _Arr(score, np.float32), _Arr(keep_out, np.uint8)
    nk = ctypes.c_int64()
    _check(load().ad_select_whole_graph_noalloc(s.ptr, int(m), float(fraction), MODES.get(mode, mode), k.ptr,
                                                ctypes.byref(nk), _stream_ptr(stream)))
    return nk.value


# --------------------------------------------------------------------------- Alg. 6
def ad_ml_build(g, R, k, omega, seed, Q=0.5, coarsest_n=1000, max_levels=64, mode="local", storage="fp32"):
    p = ad_ml_params(int(R), int(k), float(omega), int(seed) & (2**64 - 1), float(Q), int(coarsest_n),
                     int(max_levels), MODES.get(mode, mode), STORAGES.get(storage, storage))
    out = ctypes.c_void_p()
    _check(load().ad_ml_build(g, ctypes.byref(p), ctypes.byref(out)))
    return out


def ad_ml_levels(ml) -> int:
    L = ctypes.c_int32()
    _check(load().ad_ml_levels(ml, ctypes.byref(L)))
    return L.value


def ad_ml_level_size(ml, level):
    n, m = ctypes.c_int64(), ctypes.c_int64()
    _check(load().ad_ml_level_size(ml, int(level), ctypes.byref(n), ctypes.byref(m)))
    return n.value, m.value


def ad_ml_sparsify(ml, ratios, target_fraction, keep_out):
    r = np.ascontiguousarray(ratios, dtype=np.float64)
    k = _Arr(keep_out, np.uint8)
    nk = ctypes.c_int64()
    ru = ctypes.c_double()
    _check(load().ad_ml_sparsify(ml, r.ctypes.data, len(r), float(target_fraction), k.ptr, ctypes.byref(nk),
                                 ctypes.byref(ru)))
    return nk.value, ru.value


def ad_ml_segment_ratios(n_levels, segment, level_span, value):
    seg = {"coarse": 1, "middle": 2, "fine": 3}.get(segment, segment)
    out = np.zeros(n_levels, dtype=np.float64)
    _check(load().ad_ml_segment_ratios(int(n_levels), int(seg), int(level_span), float(value), out.ctypes.data))
    return out


def ad_ml_destroy(ml):
    if ml is not None:
        _check(load().ad_ml_destroy(ml))


def ad_ml_level_export(ml, level):
    """Level `level` of a hierarchy: dict with row_ptr, col, weight (None: unit), rho
    (downward distances) and, below the coarsest level, agg and f2c."""
    n, m = ad_ml_level_size(ml, level)
    L = ad_ml_levels(ml)
    rp = np.zeros(n + 1, np.int64)
    nnz = 2 * m
    ci = np.zeros(max(nnz, 1), np.int32)
    w = np.zeros(max(nnz, 1), np.float32)
    hw = ctypes.c_int32()
    rho = np.zeros(max(m, 1), np.float32)
    agg = np.zeros(max(n, 1), np.int32) if level < L - 1 else None
    f2c = np.zeros(max(m, 1), np.int64) if level < L - 1 else None
    _check(load().ad_ml_level_export(ml, int(level), rp.ctypes.data, ci.ctypes.data, w.ctypes.data, ctypes.byref(hw),
                                     rho.ctypes.data, None if agg is None else agg.ctypes.data,
                                     None if f2c is None else f2c.ctypes.data))
    return {"row_ptr": rp, "col": ci[:nnz], "weight": w[:nnz] if hw.value else None, "rho": rho[:m],
            "agg": None if agg is None else agg[:n], "f2c": None if f2c is None else f2c[:m]}


def ad_ml_set_trace(ml, enable=True):
    _check(load().ad_ml_set_trace(ml, int(bool(enable))))


def ad_ml_level_trace(ml, level):
    """(inherited, kept, rho_up) of one level from the last traced ad_ml_sparsify call."""
    _, m = ad_ml_level_size(ml, level)
    inh = np.zeros(max(m, 1), np.uint8)
    kp = np.zeros(max(m, 1), np.uint8)
    ru = np.zeros(max(m, 1), np.float32)
    _check(load().ad_ml_level_trace(ml, int(level), inh.ctypes.data, kp.ctypes.data, ru.ctypes.data))
    return inh[:m], kp[:m], ru[:m]


def ad_multilevel(g, ratios, target_fraction, keep_out, *, R, k, omega, seed, Q=0.5, coarsest_n=1000, max_levels=64,
                  mode="local", storage="fp32"):
    """Alg. 6 in one call; ratios[0] belongs to the coarsest level.  Returns the number of levels."""
    p = ad_ml_params(int(R), int(k), float(omega), int(seed) & (2**64 - 1), float(Q), int(coarsest_n),
                     int(max_levels), MODES.get(mode, mode), STORAGES.get(storage, storage))
    r = None if ratios is None else np.ascontiguousarray(ratios, dtype=np.float64)
    kk = _Arr(keep_out, np.uint8)
    nl = ctypes.c_int32()
    _check(load().ad_multilevel(g, ctypes.byref(p), None if r is None else r.ctypes.data,
                                0 if r is None else len(r), float(target_fraction), kk.ptr, ctypes.byref(nl)))
    return nl.value


def ad_coarsen(g, score, Q, agg_out, fine_to_coarse_out=None, want_graph=True):
    s, a = _Arr(score, np.float32), _Arr(agg_out, np.int32)
    f = _Arr(fine_to_coarse_out, np.int64)
    nc = ctypes.c_int64()
    cg = ctypes.c_void_p()
    _check(load().ad_coarsen(g, s.ptr, float(Q), a.ptr, ctypes.byref(nc), ctypes.byref(cg) if want_graph else None,
                             f.ptr))
    return nc.value, (cg if want_graph else None)
