"""FP64 CPU oracle for sparsification by algebraic distance (arXiv 1601.05527).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
(``paper_1601_05527_gb300``) never imports this package and has no CPU
fallback.  The C source ``ad_oracle.c`` shares no code with the CUDA sources.

Functions follow the paper's algorithms (Alg. 1 ComputeAlgDist, Alg. 2
Sparsify, Sec. 5 / Alg. 6 MLSparsify with Eq. (P) and the Galerkin product)
in FP64; see the header of ``ad_oracle.c`` for the readings R1-R12 of points
the paper leaves open.  Damping is passed as ``omega`` (the weight of the
neighbour average) and handed to the C code as the paper's alpha = 1 - omega.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ad_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

I64P = ctypes.POINTER(ctypes.c_int64)
I32P = ctypes.POINTER(ctypes.c_int32)
U32P = ctypes.POINTER(ctypes.c_uint32)
U8P = ctypes.POINTER(ctypes.c_uint8)
F64P = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ad_oracle.c into liboracle.so (plain gcc, no target-specific flags),
    with OpenMP where the compiler has it (the row loops of Alg. 1 then run on
    several host threads, with results that do not depend on the thread count)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        base = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-Wall", "-Wextra"]
        if subprocess.call(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base + [_SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            sig = {
                "orc_philox4x32_10": (None, [U32P, U32P, U32P]),
                "orc_set_threads": (None, [ctypes.c_int32]),
                "orc_max_threads": (ctypes.c_int32, []),
                "orc_last_phase_seconds": (None, [F64P]),
                "orc_test_value": (ctypes.c_double, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int32]),
                "orc_init_vectors": (None, [ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32, F64P]),
                "orc_count_edges": (ctypes.c_int64, [ctypes.c_int64, I64P, I32P]),
                "orc_edge_list": (None, [ctypes.c_int64, I64P, I32P, I32P, I32P]),
                "orc_entry_edge_ids": (None, [ctypes.c_int64, I64P, I32P, I64P]),
                "orc_weighted_degree": (None, [ctypes.c_int64, I64P, F64P, F64P]),
                "orc_algebraic_distance": (ctypes.c_int, [ctypes.c_int64, I64P, I32P, F64P, ctypes.c_int32,
                                                          ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                                          ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32,
                                                          F64P, F64P, F64P]),
                "orc_select_whole_graph": (ctypes.c_int64, [ctypes.c_int64, F64P, ctypes.c_int32, ctypes.c_int64, U8P]),
                "orc_degree_target": (ctypes.c_int64, [ctypes.c_int64, ctypes.c_double]),
                "orc_select_per_node": (ctypes.c_int64, [ctypes.c_int64, I64P, I32P, F64P, ctypes.c_int32,
                                                         ctypes.c_double, U8P]),
                "orc_target_count": (ctypes.c_int64, [ctypes.c_int64, ctypes.c_double]),
                "orc_sparsify": (ctypes.c_int, [ctypes.c_int64, I64P, I32P, F64P, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_double, U8P, I64P, F64P]),
                "orc_binned_ranks": (ctypes.c_int, [ctypes.c_int64, I64P, I32P, F64P, ctypes.c_uint64, I64P, I64P]),
                "orc_sparsify_binned": (ctypes.c_int, [ctypes.c_int64, I64P, I32P, F64P, ctypes.c_uint64,
                                                       ctypes.c_double, U8P, I64P, F64P]),
                "orc_sparsify_local_degree": (ctypes.c_int, [ctypes.c_int64, I64P, I32P, ctypes.c_double, U8P, I64P,
                                                             F64P]),
                "orc_create_seeds": (ctypes.c_int, [ctypes.c_int64, I64P, I32P, F64P, ctypes.c_double, U8P]),
                "orc_aggregate": (ctypes.c_int64, [ctypes.c_int64, I64P, I32P, F64P, U8P, I32P]),
                "orc_galerkin": (ctypes.c_int64, [ctypes.c_int64, I64P, I32P, F64P, I32P, ctypes.c_int64,
                                                  I64P, I32P, F64P, I64P]),
                "orc_uncoarsen": (None, [ctypes.c_int64, I64P, U8P, U8P]),
                "orc_ml_build": (ctypes.c_void_p, [ctypes.c_int64, I64P, I32P, F64P, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.c_double, ctypes.c_uint64, ctypes.c_double, ctypes.c_int64,
                                                   ctypes.c_int32, ctypes.c_int32]),
                "orc_ml_free": (None, [ctypes.c_void_p]),
                "orc_ml_levels": (ctypes.c_int32, [ctypes.c_void_p]),
                "orc_ml_level_size": (None, [ctypes.c_void_p, ctypes.c_int32, I64P, I64P]),
                "orc_ml_sparsify": (ctypes.c_int, [ctypes.c_void_p, F64P, ctypes.c_int32, ctypes.c_double, U8P,
                                                   I64P, F64P]),
                "orc_ml_segment_ratios": (None, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, F64P]),
                "orc_loss_grad": (ctypes.c_int, [ctypes.c_int64, I64P, I32P, F64P, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                                 I64P, F64P, F64P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _csr(rp, ci, w=None):
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    return rp, ci, w


# --------------------------------------------------------------------------- threads
def set_threads(n: int):
    """Host threads of the oracle's row loops (1 = sequential)."""
    _L().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_L().orc_max_threads())


def last_phase_seconds():
    """(init, sweeps, distance) wall seconds of the last algebraic_distance call."""
    out = np.zeros(3, dtype=np.float64)
    _L().orc_last_phase_seconds(_p(out, F64P))
    return {"init": float(out[0]), "sweeps": float(out[1]), "distance": float(out[2])}


# --------------------------------------------------------------------------- Philox / init
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _L().orc_philox4x32_10(_p(c, U32P), _p(k, U32P), _p(out, U32P))
    return out


def test_value(seed, stream, i, r):
    return _L().orc_test_value(seed, stream, i, r)


def init_vectors(n, R, seed, stream=0):
    x = np.zeros((n, R), dtype=np.float64)
    _L().orc_init_vectors(n, R, seed, stream, _p(x, F64P))
    return x


# --------------------------------------------------------------------------- graph helpers
def count_edges(rp, ci):
    rp, ci, _ = _csr(rp, ci)
    return int(_L().orc_count_edges(len(rp) - 1, _p(rp, I64P), _p(ci, I32P)))


def edge_list(rp, ci):
    rp, ci, _ = _csr(rp, ci)
    m = count_edges(rp, ci)
    eu = np.zeros(m, dtype=np.int32)
    ev = np.zeros(m, dtype=np.int32)
    _L().orc_edge_list(len(rp) - 1, _p(rp, I64P), _p(ci, I32P), _p(eu, I32P), _p(ev, I32P))
    return eu, ev


def entry_edge_ids(rp, ci):
    rp, ci, _ = _csr(rp, ci)
    eid = np.zeros(len(ci), dtype=np.int64)
    _L().orc_entry_edge_ids(len(rp) - 1, _p(rp, I64P), _p(ci, I32P), _p(eid, I64P))
    return eid


def weighted_degree(rp, ci, w=None):
    rp, ci, w = _csr(rp, ci, w)
    D = np.zeros(len(rp) - 1, dtype=np.float64)
    _L().orc_weighted_degree(len(rp) - 1, _p(rp, I64P), _p(w, F64P), _p(D, F64P))
    return D


# --------------------------------------------------------------------------- Alg. 1
def algebraic_distance(rp, ci, w=None, *, R, k, omega, seed, stream=0, rescale="per_sweep",
                       normalize=False, x0=None, return_x=False):
    """rho[m] (edge-id order) of Alg. 1; optionally also the final rescaled vectors [n][R]."""
    rp, ci, w = _csr(rp, ci, w)
    n = len(rp) - 1
    m = count_edges(rp, ci)
    rho = np.zeros(m, dtype=np.float64)
    xf = np.zeros((n, R), dtype=np.float64) if return_x else None
    if x0 is not None:
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        assert x0.shape == (n, R)
    mode = {"per_sweep": 0, "end": 1}[rescale]
    st = _L().orc_algebraic_distance(n, _p(rp, I64P), _p(ci, I32P), _p(w, F64P), R, k, 1.0 - omega,
                                     seed, stream, mode, int(bool(normalize)), _p(x0, F64P),
                                     _p(xf, F64P), _p(rho, F64P))
    if st != 0:
        raise RuntimeError(f"oracle algebraic_distance failed ({st})")
    return (rho, xf) if return_x else rho


# --------------------------------------------------------------------------- Alg. 2
MODES = {"local": 0, "global": 1}
SCOPES = {"per_node": 0, "whole_graph": 1}


def select_whole_graph(score, mode, K):
    s = np.ascontiguousarray(score, dtype=np.float64)
    keep = np.zeros(len(s), dtype=np.uint8)
    _L().orc_select_whole_graph(len(s), _p(s, F64P), MODES[mode], K, _p(keep, U8P))
    return keep


def degree_target(d, e):
    return int(_L().orc_degree_target(d, e))


def target_count(m, fraction):
    return int(_L().orc_target_count(m, fraction))


def select_per_node(rp, ci, score, mode, e):
    rp, ci, _ = _csr(rp, ci)
    s = np.ascontiguousarray(score, dtype=np.float64)
    keep = np.zeros(len(s), dtype=np.uint8)
    c = _L().orc_select_per_node(len(rp) - 1, _p(rp, I64P), _p(ci, I32P), _p(s, F64P), MODES[mode], e,
                                 _p(keep, U8P))
    return keep, int(c)


def sparsify(rp, ci, score, mode, scope, fraction):
    """(keep[m] uint8, n_kept, e_used) — e_used is -1 for the whole-graph scope."""
    rp, ci, _ = _csr(rp, ci)
    s = np.ascontiguousarray(score, dtype=np.float64)
    keep = np.zeros(len(s), dtype=np.uint8)
    nk = ctypes.c_int64(0)
    eu = ctypes.c_double(0)
    st = _L().orc_sparsify(len(rp) - 1, _p(rp, I64P), _p(ci, I32P), _p(s, F64P), MODES[mode], SCOPES[scope],
                           fraction, _p(keep, U8P), ctypes.byref(nk), ctypes.byref(eu))
    if st != 0:
        raise RuntimeError(f"oracle sparsify failed ({st})")
    return keep, nk.value, eu.value


def binned_ranks(rp, ci, score, seed, return_bins=False):
    """Selection rank of every CSR entry under SparsifyB (Alg. 3, reading R13);
    with return_bins also the bin of every entry."""
    rp, ci, _ = _csr(rp, ci)
    s = np.ascontiguousarray(score, dtype=np.float64)
    rank = np.zeros(int(rp[-1]), dtype=np.int64)
    bins = np.zeros(int(rp[-1]), dtype=np.int64)
    if _L().orc_binned_ranks(len(rp) - 1, _p(rp, I64P), _p(ci, I32P), _p(s, F64P), int(seed) & (2**64 - 1),
                             _p(rank, I64P), _p(bins, I64P)) != 0:
        raise RuntimeError("oracle binned ranks failed")
    return (rank, bins) if return_bins else rank


def sparsify_binned(rp, ci, score, seed, fraction):
    """SparsifyB to a target fraction: (keep[m] uint8, n_kept, e_used)."""
    rp, ci, _ = _csr(rp, ci)
    s = np.ascontiguousarray(score, dtype=np.float64)
    keep = np.zeros(len(s), dtype=np.uint8)
    nk = ctypes.c_int64(0)
    eu = ctypes.c_double(0)
    st = _L().orc_sparsify_binned(len(rp) - 1, _p(rp, I64P), _p(ci, I32P), _p(s, F64P), int(seed) & (2**64 - 1),
                                  fraction, _p(keep, U8P), ctypes.byref(nk), ctypes.byref(eu))
    if st != 0:
        raise RuntimeError(f"oracle binned sparsify failed ({st})")
    return keep, nk.value, eu.value


def sparsify_local_degree(rp, ci, fraction):
    """Local Degree (the comparison method of Sec. 6): (keep[m] uint8, n_kept, e_used)."""
    rp, ci, _ = _csr(rp, ci)
    m = int(_L().orc_count_edges(len(rp) - 1, _p(rp, I64P), _p(ci, I32P)))
    keep = np.zeros(m, dtype=np.uint8)
    nk = ctypes.c_int64(0)
    eu = ctypes.c_double(0)
    st = _L().orc_sparsify_local_degree(len(rp) - 1, _p(rp, I64P), _p(ci, I32P), fraction, _p(keep, U8P),
                                        ctypes.byref(nk), ctypes.byref(eu))
    if st != 0:
        raise RuntimeError(f"oracle local degree failed ({st})")
    return keep, nk.value, eu.value


# --------------------------------------------------------------------------- Sec. 5 / Alg. 6
def create_seeds(rp, ci, w=None, Q=0.5):
    rp, ci, w = _csr(rp, ci, w)
    s = np.zeros(len(rp) - 1, dtype=np.uint8)
    _L().orc_create_seeds(len(rp) - 1, _p(rp, I64P), _p(ci, I32P), _p(w, F64P), Q, _p(s, U8P))
    return s


def aggregate(rp, ci, score, is_seed):
    rp, ci, _ = _csr(rp, ci)
    s = np.ascontiguousarray(score, dtype=np.float64)
    seeds = np.ascontiguousarray(is_seed, dtype=np.uint8)
    agg = np.zeros(len(rp) - 1, dtype=np.int32)
    nc = _L().orc_aggregate(len(rp) - 1, _p(rp, I64P), _p(ci, I32P), _p(s, F64P), _p(seeds, U8P), _p(agg, I32P))
    if nc < 0:
        raise RuntimeError("oracle aggregate: F vertex without seed neighbour")
    return agg, int(nc)


def galerkin(rp, ci, w, agg, nc):
    """(rp_c, ci_c, w_c, fine_to_coarse[m_f]) of L_c = P^T L_f P."""
    rp, ci, w = _csr(rp, ci, w)
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    nnz = len(ci)
    m = count_edges(rp, ci)
    rpc = np.zeros(nc + 1, dtype=np.int64)
    cic = np.zeros(max(nnz, 1), dtype=np.int32)
    wc = np.zeros(max(nnz, 1), dtype=np.float64)
    f2c = np.zeros(max(m, 1), dtype=np.int64)
    nnzc = _L().orc_galerkin(len(rp) - 1, _p(rp, I64P), _p(ci, I32P), _p(w, F64P), _p(agg, I32P), nc,
                             _p(rpc, I64P), _p(cic, I32P), _p(wc, F64P), _p(f2c, I64P))
    if nnzc < 0:
        raise RuntimeError("oracle galerkin failed")
    return rpc, cic[:nnzc].copy(), wc[:nnzc].copy(), f2c[:m].copy()


def uncoarsen(fine_to_coarse, keep_c):
    f2c = np.ascontiguousarray(fine_to_coarse, dtype=np.int64)
    kc = np.ascontiguousarray(keep_c, dtype=np.uint8)
    kf = np.zeros(len(f2c), dtype=np.uint8)
    _L().orc_uncoarsen(len(f2c), _p(f2c, I64P), _p(kc, U8P), _p(kf, U8P))
    return kf


SEGMENTS = {"coarse": 1, "middle": 2, "fine": 3}


def segment_ratios(L, segment, level_span, value):
    r = np.zeros(L, dtype=np.float64)
    _L().orc_ml_segment_ratios(L, SEGMENTS[segment], level_span, value, _p(r, F64P))
    return r


class Multilevel:
    """Hierarchy of Alg. 6 (downward half) plus the upward sparsification."""

    def __init__(self, rp, ci, w=None, *, R, k, omega, seed, Q=0.5, coarsest_n=1000, max_levels=64,
                 mode="local"):
        self._rp, self._ci, self._w = _csr(rp, ci, w)   # borrowed by the C handle
        self._h = _L().orc_ml_build(len(self._rp) - 1, _p(self._rp, I64P), _p(self._ci, I32P),
                                    _p(self._w, F64P), R, k, 1.0 - omega, seed, Q, coarsest_n,
                                    max_levels, MODES[mode])
        if not self._h:
            raise RuntimeError("oracle ml_build failed")
        self.m0 = count_edges(self._rp, self._ci)

    @property
    def levels(self):
        return int(_L().orc_ml_levels(self._h))

    def level_size(self, l):
        n = ctypes.c_int64(0)
        m = ctypes.c_int64(0)
        _L().orc_ml_level_size(self._h, l, ctypes.byref(n), ctypes.byref(m))
        return n.value, m.value

    def sparsify(self, ratios, target_fraction=-1.0):
        r = np.ascontiguousarray(ratios, dtype=np.float64)
        keep = np.zeros(max(self.m0, 1), dtype=np.uint8)
        nk = ctypes.c_int64(0)
        ru = ctypes.c_double(0)
        st = _L().orc_ml_sparsify(self._h, _p(r, F64P), len(r), target_fraction, _p(keep, U8P),
                                  ctypes.byref(nk), ctypes.byref(ru))
        if st != 0:
            raise RuntimeError(f"oracle ml_sparsify failed ({st})")
        return keep[:self.m0], nk.value, ru.value

    def close(self):
        if self._h:
            _L().orc_ml_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- reverse mode
def loss_grad(rp, ci, w, S, *, R, k, omega, seed, stream=0):
    """(L, dL/dw_e[m]) for L = sum_{e in S} rho_e^2 (per-sweep rescale form of Alg. 1)."""
    rp, ci, w = _csr(rp, ci, w)
    S = np.ascontiguousarray(S, dtype=np.int64)
    m = count_edges(rp, ci)
    g = np.zeros(max(m, 1), dtype=np.float64)
    loss = ctypes.c_double(0)
    st = _L().orc_loss_grad(len(rp) - 1, _p(rp, I64P), _p(ci, I32P), _p(w, F64P), R, k, 1.0 - omega, seed,
                            stream, len(S), _p(S, I64P), ctypes.byref(loss), _p(g, F64P))
    if st != 0:
        raise RuntimeError(f"oracle loss_grad failed ({st})")
    return loss.value, g[:m]
