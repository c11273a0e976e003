"""GPU parity of ComputeAlgDist (Alg. 1): Philox init, JOR sweeps with the
per-sweep rescale, edge distances, through the C ABI, against the FP64 oracle
on the same seeded inputs."""
import numpy as np
import pytest

import oracle
from paper_1601_05527_gb300 import graphgen
from gpu_util import assert_rho_close, entry_weights_f64, jaccard, lib, rho_error

pytestmark = pytest.mark.gpu


def gpu_rho(g, R, k, omega, seed, stream_id=0, storage="fp32", normalize=False):
    L = lib()
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, g.weight)
    try:
        rho = np.zeros(g.m, dtype=np.float32)
        L.ad_algebraic_distance(h, R, k, omega, seed, stream_id, storage, L.AD_DIST_NORMALIZE if normalize else 0,
                                rho)
        return rho
    finally:
        L.ad_graph_destroy(h)


def ref_rho(g, R, k, omega, seed, stream_id=0, normalize=False, x0=None):
    return oracle.algebraic_distance(g.row_ptr, g.col, entry_weights_f64(g), R=R, k=k, omega=omega, seed=seed,
                                     stream=stream_id, normalize=normalize, x0=x0)


def weighted(g, seed=1):
    return graphgen.with_edge_weights(g, graphgen.lognormal_edge_weights(g.m, seed=seed))


GRAPHS = {
    "grid64": lambda: graphgen.grid2d(64, 64),
    "rmat12": lambda: graphgen.rmat(12, 16, seed=3),
    "rmat11w": lambda: weighted(graphgen.rmat(11, 16, seed=4)),
    "ba3000": lambda: graphgen.barabasi_albert(3000, 8, seed=5),
    "ws4000": lambda: graphgen.watts_strogatz(4000, 10, 0.1, seed=6),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_rho_matches_oracle_fp32(name):
    g = GRAPHS[name]()
    R, k = (8, 20) if name == "grid64" else (32, 20)
    rho = gpu_rho(g, R, k, 0.5, seed=0x1601055270000000)
    assert_rho_close(rho, ref_rho(g, R, k, 0.5, seed=0x1601055270000000))


@pytest.mark.parametrize("R", [1, 3, 10, 16, 24, 40, 64, 100, 128, 256])
def test_ragged_vector_counts(R):
    g = graphgen.rmat(10, 8, seed=7)
    assert_rho_close(gpu_rho(g, R, 6, 0.5, seed=R), ref_rho(g, R, 6, 0.5, seed=R))


@pytest.mark.parametrize("omega,k", [(0.3, 9), (0.8, 5), (1.0, 4), (0.5, 1), (0.5, 0)])
def test_damping_and_sweep_counts(omega, k):
    g = weighted(graphgen.barabasi_albert(2000, 5, seed=8), seed=9)
    assert_rho_close(gpu_rho(g, 16, k, omega, seed=3, stream_id=5), ref_rho(g, 16, k, omega, seed=3, stream_id=5))


def test_init_is_bit_identical_to_oracle():
    # k = 0: rho of the raw Philox vectors; only FP32 rounding of sum/sqrt remains
    g = graphgen.rmat(11, 8, seed=1)
    rho = gpu_rho(g, 32, 0, 0.5, seed=77, stream_id=9)
    ref = ref_rho(g, 32, 0, 0.5, seed=77, stream_id=9)
    assert np.max(np.abs(rho - ref) / np.maximum(ref, 1e-30)) < 2e-6


def test_normalized_scores():
    g = weighted(graphgen.rmat(11, 16, seed=2), seed=3)
    assert_rho_close(gpu_rho(g, 16, 10, 0.5, seed=4, normalize=True), ref_rho(g, 16, 10, 0.5, seed=4, normalize=True))


def test_single_edge_components_and_isolated_vertices():
    u = np.array([0, 2, 4, 6, 6, 7])
    v = np.array([1, 3, 5, 7, 8, 8])
    g = graphgen.from_edges(12, u, v)          # vertices 9..11 isolated
    rho = gpu_rho(g, 8, 4, 0.5, seed=1)
    assert np.all(rho[:3] == 0.0) and np.all(rho[3:] > 0)
    g1 = graphgen.from_edges(2, [0], [1])
    r1 = gpu_rho(g1, 8, 3, 0.3, seed=1)
    np.testing.assert_allclose(r1, np.sqrt(8), rtol=1e-6)


def test_isolated_vertices_do_not_change_distances():
    g = graphgen.rmat(10, 8, seed=3)
    eu, ev = g.edges_upper()
    g2 = graphgen.from_edges(g.n + 500, eu, ev)
    np.testing.assert_array_equal(gpu_rho(g, 16, 8, 0.5, seed=2), gpu_rho(g2, 16, 8, 0.5, seed=2))


def test_deterministic():
    g = graphgen.rmat(12, 16, seed=3)
    a = gpu_rho(g, 32, 10, 0.5, seed=5)
    b = gpu_rho(g, 32, 10, 0.5, seed=5)
    np.testing.assert_array_equal(a, b)


def test_empty_and_edgeless_graphs():
    L = lib()
    for n in (0, 7):
        h = L.ad_graph_create(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32))
        info = L.ad_graph_info(h)
        assert info["m"] == 0 and info["n_active"] == 0
        L.ad_algebraic_distance(h, 8, 5, 0.5, 1, 0, "fp32", 0, np.zeros(0, np.float32))
        keep = np.zeros(0, np.uint8)
        assert L.ad_sparsify(h, 0.5, "local", "whole_graph", keep)[0] == 0
        assert L.ad_sparsify(h, 0.5, "global", "per_node", keep)[0] == 0
        L.ad_graph_destroy(h)


# Error of the 16-bit storage formats against the FP64 oracle on R-MAT scale 12,
# R = 32, k = 20 (rms rho ~ 0.02 of the [-1/2, 1/2] range).  For scale: two FP64
# runs with different seeds differ by 0.97 on this measure.  The bounds are set
# from measurement on GB300 with a margin.
STORAGE_BOUNDS = {"q16": 0.02, "fp16": 0.25, "bf16": 0.6}


@pytest.mark.parametrize("storage", list(STORAGE_BOUNDS))
def test_16bit_storage_error_against_fp64(storage):
    g = graphgen.rmat(12, 16, seed=3)
    ref = ref_rho(g, 32, 20, 0.5, seed=11)
    err = rho_error(gpu_rho(g, 32, 20, 0.5, seed=11, storage=storage), ref)
    assert err < STORAGE_BOUNDS[storage], err


def test_torch_device_tensors_in_and_out():
    import torch
    L = lib()
    g = graphgen.rmat(10, 8, seed=3)
    dev = torch.device("cuda")
    h = L.ad_graph_create(g.n, torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev), None)
    out = torch.zeros(g.m, dtype=torch.float32, device=dev)
    L.ad_algebraic_distance(h, 16, 5, 0.5, 3, 0, "fp32", 0, out)
    torch.cuda.synchronize()
    L.ad_graph_destroy(h)
    np.testing.assert_array_equal(out.cpu().numpy(), gpu_rho(g, 16, 5, 0.5, seed=3))


@pytest.mark.parametrize("bad", ["asym", "self", "dup", "unsorted", "negw", "nanw", "asymw", "range", "rowptr"])
def test_invalid_graphs_are_rejected(bad):
    L = lib()
    g = graphgen.grid2d(3, 3)
    rp, col = g.row_ptr.copy(), g.col.copy()
    w = np.ones(g.nnz, np.float32)
    expect = {"asym": 2, "self": 3, "dup": 4, "unsorted": 4, "negw": 5, "nanw": 5, "asymw": 2, "range": 10,
              "rowptr": 10}[bad]
    if bad == "asym":
        col[1] = 5 if col[1] != 5 else 7          # row 0 gets an entry without its mirror
        col[:2] = np.sort(col[:2])
    elif bad == "self":
        col[0] = 0
    elif bad in ("dup", "unsorted"):
        col[1] = col[0] if bad == "dup" else col[1]
        if bad == "unsorted":
            col[0], col[1] = col[1], col[0]
    elif bad == "negw":
        w[3] = -1.0
    elif bad == "nanw":
        w[3] = np.nan
    elif bad == "asymw":
        w[0] = 2.0
    elif bad == "range":
        col[-1] = 99
    elif bad == "rowptr":
        rp[4] = rp[3] - 1
    with pytest.raises(L.ADError) as ei:
        L.ad_graph_create(g.n, rp, col, w)
    assert ei.value.status == expect, (bad, ei.value)


def test_edge_across_batch_is_rejected():
    L = lib()
    g = graphgen.from_edges(6, [0, 1, 3, 2], [1, 2, 4, 3])     # edge (2,3) joins the two graphs
    with pytest.raises(L.ADError) as ei:
        L.ad_graph_create_batched([0, 3, 6], g.n, g.row_ptr, g.col)
    assert ei.value.status == 1


def test_full_size_rmat20_benchmark_configuration():
    """The benchmark's own workload: R-MAT scale 20, R = 32, k = 20, omega = 1/2.

    FP32 storage: every edge within the tolerance of the FP64 oracle, and the
    30% per-node selections (local and global) at Jaccard >= 0.999 against
    the oracle's selection on its own FP64 distances (and exactly equal to the
    oracle's selection on the GPU's FP32 distances).  BF16 and FP16 storage
    (FP32 accumulation): their error against the FP64 oracle is stated and
    bounded -- RMS and worst edge relative to the RMS distance, Jaccard of the
    30% local set."""
    L = lib()
    g = graphgen.rmat(20, 16, seed=2)
    seed = 0x1601055270000000
    ref = ref_rho(g, 32, 20, 0.5, seed=seed)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    rho = np.zeros(g.m, np.float32)
    L.ad_algebraic_distance(h, 32, 20, 0.5, seed, 0, "fp32", 0, rho)
    err = assert_rho_close(rho, ref)
    rms = float(np.sqrt(np.mean(ref ** 2)))
    keeps = {}
    for mode in ("local", "global"):
        keep = np.zeros(g.m, np.uint8)
        L.ad_sparsify(h, 0.3, mode, "per_node", keep)
        own, _, _ = oracle.sparsify(g.row_ptr, g.col, rho.astype(np.float64), mode, "per_node", 0.3)
        np.testing.assert_array_equal(keep, own)
        rk, _, _ = oracle.sparsify(g.row_ptr, g.col, ref, mode, "per_node", 0.3)
        assert jaccard(keep, rk) >= 0.999, (mode, jaccard(keep, rk))
        keeps[mode] = rk
    report = {"fp32": {"max_err_tol_units": err}}
    bounds = {"fp16": (1e-3, 0.5, 0.99), "bf16": (1e-2, 3.0, 0.95)}   # RMS / RMS, max / RMS, Jaccard
    for st, (b_rms, b_max, b_jac) in bounds.items():
        r16 = np.zeros(g.m, np.float32)
        L.ad_algebraic_distance(h, 32, 20, 0.5, seed, 0, st, 0, r16)
        keep = np.zeros(g.m, np.uint8)
        L.ad_sparsify(h, 0.3, "local", "per_node", keep)
        d = r16.astype(np.float64) - ref
        e_rms = float(np.sqrt(np.mean(d ** 2))) / rms
        e_max = float(np.max(np.abs(d))) / rms
        jac = jaccard(keep, keeps["local"])
        report[st] = {"rms_err_over_rms": e_rms, "max_err_over_rms": e_max, "jaccard_local_30": jac}
        assert e_rms <= b_rms and e_max <= b_max and jac >= b_jac, (st, report[st])
    L.ad_graph_destroy(h)
    print("storage error against the FP64 oracle:", report)


def test_repeated_calls_replay_the_same_results():
    """On a handle bound to a capturable stream the second identical call is
    recorded as a CUDA graph and later ones replay it: every call must give
    the same distances, and a change of seed, storage or edge weights must be
    seen by the next call."""
    import torch
    L = lib()
    base = graphgen.rmat(11, 8, seed=4)
    g = graphgen.with_edge_weights(base, graphgen.uniform_edge_weights(base.m, seed=5))
    s = torch.cuda.Stream()
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, g.weight, 0, s)
    w64 = g.weight.astype(np.float64)
    ref = oracle.algebraic_distance(g.row_ptr, g.col, w64, R=16, k=12, omega=0.5, seed=3)
    outs = []
    for _ in range(4):
        rho = np.zeros(g.m, np.float32)
        L.ad_algebraic_distance(h, 16, 12, 0.5, 3, 0, "fp32", 0, rho)
        outs.append(rho)
    for r in outs:
        np.testing.assert_array_equal(r, outs[0])
    assert_rho_close(outs[0], ref)
    rho = np.zeros(g.m, np.float32)
    L.ad_algebraic_distance(h, 16, 12, 0.5, 4, 0, "fp32", 0, rho)          # new seed
    assert_rho_close(rho, oracle.algebraic_distance(g.row_ptr, g.col, w64, R=16, k=12, omega=0.5, seed=4))
    new_w = graphgen.uniform_edge_weights(g.m, seed=9)
    L.ad_graph_set_edge_weights(h, new_w)
    g2 = graphgen.with_edge_weights(g, new_w)
    for _ in range(3):                                                       # same call, new weights
        L.ad_algebraic_distance(h, 16, 12, 0.5, 4, 0, "fp32", 0, rho)
    assert_rho_close(rho, oracle.algebraic_distance(g2.row_ptr, g2.col, g2.weight.astype(np.float64), R=16, k=12,
                                                    omega=0.5, seed=4))
    L.ad_graph_destroy(h)


@pytest.mark.parametrize("storage,R", [("fp32", 32), ("fp16", 32), ("bf16", 16), ("fp32", 8)])
def test_autotuned_shape_keeps_the_distances(storage, R):
    """After ad_graph_autotune the handle uses the chosen sweep shape; the
    distances stay within tolerance of the oracle (FP32) or equal to the
    untuned run up to FP32 summation order (16-bit storage)."""
    L = lib()
    g = graphgen.rmat(13, 16, seed=4)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    before = np.zeros(g.m, np.float32)
    L.ad_algebraic_distance(h, R, 12, 0.5, 3, 0, storage, 0, before)
    lpr, cpl, per_sm = L.ad_graph_autotune(h, R, storage)
    assert lpr >= 1 and cpl in (1, 2) and per_sm in (0, 4, 5)
    after = np.zeros(g.m, np.float32)
    L.ad_algebraic_distance(h, R, 12, 0.5, 3, 0, storage, 0, after)
    L.ad_graph_destroy(h)
    if storage == "fp32":
        assert_rho_close(after, ref_rho(g, R, 12, 0.5, seed=3))
    else:
        assert rho_error(after, before.astype(np.float64)) < 0.05


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_persistent_launch_equals_separate_launches(storage):
    """AD_DIST_PERSISTENT relaxes a single graph in one cooperative launch
    (init, k sweeps with grid-wide barriers, distances); profiling forces one
    launch per sweep.  The arithmetic is the same, so the distances must be
    bit-identical, and the FP32 ones within tolerance of the oracle."""
    L = lib()
    g = weighted(graphgen.rmat(13, 16, seed=12), seed=3)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, g.weight)
    a = np.zeros(g.m, np.float32)
    L.ad_algebraic_distance(h, 32, 20, 0.5, 7, 0, storage, L.AD_DIST_PERSISTENT, a)
    L.ad_graph_set_profiling(h, True)
    b = np.zeros(g.m, np.float32)
    L.ad_algebraic_distance(h, 32, 20, 0.5, 7, 0, storage, 0, b)
    L.ad_graph_set_profiling(h, False)
    L.ad_graph_destroy(h)
    np.testing.assert_array_equal(a, b)
    if storage == "fp32":
        assert_rho_close(a, ref_rho(g, 32, 20, 0.5, seed=7))


def test_persistent_launch_on_a_larger_graph():
    """AD_DIST_PERSISTENT on a graph whose sweeps use every SM."""
    L = lib()
    g = graphgen.rmat(17, 16, seed=5)
    assert g.nnz > (1 << 21)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    a = np.zeros(g.m, np.float32)
    L.ad_algebraic_distance(h, 32, 6, 0.5, 3, 0, "fp32", L.AD_DIST_PERSISTENT, a)
    b = np.zeros(g.m, np.float32)
    L.ad_algebraic_distance(h, 32, 6, 0.5, 3, 0, "fp32", 0, b)
    L.ad_graph_destroy(h)
    np.testing.assert_array_equal(a, b)
    assert_rho_close(a, ref_rho(g, 32, 6, 0.5, seed=3))


def test_grid_barrier_wait_is_bounded():
    """A grid-wide barrier that can never complete ends with AD_ERR_TIMEOUT
    after its poll limit instead of hanging, and the context stays usable."""
    L = lib()
    assert L.ad_selftest_barrier_timeout(polls=2000) == 8      # AD_ERR_TIMEOUT
    g = graphgen.grid2d(16, 16)
    assert_rho_close(gpu_rho(g, 8, 10, 0.5, seed=2), ref_rho(g, 8, 10, 0.5, seed=2))
