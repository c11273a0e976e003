"""Pins of the oracle's SparsifyB (Alg. 3, reading R13): Scott-rule bins of
each node's incident distances (h = 3.5 sigma / d^(1/3), Sec. 4), a
stratified draw over the bins, and the fit of e of Alg. 2.

The pins use closed forms (sigma of an arithmetic progression and of two
point masses), the round-robin structure that "sampling the edges from all
bins" asks for, the Philox words (pinned elsewhere against cuRAND), and a
brute-force union on small graphs."""
import math

import numpy as np
import pytest

import oracle
from paper_1601_05527_gb300 import graphgen

BIN_STREAM = 0xB1000000


def star(d):
    """Centre 0 joined to leaves 1..d; edge t is (0, t + 1)."""
    return graphgen.from_edges(d + 1, np.zeros(d, np.int64), np.arange(1, d + 1))


def entry_word(seed, e):
    return int(oracle.philox4x32_10([e & 0xFFFFFFFF, e >> 32, 0, BIN_STREAM], [seed & 0xFFFFFFFF, seed >> 32])[0])


def test_bins_of_an_arithmetic_progression():
    d, c = 64, 1.0 / 64
    g = star(d)
    scores = c * np.arange(d, dtype=np.float64)
    rank, bins = oracle.binned_ranks(g.row_ptr, g.col, scores, seed=5, return_bins=True)
    sigma = c * math.sqrt((d * d - 1) / 12.0)          # population sigma of 0, c, ..., (d-1) c
    h = 3.5 * sigma / d ** (1.0 / 3.0)
    expect = np.floor(scores / h).astype(np.int64)
    assert expect.max() == 3                           # four bins, no value near a boundary
    np.testing.assert_array_equal(bins[:d], expect)
    assert (bins[d:] == 0).all()                       # leaves: a single distance, one bin
    assert (rank[d:] == 0).all()


def test_two_clusters_alternate():
    a, b = 10, 30
    g = star(a + b)
    scores = np.r_[np.full(a, 0.1), np.full(b, 0.9)]
    rank, bins = oracle.binned_ranks(g.row_ptr, g.col, scores, seed=11, return_bins=True)
    sigma = 0.8 * math.sqrt(a * b) / (a + b)
    h = 3.5 * sigma / (a + b) ** (1.0 / 3.0)
    assert set(bins[:a]) == {0} and set(bins[a:a + b]) == {int(math.floor(0.8 / h))}
    order = np.argsort(rank[:a + b])                   # entries of the centre in selection order
    first = order < a
    for q in range(1, a + 1):                          # every prefix of 2q takes q from each cluster
        assert first[:2 * q].sum() == q
    assert not first[2 * a:].any()


def test_equal_distances_follow_the_random_words():
    d, seed = 50, 123
    g = star(d)
    rank = oracle.binned_ranks(g.row_ptr, g.col, np.full(d, 0.25), seed=seed)
    words = np.array([entry_word(seed, e) for e in range(d)], dtype=np.uint64)
    np.testing.assert_array_equal(rank[:d], np.argsort(np.argsort(words, kind="stable"), kind="stable"))


@pytest.mark.parametrize("seed", [1, 2])
def test_round_robin_over_bins(seed):
    g = graphgen.rmat(9, 12, seed=seed)
    scores = graphgen.random_scores(g.m, None, seed=seed).astype(np.float64) ** 3   # skewed distances
    rank, bins = oracle.binned_ranks(g.row_ptr, g.col, scores, seed=seed, return_bins=True)
    eid = oracle.entry_edge_ids(g.row_ptr, g.col)
    for i in range(g.n):
        p0, p1 = g.row_ptr[i], g.row_ptr[i + 1]
        if p1 - p0 < 2:
            continue
        r, bn, e = rank[p0:p1], bins[p0:p1], eid[p0:p1]
        assert sorted(r) == list(range(p1 - p0))
        seq = bn[np.argsort(r)]
        sizes = {int(x): int((bn == x).sum()) for x in set(bn)}
        taken = {x: 0 for x in sizes}
        for x in seq:
            taken[int(x)] += 1
            rnd = taken[int(x)]                        # round of this entry (1-based)
            # every bin that still had entries in an earlier round has given them already
            assert all(taken[y] >= min(sizes[y], rnd - 1) for y in sizes)
        for x in sizes:                                # inside a bin: ascending Philox word
            members = np.flatnonzero(bn == x)
            by_rank = members[np.argsort(r[members])]
            w = [entry_word(seed, int(e[j])) for j in by_rank]
            assert w == sorted(w)


def test_fit_is_the_brute_force_union():
    g = graphgen.rmat(8, 8, seed=4)
    scores = graphgen.random_scores(g.m, 20, seed=4).astype(np.float64)
    rank = oracle.binned_ranks(g.row_ptr, g.col, scores, seed=9)
    eid = oracle.entry_edge_ids(g.row_ptr, g.col)
    d = np.diff(g.row_ptr)

    def union(e):
        keep = np.zeros(g.m, np.uint8)
        for i in range(g.n):
            T = oracle.degree_target(int(d[i]), e)
            for p in range(g.row_ptr[i], g.row_ptr[i + 1]):
                if rank[p] < T:
                    keep[eid[p]] = 1
        return keep

    for f in (0.0, 0.35, 0.7, 1.0):
        keep, kept, e = oracle.sparsify_binned(g.row_ptr, g.col, scores, 9, f)
        K = oracle.target_count(g.m, f)
        np.testing.assert_array_equal(keep, union(e))
        assert kept == keep.sum() >= K
        if e > 2.0 ** -40:
            assert union(e - 2.0 ** -40).sum() < K
    assert oracle.sparsify_binned(g.row_ptr, g.col, scores, 9, 1.0)[1] == g.m


def expected_bins(scores, d):
    """floor((x - min) / h), h = 3.5 sigma / d^(1/3) with the population sigma."""
    sigma = float(np.std(scores))                      # population (divides by d)
    h = 3.5 * sigma / d ** (1.0 / 3.0)
    frac = (scores - scores.min()) / h
    nz = frac[frac > 0]
    assert np.min(np.abs(nz - np.round(nz))) > 1e-3    # no value near a bin edge
    return np.floor(frac).astype(np.int64)


def test_bins_measure_from_the_smallest_distance():
    """The same progression shifted away from 0: bins count from the row minimum."""
    d = 64
    g = star(d)
    scores = 0.37 + np.arange(d, dtype=np.float64) / 64
    _, bins = oracle.binned_ranks(g.row_ptr, g.col, scores, seed=5, return_bins=True)
    np.testing.assert_array_equal(bins[:d], expected_bins(scores, d))


def test_bins_use_the_population_sigma():
    """d = 12 equally spaced distances: the sample sigma (divide by d - 1) would
    move one value into the next bin; the population sigma is the rule's."""
    d = 12
    g = star(d)
    scores = np.arange(d, dtype=np.float64) / 16
    _, bins = oracle.binned_ranks(g.row_ptr, g.col, scores, seed=5, return_bins=True)
    expect = expected_bins(scores, d)
    sample = np.floor((scores - scores.min()) / (3.5 * np.std(scores, ddof=1) / d ** (1.0 / 3.0)))
    assert (sample != expect).any()                    # the case tells the two apart
    np.testing.assert_array_equal(bins[:d], expect)


def bin_word(seed, i, b):
    return int(oracle.philox4x32_10([i & 0xFFFFFFFF, i >> 32, 1 + b, BIN_STREAM], [seed & 0xFFFFFFFF, seed >> 32])[0])


@pytest.mark.parametrize("seed", [1, 2])
def test_bins_of_a_round_follow_their_random_words(seed):
    """Within a round the bins give their entries in ascending Philox word of
    (vertex, 1 + bin) -- the random order of the bins."""
    g = graphgen.rmat(9, 12, seed=seed)
    scores = graphgen.random_scores(g.m, None, seed=seed).astype(np.float64) ** 3
    rank, bins = oracle.binned_ranks(g.row_ptr, g.col, scores, seed=seed, return_bins=True)
    checked = 0
    for i in range(g.n):
        p0, p1 = g.row_ptr[i], g.row_ptr[i + 1]
        bn = bins[p0:p1]
        if len(set(bn.tolist())) < 2:
            continue
        seq = bn[np.argsort(rank[p0:p1])]              # bins in selection order
        taken, rounds = {}, {}
        for b in seq.tolist():
            taken[b] = taken.get(b, 0) + 1
            rounds.setdefault(taken[b], []).append(b)
        for r, bs in rounds.items():
            words = [bin_word(seed, i, b) for b in bs]
            assert words == sorted(words), (i, r, bs)
        checked += 1
    assert checked > 20
