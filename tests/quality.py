"""Quality measures the paper compares sparsified graphs with (Sec. 2): the
clustering coefficient of Eq. (cc) and the Spearman rank correlation of two
node distributions.  Test helpers on the CPU; not part of the method."""
import numpy as np

from paper_1601_05527_gb300 import graphgen


def local_clustering(g):
    """c_i = (edges among the neighbours of i) / (d_i (d_i - 1) / 2) for d_i > 1,
    NaN where d_i <= 1 (those nodes are outside V' of Eq. (cc))."""
    nb = [set(g.col[g.row_ptr[i]:g.row_ptr[i + 1]].tolist()) for i in range(g.n)]
    c = np.full(g.n, np.nan)
    for i in range(g.n):
        d = len(nb[i])
        if d < 2:
            continue
        links = sum(len(nb[i] & nb[j]) for j in nb[i]) / 2     # each neighbour pair counted from both ends
        c[i] = links / (d * (d - 1) / 2)
    return c


def clustering_coefficient(g):
    """C_G = mean of c_i over V' = {i : d_i > 1} (Eq. (cc))."""
    c = local_clustering(g)
    return float(np.nanmean(c)) if np.isfinite(c).any() else 0.0


def average_ranks(x):
    """Ranks 1..n, tied values sharing the mean of their positions."""
    x = np.asarray(x)
    order = np.argsort(x, kind="stable")
    r = np.empty(len(x), dtype=np.float64)
    xs = x[order]
    i = 0
    while i < len(x):
        j = i
        while j + 1 < len(x) and xs[j + 1] == xs[i]:
            j += 1
        r[order[i:j + 1]] = (i + j) / 2 + 1
        i = j + 1
    return r


def spearman(x, y):
    """rho = 1 - 6 sum p_i^2 / (n (n^2 - 1)), p_i the difference of the ranks (Sec. 2)."""
    n = len(x)
    p = average_ranks(x) - average_ranks(y)
    return 1.0 - 6.0 * float(np.sum(p * p)) / (n * (n * n - 1.0))


def kept_graph(g, keep):
    """The graph of the kept edges (same vertex set)."""
    eu, ev = g.edges_upper()
    k = np.asarray(keep).astype(bool)
    return graphgen.from_edges(g.n, eu[k], ev[k])
