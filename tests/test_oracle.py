"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: the paper's definitions or theorems, a closed
form, brute force over all spanning trees, an independent algorithm, a library routine for a
special case, or exact rational arithmetic.  None of these tests needs a GPU.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthdata

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers (independent code)

def _all_edges_sorted(x, cd2=None):
    """All n(n-1)/2 edges sorted by K, w2 computed here term by term in dimension order."""
    n, d = x.shape
    iu, iv = np.triu_indices(n, 1)
    w2 = np.zeros(len(iu))
    for k in range(d):
        t = x[iu, k] - x[iv, k]
        w2 = w2 + t * t
    if cd2 is not None:
        w2 = np.maximum(np.maximum(w2, cd2[iu]), cd2[iv])
    order = np.lexsort((iv, iu, w2))
    return iu[order], iv[order], w2[order]


def _kruskal_all(n, iu, iv, w2):
    par = list(range(n))

    def find(a):
        while par[a] != a:
            par[a] = par[par[a]]
            a = par[a]
        return a
    out = []
    for a, b, w in zip(iu.tolist(), iv.tolist(), w2.tolist()):
        ra, rb = find(a), find(b)
        if ra != rb:
            par[ra] = rb
            out.append((a, b, w))
            if len(out) == n - 1:
                break
    return out


def _prufer_trees(n):
    """All n^(n-2) labelled trees on n vertices via Pruefer sequences."""
    for seq in itertools.product(range(n), repeat=n - 2):
        degree = [1] * n
        for s in seq:
            degree[s] += 1
        edges = []
        for s in seq:
            leaf = min(i for i in range(n) if degree[i] == 1)
            edges.append((min(leaf, s), max(leaf, s)))
            degree[leaf] -= 1
            degree[s] -= 1
        u, v = [i for i in range(n) if degree[i] == 1]
        edges.append((u, v))
        yield edges


def _edge_set(u, v):
    return set(zip(np.minimum(u, v).tolist(), np.maximum(u, v).tolist()))


# ------------------------------------------------------------------------ distance (Sec. 2.1)

@pytest.mark.parametrize("d", [1, 2, 3, 5, 7, 16])
def test_sqdist_within_fp64_error_bound_of_exact_value(d):
    """D(p,q) agrees with the exact rational sum of squares within (d+2) units of 2^-53."""
    x = synthdata.uniform(40, d, seed=d) * 7.0 - 3.0
    u = 2.0 ** -53
    for i in range(0, 40, 3):
        for j in range(1, 40, 7):
            exact = sum((Fraction(x[i, k]) - Fraction(x[j, k])) ** 2 for k in range(d))
            got = Fraction(oracle.sqdist(x, i, j))
            if exact == 0:
                assert got == 0
            else:
                assert abs(got - exact) / exact <= (d + 2) * u


def test_sqdist_is_exact_on_integers():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 2.0], [-3.0, 4.0, 12.0]])
    assert oracle.sqdist(x, 0, 1) == 9.0
    assert oracle.sqdist(x, 0, 2) == 169.0
    assert oracle.sqdist(x, 1, 2) == 16.0 + 4.0 + 100.0


# --------------------------------------------------------------------------- EMST (Sec. 2.1)

@pytest.mark.parametrize("n,d,seed", [(5, 2, 0), (6, 3, 1), (7, 2, 2), (7, 5, 3)])
def test_emst_equals_brute_force_over_all_spanning_trees(n, d, seed):
    """The unique K-minimum spanning tree is the minimiser of the sum of K-ranks over all trees."""
    x = synthdata.uniform(n, d, seed)
    iu, iv, _ = _all_edges_sorted(x)
    rank = {(a, b): r for r, (a, b) in enumerate(zip(iu.tolist(), iv.tolist()))}
    best = min(_prufer_trees(n), key=lambda es: sum(rank[e] for e in es))
    r = oracle.emst(x)
    assert _edge_set(r["u"], r["v"]) == set(best)


@pytest.mark.parametrize("n,d,seed,kind", [(300, 2, 0, "uniform"), (500, 3, 1, "uniform"),
                                           (400, 7, 2, "uniform"), (600, 3, 3, "gmm"),
                                           (700, 2, 4, "varden")])
def test_emst_equals_independent_kruskal_on_all_edges(n, d, seed, kind):
    x = synthdata.generate(kind, n, d, seed).astype(np.float64)
    iu, iv, w2 = _all_edges_sorted(x)
    kr = _kruskal_all(n, iu, iv, w2)
    r = oracle.emst(x)
    # Kruskal emits edges in K order, so the oracle's K-sorted list must agree entry by entry.
    assert [(a, b) for a, b, _ in kr] == list(zip(r["u"].tolist(), r["v"].tolist()))
    assert np.array_equal(np.array([w for _, _, w in kr]), r["w2"])


@pytest.mark.parametrize("n,d,seed", [(200, 2, 5), (300, 3, 6), (250, 5, 7)])
def test_emst_total_weight_matches_scipy_csgraph(n, d, seed):
    from scipy.sparse.csgraph import minimum_spanning_tree
    from scipy.spatial.distance import cdist
    x = synthdata.uniform(n, d, seed)
    ref = minimum_spanning_tree(cdist(x, x)).sum()
    assert abs(oracle.emst(x)["total"] - ref) <= 1e-12 * ref


def test_emst_cut_property_on_every_tree_edge():
    """Each tree edge is the K-minimum edge crossing the cut it defines in the tree."""
    x = synthdata.gaussian_mixture(160, 2, seed=3).astype(np.float64)
    n = len(x)
    r = oracle.emst(x)
    iu, iv, w2 = _all_edges_sorted(x)
    for k in range(n - 1):
        # side of r.u[k] after removing edge k
        adj = [[] for _ in range(n)]
        for j in range(n - 1):
            if j != k:
                adj[r["u"][j]].append(r["v"][j])
                adj[r["v"][j]].append(r["u"][j])
        side = np.zeros(n, bool)
        stack = [r["u"][k]]
        side[r["u"][k]] = True
        while stack:
            a = stack.pop()
            for b in adj[a]:
                if not side[b]:
                    side[b] = True
                    stack.append(b)
        crossing = side[iu] != side[iv]
        first = np.flatnonzero(crossing)[0]   # edges are K-sorted
        assert (iu[first], iv[first]) == (r["u"][k], r["v"][k])


@pytest.mark.parametrize("n", [2, 17, 100, 1000])
def test_emst_collinear_closed_form(n):
    """n unit-spaced collinear points: every MST has n-1 unit edges, total n-1."""
    r = oracle.emst(synthdata.collinear(n, d=2, seed=n))
    assert len(r["u"]) == n - 1
    assert np.all(r["w2"] == 1.0)
    assert r["total"] == float(n - 1)


@pytest.mark.parametrize("k,d", [(2, 2), (7, 2), (20, 2), (5, 3)])
def test_emst_unit_grid_closed_form(k, d):
    """The unit grid {0..k-1}^d: total weight k^d - 1, every edge of length 1."""
    r = oracle.emst(synthdata.unit_grid(k, d, seed=k))
    assert np.all(r["w2"] == 1.0)
    assert r["total"] == float(k ** d - 1)


def test_emst_single_point_and_duplicates():
    r = oracle.emst(np.zeros((1, 3)))
    assert len(r["u"]) == 0 and r["total"] == 0.0
    x = np.array([[0.5, 0.5]] * 4 + [[2.0, 0.5]])
    r = oracle.emst(x)
    # duplicates: zero-weight edges ordered by ids, then the unit-and-a-half edge
    assert list(zip(r["u"].tolist(), r["v"].tolist()))[:3] == [(0, 1), (0, 2), (0, 3)]
    assert r["w2"][-1] == 2.25


def test_tie_certificate():
    assert oracle.emst(synthdata.unit_grid(4, 2, 0))["tie"]
    assert not oracle.emst(synthdata.uniform(500, 2, 0))["tie"]


# -------------------------------------------------------------- core distances (Sec. 2.1)

def test_core_distance_min_pts_one_is_zero():
    assert np.all(oracle.core_dist2(synthdata.uniform(100, 3, 0), 1) == 0.0)


@pytest.mark.parametrize("min_pts", [2, 3, 10, 50])
def test_core_distance_matches_scipy_kdtree(min_pts):
    """cd(p) = distance to the min_pts-th nearest neighbour counting p itself (k = min_pts)."""
    from scipy.spatial import cKDTree
    x = synthdata.gaussian_mixture(800, 3, seed=min_pts).astype(np.float64)
    dist, _ = cKDTree(x).query(x, k=min_pts)
    ref = dist[:, -1] if min_pts > 1 else dist
    got = np.sqrt(oracle.core_dist2(x, min_pts))
    assert np.allclose(got, ref, rtol=1e-13, atol=0)


def test_core_distance_with_duplicates_counts_multiplicity():
    x = np.array([[0.0], [0.0], [0.0], [3.0]])
    assert oracle.core_dist2(x, 3).tolist() == [0.0, 0.0, 0.0, 9.0]
    assert oracle.core_dist2(x, 4).tolist() == [9.0, 9.0, 9.0, 9.0]


# ------------------------------------------------------- HDBSCAN* MST (Sec. 2.1, App. theorem)

@pytest.mark.parametrize("min_pts", [1, 2])
def test_hdbscan_mst_equals_emst_for_min_pts_at_most_two(min_pts):
    """For minPts <= 2 every mutual reachability weight is the Euclidean distance."""
    x = synthdata.uniform(400, 3, 11)
    e = oracle.emst(x)
    h = oracle.hdbscan(x, min_pts)
    assert np.array_equal(e["u"], h["u"]) and np.array_equal(e["v"], h["v"])
    assert np.array_equal(e["w2"], h["w2"])


@pytest.mark.parametrize("seed", [12, 13])
def test_hdbscan_min_pts_three_emst_edges_form_an_mst_of_gmr(seed):
    """The EMST's edge set is an MST of G_MR when minPts = 3 (appendix theorem): weighed with
    d_m, the EMST edges have the same total as the oracle's MST of G_MR."""
    x = synthdata.uniform(500, 2, seed)
    e = oracle.emst(x)
    h = oracle.hdbscan(x, 3)
    cd2 = h["cd2"]
    dm2 = np.maximum(np.maximum(e["w2"], cd2[e["u"]]), cd2[e["v"]])
    assert abs(np.sort(np.sqrt(dm2)).sum() - np.sort(h["w"]).sum()) <= 1e-12 * h["total"]
    # and for minPts = 4 the paper gives a counterexample, so no such check is made there.


@pytest.mark.parametrize("n,d,min_pts,seed", [(300, 2, 5, 0), (400, 3, 10, 1), (250, 5, 4, 2)])
def test_hdbscan_mst_equals_independent_kruskal(n, d, min_pts, seed):
    x = synthdata.gaussian_mixture(n, d, seed).astype(np.float64)
    cd2 = oracle.core_dist2(x, min_pts)
    iu, iv, w2 = _all_edges_sorted(x, cd2)
    kr = _kruskal_all(n, iu, iv, w2)
    h = oracle.hdbscan(x, min_pts)
    assert [(a, b) for a, b, _ in kr] == list(zip(h["u"].tolist(), h["v"].tolist()))


# ------------------------------------------------------ dendrogram and plot (Sec. 2.1, Sec. 4)

def _cluster_sets(n, left, right):
    sets = {i: frozenset([i]) for i in range(n)}
    out = []
    for i, (a, b) in enumerate(zip(left.tolist(), right.tolist())):
        s = sets[a] | sets[b]
        sets[n + i] = s
        out.append((sets[a], sets[b]))
    return out


def test_single_linkage_dendrogram_matches_scipy_linkage():
    from scipy.cluster.hierarchy import linkage
    x = synthdata.uniform(300, 2, 21)
    n = len(x)
    e = oracle.emst(x)
    sl = oracle.single_linkage(n, e["u"], e["v"], e["w2"], s=0)
    Z = linkage(x, method="single")
    assert np.allclose(Z[:, 2], sl["height"], rtol=1e-12, atol=0)
    # merge i joins the same two clusters (as unordered sets of points)
    zsets = {i: frozenset([i]) for i in range(n)}
    mine = _cluster_sets(n, sl["left"], sl["right"])
    for i, row in enumerate(Z):
        a, b = zsets[int(row[0])], zsets[int(row[1])]
        zsets[n + i] = a | b
        assert {a, b} == set(mine[i])
        assert int(row[3]) == sl["size"][i]


@pytest.mark.parametrize("s", [0, 7, 199])
def test_ordered_dendrogram_inorder_equals_prim_order(s):
    """The in-order leaves of the ordered dendrogram are the reachability-plot order (Sec. 4.1)."""
    x = synthdata.gaussian_mixture(200, 3, seed=s).astype(np.float64)
    h = oracle.hdbscan(x, 5, s=s)
    assert h["order"][0] == s
    assert np.array_equal(h["order"], h["inorder"])


def test_reachability_bar_is_min_mutual_reachability_to_earlier_points():
    """Bar i = min over j < i of d_m(p_i, p_j), straight from the definition (Sec. 2.1)."""
    x = synthdata.gaussian_mixture(250, 2, seed=4).astype(np.float64)
    mp = 6
    h = oracle.hdbscan(x, mp, s=3)
    cd2 = h["cd2"]
    order = h["order"]
    for i in range(1, len(order)):
        p = order[i]
        q = order[:i]
        dd = np.zeros(len(q))
        for k in range(x.shape[1]):
            t = x[p, k] - x[q, k]
            dd = dd + t * t
        dm2 = np.maximum(np.maximum(dd, cd2[p]), cd2[q])
        assert h["reach"][i] == math.sqrt(dm2.min())
    assert h["reach"][0] == math.inf


def test_reachability_bar_is_height_of_inorder_internal_node():
    """Leaves i-1 and i of the ordered dendrogram meet at the internal node of height reach[i]."""
    x = synthdata.uniform(150, 2, 9)
    n = len(x)
    h = oracle.hdbscan(x, 4, s=0)
    pos = np.empty(n, int)
    pos[h["inorder"]] = np.arange(n)
    # in-order interval of each node
    lo = list(range(n)) + [0] * (n - 1)
    hi = list(range(n)) + [0] * (n - 1)
    lo = [pos[i] for i in range(n)] + [0] * (n - 1)
    hi = [pos[i] for i in range(n)] + [0] * (n - 1)
    sep = {}
    for i in range(n - 1):
        a, b = h["left"][i], h["right"][i]
        lo[n + i], hi[n + i] = lo[a], hi[b]
        assert hi[a] + 1 == lo[b]
        sep[lo[b]] = h["height"][i]
    for i in range(1, n):
        assert h["reach"][i] == sep[i]


def test_dendrogram_heights_monotone_and_sizes_consistent():
    x = synthdata.varden_blobs(400, 3, seed=2).astype(np.float64)
    n = len(x)
    h = oracle.hdbscan(x, 10)
    size = np.concatenate([np.ones(n, int), h["size"]])
    height = np.concatenate([np.zeros(n), h["height"]])
    for i in range(n - 1):
        a, b = h["left"][i], h["right"][i]
        assert height[a] <= h["height"][i] and height[b] <= h["height"][i]
        assert size[a] + size[b] == h["size"][i]
    assert h["size"][-1] == n


def test_cut_at_eps_equals_components_of_light_tree_edges():
    """Cutting the dendrogram at eps = removing MST edges heavier than eps (Sec. 2.1)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    x = synthdata.gaussian_mixture(300, 2, seed=8).astype(np.float64)
    n = len(x)
    h = oracle.hdbscan(x, 5)
    eps = float(np.quantile(h["w"], 0.8))
    keep = h["w"] <= eps
    g = coo_matrix((np.ones(keep.sum()), (h["u"][keep], h["v"][keep])), shape=(n, n))
    _, lab = connected_components(g, directed=False)
    # dendrogram cut: climb from each leaf while the parent's height <= eps
    parent = np.full(2 * n - 1, -1)
    for i in range(n - 1):
        parent[h["left"][i]] = n + i
        parent[h["right"][i]] = n + i
    height = np.concatenate([np.zeros(n), h["height"]])
    top = []
    for p in range(n):
        a = p
        while parent[a] >= 0 and height[parent[a]] <= eps:
            a = parent[a]
        top.append(a)
    top = np.array(top)
    for p in range(n):
        assert np.array_equal(lab == lab[p], top == top[p])


# ------------------------------------------------------- the paper's worked example (Fig. 1)

def test_figure1_caption_facts():
    with open(os.path.join(GOLDEN, "fig1_worked_example.json")) as f:
        g = json.load(f)
    names = g["names"]
    idx = {k: i for i, k in enumerate(names)}
    x = np.array(g["points"], float)
    facts = g["facts"]
    h = oracle.hdbscan(x, g["min_pts"], s=idx[g["start"]])
    cd = h["cd"]
    assert cd[idx["a"]] == facts["core_distance_a"]
    dist_a = np.sqrt([oracle.sqdist(x, idx["a"], j) for j in range(len(x))])
    third = np.argsort(dist_a, kind="stable")[g["min_pts"] - 1]
    assert names[third] == facts["third_nn_of_a_including_itself"]
    assert dist_a[idx["b"]] == facts["dist_a_b"]
    t = facts["edge_a_d_terms"]
    assert cd[idx["a"]] == t["cd_a"] and h["cd2"][idx["d"]] == t["cd_d_squared"]
    assert oracle.sqdist(x, idx["a"], idx["d"]) == t["dist_a_d_squared"]
    a, d = idx["a"], idx["d"]
    w_ad = math.sqrt(max(h["cd2"][a], h["cd2"][d], oracle.sqdist(x, a, d)))
    assert w_ad == facts["edge_a_d_weight"]
    assert (min(a, d), max(a, d)) in _edge_set(h["u"], h["v"])
    eps = facts["cut_eps"]
    core = cd <= eps
    assert sorted(names[i] for i in np.flatnonzero(~core)) == sorted(facts["noise_at_cut"])
    # clusters: components of MST edges <= eps among core points
    par = list(range(len(x)))

    def find(q):
        while par[q] != q:
            q = par[q]
        return q
    for u, v, w in zip(h["u"], h["v"], h["w"]):
        if w <= eps and core[u] and core[v]:
            par[find(u)] = find(v)
    groups = {}
    for i in np.flatnonzero(core):
        groups.setdefault(find(i), set()).add(names[i])
    assert sorted(map(sorted, groups.values())) == sorted(map(sorted, facts["clusters_at_cut"]))
    order = [names[i] for i in h["order"]]
    k = 0
    for valley in facts["plot_valleys_in_order"]:
        assert set(order[k:k + len(valley)]) == set(valley)
        k += len(valley)


def test_core_dist_subset_and_nearest_edge_agree_with_full_oracle():
    x = synthdata.gaussian_mixture(500, 3, seed=3).astype(np.float64)
    idx = np.array([0, 7, 123, 499])
    assert np.array_equal(oracle.core_dist2_subset(x, 7, idx), oracle.core_dist2(x, 7)[idx])
    e = oracle.emst(x)
    es = _edge_set(e["u"], e["v"])
    iu, iv, w2 = _all_edges_sorted(x)
    for p in (0, 11, 250):
        q, w = oracle.nearest_edge(x, p)
        assert (min(p, q), max(p, q)) in es            # cut property of the singleton {p}
        first = np.flatnonzero((iu == p) | (iv == p))[0]
        assert (iu[first], iv[first]) == (min(p, q), max(p, q)) and w2[first] == w


# ---------------------------------------------------------------- the solvers used at scale
# k-d tree Boruvka and k-d tree k-NN compute the same trees and core distances as the brute-force
# definitions above by other algorithms; every case must agree exactly (edge list in K order and
# bit-identical w2), including fully tied inputs (grids, duplicates) where only K decides.

@pytest.mark.parametrize("kind,n,d,seed", [("uniform", 1200, 2, 0), ("gmm", 1500, 3, 1), ("varden", 1500, 5, 2),
                                           ("uniform", 700, 7, 3), ("varden", 900, 3, 4)])
def test_boruvka_equals_prim_emst(kind, n, d, seed):
    x = synthdata.generate(kind, n, d, seed=seed)
    e = oracle.emst(x)
    u, v, w2 = oracle.boruvka(x)
    assert np.array_equal(u, e["u"]) and np.array_equal(v, e["v"]) and np.array_equal(w2, e["w2"])


@pytest.mark.parametrize("k,d", [(12, 2), (6, 3)])
def test_boruvka_equals_prim_on_tied_grid(k, d):
    x = synthdata.unit_grid(k, d, seed=k)
    e = oracle.emst(x)
    u, v, w2 = oracle.boruvka(x)
    assert np.array_equal(u, e["u"]) and np.array_equal(v, e["v"]) and np.array_equal(w2, e["w2"])
    assert math.isclose(oracle.total_weight(w2), k ** d - 1, rel_tol=1e-12)


def test_boruvka_with_duplicate_points():
    x = np.repeat(synthdata.uniform(200, 3, seed=5), 3, axis=0)
    e = oracle.emst(x)
    u, v, w2 = oracle.boruvka(x)
    assert np.array_equal(u, e["u"]) and np.array_equal(v, e["v"]) and np.array_equal(w2, e["w2"])
    assert np.count_nonzero(w2 == 0.0) == 400


@pytest.mark.parametrize("kind,n,d,min_pts,seed", [("gmm", 1500, 3, 10, 0), ("uniform", 1000, 2, 5, 1),
                                                   ("varden", 1200, 5, 4, 2), ("uniform", 600, 7, 20, 3)])
def test_kdtree_core_distances_and_boruvka_gmr_equal_brute_force(kind, n, d, min_pts, seed):
    x = synthdata.generate(kind, n, d, seed=seed)
    cd2 = oracle.core_dist2(x, min_pts)
    assert np.array_equal(oracle.core_dist2_kdtree(x, min_pts), cd2)
    pu, pv, pw, _ = oracle.prim_complete(x, cd2)
    pu, pv, pw = oracle.sort_edges(pu, pv, pw)
    u, v, w2 = oracle.boruvka(x, cd2)
    assert np.array_equal(u, pu) and np.array_equal(v, pv) and np.array_equal(w2, pw)


def test_hdbscan_at_scale_equals_hdbscan():
    x = synthdata.gaussian_mixture(1200, 3, seed=7)
    a = oracle.hdbscan(x, 10, 5)
    b = oracle.hdbscan_at_scale(x, 10, 5)
    for key in ("cd2", "u", "v", "w2", "left", "right", "height", "size", "order", "reach"):
        assert np.array_equal(a[key], b[key]), key


def test_kdtree_solvers_fail_loudly_when_a_search_stack_overflows():
    # A median-split tree never fills the 256-entry search stacks; with the capacity lowered, a
    # search that would have to drop a subtree must fail instead of returning a wrong value.
    x = synthdata.uniform(5000, 3, seed=11)
    oracle.set_kd_stack_cap(6)
    try:
        with pytest.raises(RuntimeError, match="code -3"):
            oracle.core_dist2_kdtree(x, 10)
        with pytest.raises(RuntimeError, match="code -3"):
            oracle.boruvka(x)
    finally:
        oracle.set_kd_stack_cap(256)
    assert np.array_equal(oracle.core_dist2_kdtree(x, 10), oracle.core_dist2(x, 10))
