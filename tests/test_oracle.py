"""Pins for the CPU oracle against facts that do not come from the oracle:
hand-derived values, closed forms, library routines and a brute force."""
from __future__ import annotations

import math
from fractions import Fraction

import networkx as nx
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_20403_gb300 import workloads as W
from tests import bruteforce as BF
from tests.helpers import handtree, random_small_graph, graph_from_edges


# ---------------------------------------------------------------- exact sums

def test_exact_sum_matches_fsum_random():
    rng = np.random.default_rng(1)
    for _ in range(300):
        cnt = int(rng.integers(1, 60))
        xs = np.power(10.0, rng.uniform(-20, 20, cnt)) * rng.random(cnt)
        assert O.exact_sum(xs) == math.fsum(xs)


def test_exact_sum_rounding_cases():
    eps = 2.0 ** -53
    # exact tie -> even
    assert O.exact_sum([1.0, eps]) == 1.0
    assert O.exact_sum([1.0 + 2 * eps, eps]) == 1.0 + 4 * eps
    # just above the tie -> up
    assert O.exact_sum([1.0, eps, 2.0 ** -105]) == 1.0 + 2 * eps
    # subnormals and the smallest double
    tiny = 5e-324
    assert O.exact_sum([tiny] * 7) == 7 * tiny
    # far-apart magnitudes
    xs = [1e300, 1.0, 1e-300]
    assert O.exact_sum(xs) == math.fsum(xs)
    # rounding carry into a new binade
    xs = [2.0 ** 53 - 1, 0.5, 0.25]
    assert O.exact_sum(xs) == float(Fraction(2 ** 53 - 1) + Fraction(3, 4))


# ---------------------------------------------------------------- hand-worked example

def test_handtree_scores():
    g, d = handtree()
    s = O.offtree_scores(g, c=2)
    assert sorted(int(i) for i in s["id"]) == sorted(int(k) for k in d["offtree"])
    for j, i in enumerate(s["id"]):
        exp = d["offtree"][str(int(i))]
        assert (int(s["u"][j]), int(s["v"][j])) == (exp["u"], exp["v"])
        assert int(s["lca"][j]) == exp["lca"]
        assert float(s["resistance"][j]) == exp["R"]
        assert float(s["score"][j]) == exp["stretch"]
        assert int(s["beta"][j]) == min(exp["hops"][0], exp["hops"][1], 2)


@pytest.mark.parametrize("key,c,mode", [("stretch_c2", 2, O.SCORE_STRETCH), ("stretch_c1", 1, O.SCORE_STRETCH),
                                         ("stretch_c0", 0, O.SCORE_STRETCH),
                                         ("resistance_c2", 2, O.SCORE_RESISTANCE)])
def test_handtree_recovered(key, c, mode):
    g, d = handtree()
    st, ids, _, _ = O.recover(g, alpha=0.0, c=c, score_mode=mode, k_override=8)
    assert ids.tolist() == d["recovered"][key]
    # a budget cut takes a prefix
    st, ids2, _, _ = O.recover(g, alpha=0.2, c=c, score_mode=mode)
    assert ids2.tolist() == d["recovered"][key][:2]


def test_handtree_noncommutative_bruteforce():
    g, d = handtree()
    a, b = d["noncommutative"]["pair"]
    first, _ = BF.greedy(g, 8, 2, sequence=[a, b])
    second, _ = BF.greedy(g, 8, 2, sequence=[b, a])
    assert first == d["noncommutative"]["first_then_second_recovers"]
    assert sorted(second) == d["noncommutative"]["second_then_first_recovers"]


# ---------------------------------------------------------------- closed forms

def _exact_grounded_resistance(n, tree_edges, root, pairs):
    """Effective resistance by exact rational Gaussian elimination on the
    grounded Laplacian (root row/column removed)."""
    idx = {x: i for i, x in enumerate(y for y in range(n) if y != root)}
    N = n - 1
    L = [[Fraction(0)] * N for _ in range(N)]
    for (a, b, w) in tree_edges:
        c = Fraction(w)
        for x in (a, b):
            if x != root:
                L[idx[x]][idx[x]] += c
        if a != root and b != root:
            L[idx[a]][idx[b]] -= c
            L[idx[b]][idx[a]] -= c
    # invert by Gauss-Jordan on [L | I]
    A = [row[:] + [Fraction(int(i == j)) for j in range(N)] for i, row in enumerate(L)]
    for col in range(N):
        piv = next(r for r in range(col, N) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        inv = 1 / A[col][col]
        A[col] = [x * inv for x in A[col]]
        for r in range(N):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
    Linv = [row[N:] for row in A]
    out = []
    for (u, v) in pairs:
        x = [Fraction(0)] * N
        if u != root:
            x[idx[u]] += 1
        if v != root:
            x[idx[v]] -= 1
        out.append(sum(x[i] * sum(Linv[i][j] * x[j] for j in range(N)) for i in range(N)))
    return out


def test_resistance_equals_effective_resistance():
    """In a tree, the path resistance is the effective resistance
    (e_u - e_v)^T L_T^+ (e_u - e_v).  Checked with numpy's pinv on moderate
    weights (1e-9 relative) and, on weights spanning six decades, with exact
    rational elimination on the grounded Laplacian rounded once, which must
    agree bit for bit (the oracle sums the fl(1/w) values, so the exact
    solve uses those same reciprocals as conductances' inverses)."""
    rng = np.random.default_rng(2)
    for trial in range(16):
        wide = trial % 2 == 1
        g = random_small_graph(rng, n_lo=5, n_hi=22 if wide else 60, tree="mixed",
                               weights="wide" if wide else "uniform")
        s = O.offtree_scores(g, c=2)
        if len(s["u"]) == 0:
            continue
        root = int(np.flatnonzero(g.parent < 0)[0])
        if wide:
            # conductance = 1 / fl(1/w), so the resistance of a tree edge is fl(1/w) exactly
            tree_edges = [(v, int(g.parent[v]), 1 / Fraction(1.0 / BF.tree_weight(g, v)))
                          for v in range(g.n) if g.parent[v] >= 0]
            pairs = [(int(a), int(b)) for a, b in zip(s["u"], s["v"])]
            exact = _exact_grounded_resistance(g.n, tree_edges, root, pairs)
            for j in range(len(pairs)):
                assert float(s["resistance"][j]) == float(exact[j])
        else:
            tree_edges = [(v, int(g.parent[v]), BF.tree_weight(g, v)) for v in range(g.n) if g.parent[v] >= 0]
            Lp = np.linalg.pinv(BF.laplacian(g.n, tree_edges), rcond=1e-10)  # one-dim null space
            for j in range(len(s["u"])):
                x = np.zeros(g.n)
                x[int(s["u"][j])], x[int(s["v"][j])] = 1.0, -1.0
                reff = x @ Lp @ x
                assert abs(float(s["resistance"][j]) - reff) <= 1e-9 * reff


def test_path_graph_prefix_sums():
    """Path 0-1-...-(n-1) as the tree plus chords (0, j): R = prefix sum."""
    n = 40
    rng = np.random.default_rng(3)
    wt = np.power(2.0, rng.integers(-6, 6, n - 1)).astype(float)  # exact reciprocals
    edges = [(i, i + 1, float(wt[i])) for i in range(n - 1)]
    edges += [(0, j, 1.0) for j in range(2, n)]
    parent = [-1] + list(range(n - 1))
    g = graph_from_edges(n, edges, parent)
    s = O.offtree_scores(g, c=2)
    for j in range(len(s["u"])):
        u, v = int(s["u"][j]), int(s["v"][j])
        assert u == 0
        assert float(s["resistance"][j]) == float(sum(Fraction(1.0 / wt[i]) for i in range(v)))
        assert int(s["lca"][j]) == 0
        assert int(s["beta"][j]) == 0  # u is its own LCA


# ---------------------------------------------------------------- brute force

def _check_scores_vs_bruteforce(g, c, mode):
    s = O.offtree_scores(g, c=c, score_mode=O.SCORE_RESISTANCE if mode == "resistance" else O.SCORE_STRETCH)
    facts = BF.edge_facts(g, c, mode)
    assert sorted(facts) == sorted(int(i) for i in s["id"])
    for j, i in enumerate(s["id"]):
        f = facts[int(i)]
        assert int(s["lca"][j]) == f["lca"]
        assert float(s["resistance"][j]) == f["R"]
        assert float(s["score"][j]) == f["score"]
        assert int(s["beta"][j]) == f["beta"]


def test_scores_vs_bruteforce_random():
    rng = np.random.default_rng(4)
    for trial in range(60):
        g = random_small_graph(rng, tree="mixed")
        _check_scores_vs_bruteforce(g, int(rng.integers(0, 4)), ["stretch", "resistance"][trial % 2])


def test_lca_vs_networkx():
    rng = np.random.default_rng(5)
    for _ in range(20):
        g = random_small_graph(rng, n_lo=10, n_hi=40, tree="random")
        s = O.offtree_scores(g, c=2)
        root = int(np.flatnonzero(g.parent < 0)[0])
        T = nx.DiGraph()
        T.add_nodes_from(range(g.n))
        for v in range(g.n):
            if g.parent[v] >= 0:
                T.add_edge(int(g.parent[v]), v)
        pairs = [(int(a), int(b)) for a, b in zip(s["u"], s["v"])]
        want = dict(nx.tree_all_pairs_lowest_common_ancestor(T, root=root, pairs=pairs))
        for j, p in enumerate(pairs):
            assert int(s["lca"][j]) == want[p]


@pytest.mark.parametrize("seed", range(6))
def test_recover_vs_bruteforce_random(seed):
    rng = np.random.default_rng(100 + seed)
    for trial in range(40):
        g = random_small_graph(rng, tree="mixed")
        c = int(rng.integers(0, 4))
        mode = ["stretch", "resistance"][int(rng.integers(2))]
        k = int(rng.integers(0, g.m + 1))
        st, ids, _, _ = O.recover(g, 0.0, c=c, k_override=k,
                                  score_mode=O.SCORE_RESISTANCE if mode == "resistance" else O.SCORE_STRETCH)
        want, _ = BF.greedy(g, k, c, mode)
        assert ids.tolist() == want, (g.n, c, k, mode)
        assert st == (O.UNDER_BUDGET if len(want) < k else O.OK)


def test_recover_with_alpha_budget():
    rng = np.random.default_rng(7)
    for _ in range(20):
        g = random_small_graph(rng, n_lo=8, n_hi=14)
        alpha = float(rng.uniform(0, 0.6))
        st, ids, _, _ = O.recover(g, alpha, c=2)
        want, _ = BF.greedy(g, BF.budget(g.n, alpha), 2)
        assert ids.tolist() == want


def test_c0_is_topk_by_score():
    """c = 0 makes every neighbourhood a single vertex, so nothing is ever
    marked (simple graph): the output is the top-k of (score desc, id asc),
    which numpy's lexsort gives independently."""
    g = W.grid_graph(20, seed=11)
    s = O.offtree_scores(g, c=0)
    k = 60
    order = np.lexsort((s["id"], -s["score"]))
    st, ids, sc, _ = O.recover(g, 0.0, c=0, k_override=k)
    assert ids.tolist() == s["id"][order[:k]].tolist()
    assert sc.tolist() == s["score"][order[:k]].tolist()


def test_ties_break_by_smaller_id():
    """Unit weights on a grid give massive score ties."""
    n_side = 8
    eu, ev = W.grid2d_edges(n_side, n_side)
    ew = np.ones(eu.shape[0])
    g = W.build_graph(n_side * n_side, eu, ev, ew)
    st, ids, sc, _ = O.recover(g, 0.0, c=0, k_override=20)
    for a, b, sa, sb in zip(ids[:-1], ids[1:], sc[:-1], sc[1:]):
        assert sa > sb or (sa == sb and a < b)
    want, _ = BF.greedy(g, 20, 0)
    assert ids.tolist() == want


# ---------------------------------------------------------------- invariants

def _invariants(g, c, ids, k, full):
    T = BF.tree_graph(g)
    facts = BF.edge_facts(g, c)
    order = BF.order(facts)
    acc = set(int(i) for i in ids)
    accepted_seq = [i for i in order if i in acc]
    assert accepted_seq == [int(i) for i in ids]  # recovery order = score order
    last = order.index(int(ids[-1])) if len(ids) else -1
    prefix_acc = []
    for pos in range(last + 1):
        i = order[pos]
        sim = any(BF.strictly_similar(T, facts[i], facts[a]) for a in prefix_acc)
        if i in acc:
            assert not sim  # independence
            prefix_acc.append(i)
        else:
            assert sim  # maximality
            # Lemma share-LCA: any marker has the same LCA
            assert any(facts[a]["lca"] == facts[i]["lca"] and BF.strictly_similar(T, facts[i], facts[a])
                       for a in prefix_acc)
    assert len(ids) == min(k, full)
    # T plus the recovered edges is connected with n - 1 + |A| edges
    P = nx.Graph(T)
    for i in ids:
        P.add_edge(facts[int(i)]["u"], facts[int(i)]["v"])
    assert nx.is_connected(P) and P.number_of_edges() == g.n - 1 + len(ids)


def test_invariants_random_medium():
    rng = np.random.default_rng(8)
    for _ in range(6):
        g = random_small_graph(rng, n_lo=20, n_hi=40, tree="max", weights="uniform")
        k = g.n // 4
        st, ids, _, full = O.recover(g, 0.0, c=2, k_override=k, full_count=True)
        _invariants(g, 2, ids, k, full)


def test_invariants_grid():
    g = W.grid_graph(12, seed=9)
    st, ids, _, full = O.recover(g, 0.1, c=2, full_count=True)
    _invariants(g, 2, ids, BF.budget(g.n, 0.1), full)


def test_spectral_monotone():
    """L_P <= L_G for a subgraph P with the same weights, so every generalised
    eigenvalue of (L_G, L_P) is >= 1, and adding recovered edges to the tree
    cannot raise lambda_max (Sec. 2.1, relative condition number)."""
    rng = np.random.default_rng(10)
    for _ in range(4):
        g = random_small_graph(rng, n_lo=25, n_hi=45, tree="max", weights="uniform")
        edges = [(u, v, w) for (_, u, v, w) in BF.canonical_edges(g)]
        LG = BF.laplacian(g.n, edges)
        facts = BF.edge_facts(g, 2)
        tree_edges = [(v, int(g.parent[v]), BF.tree_weight(g, v)) for v in range(g.n) if g.parent[v] >= 0]
        st, ids, _, _ = O.recover(g, 0.0, c=2, k_override=g.n // 3)
        prev = None
        for t in range(len(ids) + 1):
            P = tree_edges + [(facts[int(i)]["u"], facts[int(i)]["v"], facts[int(i)]["w"]) for i in ids[:t]]
            ev = BF.generalized_eigs(LG, BF.laplacian(g.n, P))
            assert ev[0] >= 1 - 1e-8
            if prev is not None:
                assert ev[-1] <= prev * (1 + 1e-8)
            prev = ev[-1]


def test_under_budget_on_tree_only_graph():
    n = 12
    edges = [(i, i + 1, 1.0 + i) for i in range(n - 1)]
    g = graph_from_edges(n, edges, [-1] + list(range(n - 1)))
    st, ids, _, _ = O.recover(g, 0.5, c=2)
    assert st == O.UNDER_BUDGET and len(ids) == 0


def test_oracle_rejects_non_tree():
    g, _ = handtree()
    bad = g.parent.copy()
    bad[1] = 7  # 1 -> 7 -> 3 -> 1 is a cycle
    g2 = W.Graph(n=g.n, row_ptr=g.row_ptr, col=g.col, w=g.w, parent=bad)
    with pytest.raises(RuntimeError):
        O.recover(g2, 0.1)


# ---------------------------------------------------------------- the two scoring methods

@pytest.mark.parametrize("maker", [lambda: W.mesh3d_graph(14, seed=21), lambda: W.rmat_graph(12, seed=22),
                                   lambda: W.grid_graph(40, seed=23)])
def test_walk_and_dists_methods_agree(maker):
    """Algorithm 1's route (dists + skip table) equals the path-walk definition bit for bit."""
    g = maker()
    for mode in (O.SCORE_STRETCH, O.SCORE_RESISTANCE):
        a = O.offtree_scores(g, c=2, score_mode=mode, method=O.METHOD_WALK)
        b = O.offtree_scores(g, c=2, score_mode=mode, method=O.METHOD_DISTS)
        for key in a:
            assert np.array_equal(a[key], b[key]), key


def test_dists_method_wide_weights_random():
    rng = np.random.default_rng(31)
    for _ in range(30):
        g = random_small_graph(rng, n_lo=3, n_hi=30, tree="mixed", weights="wide")
        a = O.offtree_scores(g, c=3, method=O.METHOD_WALK)
        b = O.offtree_scores(g, c=3, method=O.METHOD_DISTS)
        for key in a:
            assert np.array_equal(a[key], b[key]), key


def test_prefix_restart_matches_full_pass():
    """The prefix-bounded greedy returns the same edges as a run over the whole order."""
    g = W.mesh3d_graph(12, seed=24)
    for k in (5, 50, 400, 2000):
        st, ids, _, full = O.recover(g, 0.0, c=2, k_override=k, full_count=True)
        st2, ids2, _, _ = O.recover(g, 0.0, c=2, k_override=k)
        assert ids.tolist() == ids2.tolist()
