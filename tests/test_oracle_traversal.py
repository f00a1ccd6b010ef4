"""Pins of the oracle's dual tree traversal (section "Dual tree traversal").

* The paper states that theta = 0.5 with its MAC is equivalent to a typical FMM
  with a 3x3x3 neighbour list (Results section).
* The interaction stencil is "mutually exclusive at each level": every ordered
  pair of particles is accounted for exactly once, either by a particle-particle
  leaf pair or by exactly one cell-cell pair of cells containing them.
* The dual traversal is O(N): interaction counts per particle stay bounded."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_5815_gb300 import inputs
from tests.oracle_helpers import cell_index, coverage_matrix


def _lattice(m, seed=0):
    """One jittered point in each cell of an m^3 grid (m a power of two)."""
    rng = np.random.default_rng(seed)
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1)
    g = g.reshape(-1, 3).astype(np.float64)
    x = (g + 0.25 + 0.5 * rng.random(g.shape)) / m
    # pin the box to exactly [0,1]^3 with two corner points
    x = np.vstack([x, [[0, 0, 0], [1, 1, 1]]])
    return x.astype(np.float32), rng.uniform(-1, 1, len(x)).astype(np.float32)


def test_theta_half_is_3x3x3_neighbour_list():
    m = 8
    x, q = _lattice(m)
    # ncrit = 1 except the two corner cells which hold 2 points; max_depth 3
    f = O.Fmm(x, q, 2, 0.5, 1, max_depth=3)
    c, L = f.cells(), f.lists()
    k = cell_index(c["level"], c["prefix"])
    leaves = np.flatnonzero(c["nchild"] == 0)
    assert np.all(c["level"][leaves] == 3) and len(leaves) == m ** 3
    near = {}
    for t, s in zip(L["p2p_t"], L["p2p_s"]):
        near.setdefault(t, set()).add(s)
    for t in leaves:
        got = {tuple(k[s]) for s in near[t]}
        expect = {(a, b, d) for a in range(k[t][0] - 1, k[t][0] + 2)
                  for b in range(k[t][1] - 1, k[t][1] + 2) for d in range(k[t][2] - 1, k[t][2] + 2)
                  if 0 <= a < m and 0 <= b < m and 0 <= d < m}
        assert got == expect
    # and no same-level cell-cell pair is a neighbour
    same = c["level"][L["m2l_t"]] == c["level"][L["m2l_s"]]
    cheb = np.abs(k[L["m2l_t"][same]] - k[L["m2l_s"][same]]).max(axis=1)
    assert np.all(cheb >= 2)


@pytest.mark.parametrize("dist,theta,ncrit,leaf_first", [("uniform", 0.5, 8, False),
                                                         ("uniform", 0.4, 16, False),
                                                         ("plummer", 0.6, 4, False),
                                                         ("shell", 0.5, 8, False),
                                                         ("plummer", 0.5, 8, True)])
def test_exclusive_coverage(dist, theta, ncrit, leaf_first):
    x, q = inputs.make(dist, 1200, 21)
    f = O.Fmm(x, q, 2, theta, ncrit, leaf_first=leaf_first)
    cov = coverage_matrix(f.N, f.cells(), f.lists())
    assert np.all(cov == 1)


def test_mac_pairs_satisfy_mac_and_p2p_pairs_are_leaves():
    x, q = inputs.plummer(2000, 4)
    theta = 0.45
    f = O.Fmm(x, q, 2, theta, 8)
    c, L = f.cells(), f.lists()
    k = cell_index(c["level"], c["prefix"])
    h = (1 << (21 - c["level"])).astype(np.int64)
    C = (2 * k + 1) * h[:, None]
    t, s = L["m2l_t"], L["m2l_s"]
    R2 = ((C[t] - C[s]) ** 2).sum(axis=1).astype(np.float64)
    assert np.all(((h[t] + h[s]).astype(np.float64)) ** 2 <= theta * theta * R2)
    assert np.all(c["nchild"][L["p2p_t"]] == 0) and np.all(c["nchild"][L["p2p_s"]] == 0)


def test_lists_are_order_n():
    per = []
    for n in (4096, 32768, 262144):
        x, q = inputs.uniform_cube(n, 99)
        f = O.Fmm(x, q, 2, 0.5, 32)
        c, L = f.cells(), f.lists()
        sz = c["end"] - c["begin"]
        p2p_inter = np.sum(sz[L["p2p_t"]] * sz[L["p2p_s"]])
        per.append((f.nm2l / n, p2p_inter / n))
    m2l = [a for a, _ in per]
    p2p = [b for _, b in per]
    assert max(m2l) < 2.0 * min(m2l) and max(p2p) < 2.0 * min(p2p)


def _chain6():
    """The hand-built adaptive tree of tests/golden/split_rule_chain6.json."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "split_rule_chain6.json")))
    x = np.zeros((len(g["points_x"]), 3), dtype=np.float32)
    x[:, 0] = g["points_x"]
    x[:, 1:] = g["points_yz"]
    q = np.linspace(-1.0, 1.0, len(x)).astype(np.float32)
    return g, x, q


def _named_pairs(level, prefix, t, s, names):
    k = cell_index(level, prefix)
    name = {}
    for c in range(len(level)):
        assert k[c][1] == 0 and k[c][2] == 0
        name[c] = names[(int(level[c]), int(k[c][0]))]
    return sorted((name[a], name[b]) for a, b in zip(t, s))


def chain6_expected():
    g, _, _ = _chain6()
    names = {tuple(v): n for n, v in g["cells"].items()}
    return g, names, sorted(map(tuple, g["m2l"])), sorted(map(tuple, g["p2p"]))


def test_split_rule_matches_hand_derived_lists():
    # The split rule (the larger cell; the target on a tie; the other cell when the
    # chosen one is a leaf) fixes which pairs reach the lists; the expected lists
    # were derived by hand for a six-particle adaptive tree.
    g, x, q = _chain6()
    _, names, m2l, p2p = chain6_expected()
    f = O.Fmm(x, q, 2, g["theta"], g["ncrit"], max_depth=g["max_depth"])
    c, L = f.cells(), f.lists()
    assert sorted(names) == sorted((int(a), int(b)) for a, b in
                                   zip(c["level"], cell_index(c["level"], c["prefix"])[:, 0]))
    assert _named_pairs(c["level"], c["prefix"], L["m2l_t"], L["m2l_s"], names) == m2l
    assert _named_pairs(c["level"], c["prefix"], L["p2p_t"], L["p2p_s"], names) == p2p


@pytest.mark.parametrize("rule", ["smaller", "source_on_tie"])
def test_wrong_split_rules_fail_the_hand_derived_lists(rule):
    # A traversal that splits the smaller cell, or the source on a tie, still
    # covers every particle pair exactly once (so the coverage pins cannot tell
    # it apart), but its lists differ from the hand-derived ones.
    g, x, q = _chain6()
    _, names, m2l, p2p = chain6_expected()
    f = O.Fmm(x, q, 2, g["theta"], g["ncrit"], max_depth=g["max_depth"], split_rule=rule)
    c, L = f.cells(), f.lists()
    assert np.all(coverage_matrix(f.N, c, L) == 1)
    got = (_named_pairs(c["level"], c["prefix"], L["m2l_t"], L["m2l_s"], names),
           _named_pairs(c["level"], c["prefix"], L["p2p_t"], L["p2p_s"], names))
    assert got != (m2l, p2p)


@pytest.mark.parametrize("rule", ["smaller", "source_on_tie"])
def test_wrong_split_rules_change_lists_on_random_trees(rule):
    # the same on a Plummer tree: some (target, source) pair set differs
    x, q = inputs.plummer(3000, 31)
    a = O.Fmm(x, q, 2, 0.6, 8)
    b = O.Fmm(x, q, 2, 0.6, 8, split_rule=rule)
    la, lb = a.lists(), b.lists()
    ka = set(zip(la["m2l_t"].tolist(), la["m2l_s"].tolist()))
    kb = set(zip(lb["m2l_t"].tolist(), lb["m2l_s"].tolist()))
    assert ka != kb
