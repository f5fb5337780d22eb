"""Pins of the oracle's single-node evaluators (no GPU).

``Grid.sharing``, ``rhs_at``, ``jac_at`` and ``jacT_at`` evaluate the assembled
operators of Sec. 3.3 (eqs. rhsvec, jacvec, jactransvec) at chosen global nodes
from the elements that share each node only.  They are the checker of the
full-size sampled parity tests, so they are pinned here against something other
than themselves:

* ``sharing`` against a brute-force scan of every (element, local node) pair of
  the grid through the periodic scatter Q;
* the three evaluators against the full operators (``rhs``, ``jac``, ``jacT``),
  which sum every element with ``np.add.at``, at every node class: interior,
  face (2 sharing elements), edge (4), corner (8), both sides of the periodic
  seam (g = 0 and g = G-1), and a grid of one element per direction, where an
  element shares a node with itself across the seam.
"""
import itertools

import numpy as np
import pytest

from oracle.sem import Grid


def _brute_sharing(g, node):
    """Every (element id, local index) whose scatter Q lands on `node`, by scanning the grid."""
    hits = []
    for e in range(g.nelem):
        # element ids count x_0 fastest, so the array-order coordinates are a C-order unravel
        ec = np.unravel_index(e, (g.E,) * g.d)
        for loc in itertools.product(range(g.n), repeat=g.d):
            if all((ec[p] * g.N + loc[p]) % g.G == node[p] for p in range(g.d)):
                hits.append((e, tuple(loc)))
    return sorted(hits)


def _node_classes(g):
    """Nodes of every class, by the number of element boundaries they lie on, plus the seam."""
    N, G = g.N, g.G
    inner = [i for i in range(G) if i % N != 0]
    bound = [i for i in range(G) if i % N == 0]
    picks = set()
    for nb in range(g.d + 1):
        for axes in itertools.combinations(range(g.d), nb):
            node = tuple((bound[-1] if p in axes else inner[len(inner) // 2]) for p in range(g.d))
            picks.add(node)
            node = tuple((0 if p in axes else inner[0]) for p in range(g.d))
            picks.add(node)
    picks.add((G - 1,) * g.d)
    picks.add((0,) * g.d)
    picks.add(tuple(G - 1 if p % 2 else 0 for p in range(g.d)))
    return sorted(picks)


CASES = [(2, 3, 3), (2, 1, 4), (3, 2, 3), (3, 3, 2), (3, 1, 3), (1, 4, 5), (1, 1, 4)]


@pytest.mark.parametrize("dim,E,N", CASES)
def test_sharing_equals_brute_force_scan(dim, E, N):
    g = Grid(dim, E, N, 0.05)
    for node in _node_classes(g):
        got = sorted((int(e), tuple(int(i) for i in loc)) for e, loc in g.sharing(node))
        want = _brute_sharing(g, node)
        assert got == want, (node, got, want)
        nb = sum(1 for p in range(dim) if node[p] % N == 0)
        assert len(got) == 2 ** nb


@pytest.mark.parametrize("dim,E,N", CASES)
def test_sampled_evaluators_equal_full_operators(dim, E, N):
    g = Grid(dim, E, N, 0.05)
    rng = np.random.default_rng(100 * dim + 10 * E + N)
    shape = (dim,) + g.global_shape()
    u, w, v = (rng.standard_normal(shape) for _ in range(3))
    nodes = _node_classes(g)
    F, Jw, JTv = g.rhs(u), g.jac(u, w), g.jacT(u, v)
    at = lambda X: np.array([[X[c][nd] for nd in nodes] for c in range(dim)])
    for full, sampled in ((F, g.rhs_at(u, nodes)), (Jw, g.jac_at(u, w, nodes)), (JTv, g.jacT_at(u, v, nodes))):
        ref = at(full)
        scale = np.max(np.abs(full))
        assert np.max(np.abs(sampled - ref)) <= 1e-13 * scale


def test_sampled_evaluators_see_a_planted_sharing_mistake():
    """A sharing list that drops one element of a corner node changes the sampled value."""
    g = Grid(3, 2, 3, 0.05)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((3,) + g.global_shape())
    corner = (0, 0, 0)
    good = g.rhs_at(u, [corner])
    orig = g.sharing
    g.sharing = lambda node: orig(node)[:-1]
    try:
        bad = g.rhs_at(u, [corner])
    finally:
        g.sharing = orig
    assert np.max(np.abs(bad - good)) > 1e-6 * np.max(np.abs(good))
