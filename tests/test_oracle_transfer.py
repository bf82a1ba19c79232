"""Pins of the oracle's point location, P1 transfer I_h^FD and mesh quantities.

Section 3.1 of the paper: (IhFD-1), Lemma 3.1 (i)-(v), Theorem 3.2.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import meshgen as mg
from oracle import gofd as o

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _pure_fraction_locate(verts, simp, lo, h, n):
    """Brute force with exact rationals only (no float filter at all)."""
    d = verts.shape[1]
    owner = []
    X = o.grid_node_coords(lo, h, n, np.arange(int(np.prod(n))))
    for x in X:
        own = -1
        for e, s in enumerate(simp):
            V = verts[s]
            full = o.orient_exact(V)
            ok = True
            for i in range(d + 1):
                P = V.copy()
                P[i] = x
                di = o.orient_exact(P)
                if di * full < 0:
                    ok = False
                    break
            if ok:
                own = e
                break
        owner.append(own)
    return np.array(owner)


def test_golden_two_triangles():
    g = json.load(open(os.path.join(GOLD, "two_triangles.json")))
    v = np.array(g["vertices"])
    s = np.array(g["simplices"])
    lo = np.array(g["box_lo"])
    n = o.grid_shape(lo, g["box_hi"], g["h"])
    own = o.locate(v, s, lo, g["h"], n)
    assert own.tolist() == g["owner"]
    nodes, idx, w = o.ell_layout(v, s, lo, g["h"], n, own)
    assert idx.tolist() == g["ell_idx"]
    assert np.array_equal(w, np.array(g["ell_w"]))
    assert o.boundary_vertices(s, 4).tolist() == g["boundary"]


@pytest.mark.parametrize("d,cells,n", [(2, 3, 7), (2, 4, 9), (3, 2, 5)])
def test_locate_matches_pure_rationals_on_aligned_meshes(d, cells, n):
    # mesh vertices coincide with grid nodes: every node sits on facets, the
    # hardest case for the sign decisions and the tie rule
    lo, hi, h = mg.grid_box(d, n, -1.0, 1.0)
    verts, simp = mg.grid_aligned_mesh(d, -1.0, h, cells, origin_cells=1)
    shape = o.grid_shape(lo, hi, h)
    a = o.locate(verts, simp, lo, h, shape)
    b = _pure_fraction_locate(verts, simp, lo, h, shape)
    assert np.array_equal(a, b)
    assert (a >= 0).sum() == (cells + 1) ** d


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_locate_matches_pure_rationals_random_2d(seed):
    v, s = mg.disk_ring_mesh(rings=3, seed=seed)
    lo, hi, h = mg.grid_box(2, 9)
    n = o.grid_shape(lo, hi, h)
    assert np.array_equal(o.locate(v, s, lo, h, n), _pure_fraction_locate(v, s, lo, h, n))


def test_locate_matches_pure_rationals_3d():
    v, s = mg.ball_shell_mesh(shells=2, seed=7)
    lo, hi, h = mg.grid_box(3, 5)
    n = o.grid_shape(lo, hi, h)
    assert np.array_equal(o.locate(v, s, lo, h, n), _pure_fraction_locate(v, s, lo, h, n))


@pytest.mark.parametrize("d,cells,n", [(2, 4, 9), (3, 2, 5)])
def test_aligned_mesh_transfer_is_selection(d, cells, n):
    # (IhFD-1) with every grid node a mesh vertex: I_h^FD selects vertex values
    lo, hi, h = mg.grid_box(d, n)
    verts, simp = mg.grid_aligned_mesh(d, -1.0, h, cells, origin_cells=2)
    shape = o.grid_shape(lo, hi, h)
    own = o.locate(verts, simp, lo, h, shape)
    nodes, idx, w = o.ell_layout(verts, simp, lo, h, shape, own)
    X = o.grid_node_coords(lo, h, shape, nodes)
    for r in range(len(nodes)):
        one = np.nonzero(w[:, r] == 1.0)[0]
        assert len(one) == 1 and np.all(np.delete(w[:, r], one) == 0.0)
        assert np.array_equal(verts[idx[one[0], r]], X[r])


def _disk_problem(rings=6, n=17, seed=3, alpha=1.0):
    v, s = mg.disk_ring_mesh(rings=rings, seed=seed)
    lo, hi, h = mg.grid_box(2, n)
    return o.build(2, v, s, alpha, h, lo, hi, M=2 ** 10)


def test_lemma31_invariants():
    P = _disk_problem()
    w = P.ell_w
    # (i) 0 <= I <= 1
    assert w.min() >= 0.0 and w.max() <= 1.0
    # (iii) row sums are 1 on located nodes, 0 elsewhere
    rs = np.asarray(P.I.sum(axis=1)).ravel()
    assert np.allclose(rs[P.nodes], 1.0, atol=1e-14)
    mask = np.ones(P.n_grid, dtype=bool)
    mask[P.nodes] = False
    assert np.all(rs[mask] == 0.0)
    # linear precision of P1 interpolation: sum_j phi_j(x) x_j = x
    X = o.grid_node_coords(P.box_lo, P.h, P.n, P.nodes)
    rec = np.einsum("an,and->nd", w, P.verts[P.ell_idx])
    assert np.abs(rec - X).max() < 1e-14
    # (ii) sparsity: x_k lies in the patch of every vertex it uses
    # (iv) max phi <= D_h <= N_val N_FD^h and (v) lambda_max(I^T I) <= N_val N_FD^h
    nval = np.bincount(P.simp.ravel()).max()
    nfd = np.bincount(P.owner[P.owner >= 0]).max()
    # N_FD^h counts nodes in the closed element, which can exceed the owned count
    nfd_closed = 0
    for e in range(len(P.simp)):
        nfd_closed = max(nfd_closed, int(np.sum(_in_closed(P, e))))
    assert nfd <= nfd_closed
    maxphi = np.zeros(len(P.verts))
    np.maximum.at(maxphi, P.ell_idx.ravel(), w.ravel())
    assert np.all(maxphi <= P.Dh + 1e-15)
    assert np.all(P.Dh <= nval * nfd_closed)
    ItI = (P.I.T @ P.I).toarray()
    assert np.linalg.eigvalsh(ItI).max() <= nval * nfd_closed
    IIt = (P.I @ P.I.T).toarray()
    assert np.linalg.eigvalsh(IIt).max() <= nval * nfd_closed + 1e-12


def _in_closed(P, e):
    X = o.grid_node_coords(P.box_lo, P.h, P.n, np.arange(P.n_grid))
    V = P.verts[P.simp[e]]
    full = o.orient_exact(V)
    res = []
    for x in X:
        if np.any(x < V.min(axis=0) - 1e-12) or np.any(x > V.max(axis=0) + 1e-12):
            res.append(False)
            continue
        ok = True
        for i in range(len(V)):
            Q = V.copy()
            Q[i] = x
            if o.orient_exact(Q) * full < 0:
                ok = False
        res.append(ok)
    return np.array(res)


def test_theorem32_under_grid_bound():
    # (hFD-1): h_FD <= a_h / ((d+1) sqrt(d))  =>  D_h >= a_h / ((d+1) sqrt(d) h)
    # and I_h^FD has full column rank.
    v, s = mg.disk_ring_mesh(rings=2, jitter=0.1, seed=11)
    a_h = o.element_heights(v, s).min()
    bound = a_h / (3.0 * np.sqrt(2.0))
    n = int(np.ceil(2.0 / bound)) + 1
    lo, hi, h = mg.grid_box(2, n)
    assert h <= bound
    P = o.build(2, v, s, 1.0, h, lo, hi, M=2 ** 10, exact_weights=False)
    # h in (thm:IhFD:0) is the maximum element diameter (longest edge)
    diam = max(np.max(np.linalg.norm(v[s[:, a]] - v[s[:, b]], axis=1))
               for a, b in itertools.combinations(range(3), 2))
    assert np.all(P.Dh >= a_h / (3.0 * np.sqrt(2.0) * diam) - 1e-14)
    ItI = (P.I.T @ P.I).toarray()
    assert np.linalg.eigvalsh(ItI).min() > 0.0


def test_heights_equilateral_and_right_triangle():
    # equilateral triangle of side 1: every height is sqrt(3)/2
    v = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, np.sqrt(3) / 2]])
    assert abs(o.element_heights(v, np.array([[0, 1, 2]]))[0] - np.sqrt(3) / 2) < 1e-15
    # right isosceles tetrahedron corner: min height = 1/sqrt(3)
    v3 = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    assert abs(o.element_heights(v3, np.array([[0, 1, 2, 3]]))[0] - 1 / np.sqrt(3)) < 1e-15


def test_outside_nodes_and_degenerate_simplex():
    v = np.array([[0.0, 0.0], [0.5, 0.0], [0.0, 0.5]])
    lo, hi, h = mg.grid_box(2, 5)
    n = o.grid_shape(lo, hi, h)
    own = o.locate(v, np.array([[0, 1, 2]]), lo, h, n)
    X = o.grid_node_coords(lo, h, n, np.arange(25))
    inside = (X[:, 0] >= 0) & (X[:, 1] >= 0) & (X[:, 0] + X[:, 1] <= 0.5)
    assert np.array_equal(own >= 0, inside)
    flat = np.array([[0.0, 0.0], [0.5, 0.5], [1.0, 1.0]])
    with pytest.raises(o.OracleError):
        o.locate(flat, np.array([[0, 1, 2]]), lo, h, n)


def test_exact_weights_are_rounded_rationals():
    v, s = mg.disk_ring_mesh(rings=3, seed=4)
    x = np.array([0.1, 0.05])
    e = 0
    for e in range(len(s)):
        V = v[s[e]]
        full = o.orient_exact(V)
        ds = []
        for i in range(3):
            Q = V.copy()
            Q[i] = x
            ds.append(o.orient_exact(Q))
        if all(di * full >= 0 for di in ds):
            break
    w = o.barycentric_exact(v, s[e], x)
    full = o.orient_exact(v[s[e]])
    for i in range(3):
        Q = v[s[e]].copy()
        Q[i] = x
        assert w[i] == float(o.orient_exact(Q) / full)
    assert abs(Fraction(w.sum()) - 1) < Fraction(1, 2 ** 50)


def test_grid_rejects_non_integral_box():
    with pytest.raises(o.OracleError):
        o.grid_shape([-1.0, -1.0], [1.0, 1.0], 0.3)


@pytest.mark.parametrize("case", ["disk", "aligned2", "aligned3", "ball"])
def test_pruned_locate_equals_brute_force(case):
    if case == "disk":
        v, s = mg.disk_ring_mesh(rings=8, seed=2)
        lo, hi, h = mg.grid_box(2, 33)
    elif case == "aligned2":
        lo, hi, h = mg.grid_box(2, 9)
        v, s = mg.grid_aligned_mesh(2, -1.0, h, 4, origin_cells=2)
    elif case == "aligned3":
        lo, hi, h = mg.grid_box(3, 5)
        v, s = mg.grid_aligned_mesh(3, -1.0, h, 2, origin_cells=1)
    else:
        v, s = mg.ball_shell_mesh(shells=3, seed=4)
        lo, hi, h = mg.grid_box(3, 9)
    n = o.grid_shape(lo, hi, h)
    assert np.array_equal(o.locate_pruned(v, s, lo, h, n), o.locate(v, s, lo, h, n))


@pytest.mark.parametrize("case", ["disk", "aligned2", "aligned3", "ball"])
def test_mixed_orientations_permute_slots_only(case):
    # containment in a closed simplex does not depend on its orientation: with
    # half of the simplices flipped (first two local vertices swapped) every
    # owner is the same, the ELL row lists the same vertices in the new local
    # order, the exact weights follow their vertices, and the pure-rational
    # brute force agrees
    if case == "disk":
        v, s = mg.disk_ring_mesh(rings=4, seed=5)
        lo, hi, h = mg.grid_box(2, 13)
    elif case == "aligned2":
        lo, hi, h = mg.grid_box(2, 9)
        v, s = mg.grid_aligned_mesh(2, -1.0, h, 4, origin_cells=2)
    elif case == "aligned3":
        lo, hi, h = mg.grid_box(3, 5)
        v, s = mg.grid_aligned_mesh(3, -1.0, h, 2, origin_cells=1)
    else:
        v, s = mg.ball_shell_mesh(shells=2, seed=6)
        lo, hi, h = mg.grid_box(3, 5)
    f = mg.flip_orientations(s, seed=11)
    flipped = np.any(f != s, axis=1)
    assert 0.3 < flipped.mean() < 0.7
    assert np.all(o.element_orientations(v, f)[flipped] == -1)
    n = o.grid_shape(lo, hi, h)
    own_s = o.locate(v, s, lo, h, n)
    own_f = o.locate(v, f, lo, h, n)
    assert np.array_equal(own_s, own_f)
    assert np.array_equal(own_f, _pure_fraction_locate(v, f, lo, h, n))
    assert np.array_equal(own_f, o.locate_pruned(v, f, lo, h, n))
    _, idx_s, w_s = o.ell_layout(v, s, lo, h, n, own_s)
    _, idx_f, w_f = o.ell_layout(v, f, lo, h, n, own_f)
    swap = flipped[own_f[own_f >= 0]]
    perm = np.arange(len(idx_s))
    perm[:2] = [1, 0]
    assert np.array_equal(idx_f[:, swap], idx_s[perm][:, swap])
    assert np.array_equal(idx_f[:, ~swap], idx_s[:, ~swap])
    assert np.array_equal(w_f[:, swap], w_s[perm][:, swap])
    assert np.array_equal(w_f[:, ~swap], w_s[:, ~swap])
    # float weights (the large-case route) follow their vertices too
    _, _, wf_f = o.ell_layout(v, f, lo, h, n, own_f, exact=False)
    assert np.abs(wf_f - w_f).max() < 1e-14
