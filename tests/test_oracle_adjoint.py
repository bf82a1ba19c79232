"""Pins of the oracle's adjoint (gradients of the (GoFD-3) solve) by central
finite differences of the oracle's own solves."""
import numpy as np
import pytest

import meshgen as mg
from oracle import gofd as o


def _setup(seed=3):
    # the box leaves room around the disk so that perturbed vertices stay inside
    v, s = mg.disk_ring_mesh(rings=5, seed=seed)
    # and is shifted so that no grid node sits on a vertex (owners stay fixed
    # under the small perturbations of the finite differences)
    lo, hi, h = mg.grid_box(2, 23, -1.1037, 1.0963)
    return v, s, lo, hi, h


def _loss(v, s, lo, hi, h, f, ut, alpha=1.2):
    P = o.build(2, v, s, alpha, h, lo, hi, M=2 ** 10, exact_weights=False)
    b = o.rhs_vertex(P, f)
    u, _ = o.solve(P, b, tol=1e-14)
    return 0.5 * np.sum((u - ut) ** 2), P, u


def test_gradient_wrt_vertex_data_matches_central_differences():
    v, s, lo, hi, h = _setup()
    rng = np.random.default_rng(1)
    f = mg.target_bump(v) + 0.3
    ut = 0.05 * rng.standard_normal(len(v))
    L0, P, u = _loss(v, s, lo, hi, h, f, ut)
    gf, _ = o.adjoint_vertex(P, f, u, u - ut)
    for k in range(4):
        d = rng.standard_normal(len(v))
        eps = 1e-3
        Lp = _loss(v, s, lo, hi, h, f + eps * d, ut)[0]
        Lm = _loss(v, s, lo, hi, h, f - eps * d, ut)[0]
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - gf @ d) <= 1e-7 * max(1.0, abs(fd)), (fd, gf @ d)


def test_gradient_wrt_vertices_matches_central_differences():
    v, s, lo, hi, h = _setup()
    rng = np.random.default_rng(2)
    f = mg.target_bump(v) + 0.3
    ut = 0.05 * rng.standard_normal(len(v))
    L0, P, u = _loss(v, s, lo, hi, h, f, ut)
    _, gx = o.adjoint_vertex(P, f, u, u - ut)
    checked = 0
    for k in range(12):
        d = rng.standard_normal(v.shape)
        eps = 1e-7
        Lp, Pp, _ = _loss(v + eps * d, s, lo, hi, h, f, ut)
        Lm, Pm, _ = _loss(v - eps * d, s, lo, hi, h, f, ut)
        if not (np.array_equal(Pp.owner, P.owner) and np.array_equal(Pm.owner, P.owner)):
            continue                     # the owner map changed: not differentiable there
        fd = (Lp - Lm) / (2 * eps)
        an = float(np.sum(gx * d))
        assert abs(fd - an) <= 1e-5 * max(abs(fd), 1e-8), (k, fd, an)
        checked += 1
    assert checked >= 6


def test_dropping_a_term_breaks_the_vertex_gradient(monkeypatch):
    # a planted mistake (the D_h(X) part of the right-hand side left out)
    # must disagree with finite differences
    v, s, lo, hi, h = _setup()
    rng = np.random.default_rng(2)
    f = mg.target_bump(v) + 0.3
    ut = 0.05 * rng.standard_normal(len(v))
    L0, P, u = _loss(v, s, lo, hi, h, f, ut)
    _, gx = o.adjoint_vertex(P, f, u, u - ut)
    _, gx_bad = o.adjoint_vertex(P, np.zeros_like(f), u, u - ut)   # lambda*f term removed
    d = rng.standard_normal(v.shape)
    eps = 1e-7
    fd = (_loss(v + eps * d, s, lo, hi, h, f, ut)[0] - _loss(v - eps * d, s, lo, hi, h, f, ut)[0]) / (2 * eps)
    assert abs(fd - np.sum(gx * d)) < abs(fd - np.sum(gx_bad * d))
