"""Pins of the oracle's A_FD, stiffness operator S = I^T A_FD I, RHS and solve.

Section 2.2 ((AFD-1), Proposition 2.1, (FD-1)), Section 3.2 ((GoFD-1..3),
Theorem 3.1), Section 3.3 ((Ah-4)), Section 5 ((exam-0), (exam-2)).
"""
import numpy as np
import pytest
from scipy.special import gamma as G

import meshgen as mg
from oracle import gofd as o


@pytest.mark.parametrize("d,n,s", [(2, 9, 0.75), (2, 12, 0.3), (3, 5, 0.6), (1, 17, 0.4)])
def test_fft_apply_matches_direct_toeplitz_sum(d, n, s):
    T = o.coefficients(d, s, n, M=2 ** 10 if d < 3 else 2 ** 8)
    P = o.circulant_size(n)
    lam = o.symbol(T, P)
    v = np.random.default_rng(3).uniform(-1, 1, size=(n,) * d)
    w1 = o.afd_apply_direct(T, v)
    w2 = o.afd_apply_fft(lam, v, P)
    assert np.linalg.norm(w1 - w2) / np.linalg.norm(w1) < 1e-13


def test_s1_afd_is_five_point_laplacian():
    n = 9
    T = o.coefficients(2, 1.0, n, M=2 ** 10)
    v = np.random.default_rng(1).uniform(-1, 1, size=(n, n))
    pad = np.zeros((n + 2, n + 2))
    pad[1:-1, 1:-1] = v
    lap = 4 * v - pad[:-2, 1:-1] - pad[2:, 1:-1] - pad[1:-1, :-2] - pad[1:-1, 2:]
    w = o.afd_apply_fft(o.symbol(T, o.circulant_size(n)), v, o.circulant_size(n))
    assert np.abs(w - lap).max() < 1e-13


def test_afd_symmetric_positive_definite():
    # Proposition 2.1: A_FD is SPD; its smallest eigenvalue is bounded below
    n = 8
    for s in (0.25, 0.75):
        T = o.coefficients(2, s, n, M=2 ** 10)
        N = n * n
        A = np.zeros((N, N))
        for j in range(N):
            e = np.zeros(N)
            e[j] = 1
            A[:, j] = o.afd_apply_direct(T, e.reshape(n, n)).ravel()
        assert np.abs(A - A.T).max() < 1e-15
        assert np.linalg.eigvalsh(A).min() > 0


def _disk(rings=6, n=17, alpha=1.0, seed=3):
    v, s = mg.disk_ring_mesh(rings=rings, seed=seed)
    lo, hi, h = mg.grid_box(2, n)
    return o.build(2, v, s, alpha, h, lo, hi, M=2 ** 10)


def test_stiffness_symmetric_positive_definite():
    # Theorem 3.1 with D_h > 0 and full column rank
    P = _disk()
    u = mg.random_vector(len(P.verts), 1)
    w = mg.random_vector(len(P.verts), 2)
    Su = o.stiffness_apply(P, u)
    Sw = o.stiffness_apply(P, w)
    assert abs(w @ Su - u @ Sw) < 1e-13 * np.linalg.norm(Su) * np.linalg.norm(w)
    uu = u.copy()
    uu[P.boundary] = 0
    assert uu @ Su > 0
    assert np.all(Su[P.boundary] == 0.0)


def test_stiffness_direct_equals_fft():
    P = _disk()
    u = mg.random_vector(len(P.verts), 5)
    a = o.stiffness_apply(P, u, "direct")
    b = o.stiffness_apply(P, u, "fft")
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-13


@pytest.mark.parametrize("d,n,cells,off", [(2, 11, 6, 2), (3, 7, 4, 1)])
def test_grid_aligned_mesh_reduces_to_uniform_fd(d, n, cells, off):
    # With every mesh vertex on a grid node, I_h^FD is a 0/1 selection and
    # S = A_FD restricted to the interior nodes: the square-domain scheme (FD-1)
    lo, hi, h = mg.grid_box(d, n)
    verts, simp = mg.grid_aligned_mesh(d, -1.0, h, cells, origin_cells=off)
    P = o.build(d, verts, simp, 1.2, h, lo, hi, M=2 ** 10 if d == 2 else 2 ** 8)
    u = mg.random_vector(len(verts), 9)
    u[P.boundary] = 0.0
    # place the interior values on their grid nodes
    k = np.rint((verts - lo) / h).astype(np.int64)
    lin = k[:, 0] + n * k[:, 1] + (n * n * k[:, 2] if d == 3 else 0)
    v = np.zeros(P.n_grid)
    v[lin] = u
    w = o.afd_apply_direct(P.T, v.reshape((n,) * d)).ravel()
    y = o.stiffness_apply(P, u)
    ref = np.where(P.boundary, 0.0, w[lin])
    assert np.abs(y - ref).max() < 1e-13


def test_rhs_grid_and_vertex_agree_for_constant_f():
    # (GoFD-2) with f = 1: h^{2s} I^T 1 = h^{2s} D_h, which is (GoFD-3) with f_h = 1
    P = _disk()
    a = o.rhs_grid(P, np.ones(P.n_grid))
    b = o.rhs_vertex(P, np.ones(len(P.verts)))
    assert np.abs(a - b).max() < 1e-15


def test_constant_preservation_of_fd_to_mesh_transfer():
    # Remark 3.1: rows of D_h^{-1} I^T sum to one
    # (every interior vertex has D_h > 0 here; a boundary vertex may not)
    P = _disk()
    assert np.all(P.Dh[P.interior] > 0)
    pos = P.Dh > 0
    rs = (P.I.T @ np.ones(P.n_grid))[pos] / P.Dh[pos]
    assert np.abs(rs - 1).max() < 1e-14


def test_fraclap_is_scaled_stiffness():
    P = _disk()
    u = mg.random_vector(len(P.verts), 4)
    y = o.fraclap_apply(P, u)
    S = o.stiffness_apply(P, u)
    ii = P.interior
    assert np.allclose(y[ii] * P.Dh[ii] * P.h ** (2 * P.s), S[ii], rtol=1e-14, atol=0)


def test_cg_matches_dense_solve():
    P = _disk(rings=4, n=13)
    ii = P.interior
    N = len(P.verts)
    S = np.zeros((len(ii), len(ii)))
    for c, j in enumerate(ii):
        e = np.zeros(N)
        e[j] = 1
        S[:, c] = o.stiffness_apply(P, e)[ii]
    b = o.rhs_grid(P, np.ones(P.n_grid))
    x, info = o.solve(P, b, tol=1e-13)
    ref = np.linalg.solve(S, b[ii])
    assert info["rel_res"] < 1e-13
    assert np.abs(x[ii] - ref).max() < 1e-10 * np.abs(ref).max()


def test_ball_constant_closed_forms():
    # (exam-0) with k = 0: C = Gamma(d/2) / (2^{2s} Gamma(1+s) Gamma(d/2+s))
    assert abs(o.ball_constant(2, 0.5) - 2 / np.pi) < 1e-15
    assert abs(o.ball_constant(3, 0.5) - 0.5) < 1e-15
    # d = 1: C = Gamma(1/2)/(2^{2s} Gamma(1+s) Gamma(1/2+s))
    assert abs(o.ball_constant(1, 0.5) - np.sqrt(np.pi) / (2 * G(1.5) * G(1.0))) < 1e-15


@pytest.mark.parametrize("s", [0.5, 0.75])
def test_disk_convergence_order(s):
    # Remark 3.6 / Example 5.2: L2 error ~ O(h^{min(1, s+1/2)}) on fixed meshes
    errs, hb = [], []
    for rings, n in [(6, 17), (12, 33), (24, 65)]:
        v, simp = mg.disk_ring_mesh(rings=rings, seed=5)
        lo, hi, h = mg.grid_box(2, n)
        P = o.build(2, v, simp, 2 * s, h, lo, hi, M=2 ** 11, exact_weights=False)
        b = o.rhs_grid(P, np.ones(P.n_grid))
        x, info = o.solve(P, b, 1e-11)
        assert info["rel_res"] < 1e-11
        errs.append(o.lumped_l2(v, simp, x - o.ball_exact(v, s)))
        hb.append(len(simp) ** -0.5)
    slope = np.polyfit(np.log(hb), np.log(errs), 1)[0]
    assert abs(slope - min(1.0, s + 0.5)) < 0.25, slope
    assert errs[-1] < errs[0]


def test_interval_convergence_1d():
    # Example 5.1 setting (d = 1): FM error in L2 decreases ~ h^{min(1, s+1/2)}
    s = 0.5
    errs = []
    hs = []
    for cells, n in [(16, 33), (32, 65), (64, 129)]:
        v, simp = mg.interval_mesh(cells, seed=2)
        lo, hi, h = mg.grid_box(1, n)
        P = o.build(1, v, simp, 2 * s, h, lo, hi, M=2 ** 13)
        b = o.rhs_grid(P, np.ones(P.n_grid))
        x, _ = o.solve(P, b, 1e-12)
        errs.append(o.lumped_l2(v, simp, x - o.ball_exact(v, s)))
        hs.append(1.0 / cells)
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert abs(slope - 1.0) < 0.25, slope
