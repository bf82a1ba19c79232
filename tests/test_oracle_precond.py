"""Pins of the oracle's sparse preconditioner (Section 3.3, (Ah-4)) and PCG."""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen as mg
from oracle import gofd as o


def _spd_matrix(N, seed, density=0.15):
    rng = np.random.default_rng(seed)
    A = sp.random(N, N, density=density, random_state=rng)
    A = A + A.T
    A = A + sp.diags(np.abs(A).sum(axis=1).A.ravel() + 1.0)
    return A.tocsr()


def test_full_fill_level_is_exact_cholesky():
    A = _spd_matrix(30, 1)
    L, shift = o.ic_factor(A, level=100)
    assert shift == 0.0
    ref = np.linalg.cholesky(A.toarray())
    assert np.abs(L.toarray() - ref).max() < 1e-12


def test_tridiagonal_needs_no_fill():
    N = 20
    A = sp.diags([-np.ones(N - 1), 2.5 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1]).tocsr()
    L0, _ = o.ic_factor(A, level=0)
    assert np.abs(L0.toarray() - np.linalg.cholesky(A.toarray())).max() < 1e-14


def test_ic1_reproduces_a_on_the_kept_pattern():
    A = _spd_matrix(40, 2, density=0.08)
    pat = o.ic_symbolic(A, 1)
    L = o.ic_numeric(A, pat)
    R = (L @ L.T).toarray()
    Ad = A.toarray()
    for i, cols in enumerate(pat):
        for j in cols:
            assert abs(R[i, j] - Ad[i, j]) < 1e-12 * abs(Ad[i, i])


def test_ic1_pattern_by_hand():
    # arrow-free 4-cycle 0-1-2-3-0: eliminating 0 creates fill (3,1) at level 1
    A = sp.csr_matrix(np.array([[4, -1, 0, -1], [-1, 4, -1, 0], [0, -1, 4, -1], [-1, 0, -1, 4.0]]))
    assert o.ic_symbolic(A, 0) == [[0], [0, 1], [1, 2], [0, 2, 3]]
    assert o.ic_symbolic(A, 1) == [[0], [0, 1], [1, 2], [0, 1, 2, 3]]


def _disk(alpha):
    v, s = mg.disk_ring_mesh(rings=8, seed=3)
    lo, hi, h = mg.grid_box(2, 25)
    return o.build(2, v, s, alpha, h, lo, hi, M=2 ** 10, exact_weights=False)


def test_preconditioner_matrix_is_stencil_galerkin():
    P = _disk(1.5)
    A9 = o.preconditioner_matrix(P, 9)
    assert abs(A9 - A9.T).max() < 1e-15
    # the 9-point stencil keeps T_0, T_(1,0), T_(0,1), T_(1,1)
    S9 = o.stencil_matrix(P, 9)
    assert S9.nnz <= 9 * P.n_grid
    assert np.isclose(S9[P.n_grid // 2, P.n_grid // 2], P.T[0, 0])


@pytest.mark.parametrize("alpha", [1.0, 1.8])
def test_ic1_preconditioner_reduces_iterations(alpha):
    # Section 5.2: the IC(1) preconditioner reduces the CG iteration count
    P = _disk(alpha)
    b = o.rhs_grid(P, np.ones(P.n_grid))
    _, plain = o.solve(P, b, 1e-10)
    x, pc = o.pcg_ic(P, b, pattern=9, tol=1e-10)
    assert pc["rel_res"] < 1e-10
    assert pc["iters"] < plain["iters"]


def test_jacobi_diagonal_is_the_diagonal_of_s():
    # S assembled column by column from the stiffness product (an independent
    # route through A_FD by FFT), against the row-by-row double sum
    for d, v, s, n, alpha in (
            (2,) + mg.disk_ring_mesh(rings=4, seed=mg.seed_for(1, 9)) + (13, 1.3),
            (1,) + mg.interval_mesh(9, seed=mg.seed_for(0, 9)) + (19, 0.7)):
        lo, hi, h = mg.grid_box(d, n)
        ref = o.build(d, v, s, alpha, h, lo, hi, M=2 ** 9)
        ii = ref.interior
        want = np.empty(len(ii))
        for r, j in enumerate(ii):
            e = np.zeros(len(v))
            e[j] = 1.0
            want[r] = o.stiffness_apply(ref, e)[j]
        got = o.jacobi_diagonal(ref)
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_jacobi_pcg_matches_plain_cg():
    v, s = mg.disk_ring_mesh(rings=5, seed=mg.seed_for(1, 8))
    lo, hi, h = mg.grid_box(2, 17)
    ref = o.build(2, v, s, 1.1, h, lo, hi, M=2 ** 9)
    b = o.rhs_grid(ref, np.ones(ref.n_grid))
    x1, _ = o.solve(ref, b, tol=1e-13)
    x2, _ = o.pcg_jacobi(ref, b, tol=1e-13)
    assert np.linalg.norm(x1 - x2) <= 1e-10 * np.linalg.norm(x1)


# ---------------------------------------------------------------------------
# the circulant alternative of Section 3.3 (reading R24)
# ---------------------------------------------------------------------------
def _dense_circulant(c):
    """The circulant matrix with first column c (shape (P,)*d), entry by entry:
    C[(i), (j)] = c[(i - j) mod P] per axis."""
    P = c.shape[0]
    d = c.ndim
    idx = np.array(np.unravel_index(np.arange(P ** d), (P,) * d)).T
    diff = (idx[:, None, :] - idx[None, :, :]) % P
    return c[tuple(diff[..., a] for a in range(d))]


@pytest.mark.parametrize("d,n", [(1, 9), (2, 5)])
def test_circulant_inverse_is_a_dense_circulant_solve(d, n):
    T = o.coefficients(d, 0.6, n, 2 ** 10)
    P = o.circulant_size(n)
    C = _dense_circulant(o.circulant_first_column(T, P))
    rng = np.random.default_rng(7)
    vg = rng.standard_normal((n,) * d)
    vp = np.zeros((P,) * d)
    vp[(slice(0, n),) * d] = vg
    want = np.linalg.solve(C, vp.ravel()).reshape((P,) * d)[(slice(0, n),) * d].ravel()

    class _G:   # the fields circulant_inverse_apply reads
        pass
    g = _G()
    g.d, g.n, g.P, g.lam = d, (n,) * d, P, o.symbol(T, P)
    g.grid_vector = lambda f: f.reshape((n,) * d)
    got = o.circulant_inverse_apply(g, vg.ravel())
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_symbol_of_the_fractional_stencil_is_positive_with_minimum_at_zero():
    # T_0 > 0 and T_m < 0 otherwise (the kernel of (T-1) is positive off the
    # origin), so lambda_k >= lambda_0 = sum of the embedded T > 0: C is SPD
    for d, n, s in [(1, 33, 0.3), (2, 17, 0.75), (3, 9, 0.5)]:
        T = o.coefficients(d, s, n, 2 ** 10 if d < 3 else 2 ** 8)
        off = T.ravel()[1:]
        assert T.ravel()[0] > 0 and np.all(off < 0)
        lam = o.symbol(T, o.circulant_size(n))
        assert lam.min() > 0 and np.argmin(lam) == 0


def test_circulant_precond_on_a_grid_aligned_mesh_is_the_restricted_inverse():
    # every vertex on a grid node: I is a 0/1 selection, D_h = 1, so
    # M^{-1} r = (R C^{-1} R^T r) at the vertices' nodes (dense solve)
    n, cells, off = 11, 6, 2
    lo, hi, h = mg.grid_box(2, n)
    verts, simp = mg.grid_aligned_mesh(2, -1.0, h, cells, origin_cells=off)
    P = o.build(2, verts, simp, 1.2, h, lo, hi, M=2 ** 10)
    assert np.allclose(P.Dh, 1.0)
    r = mg.random_vector(len(verts), 11)
    r[P.boundary] = 0.0
    k = np.rint((verts - lo) / h).astype(np.int64)
    vp = np.zeros((P.P, P.P))
    vp[k[:, 1], k[:, 0]] = r
    C = _dense_circulant(o.circulant_first_column(P.T, P.P))
    w = np.linalg.solve(C, vp.ravel()).reshape(P.P, P.P)
    want = np.where(P.boundary, 0.0, w[k[:, 1], k[:, 0]])
    got = o.circulant_precond(P, r)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_circulant_precond_is_symmetric_positive_definite():
    P = _disk(1.5)
    a = mg.random_vector(len(P.verts), 12)
    b = mg.random_vector(len(P.verts), 13)
    a[P.boundary] = 0.0
    b[P.boundary] = 0.0
    Ma, Mb = o.circulant_precond(P, a), o.circulant_precond(P, b)
    assert abs(a @ Mb - b @ Ma) <= 1e-12 * abs(a @ Mb)
    assert a @ Ma > 0 and b @ Mb > 0
    assert np.all(Ma[P.boundary] == 0.0)


def test_circulant_pcg_reaches_the_plain_cg_solution():
    P = _disk(1.0)
    b = o.rhs_grid(P, np.ones(P.n_grid))
    x0, i0 = o.solve(P, b, tol=1e-12)
    x1, i1 = o.pcg_circulant(P, b, tol=1e-12)
    assert i1["rel_res"] <= 1e-12
    assert np.linalg.norm(x1 - x0) <= 1e-9 * np.linalg.norm(x0)
