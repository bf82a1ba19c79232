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
