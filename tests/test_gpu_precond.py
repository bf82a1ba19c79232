"""Parity of the GPU incomplete Cholesky preconditioner (Section 3.3, (Ah-4))
with the oracle's IC(1) under the same unknown order, and its effect on PCG."""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen as mg
from oracle import gofd as o

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2307_14437_gb300 import build_native
    build_native.build()


def _case(name):
    if name == "disk":
        v, s = mg.disk_ring_mesh(rings=8, seed=mg.seed_for(1, 4))
        return 2, v, s, 25, 1.5, 2 ** 10
    if name == "lshape":
        v, s = mg.lshape_mesh(spacing=0.12, seed=mg.seed_for(2, 2))
        return 2, v, s, 33, 1.0, 2 ** 10
    if name == "ball":
        v, s = mg.ball_shell_mesh(shells=3, seed=mg.seed_for(3, 3))
        return 3, v, s, 11, 1.5, 2 ** 8
    if name == "interval":
        v, s = mg.interval_mesh(24, seed=mg.seed_for(0, 2))
        return 1, v, s, 49, 1.2, 2 ** 12
    raise KeyError(name)


CASES = [("disk", 9), ("disk", 5), ("lshape", 9), ("ball", 27), ("ball", 7), ("interval", 3)]


@pytest.mark.parametrize("ordering", [0, 1])
@pytest.mark.parametrize("name,pattern", CASES)
def test_ic1_factor_matches_oracle(name, pattern, ordering):
    from paper_2307_14437_gb300 import Problem
    d, v, s, n, alpha, M = _case(name)
    lo, hi, h = mg.grid_box(d, n)
    gp = Problem(v, s, alpha, h, lo, hi, filon_M=M, precond=pattern, ordering=ordering)
    ref = o.build(d, v, s, alpha, h, lo, hi, M=M, exact_weights=False)
    perm, lptr, lcol, lval = gp.export_precond()
    assert sorted(perm.tolist()) == list(range(len(ref.interior)))
    A = o.preconditioner_matrix(ref, pattern)
    Ap = A[perm][:, perm].tocsr()
    L, shift = o.ic_factor(Ap, 1)
    assert gp.info()["ic_shift"] == shift
    L = L.tocsr()
    L.sort_indices()
    assert np.array_equal(lptr, L.indptr.astype(np.int32))
    assert np.array_equal(lcol, L.indices.astype(np.int32))
    assert np.abs(lval - L.data).max() <= 1e-12 * np.abs(L.data).max()
    gp.close()


@pytest.mark.parametrize("ordering", [0, 1])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_ic1_pcg_converges_with_fewer_iterations(mode, ordering):
    from paper_2307_14437_gb300 import Problem
    d, v, s, n, alpha, M = _case("disk")
    lo, hi, h = mg.grid_box(d, n)
    plain = Problem(v, s, alpha, h, lo, hi, filon_M=M, check_every=1)
    pc = Problem(v, s, alpha, h, lo, hi, filon_M=M, precond=9, ordering=ordering, check_every=1)
    ref = o.build(d, v, s, alpha, h, lo, hi, M=M, exact_weights=False)
    f = torch.ones(pc.n_grid, dtype=torch.float64, device="cuda")
    u0, i0 = plain.solve(f, mode=mode, tol=1e-10)
    u1, i1 = pc.solve(f, mode=mode, tol=1e-10)
    b = o.rhs_grid(ref, np.ones(ref.n_grid))
    res = np.linalg.norm(b - o.stiffness_apply(ref, u1.cpu().numpy())) / np.linalg.norm(b)
    assert res < 2e-10
    assert i1["inner_iters"] < i0["inner_iters"], (i0, i1)
    plain.close()
    pc.close()


def _ic_apply_oracle(L, perm, r):
    """z = P^T (L L^T)^{-1} P r in the oracle's interior order (P: the factor's
    unknown order), two triangular solves with SciPy."""
    from scipy.sparse.linalg import spsolve_triangular
    L = sp.csr_matrix(L)
    y = spsolve_triangular(L, r[perm], lower=True)
    zp = spsolve_triangular(sp.csr_matrix(L.T), y, lower=False)
    z = np.empty_like(zp)
    z[perm] = zp
    return z


@pytest.mark.parametrize("ic_solve", [0, 1])
@pytest.mark.parametrize("ordering", [0, 1])
@pytest.mark.parametrize("name,pattern", CASES)
def test_ic1_apply_matches_oracle(name, pattern, ordering, ic_solve):
    # z = M^{-1} r with M = L L^T the IC(1) factor (Section 3.3), both forms of
    # the triangular solves: one persistent launch per solve, one launch per level
    from paper_2307_14437_gb300 import Problem
    d, v, s, n, alpha, M = _case(name)
    lo, hi, h = mg.grid_box(d, n)
    gp = Problem(v, s, alpha, h, lo, hi, filon_M=M, precond=pattern, ordering=ordering, ic_solve=ic_solve)
    ref = o.build(d, v, s, alpha, h, lo, hi, M=M, exact_weights=False)
    perm, *_ = gp.export_precond()
    A = o.preconditioner_matrix(ref, pattern)
    L, _ = o.ic_factor(A[perm][:, perm].tocsr(), 1)
    ii, iv, r, rc = _interior_vectors(gp, ref, 47)
    want = _ic_apply_oracle(L, perm, r[iv])
    for dt, tol in ((torch.float64, 1e-11), (torch.float32, 1e-4)):
        z = gp.precond_apply(torch.tensor(rc, dtype=dt, device="cuda")).cpu().numpy().astype(np.float64)
        assert z[-1] == 0.0
        got = z[ii[iv]]
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want), (dt, name, pattern, ordering, ic_solve)
    gp.close()


def _lshape600():
    v, s = mg.lshape_mesh(spacing=0.03, seed=mg.seed_for(2, 31))
    lo, hi, h = mg.grid_box(2, 600)
    return v, s, lo, hi, h


@pytest.mark.parametrize("ordering", [0, 1])
def test_persistent_ic_solves_at_scale(ordering):
    # L-shape mesh on a 600^2 grid (thousands of tiles, hundreds to thousands of
    # levels): the persistent solves agree with the level-by-level ones, and the
    # result satisfies L L^T z = P r to within the rounding of the two solves
    from paper_2307_14437_gb300 import Problem
    v, s, lo, hi, h = _lshape600()
    a = Problem(v, s, 0.7, h, lo, hi, precond=9, ordering=ordering, ic_solve=0)
    b = Problem(v, s, 0.7, h, lo, hi, precond=9, ordering=ordering, ic_solve=1)
    pa, lpa, lca, lva = a.export_precond()
    pb, lpb, lcb, lvb = b.export_precond()
    assert np.array_equal(pa, pb) and np.array_equal(lpa, lpb) and np.array_equal(lca, lcb)
    assert np.array_equal(lva, lvb)
    nint = a.info()["n_interior"]
    assert a.info()["precond_levels"] > 50
    rng = np.random.default_rng(mg.seed_for(2, 61))
    r = np.zeros(nint + 1)
    r[:nint] = rng.standard_normal(nint)
    L = sp.csr_matrix((lva, lca, lpa), shape=(nint, nint))
    # (the two forms add a row's products in different orders)
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        rt = torch.tensor(r, dtype=dt, device="cuda")
        za = a.precond_apply(rt).cpu().numpy().astype(np.float64)
        zb = b.precond_apply(rt).cpu().numpy().astype(np.float64)
        assert np.isfinite(za).all() and za[-1] == 0.0
        assert np.linalg.norm(za - zb) <= tol * np.linalg.norm(zb), dt
    # componentwise backward error of the FP64 result, two triangular solves of
    # rows with k entries and the check's own products: about 4 k eps |L| |L^T| |z_p|
    z64 = a.precond_apply(torch.tensor(r, device="cuda")).cpu().numpy()[:nint]
    zp, rp = z64[pa], r[:nint][pa]
    res = rp - L @ (L.T @ zp)
    Lab = abs(L)
    bound = Lab @ (Lab.T @ np.abs(zp))
    k = int(max(np.diff(lpa).max(), np.bincount(lca).max()))   # longest row of L and of L^T
    assert np.all(np.abs(res) <= 4 * k * np.finfo(float).eps * bound + 1e-300)
    a.close()
    b.close()


def test_ic_wait_budget_runs_out_and_reports_timeout():
    # a wait budget of one cycle: the first row whose dependency is not yet
    # published gives up, the solve stops and the call returns GOFD_E_TIMEOUT;
    # the context stays usable (no device fault)
    from paper_2307_14437_gb300 import GofdError, Problem
    v, s, lo, hi, h = _lshape600()
    gp = Problem(v, s, 0.7, h, lo, hi, precond=9, ordering=0, wait_budget_cycles=1)
    nint = gp.info()["n_interior"]
    r = torch.zeros(nint + 1, dtype=torch.float64, device="cuda")
    r[:nint] = 1.0
    with pytest.raises(GofdError) as e:
        gp.precond_apply(r)
    assert e.value.code == "GOFD_E_TIMEOUT"
    f = torch.ones(gp.n_grid, dtype=torch.float64, device="cuda")
    with pytest.raises(GofdError) as e:
        gp.solve(f, mode="fp64", tol=1e-8)
    assert e.value.code == "GOFD_E_TIMEOUT"
    gp.close()
    ok = Problem(v, s, 0.7, h, lo, hi, precond=9, ordering=0)
    z = ok.precond_apply(r)
    assert torch.isfinite(z).all()
    _, info = ok.solve(f, mode="mixed", tol=1e-8)
    assert info["rel_res_fp64"] <= 1e-8
    ok.close()


def test_precond_iterations_close_to_oracle_pcg():
    # the oracle's IC(1)-PCG with the same order needs (almost) the same count
    from paper_2307_14437_gb300 import Problem
    d, v, s, n, alpha, M = _case("lshape")
    lo, hi, h = mg.grid_box(d, n)
    gp = Problem(v, s, alpha, h, lo, hi, filon_M=M, precond=9, ordering=1, check_every=1)
    ref = o.build(d, v, s, alpha, h, lo, hi, M=M, exact_weights=False)
    perm, *_ = gp.export_precond()
    b = o.rhs_grid(ref, np.ones(ref.n_grid))
    _, oi = o.pcg_ic(ref, b, pattern=9, tol=1e-10, perm=perm)
    _, gi = gp.solve(torch.ones(gp.n_grid, dtype=torch.float64, device="cuda"), mode="fp64", tol=1e-10)
    assert abs(gi["inner_iters"] - oi["iters"]) <= 2, (gi, oi)
    gp.close()


def test_bad_pattern_is_rejected():
    from paper_2307_14437_gb300 import GofdError, Problem
    d, v, s, n, alpha, M = _case("disk")
    lo, hi, h = mg.grid_box(d, n)
    with pytest.raises(GofdError) as e:
        Problem(v, s, alpha, h, lo, hi, filon_M=M, precond=27)
    assert e.value.code == "GOFD_E_ARG"


@pytest.mark.parametrize("name", ["disk", "lshape", "ball", "interval"])
def test_diagonal_of_s_matches_oracle(name):
    from paper_2307_14437_gb300 import Problem
    d, v, s, n, alpha, M = _case(name)
    lo, hi, h = mg.grid_box(d, n)
    gp = Problem(v, s, alpha, h, lo, hi, filon_M=M, precond=1)
    ref = o.build(d, v, s, alpha, h, lo, hi, M=M)
    got = gp.export_diagonal()
    want = o.jacobi_diagonal(ref)
    # FP32 products, FP64 sums
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    # the diagonal preconditioner in the solver: residual with the oracle's operator
    f = torch.ones(gp.n_grid, dtype=torch.float64, device="cuda")
    for mode in ("fp64", "mixed"):
        u, info = gp.solve(f, mode=mode, tol=1e-9)
        b = o.rhs_grid(ref, np.ones(ref.n_grid))
        assert np.linalg.norm(b - o.stiffness_apply(ref, u.cpu().numpy())) <= 1.05e-9 * np.linalg.norm(b)
    gp.close()


def test_diagonal_preconditioner_pays_on_a_graded_mesh():
    # graded disk, 385^2 grid: the diagonal of S spans two orders of magnitude;
    # scaling by it cuts the PCG iterations (the FP64 oracle: 156 -> 58)
    from paper_2307_14437_gb300 import Problem
    lo, hi, h = mg.grid_box(2, 385)
    v, s = mg.graded_disk_mesh(h, seed=mg.seed_for(4, 385))
    ft = torch.tensor(mg.target_bump(v), device="cuda")
    its = {}
    for pc in (0, 1):
        gp = Problem(v, s, 1.2, h, lo, hi, precond=pc)
        u, info = gp.solve(ft, rhs="vertex", mode="fp64", tol=1e-8)
        its[pc] = info["inner_iters"]
        assert info["rel_res_fp64"] <= 1e-8
        gp.close()
    assert its[1] < 0.6 * its[0], its


# ---------------------------------------------------------------------------
# the circulant alternative of Section 3.3 (precond = 2) through
# gofd_precond_apply, against the oracle's circulant_precond
# ---------------------------------------------------------------------------
def _interior_vectors(gp, ref, seed):
    ii, _ = gp.export_vertex_data()
    iv = np.nonzero(ii >= 0)[0]
    assert np.array_equal(iv, ref.interior)
    r = np.zeros(len(ref.verts))
    r[iv] = mg.random_vector(len(ref.verts), seed)[iv]
    rc = np.zeros(len(iv) + 1)
    rc[ii[iv]] = r[iv]
    return ii, iv, r, rc


CIRC = [("disk", 25, 1.5), ("lshape", 33, 1.0), ("lshape600", 600, 0.7)]


def _circ_case(name, n, alpha):
    if name == "lshape600":   # circulant 2048: the one-warp-per-FFT kernels in FP32
        v, s = mg.lshape_mesh(spacing=0.03, seed=mg.seed_for(2, 31))
        return v, s, 0
    d, v, s, _, _, M = _case(name)
    return v, s, M


@pytest.mark.parametrize("name,n,alpha", CIRC)
def test_circulant_precond_apply_matches_oracle(name, n, alpha):
    from paper_2307_14437_gb300 import Problem
    v, s, M = _circ_case(name, n, alpha)
    lo, hi, h = mg.grid_box(2, n)
    gp = Problem(v, s, alpha, h, lo, hi, filon_M=M, precond=2)
    inf = gp.info()
    ref = o.build(2, v, s, alpha, h, lo, hi, M=inf["filon_M"], exact_weights=False, pruned=True)
    ii, iv, r, rc = _interior_vectors(gp, ref, 41)
    want = o.circulant_precond(ref, r)[iv]
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        z = gp.precond_apply(torch.tensor(rc, dtype=dt, device="cuda")).cpu().numpy().astype(np.float64)
        assert z[-1] == 0.0
        got = z[ii[iv]]
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want), (dt, name)
    if n == 600:
        assert inf["warp_fft_path"] == 1
    gp.close()


def test_precond_apply_of_the_diagonal_matches_oracle():
    from paper_2307_14437_gb300 import Problem
    d, v, s, n, alpha, M = _case("lshape")
    lo, hi, h = mg.grid_box(d, n)
    gp = Problem(v, s, alpha, h, lo, hi, filon_M=M, precond=1)
    ref = o.build(d, v, s, alpha, h, lo, hi, M=M)
    ii, iv, r, rc = _interior_vectors(gp, ref, 43)
    want = r[iv] / o.jacobi_diagonal(ref)
    z = gp.precond_apply(torch.tensor(rc, device="cuda")).cpu().numpy()
    assert np.abs(z[ii[iv]] - want).max() <= 1e-5 * np.abs(want).max()
    gp.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_circulant_pcg_reaches_tolerance_with_oracle_iterations(mode):
    from paper_2307_14437_gb300 import Problem
    v, s, M = _circ_case("lshape", 33, 1.0)
    lo, hi, h = mg.grid_box(2, 33)
    for alpha in (1.0, 1.8):
        gp = Problem(v, s, alpha, h, lo, hi, filon_M=M, precond=2)
        ref = o.build(2, v, s, alpha, h, lo, hi, M=M, exact_weights=False)
        f = torch.ones(gp.n_grid, dtype=torch.float64, device="cuda")
        u, info = gp.solve(f, mode=mode, tol=1e-9)
        b = o.rhs_grid(ref, np.ones(ref.n_grid))
        assert np.linalg.norm(b - o.stiffness_apply(ref, u.cpu().numpy())) <= 1.05e-9 * np.linalg.norm(b)
        _, oi = o.pcg_circulant(ref, b, tol=1e-9)
        if mode == "fp64":   # one PCG run to half the tolerance, checked every 8 iterations on the device
            assert oi["iters"] - 2 <= info["inner_iters"] <= oi["iters"] + 12, (alpha, oi, info)
        gp.close()


def test_circulant_precond_is_2d_only():
    from paper_2307_14437_gb300 import GofdError, Problem
    d, v, s, n, alpha, M = _case("ball")
    lo, hi, h = mg.grid_box(d, n)
    with pytest.raises(GofdError) as e:
        Problem(v, s, alpha, h, lo, hi, filon_M=M, precond=2)
    assert e.value.code == "GOFD_E_ARG"
