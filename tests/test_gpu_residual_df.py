"""The mixed solver's FP64 residual product with its FFT convolution in
double-float arithmetic (GOFD_FP64_DF, 2D and 3D): S x (Section 3.2,
(GoFD-2); A_FD by the circulant convolution of Section 2.2) against the
oracle's FP64 product, at the bar for counting as FP64 (1e-12 relative), and
mixed solves with it.
"""
import numpy as np
import pytest

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
    if name == "disk37":        # ragged grid, circulant 128
        v, s = mg.disk_ring_mesh(rings=10, seed=mg.seed_for(1, 50))
        return v, s, 37, 1.3, 2 ** 12
    if name == "lshape200":     # circulant 512
        v, s = mg.lshape_mesh(spacing=0.05, seed=mg.seed_for(2, 50))
        return v, s, 200, 0.6, 2 ** 12
    if name == "lshape1024":    # the L-shape workload at full size, circulant 2048
        v, s = mg.lshape_mesh(seed=mg.seed_for(2))
        return v, s, 1024, 1.0, 0
    if name == "disk1100":      # circulant 4096
        v, s = mg.disk_ring_mesh(rings=30, seed=mg.seed_for(1, 51))
        return v, s, 1100, 1.5, 0
    raise KeyError(name)


@pytest.mark.parametrize("name", ["disk37", "lshape200", "lshape1024", "disk1100"])
def test_double_float_product_is_fp64_accurate(name):
    from paper_2307_14437_gb300 import Problem
    v, s, n, alpha, M = _case(name)
    lo, hi, h = mg.grid_box(2, n)
    gp = Problem(v, s, alpha, h, lo, hi, filon_M=M)
    ref = o.build(2, v, s, alpha, h, lo, hi, exact_weights=False, pruned=True, M=gp.info()["filon_M"])
    ii, _ = gp.export_vertex_data()
    iv = np.nonzero(ii >= 0)[0]
    u = np.zeros(len(v))
    u[iv] = mg.random_vector(len(v), 52)[iv]
    want = o.stiffness_apply(ref, u)[iv]
    x = np.zeros(len(iv) + 1)
    x[ii[iv]] = u[iv]
    xd = torch.tensor(x, device="cuda")
    y_df = torch.zeros(len(iv) + 1, dtype=torch.float64, device="cuda")
    y_64 = torch.zeros_like(y_df)
    gp.apply_interior(xd, y_df, prec="fp64_df")
    gp.apply_interior(xd, y_64, prec="fp64")
    got = y_df.cpu().numpy()[ii[iv]]
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 1e-12, err
    # and against the GPU's FP64 product
    g64 = y_64.cpu().numpy()[ii[iv]]
    assert np.linalg.norm(got - g64) <= 1e-12 * np.linalg.norm(g64)
    gp.close()


@pytest.mark.parametrize("n", [17, 29])
def test_double_float_product_is_fp64_accurate_in_3d(n):
    from paper_2307_14437_gb300 import Problem
    v, s = mg.ball_shell_mesh(shells=4, seed=mg.seed_for(3, 50))
    lo, hi, h = mg.grid_box(3, n)
    gp = Problem(v, s, 1.5, h, lo, hi, filon_M=2 ** 8)
    ref = o.build(3, v, s, 1.5, h, lo, hi, exact_weights=False, pruned=True, M=2 ** 8)
    ii, _ = gp.export_vertex_data()
    iv = np.nonzero(ii >= 0)[0]
    u = np.zeros(len(v))
    u[iv] = mg.random_vector(len(v), 54)[iv]
    want = o.stiffness_apply(ref, u)[iv]
    x = np.zeros(len(iv) + 1)
    x[ii[iv]] = u[iv]
    y = torch.zeros(len(iv) + 1, dtype=torch.float64, device="cuda")
    gp.apply_interior(torch.tensor(x, device="cuda"), y, prec="fp64_df")
    got = y.cpu().numpy()[ii[iv]]
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    # the mixed solve with it reaches the tolerance with the oracle's operator
    f = torch.ones(gp.n_grid, dtype=torch.float64, device="cuda")
    uu, info = gp.solve(f, mode="mixed", tol=1e-9)
    b = o.rhs_grid(ref, np.ones(ref.n_grid))
    assert np.linalg.norm(b - o.stiffness_apply(ref, uu.cpu().numpy())) <= 1.05e-9 * np.linalg.norm(b)
    gp.close()


def test_double_float_is_not_for_1d():
    from paper_2307_14437_gb300 import GofdError, Problem
    v, s = mg.interval_mesh(24, seed=mg.seed_for(0, 2))
    lo, hi, h = mg.grid_box(1, 49)
    gp = Problem(v, s, 1.2, h, lo, hi, filon_M=2 ** 12)
    x = torch.zeros(gp.n_interior + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(GofdError) as e:
        gp.apply_interior(x, torch.empty_like(x), prec="fp64_df")
    assert e.value.code == "GOFD_E_ARG"
    gp.close()


@pytest.mark.parametrize("fp64_residual", [0, 1])
def test_mixed_solves_with_either_residual(fp64_residual):
    from paper_2307_14437_gb300 import Problem
    v, s, n, alpha, M = _case("lshape200")
    lo, hi, h = mg.grid_box(2, n)
    ref = o.build(2, v, s, alpha, h, lo, hi, exact_weights=False, pruned=True, M=M)
    b = o.rhs_grid(ref, np.ones(ref.n_grid))
    for tol in (1e-8, 1e-11):
        gp = Problem(v, s, alpha, h, lo, hi, filon_M=M, fp64_residual=fp64_residual)
        f = torch.ones(gp.n_grid, dtype=torch.float64, device="cuda")
        u, info = gp.solve(f, mode="mixed", tol=tol)
        r = np.linalg.norm(b - o.stiffness_apply(ref, u.cpu().numpy())) / np.linalg.norm(b)
        assert r <= 1.05 * tol, (tol, r, info)
        # batched: every column to the tolerance
        F = torch.tensor(mg.rhs_family(mg.grid_points(lo, h, n), 3, seed=53, inside=mg.in_lshape), device="cuda")
        U, infos = gp.solve_batch(F, mode="mixed", tol=tol)
        for c in range(3):
            bc = o.rhs_grid(ref, F[c].cpu().numpy())
            rc = np.linalg.norm(bc - o.stiffness_apply(ref, U[c].cpu().numpy())) / np.linalg.norm(bc)
            assert rc <= 1.05 * tol, (c, tol, rc)
        gp.close()
