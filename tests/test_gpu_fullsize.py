"""Parity at the full sizes of the benchmark workloads, in the configuration
bench.py times (default options: paper Filon M, default circulant length).

L-shape 6.05e4 vertices / 1024^2 grid and graded disk 2.1e5 vertices / 2048^2
grid: every grid node's owner and ELL row against the exact oracle, the
coefficients and symbol, FP32 and FP64 products against the oracle's FFT
product, solves checked with the oracle's operator.  Unit ball 1.3e5 vertices
/ 256^3 grid: every owner and ELL row against the exact oracle, D_h, a seeded
sample of T against the oracle's coefficients, properties that hold at any
size (symmetry, positivity, FP32/FP64 agreement) and the closed-form solution
(exam-2).
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def lshape():
    from paper_2307_14437_gb300 import Problem
    v, s = mg.lshape_mesh(seed=mg.seed_for(2))
    lo, hi, h = mg.grid_box(2, 1024)
    gp = Problem(v, s, 1.0, h, lo, hi)
    ref = o.build(2, v, s, 1.0, h, lo, hi, exact_weights=False, pruned=True, M=gp.info()["filon_M"])
    return gp, ref


def test_lshape_transfer_coefficients_symbol(lshape):
    gp, ref = lshape
    owner, idx, w = gp.export_transfer()
    assert np.array_equal(owner, ref.owner.astype(np.int32))
    assert np.array_equal(idx, ref.ell_idx.astype(np.int32))
    assert np.abs(w - ref.ell_w).max() < 1e-12
    assert np.abs(gp.coefficients() - ref.T).max() < 1e-13
    assert gp.P == ref.P
    assert np.abs(gp.symbol() - ref.lam).max() < 1e-12 * np.abs(ref.lam).max()


def test_lshape_products(lshape):
    gp, ref = lshape
    u = mg.random_vector(len(ref.verts), 41)
    want = o.stiffness_apply(ref, u)
    y64 = gp.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    y32 = gp.apply(torch.tensor(u, device="cuda", dtype=torch.float32)).cpu().numpy().astype(np.float64)
    assert _rel(y64, want) < 1e-12
    assert _rel(y32, want) < 1e-5


_ROWS = [(8, 1), (8, 2), (8, 4), (16, 1), (16, 2), (16, 4)]
_COLS = [(8, 1), (8, 2), (8, 4), (16, 1), (16, 2), (16, 4), (32, 1), (32, 2), (32, 4)]
_SHAPES = [dict(row_elems=_ROWS[i * 5 % 6][0], lines_per_cta=_ROWS[i * 5 % 6][1], col_elems=_COLS[i][0],
                cols_per_cta=_COLS[i][1], scatter_lanes=(4, 8, 16, 32)[i % 4], batch_chunk=i % 3)
           for i in range(9)]


@pytest.mark.parametrize("shape", _SHAPES, ids=lambda d: "r%(row_elems)d.%(lines_per_cta)d-c%(col_elems)d.%(cols_per_cta)d"
                         "-s%(scatter_lanes)d-b%(batch_chunk)d" % d)
def test_lshape_products_every_launch_shape(lshape, shape):
    # every launch shape the autotuner may choose at this size (all row and
    # column shapes, every scatter width and sub-batch size) against the oracle;
    # the batched product equals the single-vector products bit for bit
    gp, ref = lshape
    gp.set_launch_shapes(**shape)
    try:
        info = gp.info()
        assert info["tune_row_elems"] == shape["row_elems"] and info["tune_col_elems"] == shape["col_elems"]
        u = mg.random_vector(len(ref.verts), 41)
        want = o.stiffness_apply(ref, u)
        y32 = gp.apply(torch.tensor(u, device="cuda", dtype=torch.float32)).cpu().numpy().astype(np.float64)
        y64 = gp.apply(torch.tensor(u, device="cuda")).cpu().numpy()
        assert _rel(y32, want) < 1e-5
        assert _rel(y64, want) < 1e-12
        ii, _ = gp.export_vertex_data()
        iv = np.nonzero(ii >= 0)[0]
        X = np.zeros((3, len(iv) + 1))
        for c in range(3):
            X[c, :len(iv)] = mg.random_vector(len(ref.verts), 50 + c)[iv]
        Xd = torch.tensor(X, device="cuda", dtype=torch.float32)
        Yd = torch.empty_like(Xd)
        gp.apply_interior_batch(Xd, Yd)
        for c in range(3):
            y1 = torch.empty(len(iv), device="cuda", dtype=torch.float32)
            gp.apply_interior(Xd[c].contiguous(), y1)
            assert torch.equal(Yd[c, :len(iv)], y1), c
    finally:
        gp.set_launch_shapes()


def test_launch_shape_arguments_are_checked(lshape):
    from paper_2307_14437_gb300 import GofdError
    gp, _ = lshape
    for bad in (dict(lines_per_cta=3), dict(cols_per_cta=8), dict(scatter_lanes=2), dict(col_elems=4),
                dict(row_elems=32), dict(batch_chunk=-1)):
        with pytest.raises(GofdError):
            gp.set_launch_shapes(**bad)
    assert gp.info()["tune_row_elems"] == 0


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5])
def test_lshape_solves_reach_1e8(lshape, alpha):
    from paper_2307_14437_gb300 import Problem
    gp0, ref0 = lshape
    if alpha == 1.0:
        gp, ref = gp0, ref0
    else:
        gp = Problem(ref0.verts, ref0.simp, alpha, ref0.h, ref0.box_lo, ref0.box_hi)
        ref = o.build(2, ref0.verts, ref0.simp, alpha, ref0.h, ref0.box_lo, ref0.box_hi, exact_weights=False,
                      pruned=True, M=gp.info()["filon_M"])
    b = o.rhs_grid(ref, np.ones(ref.n_grid))
    f = torch.ones(gp.n_grid, dtype=torch.float64, device="cuda")
    for mode in ("mixed", "fp64"):
        u, info = gp.solve(f, mode=mode, tol=1e-8)
        res = np.linalg.norm(b - o.stiffness_apply(ref, u.cpu().numpy())) / np.linalg.norm(b)
        assert res <= 1.05e-8, (mode, res, info)


def test_lshape_ic1_pcg(lshape):
    from paper_2307_14437_gb300 import Problem
    _, ref = lshape
    gp = Problem(ref.verts, ref.simp, 1.0, ref.h, ref.box_lo, ref.box_hi, precond=9, ordering=1)
    f = torch.ones(gp.n_grid, dtype=torch.float64, device="cuda")
    u, info = gp.solve(f, mode="mixed", tol=1e-8)
    b = o.rhs_grid(ref, np.ones(ref.n_grid))
    assert np.linalg.norm(b - o.stiffness_apply(ref, u.cpu().numpy())) / np.linalg.norm(b) <= 1.05e-8
    gp.close()


def test_graded_disk_2048(request):
    from paper_2307_14437_gb300 import Problem
    lo, hi, h = mg.grid_box(2, 2048)
    v, s = mg.graded_disk_mesh(h, seed=mg.seed_for(4))
    gp = Problem(v, s, 1.2, h, lo, hi)
    ref = o.build(2, v, s, 1.2, h, lo, hi, exact_weights=False, pruned=True, M=gp.info()["filon_M"])
    owner, idx, w = gp.export_transfer()
    assert np.array_equal(owner, ref.owner.astype(np.int32))
    assert np.array_equal(idx, ref.ell_idx.astype(np.int32))
    assert np.abs(w - ref.ell_w).max() < 1e-12
    assert np.abs(gp.coefficients() - ref.T).max() < 1e-13
    u = mg.random_vector(len(v), 43)
    want = o.stiffness_apply(ref, u)
    y32 = gp.apply(torch.tensor(u, device="cuda", dtype=torch.float32)).cpu().numpy().astype(np.float64)
    assert _rel(y32, want) < 1e-5
    # GoFD-3 right-hand side from vertex values of f_target (Section 3.2)
    ft = mg.target_bump(v)
    uu, info = gp.solve(torch.tensor(ft, device="cuda"), rhs="vertex", mode="mixed", tol=1e-8)
    b = o.rhs_vertex(ref, ft)
    assert np.linalg.norm(b - o.stiffness_apply(ref, uu.cpu().numpy())) / np.linalg.norm(b) <= 1.05e-8
    gp.close()


@pytest.fixture(scope="module")
def ball():
    from paper_2307_14437_gb300 import Problem
    v, s = mg.ball_shell_mesh(seed=mg.seed_for(3))
    lo, hi, h = mg.grid_box(3, 256)
    gp = Problem(v, s, 1.5, h, lo, hi)
    yield gp, v, s, lo, hi, h
    gp.close()


def test_ball_256_transfer_and_coefficients(ball):
    # every grid node's owner and every ELL row against the oracle's exact
    # location (bounding-box pruned, same predicate and tie rule), weights
    # within their FP64 evaluation error, D_h over every interior vertex; and
    # a seeded sample of T (M = 2^11, the paper's 3D default) against the
    # oracle's Filon + Richardson evaluated entry by entry
    gp, v, s, lo, hi, h = ball
    n = o.grid_shape(lo, hi, h)
    owner, idx, w = gp.export_transfer()
    want = o.locate_pruned(v, s, lo, h, n)
    assert np.array_equal(owner, want.astype(np.int32))
    nodes, ridx, rw = o.ell_layout(v, s, lo, h, n, want, exact=False)
    assert np.array_equal(idx, ridx.astype(np.int32))
    assert np.abs(w - rw).max() < 1e-12
    I = o.transfer_matrix(nodes, ridx, rw, int(np.prod(n)), len(v))
    Dh = o.column_sums(I)
    interior = np.nonzero(~o.boundary_vertices(s, len(v)))[0]
    ii, cs = gp.export_vertex_data()
    assert np.array_equal(np.nonzero(ii >= 0)[0], interior)
    assert np.abs(cs[interior] - Dh[interior]).max() < 1e-13 * Dh.max()
    info = gp.info()
    M = info["filon_M"]
    assert M == 2 ** 11
    rng = np.random.default_rng(mg.seed_for(3, 9))
    ps = np.vstack([[0, 0, 0], [1, 0, 0], [1, 1, 1], [255, 0, 0], [255, 255, 255], [0, 254, 3],
                    rng.integers(0, 256, size=(26, 3))])
    Tw = o.coefficients_at(3, 0.75, ps, M)
    T = gp.coefficients().reshape((256,) * 3)
    got = np.array([T[p[2], p[1], p[0]] for p in ps])
    assert np.abs(got - Tw).max() < 1e-13, np.abs(got - Tw).max()


def test_ball_256_properties_and_closed_form(ball):
    gp, v, s, lo, hi, h = ball
    # symmetry and positivity of S (Theorem 3.1), FP32 vs FP64 agreement
    a = torch.tensor(mg.random_vector(len(v), 44), device="cuda")
    b = torch.tensor(mg.random_vector(len(v), 45), device="cuda")
    Sa, Sb = gp.apply(a), gp.apply(b)
    ab, ba = float(torch.dot(b, Sa)), float(torch.dot(a, Sb))
    assert abs(ab - ba) <= 1e-12 * float(torch.linalg.norm(Sa) * torch.linalg.norm(b))
    ii, _ = gp.export_vertex_data()
    mask = torch.tensor(ii >= 0, device="cuda", dtype=torch.float64)
    assert float(torch.dot(a * mask, Sa)) > 0
    Sa32 = gp.apply(a.float()).double()
    assert float(torch.linalg.norm(Sa32 - Sa) / torch.linalg.norm(Sa)) < 1e-5
    # (exam-2) with s = 0.75: u = C (1-|x|^2)^0.75, C = 0.300901...
    u, info = gp.solve(torch.ones(gp.n_grid, dtype=torch.float64, device="cuda"), mode="mixed", tol=1e-8)
    assert info["rel_res_fp64"] <= 1e-8
    err = o.lumped_l2(v, s, u.cpu().numpy() - o.ball_exact(v, 0.75))
    norm = o.lumped_l2(v, s, o.ball_exact(v, 0.75))
    assert err / norm < 0.05, err / norm
