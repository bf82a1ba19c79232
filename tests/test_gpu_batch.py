"""Many right-hand sides: the batched product, the lock-step block PCG, the
autotuner and concurrent independent problems, against single-vector calls
and the FP64 oracle.

Bars: the batched product equals the single-vector product bit for bit with
the default launch shapes, and the oracle within 1e-12 (FP64) / 1e-5 (FP32);
every column of a batched solve reaches ||b - S u|| <= tol ||b|| measured with
the oracle's operator.
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
    if name == "disk37_ragged":
        v, s = mg.disk_ring_mesh(rings=9, seed=mg.seed_for(1, 2))
        return 2, v, s, 37, 0.5, 2 ** 10
    if name == "lshape33":
        v, s = mg.lshape_mesh(spacing=0.15, seed=mg.seed_for(2, 1))
        return 2, v, s, 33, 1.5, 2 ** 10
    if name == "disk65":
        v, s = mg.disk_ring_mesh(rings=14, seed=mg.seed_for(1, 3))
        return 2, v, s, 65, 1.2, 2 ** 10
    if name == "ball9":
        v, s = mg.ball_shell_mesh(shells=3, seed=mg.seed_for(3, 1))
        return 3, v, s, 9, 1.5, 2 ** 8
    if name == "interval33":
        v, s = mg.interval_mesh(16, seed=mg.seed_for(0, 1))
        return 1, v, s, 33, 0.8, 2 ** 12
    raise KeyError(name)


@pytest.fixture(scope="module")
def built():
    from paper_2307_14437_gb300 import Problem
    cache = {}

    def get(name):
        if name not in cache:
            d, v, s, n, alpha, M = _case(name)
            lo, hi, h = mg.grid_box(d, n)
            ref = o.build(d, v, s, alpha, h, lo, hi, M=M)
            gp = Problem(v, s, alpha, h, lo, hi, filon_M=M)
            cache[name] = (gp, ref)
        return cache[name]

    yield get
    for gp, _ in cache.values():
        gp.close()


def _interior(gp):
    ii, _ = gp.export_vertex_data()
    return np.nonzero(ii >= 0)[0]           # interior vertices in vertex order = interior numbering


def _compact(gp, U, pad):
    """nb x N_v vertex vectors -> nb x (n_int + 1 + pad) interior rows, zero slot and padding 0."""
    iv = _interior(gp)
    X = np.zeros((U.shape[0], len(iv) + 1 + pad))
    X[:, :len(iv)] = U[:, iv]
    return X, iv


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["disk37_ragged", "lshape33", "disk65", "ball9", "interval33"])
def test_batched_product_equals_single_and_oracle(built, name, prec):
    gp, ref = built(name)
    nb = 5
    U = np.stack([mg.random_vector(len(ref.verts), 700 + c) for c in range(nb)])
    X, iv = _compact(gp, U, pad=7)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Xd = torch.tensor(X, device="cuda", dtype=dt)
    Yd = torch.full_like(Xd, 123.0)
    gp.apply_interior_batch(Xd, Yd)
    nint = len(iv)
    for c in range(nb):
        y1 = torch.empty(nint, device="cuda", dtype=dt)
        gp.apply_interior(Xd[c, :nint + 1].contiguous(), y1)
        assert torch.equal(Yd[c, :nint], y1), (name, prec, c)
        want = o.stiffness_apply(ref, U[c])[iv]
        rel = np.linalg.norm(Yd[c, :nint].double().cpu().numpy() - want) / np.linalg.norm(want)
        assert rel < (1e-12 if prec == "fp64" else 1e-5), (c, rel)
    # padding beyond the n_int outputs of each row is left alone
    assert torch.all(Yd[:, nint:] == 123.0)


def test_batch_of_one_and_large_batch(built):
    gp, ref = built("disk37_ragged")
    iv = _interior(gp)
    for nb in (1, 33):
        U = np.stack([mg.random_vector(len(ref.verts), 900 + c) for c in range(nb)])
        X, _ = _compact(gp, U, pad=0)
        Xd = torch.tensor(X, device="cuda")
        Yd = torch.empty_like(Xd)
        gp.apply_interior_batch(Xd, Yd)
        for c in (0, nb - 1):
            want = o.stiffness_apply(ref, U[c])[iv]
            got = Yd[c, :len(iv)].cpu().numpy()
            assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["disk37_ragged", "lshape33", "ball9", "interval33"])
def test_solve_batch_every_column_meets_tol(built, name, mode):
    gp, ref = built(name)
    d = ref.d
    pts = mg.grid_points(ref.box_lo, ref.h, ref.n[0])
    F = mg.rhs_family(pts, 6, seed=mg.seed_for(5, 1))
    F[3] = 0.0                                   # a zero column converges at once to u = 0
    Fd = torch.tensor(F, device="cuda")
    U, infos = gp.solve_batch(Fd, rhs="grid", mode=mode, tol=1e-8)
    U = U.cpu().numpy()
    for c in range(F.shape[0]):
        b = o.rhs_grid(ref, F[c])
        if c == 3:
            assert np.all(U[c] == 0.0) and infos[c]["rel_res_fp64"] == 0.0
            continue
        res = np.linalg.norm(b - o.stiffness_apply(ref, U[c])) / np.linalg.norm(b)
        assert res <= 1.05e-8, (name, mode, c, res, infos[c])
        assert infos[c]["rel_res_fp64"] <= 1e-8
    assert d == gp.d


def test_solve_batch_vertex_rhs_matches_single_solves(built):
    gp, ref = built("lshape33")
    F = mg.rhs_family(ref.verts, 4, seed=mg.seed_for(5, 2))
    U, _ = gp.solve_batch(torch.tensor(F, device="cuda"), rhs="vertex", mode="fp64", tol=1e-11)
    for c in range(4):
        u1, _ = gp.solve(torch.tensor(F[c], device="cuda"), rhs="vertex", mode="fp64", tol=1e-11)
        a, b = U[c].cpu().numpy(), u1.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)


def test_solve_batch_strided_rows(built):
    gp, ref = built("disk37_ragged")
    pts = mg.grid_points(ref.box_lo, ref.h, ref.n[0])
    F = mg.rhs_family(pts, 3, seed=mg.seed_for(5, 3))
    big = torch.zeros((3, ref.n_grid + 13), dtype=torch.float64, device="cuda")
    big[:, :ref.n_grid] = torch.tensor(F, device="cuda")
    U, _ = gp.solve_batch(big[:, :ref.n_grid], rhs="grid", mode="mixed", tol=1e-9)
    for c in range(3):
        b = o.rhs_grid(ref, F[c])
        assert np.linalg.norm(b - o.stiffness_apply(ref, U[c].cpu().numpy())) <= 1.05e-9 * np.linalg.norm(b)


def test_autotune_then_products_and_solves(built):
    from paper_2307_14437_gb300 import Problem
    _, ref = built("disk65")
    gp = Problem(ref.verts, ref.simp, ref.alpha, ref.h, ref.box_lo, ref.box_hi, filon_M=2 ** 10)
    ms = gp.autotune(nb=4)
    assert ms > 0.0
    iv = _interior(gp)
    U = np.stack([mg.random_vector(len(ref.verts), 1000 + c) for c in range(4)])
    X, _ = _compact(gp, U, pad=0)
    Xd = torch.tensor(X, device="cuda")
    Y1, Y2 = torch.empty_like(Xd), torch.empty_like(Xd)
    gp.apply_interior_batch(Xd, Y1)
    gp.apply_interior_batch(Xd, Y2)
    nint = len(iv)
    assert torch.equal(Y1[:, :nint], Y2[:, :nint])   # reproducible with the tuned shapes
    for c in range(4):
        want = o.stiffness_apply(ref, U[c])[iv]
        assert np.linalg.norm(Y1[c, :nint].cpu().numpy() - want) <= 1e-12 * np.linalg.norm(want)
    pts = mg.grid_points(ref.box_lo, ref.h, ref.n[0])
    F = mg.rhs_family(pts, 4, seed=mg.seed_for(5, 4))
    Us, _ = gp.solve_batch(torch.tensor(F, device="cuda"), mode="mixed", tol=1e-8)
    for c in range(4):
        b = o.rhs_grid(ref, F[c])
        assert np.linalg.norm(b - o.stiffness_apply(ref, Us[c].cpu().numpy())) <= 1.05e-8 * np.linalg.norm(b)
    gp.close()


def test_solve_many_equals_one_at_a_time(built):
    from paper_2307_14437_gb300 import solve_many
    names = ["disk37_ragged", "lshape33", "ball9"]
    probs = [built(n)[0] for n in names]
    refs = [built(n)[1] for n in names]
    Fs = []
    for k, ref in enumerate(refs):
        pts = mg.grid_points(ref.box_lo, ref.h, ref.n[0])
        Fs.append(torch.tensor(mg.rhs_family(pts, 3, seed=mg.seed_for(5, 10 + k)), device="cuda"))
    together = solve_many(probs, Fs, mode="mixed", tol=1e-9)
    for k, gp in enumerate(probs):
        alone, _ = gp.solve_batch(Fs[k], mode="mixed", tol=1e-9)
        assert torch.equal(together[k][0], alone)      # same kernels, same order: same bits
        for c in range(3):
            b = o.rhs_grid(refs[k], Fs[k][c].cpu().numpy())
            u = alone[c].cpu().numpy()
            assert np.linalg.norm(b - o.stiffness_apply(refs[k], u)) <= 1.05e-9 * np.linalg.norm(b)


def test_batch_argument_errors(built):
    from paper_2307_14437_gb300 import GofdError
    gp, ref = built("disk37_ragged")
    F = torch.zeros((2, ref.n_grid - 1), dtype=torch.float64, device="cuda")
    with pytest.raises(GofdError):
        gp.solve_batch(F, rhs="grid")           # rows shorter than the grid
    X = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(GofdError):
        gp.apply_interior_batch(X, torch.zeros_like(X))   # ld < n_int + 1


def test_tuned_batched_product_equals_single_products(built):
    # whatever shapes and sub-batch size the tuner picks, every column of the
    # batched product equals the single-vector product with the same shapes
    from paper_2307_14437_gb300 import Problem
    _, ref = built("disk65")
    gp = Problem(ref.verts, ref.simp, ref.alpha, ref.h, ref.box_lo, ref.box_hi, filon_M=2 ** 10)
    gp.autotune(nb=5)
    info = gp.info()
    assert info["tune_batch_chunk"] in (0, 1, 2, 4)
    U = np.stack([mg.random_vector(len(ref.verts), 1100 + c) for c in range(5)])
    X, iv = _compact(gp, U, pad=3)
    nint = len(iv)
    for dt in (torch.float32, torch.float64):
        Xd = torch.tensor(X, device="cuda", dtype=dt)
        Yd = torch.empty_like(Xd)
        gp.apply_interior_batch(Xd, Yd)
        for c in range(5):
            y1 = torch.empty(nint, device="cuda", dtype=dt)
            gp.apply_interior(Xd[c, :nint + 1].contiguous(), y1)
            assert torch.equal(Yd[c, :nint], y1), (dt, c, info)
    gp.close()
