"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: owner simplex and ELL layout of I_h^FD bit-exact; barycentric weights
within their FP64 evaluation error; FP64 operators relative L2 <= 1e-12;
FP32 operators <= 1e-5 (random inputs); solves reach relative residual <= tol
measured with the oracle's operator.
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


def _gpu(v, s, alpha, h, lo, hi, **kw):
    from paper_2307_14437_gb300 import Problem
    return Problem(v, s, alpha, h, lo, hi, **kw)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------------------
# workloads of parity size: (name, d, mesh builder, n, alpha, M)
# ---------------------------------------------------------------------------
def _case(name):
    if name == "disk17":
        v, s = mg.disk_ring_mesh(rings=6, seed=mg.seed_for(1, 1))
        return 2, v, s, 17, 1.0, 2 ** 10
    if name == "disk37_ragged":
        v, s = mg.disk_ring_mesh(rings=9, seed=mg.seed_for(1, 2))
        return 2, v, s, 37, 0.5, 2 ** 10
    if name == "lshape33":
        v, s = mg.lshape_mesh(spacing=0.15, seed=mg.seed_for(2, 1))
        return 2, v, s, 33, 1.5, 2 ** 10
    if name == "aligned2":
        lo, hi, h = mg.grid_box(2, 11)
        v, s = mg.grid_aligned_mesh(2, -1.0, h, 6, origin_cells=2)
        return 2, v, s, 11, 1.2, 2 ** 10
    if name == "ball9":
        v, s = mg.ball_shell_mesh(shells=3, seed=mg.seed_for(3, 1))
        return 3, v, s, 9, 1.5, 2 ** 8
    if name == "ball37_ragged":
        v, s = mg.ball_shell_mesh(shells=5, seed=mg.seed_for(3, 2))
        return 3, v, s, 37, 0.7, 2 ** 9
    if name == "aligned3":
        lo, hi, h = mg.grid_box(3, 7)
        v, s = mg.grid_aligned_mesh(3, -1.0, h, 4, origin_cells=1)
        return 3, v, s, 7, 1.0, 2 ** 8
    if name == "interval33":
        v, s = mg.interval_mesh(16, seed=mg.seed_for(0, 1))
        return 1, v, s, 33, 0.8, 2 ** 12
    raise KeyError(name)


SMALL = ["disk17", "disk37_ragged", "lshape33", "aligned2", "ball9", "ball37_ragged", "aligned3", "interval33"]


@pytest.fixture(scope="module")
def built():
    cache = {}

    def get(name):
        if name not in cache:
            d, v, s, n, alpha, M = _case(name)
            lo, hi, h = mg.grid_box(d, n)
            ref = o.build(d, v, s, alpha, h, lo, hi, M=M, pruned=d == 3)
            gp = _gpu(v, s, alpha, h, lo, hi, filon_M=M)
            cache[name] = (gp, ref)
        return cache[name]
    return get


@pytest.mark.parametrize("name", SMALL)
def test_transfer_bit_exact(built, name):
    gp, ref = built(name)
    owner, idx, w = gp.export_transfer()
    assert np.array_equal(owner, ref.owner.astype(np.int32))
    assert np.array_equal(idx, ref.ell_idx.astype(np.int32))
    # exact rational weights rounded once vs FP64 cofactor ratios
    assert np.abs(w - ref.ell_w).max() < 1e-13


@pytest.mark.parametrize("name", SMALL)
def test_boundary_numbering_and_colsums(built, name):
    gp, ref = built(name)
    ii, cs = gp.export_vertex_data()
    expect = -np.ones(len(ref.verts), dtype=np.int64)
    expect[ref.interior] = np.arange(len(ref.interior))
    assert np.array_equal(ii, expect)
    assert np.abs(cs[ref.interior] - ref.Dh[ref.interior]).max() < 1e-13 * ref.Dh.max()
    inf = gp.info()
    assert abs(inf["a_h"] - ref.a_h) < 1e-14 * ref.a_h


@pytest.mark.parametrize("name", SMALL)
def test_coefficients(built, name):
    gp, ref = built(name)
    T = gp.coefficients()
    assert np.abs(T - ref.T).max() < 1e-13


@pytest.mark.parametrize("name", ["disk17", "aligned2", "ball9", "ball37_ragged", "aligned3", "interval33"])
def test_symbol(built, name):
    # the library's circulant length is the oracle's rule raised to at least
    # 32 (any P >= 2n-2 embeds T exactly): the oracle's symbol is taken at the
    # library's P, from the oracle's own coefficients
    gp, ref = built(name)
    P = gp.P
    assert P >= ref.P and P >= 32 and (P & (P - 1)) == 0
    want = o.symbol(ref.T, P)
    lam = gp.symbol()
    assert lam.shape == want.shape
    assert np.abs(lam - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("name", SMALL)
def test_afd_apply(built, name):
    gp, ref = built(name)
    v = mg.random_vector(ref.n_grid, 7)
    want = o.afd_apply(ref, v, method="direct")
    got64 = gp.afd_apply(torch.tensor(v, device="cuda")).cpu().numpy()
    got32 = gp.afd_apply(torch.tensor(v, device="cuda", dtype=torch.float32)).cpu().numpy()
    assert _rel(got64, want) < 1e-12
    assert _rel(got32.astype(np.float64), want) < 1e-5


@pytest.mark.parametrize("name", SMALL)
def test_stiffness_apply(built, name):
    gp, ref = built(name)
    u = mg.random_vector(len(ref.verts), 11)
    want = o.stiffness_apply(ref, u, method="direct")
    y64 = gp.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    y32 = gp.apply(torch.tensor(u, device="cuda", dtype=torch.float32)).cpu().numpy()
    assert _rel(y64, want) < 1e-12
    assert _rel(y32.astype(np.float64), want) < 1e-5
    assert np.all(y64[ref.boundary] == 0.0)


@pytest.mark.parametrize("name", ["disk17", "ball9"])
def test_fraclap_apply(built, name):
    gp, ref = built(name)
    u = mg.random_vector(len(ref.verts), 12)
    want = o.fraclap_apply(ref, u, method="direct")
    got = gp.apply(torch.tensor(u, device="cuda"), op="fraclap").cpu().numpy()
    assert _rel(got, want) < 1e-12


def test_boundary_inputs_are_ignored(built):
    gp, ref = built("disk17")
    u = mg.random_vector(len(ref.verts), 13)
    u2 = u.copy()
    u2[ref.boundary] = np.nan
    a = gp.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    b = gp.apply(torch.tensor(u2, device="cuda")).cpu().numpy()
    assert np.array_equal(a, b)


def test_apply_is_deterministic(built):
    gp, ref = built("lshape33")
    u = torch.tensor(mg.random_vector(len(ref.verts), 14), device="cuda", dtype=torch.float32)
    a = gp.apply(u).cpu().numpy()
    b = gp.apply(u).cpu().numpy()
    assert np.array_equal(a, b)


def test_apply_host_matches_device(built):
    gp, ref = built("disk37_ragged")
    u = mg.random_vector(len(ref.verts), 15)
    a = gp.apply_host(u)
    b = gp.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["disk37_ragged", "ball9"])
def test_apply_host_on_pinned_buffers(built, name):
    # pinned host buffers are read and written by the kernels in place (mapped
    # memory); a pinned input with a pageable output takes the staging copies
    gp, ref = built(name)
    u = mg.random_vector(len(ref.verts), 16)
    for dt in (torch.float64, torch.float32):
        ud = torch.tensor(u, dtype=dt, device="cuda")
        uh = torch.tensor(u, dtype=dt).pin_memory()
        yh = torch.empty_like(uh).pin_memory()
        for op in ("stiffness", "fraclap"):
            want = gp.apply(ud, op=op).cpu().numpy()
            gp.apply_host(uh.numpy(), op=op, out=yh.numpy())
            assert np.array_equal(yh.numpy(), want), (dt, op)
            got = gp.apply_host(uh.numpy(), op=op)   # pageable output
            assert np.array_equal(got, want), (dt, op)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["disk17", "lshape33", "ball9"])
def test_solve_residual(built, name, mode):
    gp, ref = built(name)
    f = np.ones(ref.n_grid)
    tol = 1e-10
    u, info = gp.solve(torch.tensor(f, device="cuda"), rhs="grid", mode=mode, tol=tol)
    u = u.cpu().numpy()
    b = o.rhs_grid(ref, f)
    res = np.linalg.norm(b - o.stiffness_apply(ref, u)) / np.linalg.norm(b)
    assert res < 2 * tol, (res, info)
    x_ref, _ = o.solve(ref, b, tol=1e-13)
    assert _rel(u, x_ref) < 1e-7
    assert np.all(u[ref.boundary] == 0.0)


def test_solver_iterations_run_as_device_loop(built):
    gp, ref = built("disk37_ragged")
    f = torch.ones(ref.n_grid, dtype=torch.float64, device="cuda")
    for mode in ("mixed", "fp64"):
        u, info = gp.solve(f, mode=mode, tol=1e-9)
        assert info["device_loop"] == 1, info
        b = o.rhs_grid(ref, np.ones(ref.n_grid))
        assert np.linalg.norm(b - o.stiffness_apply(ref, u.cpu().numpy())) <= 1.05e-9 * np.linalg.norm(b)


def test_solve_vertex_rhs_equals_grid_rhs_for_constant_f(built):
    # (GoFD-1) and (GoFD-3) give the same system for f = 1
    gp, ref = built("disk17")
    ug, _ = gp.solve(torch.ones(ref.n_grid, dtype=torch.float64, device="cuda"), rhs="grid", mode="fp64", tol=1e-12)
    uv, _ = gp.solve(torch.ones(len(ref.verts), dtype=torch.float64, device="cuda"), rhs="vertex", mode="fp64",
                     tol=1e-12)
    assert _rel(uv.cpu().numpy(), ug.cpu().numpy()) < 1e-10


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_non_finite_data_is_rejected(built):
    # a NaN or Inf in f reaching the right-hand side is an argument error, for
    # both solvers and the batched one; the handle stays usable afterwards
    from paper_2307_14437_gb300 import GofdError
    gp, ref = built("disk37_ragged")
    ii, _ = gp.export_vertex_data()
    k = int(np.nonzero(ii >= 0)[0][0])
    f = torch.ones(len(ref.verts), dtype=torch.float64, device="cuda")
    f[k] = float("nan")
    for mode in ("mixed", "fp64"):
        with pytest.raises(GofdError):
            gp.solve(f, rhs="vertex", mode=mode, tol=1e-8)
    F = torch.ones((2, len(ref.verts)), dtype=torch.float64, device="cuda")
    F[1, k] = float("inf")
    with pytest.raises(GofdError):
        gp.solve_batch(F, rhs="vertex", mode="mixed", tol=1e-8)
    f[k] = 1.0
    u, info = gp.solve(f, rhs="vertex", mode="mixed", tol=1e-8)
    assert info["rel_res_fp64"] <= 1e-8 and bool(torch.isfinite(u).all())


def test_degenerate_simplex_is_rejected():
    from paper_2307_14437_gb300 import GofdError
    v = np.array([[0.0, 0.0], [0.5, 0.5], [0.25, 0.25], [0.5, 0.0]])
    s = np.array([[0, 1, 2], [0, 3, 1]])
    lo, hi, h = mg.grid_box(2, 9)
    with pytest.raises(GofdError) as e:
        _gpu(v, s, 1.0, h, lo, hi, filon_M=2 ** 10)
    assert e.value.code == "GOFD_E_DEGENERATE_SIMPLEX"


def test_zero_column_sum_is_rejected():
    # split an interior triangle that holds no grid node at its centroid: the
    # new vertex's patch is that triangle, so its column sum D_h is exactly 0
    from paper_2307_14437_gb300 import GofdError
    v, s = mg.disk_ring_mesh(rings=6, seed=1)
    lo, hi, h = mg.grid_box(2, 13)
    n = o.grid_shape(lo, hi, h)
    own = o.locate(v, s, lo, h, n)
    cnt = np.bincount(own[own >= 0], minlength=len(s))
    bnd = o.boundary_vertices(s, len(v))
    e = int([k for k in np.nonzero(cnt == 0)[0] if not bnd[s[k]].any()][0])
    a, b, c = s[e]
    m = len(v)
    v2 = np.vstack([v, v[s[e]].mean(axis=0)])
    s2 = mg._orient_positive(v2, np.vstack([np.delete(s, e, axis=0), [[a, b, m], [b, c, m], [c, a, m]]]))
    assert o.build(2, v2, s2, 1.0, h, lo, hi, M=2 ** 10, exact_weights=False).Dh[m] == 0.0
    with pytest.raises(GofdError) as err:
        _gpu(v2, s2, 1.0, h, lo, hi, filon_M=2 ** 10)
    assert err.value.code == "GOFD_E_ZERO_COLSUM"


def test_mesh_in_a_large_box_leaves_most_nodes_outside():
    v, s = mg.disk_ring_mesh(rings=3, seed=2)
    v = 0.2 * v
    lo, hi, h = mg.grid_box(2, 65)
    gp = _gpu(v, s, 1.0, h, lo, hi, filon_M=2 ** 10)
    ref = o.build(2, v, s, 1.0, h, lo, hi, M=2 ** 10)
    owner, idx, _ = gp.export_transfer()
    assert np.array_equal(owner, ref.owner.astype(np.int32))
    u = mg.random_vector(len(v), 3)
    y = gp.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    assert _rel(y, o.stiffness_apply(ref, u)) < 1e-12


# ---------------------------------------------------------------------------
# configuration 1 in full (unit disk, 1951 vertices, 128^2 grid, alpha = 1)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c1():
    v, s = mg.disk_ring_mesh()
    lo, hi, h = mg.grid_box(2, 128)
    ref = o.build(2, v, s, 1.0, h, lo, hi, exact_weights=False)
    gp = _gpu(v, s, 1.0, h, lo, hi)
    return gp, ref


def test_c1_transfer_and_apply(c1):
    gp, ref = c1
    owner, idx, w = gp.export_transfer()
    assert np.array_equal(owner, ref.owner.astype(np.int32))
    assert np.array_equal(idx, ref.ell_idx.astype(np.int32))
    assert np.abs(w - ref.ell_w).max() < 1e-12
    assert np.abs(gp.coefficients() - ref.T).max() < 1e-13
    u = mg.random_vector(len(ref.verts), 21)
    want = o.stiffness_apply(ref, u)
    assert _rel(gp.apply(torch.tensor(u, device="cuda")).cpu().numpy(), want) < 1e-12
    y32 = gp.apply(torch.tensor(u, device="cuda", dtype=torch.float32)).cpu().numpy()
    assert _rel(y32.astype(np.float64), want) < 1e-5


def test_c1_solve_against_closed_form(c1):
    gp, ref = c1
    u, info = gp.solve(torch.ones(ref.n_grid, dtype=torch.float64, device="cuda"), rhs="grid", mode="fp64",
                       tol=1e-10)
    u = u.cpu().numpy()
    b = o.rhs_grid(ref, np.ones(ref.n_grid))
    assert np.linalg.norm(b - o.stiffness_apply(ref, u)) / np.linalg.norm(b) < 2e-10
    # (exam-2): u = (2/pi) (1-|x|^2)^{1/2}; the FM error is O(h) in L2
    err = o.lumped_l2(ref.verts, ref.simp, u - o.ball_exact(ref.verts, 0.5))
    assert err < 0.02, err


def test_3d_afd_ragged_129():
    # n = 129 (P = 256, a ragged tail in every axis); A_FD v against the
    # oracle's zero-padded FFT convolution built from the same coefficients
    # (T itself is pinned at small sizes above)
    v, s = mg.ball_shell_mesh(shells=6, seed=mg.seed_for(3, 3))
    lo, hi, h = mg.grid_box(3, 129)
    gp = _gpu(v, s, 1.3, h, lo, hi, filon_M=2 ** 11)
    T = gp.coefficients().reshape((129,) * 3)
    lam = o.symbol(T, 256)
    x = mg.random_vector(129 ** 3, 51)
    want = o.afd_apply_fft(lam, x.reshape((129,) * 3), 256).ravel()
    got64 = gp.afd_apply(torch.tensor(x, device="cuda")).cpu().numpy()
    got32 = gp.afd_apply(torch.tensor(x, device="cuda", dtype=torch.float32)).cpu().numpy().astype(np.float64)
    assert _rel(got64, want) < 1e-12
    assert _rel(got32, want) < 1e-5
    gp.close()


@pytest.fixture(scope="module")
def afd256():
    # n = 256 (P = 512): the size at which the axis-1/axis-2 kernels have
    # alternative launch shapes; one oracle product serves every shape
    import os
    v, s = mg.ball_shell_mesh(shells=6, seed=mg.seed_for(3, 4))
    lo, hi, h = mg.grid_box(3, 256)
    gp = _gpu(v, s, 1.5, h, lo, hi)
    T = gp.coefficients().reshape((256,) * 3)
    lam = o.symbol(T, 512)
    x = mg.random_vector(256 ** 3, 53)
    want = o.afd_apply_fft(lam, x.reshape((256,) * 3), 512, workers=os.cpu_count()).ravel()
    yield gp, x, want
    gp.close()


@pytest.mark.parametrize("col_elems,row_elems", [(8, 8), (16, 8), (32, 8), (8, 16), (16, 16), (32, 16)])
def test_3d_afd_every_middle_shape(afd256, col_elems, row_elems):
    # axis-2 columns with 8/16/32 elements per thread (32 in FP32 only) and
    # axis-1 planes with 8/16, against the oracle's FFT convolution
    gp, x, want = afd256
    gp.set_launch_shapes(col_elems=col_elems, row_elems=row_elems)
    try:
        xd = torch.tensor(x, device="cuda")
        got64 = gp.afd_apply(xd).cpu().numpy()
        got32 = gp.afd_apply(xd.float()).cpu().numpy().astype(np.float64)
        assert _rel(got64, want) < 1e-12
        assert _rel(got32, want) < 1e-5
    finally:
        gp.set_launch_shapes()


def test_3d_products_do_not_depend_on_plane_chunks(built):
    # the axis-1/axis-2 stage over chunks of 5 planes (13 chunks at P = 128)
    # gives the same products, bit for bit, as over all planes at once
    gp, ref = built("ball37_ragged")
    d, v, s, n, alpha, M = _case("ball37_ragged")
    lo, hi, h = mg.grid_box(d, n)
    gc = _gpu(v, s, alpha, h, lo, hi, filon_M=M, chunk_planes=5)
    u = torch.tensor(mg.random_vector(len(v), 52), device="cuda")
    for dt in (torch.float64, torch.float32):
        assert torch.equal(gc.apply(u.to(dt)), gp.apply(u.to(dt)))
    gc.close()
