"""The one-warp-per-1024-point-FFT 2D product (circulant length 2048).

Grids of 514 to 1024 nodes per axis take these kernels in FP32 with the
default launch shapes.  Checked against the FP64 oracle (Section 3.2,
(GoFD-2); Section 2.2, (AU-1)) at the FP32 bar, against the general kernels,
batched against single products bit for bit, on ragged grids and on meshes
whose grid lines cross the domain in more than two runs.
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


def _three_disks():
    # three disjoint disks on the x axis: grid lines through all three cross
    # the domain in three runs
    offset = 0
    vs, ss = [], []
    for i, cx in enumerate((-0.62, 0.0, 0.62)):
        v, s = mg.disk_ring_mesh(rings=10, seed=mg.seed_for(1, 40 + i))
        vs.append(0.3 * v + np.array([cx, 0.05 * i]))
        ss.append(s + offset)
        offset += len(v)
    return np.vstack(vs), np.vstack(ss).astype(np.int32)


def _case(name):
    if name == "disk600":
        v, s = mg.disk_ring_mesh(rings=20, seed=mg.seed_for(1, 30))
        return v, s, 600, 1.2
    if name == "lshape777":
        v, s = mg.lshape_mesh(spacing=0.03, seed=mg.seed_for(2, 30))
        return v, s, 777, 0.7
    if name == "three_disks520":
        v, s = _three_disks()
        return v, s, 520, 1.0
    if name == "disk1024":
        v, s = mg.disk_ring_mesh(rings=25, seed=mg.seed_for(1, 31))
        return v, s, 1024, 1.6
    raise KeyError(name)


@pytest.mark.parametrize("name", ["disk600", "lshape777", "three_disks520", "disk1024"])
def test_warp_path_matches_oracle_and_general_kernels(name):
    from paper_2307_14437_gb300 import Problem
    v, s, n, alpha = _case(name)
    lo, hi, h = mg.grid_box(2, n)
    gp = Problem(v, s, alpha, h, lo, hi)
    info = gp.info()
    assert gp.P == 2048 and info["warp_fft_path"] == 1
    ref = o.build(2, v, s, alpha, h, lo, hi, exact_weights=False, pruned=True, M=info["filon_M"])
    if name == "three_disks520":
        # some grid line crosses the mesh in three separate runs
        own = ref.owner.reshape(n, n) >= 0
        runs = (np.diff(own.astype(np.int8), axis=1) == 1).sum(axis=1) + own[:, 0]
        assert runs.max() >= 3
    u = mg.random_vector(len(v), 71)
    want = o.stiffness_apply(ref, u)
    ud = torch.tensor(u, device="cuda", dtype=torch.float32)
    y32 = gp.apply(ud).cpu().numpy().astype(np.float64)
    assert _rel(y32, want) < 1e-5
    # the grid convolution of a grid vector (general kernels) against the
    # oracle's FFT convolution
    xg = mg.random_vector(gp.n_grid, 72)
    wg = gp.afd_apply(torch.tensor(xg, device="cuda", dtype=torch.float32)).cpu().numpy().astype(np.float64)
    assert _rel(wg, o.afd_apply(ref, xg)) < 1e-5
    # the general kernels (explicit launch shapes) give the same product
    gp.set_launch_shapes(col_elems=32)
    assert gp.info()["warp_fft_path"] == 0
    y32g = gp.apply(ud).cpu().numpy().astype(np.float64)
    assert _rel(y32g, want) < 1e-5
    gp.set_launch_shapes()
    assert gp.info()["warp_fft_path"] == 1
    # repeatable, and a batch of columns equals the single products bit for bit
    assert np.array_equal(gp.apply(ud).cpu().numpy(), y32.astype(np.float32))
    ii, _ = gp.export_vertex_data()
    iv = np.nonzero(ii >= 0)[0]
    X = np.zeros((3, len(iv) + 1))
    for c in range(3):
        X[c, :len(iv)] = mg.random_vector(len(v), 80 + c)[iv]
    Xd = torch.tensor(X, device="cuda", dtype=torch.float32)
    Yd = torch.empty_like(Xd)
    gp.apply_interior_batch(Xd, Yd)
    for c in range(3):
        y1 = torch.empty(len(iv), device="cuda", dtype=torch.float32)
        gp.apply_interior(Xd[c].contiguous(), y1)
        assert torch.equal(Yd[c, :len(iv)], y1), c
    # mixed-precision solve through the new product reaches the FP64 tolerance
    f = torch.ones(gp.n_grid, dtype=torch.float64, device="cuda")
    uu, sinfo = gp.solve(f, mode="mixed", tol=1e-8)
    b = o.rhs_grid(ref, np.ones(ref.n_grid))
    assert np.linalg.norm(b - o.stiffness_apply(ref, uu.cpu().numpy())) <= 1.05e-8 * np.linalg.norm(b)
    gp.close()
