"""Parity on meshes with mixed simplex orientations (through the C ABI).

gofd_build accepts simplices of either orientation.  Here a seeded half of the
simplices of each mesh has its first two local vertices swapped, which makes
them negatively oriented and changes the ELL slot order of every grid node
they own.  Owner and ELL indices must still equal the oracle's bit for bit,
weights within their FP64 evaluation error, D_h and the FP64 product within
1e-13 / 1e-12, the FP32 product within 1e-5 (Section 3.1, (IhFD-1); Lemma 3.4).
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


def _case(name):
    if name == "disk37":
        v, s = mg.disk_ring_mesh(rings=9, seed=mg.seed_for(1, 2))
        return 2, v, s, 37, 0.5, 2 ** 10
    if name == "lshape33":
        v, s = mg.lshape_mesh(spacing=0.15, seed=mg.seed_for(2, 1))
        return 2, v, s, 33, 1.5, 2 ** 10
    if name == "aligned2":
        lo, hi, h = mg.grid_box(2, 11)
        v, s = mg.grid_aligned_mesh(2, -1.0, h, 6, origin_cells=2)
        return 2, v, s, 11, 1.2, 2 ** 10
    if name == "ball17":
        v, s = mg.ball_shell_mesh(shells=4, seed=mg.seed_for(3, 1))
        return 3, v, s, 17, 1.5, 2 ** 8
    if name == "aligned3":
        lo, hi, h = mg.grid_box(3, 7)
        v, s = mg.grid_aligned_mesh(3, -1.0, h, 4, origin_cells=1)
        return 3, v, s, 7, 1.0, 2 ** 8
    raise KeyError(name)


@pytest.mark.parametrize("name", ["disk37", "lshape33", "aligned2", "ball17", "aligned3"])
def test_mixed_orientation_parity(name):
    from paper_2307_14437_gb300 import Problem
    d, v, s0, n, alpha, M = _case(name)
    s = mg.flip_orientations(s0, seed=mg.seed_for(0, 77))
    flipped = np.any(s != s0, axis=1)
    assert 0.3 < flipped.mean() < 0.7
    lo, hi, h = mg.grid_box(d, n)
    ref = o.build(d, v, s, alpha, h, lo, hi, M=M, pruned=d == 3)
    gp = Problem(v, s, alpha, h, lo, hi, filon_M=M)
    owner, idx, w = gp.export_transfer()
    assert np.array_equal(owner, ref.owner.astype(np.int32))
    assert np.array_equal(idx, ref.ell_idx.astype(np.int32))
    assert np.abs(w - ref.ell_w).max() < 1e-13
    # the flipped elements do own grid nodes, so their slot order is exercised
    assert flipped[owner[owner >= 0]].any() and (~flipped[owner[owner >= 0]]).any()
    ii, cs = gp.export_vertex_data()
    assert np.array_equal(ii >= 0, np.isin(np.arange(len(v)), ref.interior))
    assert np.abs(cs[ref.interior] - ref.Dh[ref.interior]).max() < 1e-13 * ref.Dh.max()
    u = mg.random_vector(len(v), 61)
    want = o.stiffness_apply(ref, u, method="direct")
    y64 = gp.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    y32 = gp.apply(torch.tensor(u, device="cuda", dtype=torch.float32)).cpu().numpy().astype(np.float64)
    assert _rel(y64, want) < 1e-12
    assert _rel(y32, want) < 1e-5
    # the same mesh with positive orientations gives the same operator
    gq = Problem(v, s0, alpha, h, lo, hi, filon_M=M)
    y0 = gq.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    assert _rel(y64, y0) < 1e-13
    gq.close()
    gp.close()
