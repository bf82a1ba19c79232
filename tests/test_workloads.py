"""Host-side logic of the benchmark workloads (no GPU): the batched
workload's instance rule, its grid rule and the mesh-height helper behind it."""
import collections

import numpy as np

import bench
import meshgen as mg
from oracle import gofd as o


def test_batch_instances_follow_the_instance_rule():
    # 16 ring disks + 16 L-shapes, vertex counts log-uniform in [5e3, 1.5e5];
    # mesh i at alpha (0.5, 1, 1.5)[i mod 3], the first 8 of each kind also at
    # the next alpha: 48 instances on 32 meshes
    specs = mg.batch_instances()
    assert len(specs) == 48
    meshes = collections.Counter((sp["kind"], sp["mesh"]) for sp in specs)
    assert len(meshes) == 32
    assert sum(1 for k in meshes if k[0] == "disk") == 16
    for (kind, i), reps in meshes.items():
        assert reps == (2 if i < 8 else 1)
        alphas = sorted(sp["alpha"] for sp in specs if (sp["kind"], sp["mesh"]) == (kind, i))
        want = sorted(mg.BATCH_ALPHAS[(i + r) % 3] for r in range(reps))
        assert alphas == want
    nv = [sp["target_vertices"] for sp in specs]
    assert min(nv) >= 5000 and max(nv) <= 150000
    assert specs == mg.batch_instances()          # deterministic


def test_min_height_equals_the_oracle_element_heights():
    for v, s in (mg.disk_ring_mesh(rings=6, seed=3), mg.lshape_mesh(spacing=0.08, seed=4)):
        assert abs(bench._min_height(v, s) - float(np.min(o.element_heights(v, s)))) <= 1e-14


def test_batch_grid_rule():
    # smallest n in {256, ..., 2048} with h = 2/(n-1) <= a_h / 2, clipped to 2048
    assert bench.batch_grid_nodes(1.0) == 256
    assert bench.batch_grid_nodes(4.0 / 255) == 256
    assert bench.batch_grid_nodes(4.0 / 255 * 0.999) == 512
    assert bench.batch_grid_nodes(4.0 / 1023) == 1024
    assert bench.batch_grid_nodes(1e-6) == 2048
    # on the 48 instances: 6 at 512^2, 20 at 1024^2, 22 at 2048^2
    n_of = {}
    counts = collections.Counter()
    for sp in mg.batch_instances():
        key = (sp["kind"], sp["mesh"])
        if key not in n_of:
            v, s = mg.batch_mesh(sp)
            n_of[key] = bench.batch_grid_nodes(bench._min_height(v, s))
        counts[n_of[key]] += 1
    assert dict(counts) == {512: 6, 1024: 20, 2048: 22}
