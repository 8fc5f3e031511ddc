"""Consistency of the seeded input generators (inputs only, no method arithmetic)."""
import numpy as np

import workloads as W


def _areas(prob):
    p = prob.xy[prob.tri]
    return 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                  - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))


def test_structured_mesh_counts_orientation_and_cover():
    xy, tri, dr = W.structured_mesh(5, 4, 0.0, 0.0, 2.0, 1.0)
    assert xy.shape == (20, 2) and tri.shape == (2 * 4 * 3, 3)
    prob = W.transformer_problem(9, 5, 4)
    a = _areas(prob)
    assert (a > 0).all() and abs(a.sum() - 2.0) < 1e-14
    assert dr.sum() == 20 - 2 * 3
    assert set(np.unique(tri)) == set(range(20))


def test_named_workloads():
    p1 = W.config_plain_fp64()
    assert p1.n_nodes == 33 * 33 and p1.n_tri == 2048 and p1.N == 32 and p1.n_free == 961
    p2a, p2b = W.config_mixed(0, n=17, N=8), W.config_mixed(0, n=17, N=8)
    assert p2a.amp[0] == p2b.amp[0] and 20 <= p2a.amp[0] <= 80
    assert W.config_mixed(1, n=17, N=8).amp[0] != p2a.amp[0]
    p3 = W.config_transformer(65, 33, 8)
    assert p3.n_coils == 2 and (p3.coil_of_elem >= 0).sum() > 0 and p3.nonlinear_e.sum() > 0
    # coils sit in the windows, never on iron
    assert not np.any(p3.nonlinear_e.astype(bool) & (p3.coil_of_elem >= 0))
    p4 = W.config_adjoint(0, n=17, N=8)
    s = p4.sigma_e[p4.nonlinear_e.astype(bool)]
    assert (s > 0).all() and abs(np.median(np.log(s)) - np.log(10)) < 0.2
    batch = W.config_batched(0, count=8)
    assert len(batch) == 8 and all(b.N in (64, 128, 256, 512) for b in batch)


def test_delaunay_mesh_is_valid():
    p = W.delaunay_problem(300, 8, seed=1)
    a = _areas(p)
    assert (a > 0).all() and abs(a.sum() - 1.0) < 1e-12
    deg = np.bincount(p.tri.ravel(), minlength=p.n_nodes)
    assert deg.max() >= 8                       # rows wider than the structured stencil
    assert p.nonlinear_e.sum() > 0 and (p.coil_of_elem >= 0).sum() > 0


def _paper_fixture():
    import math
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_transformer_section4.txt")
    labels, materials, out = [], {}, {}
    for line in open(path):
        f = line.split("#")[0].split()
        if not f:
            continue
        if f[0] == "label":
            labels.append((f[1], float(f[2]), float(f[3])))
        elif f[0] == "material":
            val = [1e7 / (4 * math.pi) if v == "nu_air" else (None if v == "-" else float(v)) for v in f[2:]]
            materials[f[1]] = val
        else:
            out[f[0]] = [float(v) for v in f[1:]]
    return labels, materials, out


def _region_of_elements(prob):
    steel = prob.nonlinear_e.astype(bool) & (prob.sigma_e > 0)
    iron = prob.nonlinear_e.astype(bool) & (prob.sigma_e == 0)
    reg = np.full(prob.n_tri, "air", dtype=object)
    reg[steel] = "steel"
    reg[iron] = "iron"
    reg[prob.coil_of_elem == 0] = "winding+"
    reg[prob.coil_of_elem == 1] = "winding-"
    return reg


def test_paper_transformer_matches_section4_figure_and_table():
    """The transformer workload against the paper's printed data: the region
    under each label arrow of the figure, the material constants of the table,
    the cos source of amplitude +-j, the period and the tank outline."""
    import math
    labels, materials, fx = _paper_fixture()
    prob = W.config_paper_transformer("32451", 8)
    mm = 1e-3
    assert np.allclose(prob.xy.max(axis=0), np.array(fx["tank"]) * mm) and np.allclose(prob.xy.min(axis=0), 0.0)
    assert prob.T == fx["period"][0]
    reg = _region_of_elements(prob)
    p = prob.xy[prob.tri]                                        # (n_tri, 3, 2)
    for name, x, y in labels:
        q = np.array([x, y]) * mm
        # triangles that contain the point (barycentric coordinates >= 0)
        a, b, c = p[:, 0], p[:, 1], p[:, 2]
        det = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1])
        l1 = ((q[0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (q[1] - a[:, 1])) / det
        l2 = ((b[:, 0] - a[:, 0]) * (q[1] - a[:, 1]) - (q[0] - a[:, 0]) * (b[:, 1] - a[:, 1])) / det
        inside = (l1 >= -1e-12) & (l2 >= -1e-12) & (l1 + l2 <= 1 + 1e-12)
        assert inside.any()
        assert set(reg[inside]) == {name}, (name, x, y, set(reg[inside]))
    for name, (sigma, a, b, c, d, j) in materials.items():
        e = np.flatnonzero(reg == name)
        assert e.size > 0
        assert np.all(prob.sigma_e[e] == sigma)
        if b is not None:                                        # iron and steel: the exponential law
            assert np.all(prob.nonlinear_e[e] == 1)
            assert np.all(prob.law_abcd[e] == np.array([a, b, c, d]))
        else:                                                    # linear: nu = d
            assert np.all(prob.nonlinear_e[e] == 0) and prob.nu_linear == d
        if j != 0:
            k = int(prob.coil_of_elem[e[0]])
            t = np.linspace(0.0, prob.T, 7)
            src = prob.amp[k] * np.sin(2 * math.pi * t / prob.T + prob.phase[k])
            assert np.allclose(src, j * np.cos(2 * math.pi * t / prob.T), rtol=0, atol=1e-9 * abs(j))
        else:
            assert np.all(prob.coil_of_elem[e] == -1)


def test_paper_transformer_mesh_sizes_match_table1():
    """The structured grids stand in for the paper's meshes: their free-node
    counts are within 2% of Table 1's N_V."""
    _, _, fx = _paper_fixture()
    for size, nv in zip(("8208", "32451"), fx["nv"]):
        assert size == str(int(nv))
        prob = W.config_paper_transformer(size, 4)
        assert abs(prob.n_free - nv) <= 0.02 * nv


def test_workload_recipes():
    """The input recipes as stated for the named workloads: the batched draw
    (grids, steps, J0 ~ U[20, 80], s_sat ~ U[0.5, 2]), the transformer-shaped
    rectangle (sigma 5 on iron, coils J0 = 60 at phases 0 and 2 pi/3, inside
    the windows) and the adjoint case (two in-phase coils, log-normal sigma)."""
    import math
    batch = W.config_batched(0, count=64)
    assert {b.grid[0] for b in batch} <= {65, 129, 257, 513} and len({b.grid[0] for b in batch}) > 1
    assert {b.N for b in batch} <= {64, 128, 256, 512} and len({b.N for b in batch}) > 1
    assert all(20.0 <= b.amp[0] <= 80.0 and 0.5 <= b.s_sat <= 2.0 for b in batch)
    assert [b.amp[0] for b in batch] == [b.amp[0] for b in W.config_batched(0, count=64)]   # seeded
    tr = W.config_transformer(65, 33, 4)
    iron = tr.nonlinear_e.astype(bool)
    assert np.all(tr.sigma_e[iron] == 5.0) and np.all(tr.sigma_e[~iron] == 0.0)
    assert np.allclose(tr.amp, 60.0) and np.allclose(tr.phase, [0.0, 2 * math.pi / 3])
    assert tr.grid[4:] == (2.0, 1.0)
    adj = W.config_adjoint(0, n=33, N=4)
    assert adj.n_coils == 2 and np.allclose(adj.phase, 0.0) and np.allclose(adj.amp, 50.0)
    ls = np.log(adj.sigma_e[adj.nonlinear_e.astype(bool)])
    assert abs(ls.mean() - math.log(10.0)) < 0.05 and abs(ls.std() - 0.3) < 0.05
