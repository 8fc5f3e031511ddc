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
