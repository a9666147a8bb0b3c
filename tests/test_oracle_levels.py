"""Pins for the oracle's decomposition levels (Sec. 2, 2.1).

* Corner / edge counts of grid decompositions follow the closed forms
  (n_s - 1)^2 corners and 2 n_s (n_s - 1) edges of H/h - 1 nodes; the
  32x32 mesh in 4x4 substructures gives 9 + 24 = 33 coarse DOFs with edge
  averages (Table 1 "c+e" structure); level 2 of a 16x16 grid grouped 4x4
  has (4-1)^2 = 9 corners.
* The stiffness weights form a partition of unity, sum_i R_i^T D_i R_i = I,
  and equal 1/2 on edges and 1/4 at cross points for k = 1.
* The substructure matrices assemble to the global matrix.
"""
import numpy as np

from oracle import bddc, levels
from paper_0911_5730_gb300 import inputs


def test_grid_counts():
    for nx, sub in [(32, 8), (24, 4), (48, 16)]:
        e2s, ns = inputs.grid_decomposition(nx, sub)
        lv = levels.level_one(nx, np.ones(nx * nx), e2s, ns)
        side = nx // sub
        assert len(lv.corners) == (side - 1) ** 2
        assert len(lv.edges) == 2 * side * (side - 1)
        assert all(len(d) == sub - 1 for _, d in lv.edges)
        assert all(len(p) == 2 for p, _ in lv.edges)


def test_unit_config_coarse_count():
    wl = inputs.two_level_unit()
    lv = levels.level_one(wl.nx, wl.k, wl.elem_to_sub, wl.n_sub1)
    assert len(bddc.coarse_dofs_for(lv, "corners+edges")) == 33


def test_partition_of_unity_and_unit_weights():
    nx, sub = 16, 4
    e2s, ns = inputs.grid_decomposition(nx, sub)
    k = inputs.block_log_uniform_coefficient(nx, 4, 7)
    lv = levels.level_one(nx, k, e2s, ns)
    tot = np.zeros(lv.n)
    for s in range(ns):
        np.add.at(tot, lv.sub_dofs[s], lv.D[s])
    assert np.allclose(tot, 1.0, atol=1e-14)
    lv1 = levels.level_one(nx, np.ones(nx * nx), e2s, ns)
    for s in range(ns):
        m = lv1.mult[lv1.sub_dofs[s]]
        assert np.allclose(lv1.D[s], 1.0 / m)


def test_substructures_assemble_to_global():
    nx, sub = 12, 4
    e2s, ns = inputs.grid_decomposition(nx, sub)
    k = inputs.channel_coefficient(nx, 3)
    lv = levels.level_one(nx, k, e2s, ns)
    A = np.zeros((lv.n, lv.n))
    for s in range(ns):
        d = lv.sub_dofs[s]
        A[np.ix_(d, d)] += lv.A_loc[s]
    assert np.allclose(A, lv.A.toarray(), atol=1e-12 * np.abs(A).max())


def test_level_two_counts():
    nx, sub, group = 64, 4, 4           # 16x16 level-1 substructures, 4x4 level-2
    e2s, ns = inputs.grid_decomposition(nx, sub)
    s2, n2 = inputs.grid_grouping(nx // sub, group)
    H = bddc.build(nx, np.ones(nx * nx), e2s, ns, 3, "corners", sub1_to_sub2=s2, nsub2=n2)
    lv2 = H.bl[1].lv
    assert H.bl[0].nc == (nx // sub - 1) ** 2
    assert len(lv2.corners) == (nx // sub // group - 1) ** 2
    # each level-2 edge holds the group - 1 level-1 corners strictly inside it
    assert all(len(d) == group - 1 for _, d in lv2.edges)
    assert len(lv2.edges) == 2 * 4 * 3
