"""Host-side classification of the elasticity problem (bddc_inspect; no GPU).

At the paper's size (768 x 768 bilinear elements, 48 x 48 substructures,
H/h = 16) the setup's own classification gives the constraint counts of
Table 1: 4794 corner DOFs and 13818 with one average per edge and component,
counted on the whole node set as the paper's DOF count 1 182 722 = 2 * 769^2
does; with the side x = 0 clamped the 47 vertices on it drop out (4700,
13724).  The oracle reproduces the same counts from its own code
(tests/test_oracle_elasticity.py); here they are checked against the paper's
numbers and the closed forms.  Also: the setup refuses the unclamped
(singular) mesh and bad Lame parameters before any device work, and the
jagged-edge generators (which stand in for the paper's missing figure) only
trade elements between the pair, keep both substructures connected and the
sizes equal, and add no corner.
"""
import numpy as np
import pytest

from paper_0911_5730_gb300 import inputs


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc
    return bddc


def test_paper_counts_at_full_size(lib):
    e2s, ns = inputs.grid_decomposition(768, 16)
    r = lib.inspect(768, e2s, ns, problem="elasticity", clamp="none")
    assert r["n_corners"] == 4794                               # Table 1, c
    assert r["n_corners"] + 2 * r["n_edges"] == 13818           # Table 1, c+e
    assert r["n_edges"] == 2 * 48 * 47 and set(r["edge_len"]) == {30}
    r = lib.inspect(768, e2s, ns, problem="elasticity")
    assert r["n_corners"] == 2 * (49 ** 2 - 4 - 47) == 4700
    assert r["n_corners"] + 2 * r["n_edges"] == 13724
    assert r["block_size"] == 32


def test_jagged_edge(lib):
    wl = inputs.elasticity(nx=768)
    r = lib.inspect(768, wl.elem_to_sub, wl.n_sub1, problem="elasticity")
    assert r["n_corners"] == 4700 and r["n_edges"] == 2 * 48 * 47
    pairs = [tuple(p) for p in r["edge_pairs"]]
    lens = dict(zip(pairs, r["edge_len"]))
    assert lens[(1, 49)] > 30                                   # the comb is longer
    assert sorted(set(r["edge_len"]))[:1] == [30]


def test_setup_refuses_before_device_work(lib):
    wl = inputs.elasticity(nx=16, sub=4, levels=2, constraints="corners", jagged=False)
    with pytest.raises(lib.BDDCError) as e:
        lib.Problem(16, wl.k, wl.elem_to_sub, wl.n_sub1, problem="elasticity", lame=(1.0, 0.0), stream=0)
    assert e.value.code == -1
    with pytest.raises(lib.BDDCError) as e:
        lib.Problem(16, wl.k, wl.elem_to_sub, wl.n_sub1, problem="elasticity", lame=(-1.0, 2.0), stream=0)
    assert e.value.code == -1


def _connected(nx, e2s, s):
    from collections import deque
    lab = e2s.reshape(nx, nx)
    cells = list(zip(*np.nonzero(lab == s)))
    seen = {cells[0]}
    q = deque([cells[0]])
    while q:
        j, i = q.popleft()
        for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)):
            a, b = j + dj, i + di
            if 0 <= a < nx and 0 <= b < nx and lab[a, b] == s and (a, b) not in seen:
                seen.add((a, b))
                q.append((a, b))
    return len(seen) == len(cells)


@pytest.mark.parametrize("nx,sub", [(64, 16), (32, 8), (768, 16)])
def test_jagged_decomposition_is_a_valid_comb(lib, nx, sub):
    e2s, ns = inputs.jagged_grid_decomposition(nx, sub, (1, 0))
    g, _ = inputs.grid_decomposition(nx, sub)
    moved = np.nonzero(e2s != g)[0]
    assert set(np.unique(g[moved])) <= {1, 1 + nx // sub}       # only the pair trades elements
    assert np.all(np.bincount(e2s, minlength=ns) == sub * sub)   # as many teeth each way
    for s in (1, 1 + nx // sub):
        assert _connected(nx, e2s, s)
    r = lib.inspect(nx, e2s, ns, problem="elasticity")
    rg = lib.inspect(nx, g, ns, problem="elasticity")
    assert r["n_corners"] == rg["n_corners"] and r["n_edges"] == rg["n_edges"]   # no new corners


def test_jagged_grouping_is_a_valid_comb():
    s2, n2 = inputs.jagged_grid_grouping(48, 16, (1, 0))
    g2, _ = inputs.grid_grouping(48, 16)
    moved = np.nonzero(s2 != g2)[0]
    assert set(np.unique(g2[moved])) <= {1, 4} and len(moved) > 0
    assert np.all(np.bincount(s2, minlength=n2) == 256)
