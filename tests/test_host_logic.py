"""Host-side logic of the C++ library against the oracle (no GPU needed).

bddc_inspect runs only the level-1 bookkeeping of bddc_setup: interface,
corners (DOFs in >= 3 substructures), edges (connected chains of the other
interface DOFs shared by one pair, numbered by pair then lowest DOF) and the
interior block size.  The oracle classifies the same decompositions in
Python; both must agree exactly, including on irregular partitions with
several chains between one pair.
"""
import numpy as np
import pytest

from oracle import levels
from paper_0911_5730_gb300 import inputs


@pytest.fixture(scope="module")
def bddc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc as b
    return b


def _nearest_seed_partition(nx, nseeds, seed):
    rng = np.random.default_rng(seed)
    seeds = rng.uniform(0, nx, size=(nseeds, 2))
    ej, ei = np.divmod(np.arange(nx * nx), nx)
    c = np.stack([ei + 0.5, ej + 0.5], axis=1)
    d = ((c[:, None, :] - seeds[None, :, :]) ** 2).sum(-1)
    lab = d.argmin(1)
    used = np.unique(lab)
    remap = -np.ones(nseeds, int)
    remap[used] = np.arange(len(used))
    return remap[lab].astype(np.int32), len(used)


CASES = [("grid32_8",) + inputs.grid_decomposition(32, 8) + (32,),
         ("grid48_16",) + inputs.grid_decomposition(48, 16) + (48,),
         ("grid24_4",) + inputs.grid_decomposition(24, 4) + (24,)]
for sd in (1, 2, 3):
    e2s, ns = _nearest_seed_partition(24, 7, sd)
    CASES.append(("seeds24_%d" % sd, e2s, ns, 24))
for nx, c in ((64, 4), (128, 8)):          # config 4's Voronoi cells, small
    e2s, ns, _, _ = inputs.voronoi_decomposition(nx, c, 4001)
    CASES.append(("voronoi%d_%d" % (nx, c), e2s, ns, nx))


@pytest.mark.parametrize("name,e2s,ns,nx", CASES, ids=[c[0] for c in CASES])
def test_classification_matches_oracle(bddc, name, e2s, ns, nx):
    lv = levels.level_one(nx, np.ones(nx * nx), e2s, ns)
    got = bddc.inspect(nx, e2s, ns)
    assert got["n_corners"] == len(lv.corners)
    assert got["n_edges"] == len(lv.edges)
    assert [tuple(p) for p in got["edge_pairs"]] == [tuple(p) for p, _ in lv.edges]
    assert list(got["edge_len"]) == [len(d) for _, d in lv.edges]


def test_block_size_power_of_two_for_grids(bddc):
    for nx, sub, bp in [(512, 16, 16), (64, 8, 8), (32, 8, 8)]:
        e2s, ns = inputs.grid_decomposition(nx, sub)
        assert bddc.inspect(nx, e2s, ns)["block_size"] == bp


def _pieces(lab):
    """Connected pieces (across element edges) of every label, by flood fill."""
    nx = lab.shape[0]
    seen = np.zeros_like(lab, dtype=bool)
    count = {}
    for j0 in range(nx):
        for i0 in range(nx):
            if seen[j0, i0]:
                continue
            c = lab[j0, i0]
            count[c] = count.get(c, 0) + 1
            stack = [(j0, i0)]
            seen[j0, i0] = True
            while stack:
                j, i = stack.pop()
                for jj, ii in ((j, i + 1), (j, i - 1), (j + 1, i), (j - 1, i)):
                    if 0 <= jj < nx and 0 <= ii < nx and not seen[jj, ii] and lab[jj, ii] == c:
                        seen[jj, ii] = True
                        stack.append((jj, ii))
    return count


@pytest.mark.parametrize("nx,cells,group", [(64, 4, 2), (128, 8, 4), (256, 16, 8)])
def test_voronoi_partition_properties(nx, cells, group):
    e2s, ns, s2, n2 = inputs.voronoi_decomposition(nx, cells, 4001, group=group)
    again = inputs.voronoi_decomposition(nx, cells, 4001, group=group)
    assert np.array_equal(e2s, again[0]) and np.array_equal(s2, again[2])     # seeded
    assert ns == cells * cells and set(np.unique(e2s)) == set(range(ns))
    pieces = _pieces(e2s.reshape(nx, nx))
    assert all(v == 1 for v in pieces.values())                                # every cell connected
    assert n2 == (cells // group) ** 2 and set(np.unique(s2)) == set(range(n2))
    assert all(np.sum(s2 == g) == group * group for g in range(n2))
    sizes = np.bincount(e2s)
    w2 = (nx // cells) ** 2
    assert sizes.min() >= 0.5 * w2 and sizes.max() <= 1.6 * w2



def test_serving_mix_arrivals():
    """The mixed serving stream's arrivals (config 5): per problem a seeded
    Poisson stream of 1-64 right-hand sides per request at its share of the
    load, the same for the same seed, inside the window, and at least one
    request for a problem too slow to draw one."""
    pytest.importorskip("torch")
    from paper_0911_5730_gb300 import serve_mix
    cap = {"fast": 2000.0, "slow": 1e-3}
    a = serve_mix.arrivals(["fast", "slow"], cap, 0.8, 3.0, 5001)
    b = serve_mix.arrivals(["fast", "slow"], cap, 0.8, 3.0, 5001)
    assert a == b
    assert len(a["slow"]) == 1
    for k, ev in a.items():
        ts = [t for t, _, _ in ev]
        assert ts == sorted(ts) or k == "slow"
        assert all(0.0 <= t < 3.0 for t in ts)
        assert all(1 <= m <= 64 for _, m, _ in ev)
    # the fast stream offers about load / problems of its rate over the window
    offered = sum(m for _, m, _ in a["fast"]) / 3.0
    assert 0.5 * 800.0 < offered < 1.5 * 800.0


def test_serving_mix_bookkeeping_with_a_fake_server(monkeypatch):
    """serve_mix.serve end to end on the CPU against a stand-in server that
    completes every request at once: every submitted right-hand side is
    counted once per problem, none is reported failed, and every problem
    (also one too slow to draw a request) gets latencies."""
    pytest.importorskip("torch")
    from paper_0911_5730_gb300 import serve_mix

    class FakeServer:
        def __init__(self, hbm_budget=0, max_slots=1):
            self.n = 0

        def submit(self, P, b, rtol=1e-8):
            self.n += 1
            return (P, 1 if np.ndim(b) == 1 else len(b))

        def wait(self, t):
            _, m = t
            return None, [{"status": 0, "iters": 1, "relres_true": 1e-9}] * m, 0.5

        def close(self):
            pass

    monkeypatch.setattr(serve_mix.bddc, "Server", FakeServer)

    class W:
        n_dof = 16

    keys = ["channels", "blocks", "voronoi"]
    cap = {"channels": 3000.0, "blocks": 600.0, "voronoi": 50.0}
    out, _ = serve_mix.serve({k: k for k in keys}, {k: W() for k in keys}, 0.8, 0.3, 7, 0, cap=cap)
    plans = serve_mix.arrivals(keys, cap, 0.8, 0.3, 7)
    for k in keys:
        name = serve_mix.PROBLEMS[k][0]
        assert out[name]["rhs"] == sum(m for _, m, _ in plans[k])
        assert out[name]["requests"] == len(plans[k]) >= 1
        assert out[name]["latency_ms"]["p50"] == 0.5
    assert out["all"]["failed_rhs"] == 0
