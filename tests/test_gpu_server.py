"""The serving loop: requests for several resident problems, each with 1-4
right-hand sides, submitted while others run.  Every result must equal the
problem's solo solve within the FP64 tolerance (1e-10 relative: each RHS is
an independent PCG with the same operators), latencies are reported, a
request larger than the HBM budget is refused with BDDC_E_BUSY, and a
bounded wait returns BDDC_E_TIMEOUT for a request that cannot finish yet."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_0911_5730_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc
    return bddc


def test_results_same_alone_and_in_the_mix(lib):
    wls = [inputs.two_level_channels(nx=64, sub=16), inputs.two_level_unit(),
           inputs.three_level_blocks(nx=64, sub=8, group=4, tau=10.0)]
    probs = [lib.Problem.from_workload(w) for w in wls]
    rng = np.random.default_rng(5)
    reqs = []
    for k in range(9):
        j = k % 3
        nrhs = 1 + (k % 4)
        b = rng.standard_normal((nrhs, wls[j].n_dof)) if nrhs > 1 else rng.standard_normal(wls[j].n_dof)
        reqs.append((j, b))
    srv = lib.Server(hbm_budget=0, max_slots=3)
    tickets = [srv.submit(probs[j], b, rtol=1e-8) for j, b in reqs]
    outs = [srv.wait(t) for t in tickets]
    for (j, b), (x, infos, lat) in zip(reqs, outs):
        assert lat > 0
        bb = np.atleast_2d(b)
        xx = np.atleast_2d(x)
        for r in range(bb.shape[0]):
            xs, info = probs[j].solve(torch.tensor(bb[r], device="cuda"), rtol=1e-8)
            assert infos[r]["status"] == 0 and infos[r]["iters"] == info[0]["iters"]
            xs = xs.cpu().numpy()
            assert np.linalg.norm(xx[r] - xs) <= 1e-10 * np.linalg.norm(xs)
    srv.close()
    for p in probs:
        p.close()


def test_budget_and_timeout(lib):
    wl = inputs.two_level_channels(nx=64, sub=16)
    P = lib.Problem.from_workload(wl)
    srv = lib.Server(hbm_budget=4096, max_slots=1)
    with pytest.raises(lib.BDDCError) as e:
        srv.submit(P, np.ones(wl.n_dof))
    assert e.value.code == -7
    srv.close()
    srv = lib.Server(hbm_budget=0, max_slots=1)
    big = inputs.normal_rhs(wl.n_dof, 3, 16)
    t = srv.submit(P, big, rtol=1e-12, maxit=500)
    with pytest.raises(lib.BDDCError) as e:
        srv.wait(t, timeout_ms=0)
    assert e.value.code == -5
    srv.close()
    P.close()


def test_continuous_batching_waves(lib):
    """Requests arrive in waves while earlier ones iterate: more right-hand
    sides than the 32 slots, with different tolerances, on a problem served by
    continuous batching (batch_width 32) beside one that needs the generic
    kernels (served by the worker threads).  Every result equals the solo
    solve: same iteration count, FP64 solution within 1e-10."""
    import time
    batch_wl = inputs.two_level_channels(nx=64, sub=16)
    generic_wl = inputs.three_level_voronoi(nx=128, cells=4, group=2, levels=2)
    Pb = lib.Problem.from_workload(batch_wl)
    Pg = lib.Problem.from_workload(generic_wl)
    srv = lib.Server(hbm_budget=0, max_slots=2)
    rng = np.random.default_rng(11)
    sent = []
    for wave in range(4):
        for r in range(12):
            rtol = 1e-8 if r % 3 else 1e-10
            b = rng.standard_normal(batch_wl.n_dof)
            sent.append((Pb, b, rtol, srv.submit(Pb, b, rtol=rtol)))
        b = rng.standard_normal(generic_wl.n_dof)
        sent.append((Pg, b, 1e-8, srv.submit(Pg, b, rtol=1e-8)))
        time.sleep(0.002)
    for P, b, rtol, t in sent:
        x, infos, lat = srv.wait(t)
        assert lat > 0 and infos[0]["status"] == 0
        assert infos[0]["batch_width"] == (32 if P is Pb else 1)
        xs, info = P.solve(torch.tensor(b, device="cuda"), rtol=rtol)
        assert infos[0]["iters"] == info[0]["iters"]
        xs = xs.cpu().numpy()
        assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
        assert infos[0]["relres_true"] <= rtol
    srv.close()
    Pb.close()
    Pg.close()


def test_continuous_batching_mixed_precision(lib):
    wl = inputs.two_level_channels(nx=96, sub=16, tau=3.0)
    P = lib.Problem.from_workload(wl)
    P.set_precision("fp32")
    srv = lib.Server(hbm_budget=0, max_slots=1)
    B = inputs.normal_rhs(wl.n_dof, 13, 40)
    tickets = [srv.submit(P, B[i:i + 1 + i % 3]) for i in range(0, 36, 3)]
    for t in tickets:
        x, infos, lat = srv.wait(t)
        for i in infos:
            assert i["status"] == 0 and i["relres_true"] <= 1e-8 and i["batch_width"] == 32
    srv.close()
    P.close()
