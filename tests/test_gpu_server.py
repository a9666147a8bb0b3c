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
    continuous batching with the staged batch kernels, one served by the
    streaming batch kernels (irregular cells of about 1000 DOFs), both with
    batch_width 32, and one whose FP64 blocks (b about 74) exceed the
    streaming kernel's shared memory, served by the worker threads.  Every
    result matches the solo solve by the same kernels (for the streaming
    problem a two-column batch of the request and a zero column, for the
    others the solve of the request alone): both meet their tolerance on the
    true residual, and the FP64 solutions agree within 1e-10.  The lanes of a
    batch are its columns, so the order of a column's dot products depends on
    the batch width and the last bits of a solve on what it was batched with;
    where that moves the stopping test across its threshold by one iteration
    the two solutions are two converged solves one step apart, and agree
    within 100 x rtol."""
    import time
    staged_wl = inputs.two_level_channels(nx=64, sub=16)
    stream_wl = inputs.three_level_voronoi(nx=128, cells=4, group=2, levels=2)
    generic_wl = inputs.three_level_voronoi(nx=160, cells=2, group=1, levels=2)
    Ps = lib.Problem.from_workload(staged_wl)
    Pt = lib.Problem.from_workload(stream_wl)
    Pg = lib.Problem.from_workload(generic_wl)
    width = {id(Ps): 32, id(Pt): 32, id(Pg): 1}
    srv = lib.Server(hbm_budget=0, max_slots=3)
    rng = np.random.default_rng(11)
    sent = []
    for wave in range(4):
        for r in range(12):
            rtol = 1e-8 if r % 3 else 1e-10
            for P, wl in ((Ps, staged_wl), (Pt, stream_wl)) if r % 2 else ((Ps, staged_wl),):
                b = rng.standard_normal(wl.n_dof)
                sent.append((P, b, rtol, srv.submit(P, b, rtol=rtol)))
        b = rng.standard_normal(generic_wl.n_dof)
        sent.append((Pg, b, 1e-8, srv.submit(Pg, b, rtol=1e-8)))
        time.sleep(0.002)
    for P, b, rtol, t in sent:
        x, infos, lat = srv.wait(t)
        assert lat > 0 and infos[0]["status"] == 0, (rtol, lat, infos[0])
        assert infos[0]["batch_width"] == width[id(P)]
        if P is Pt:
            pair = np.zeros((2, b.size))
            pair[0] = b
            xs, info = P.solve(torch.tensor(pair, device="cuda"), rtol=rtol)
            assert info[0]["batch_width"] == 2
            xs = xs[0]
        else:
            xs, info = P.solve(torch.tensor(b, device="cuda"), rtol=rtol)
        name = "staged" if P is Ps else ("stream" if P is Pt else "generic")
        d_it = abs(infos[0]["iters"] - info[0]["iters"])
        assert d_it <= 1, (name, rtol, infos[0], info[0])
        xs = xs.cpu().numpy()
        tol = 1e-10 if d_it == 0 else 100 * rtol
        assert np.linalg.norm(x - xs) <= tol * np.linalg.norm(xs), (name, rtol, d_it)
        assert infos[0]["relres_true"] <= rtol and info[0]["relres_true"] <= rtol
    srv.close()
    Ps.close()
    Pt.close()
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
