"""Concurrent serving under load: client threads submit and wait on many
requests (1-40 right-hand sides each) for three resident problems at once --
two-level channels in FP32, three-level blocks switching between FP32 and
FP64 between submits, plane elasticity in FP32 -- under an HBM budget that
makes admission queue, while another thread runs multi-group host solves on a
fourth problem (the helper threads of the batched solve).

Every right-hand side is its own PCG column of the batch kernels, so each
result must meet the tolerance by its true residual and agree with the same
right-hand side solved again on a quiet server (up to the order of the FP64
atomic sums: 1e-7 of the solution's norm, and at most one iteration apart).

The stress functions use only numpy and the ctypes binding, so that a
sanitizer build of the library can run them from a plain Python process."""
import random
import threading
import time

import numpy as np
import pytest

from paper_0911_5730_gb300 import inputs

RTOL = 1e-8
BUDGET = 32 << 20          # bytes of requests in flight (2 n nrhs doubles each)


def make_problems(bddc):
    """The three served problems and the host-solve one (stream 0: no torch)."""
    wls = {
        "channels": (inputs.two_level_channels(nx=128, sub=16), "fp32"),
        "blocks": (inputs.three_level_blocks(nx=128, sub=8, group=4, tau=10.0), "fp64"),
        "elastic": (inputs.elasticity(nx=64, sub=16, levels=2, constraints="adaptive", tau=3.0), "fp32"),
        "host": (inputs.two_level_channels(nx=96, sub=16), "fp32"),
    }
    return {k: (bddc.Problem.from_workload(w, precision=p, stream=0), w) for k, (w, p) in wls.items()}


def stress(bddc, probs, n_clients=6, per_client=10, seed=11):
    """Runs the load; returns the records (name, precision, b, x, infos) and
    the host-solve results."""
    srv = bddc.Server(hbm_budget=BUDGET, max_slots=2)
    records, lock, errors = [], threading.Lock(), []
    prec_lock = threading.Lock()
    served = ["channels", "blocks", "elastic"]

    def client(c):
        try:
            rng = np.random.default_rng(seed + c)
            rnd = random.Random(seed + c)
            mine = []
            for q in range(per_client):
                name = served[(c + q) % 3]
                P, wl = probs[name]
                nrhs = int(rng.integers(1, 41))
                b = rng.standard_normal((nrhs, wl.n_dof)) if nrhs > 1 else rng.standard_normal(wl.n_dof)
                with prec_lock:
                    prec = "fp64"
                    if name == "blocks":
                        prec = "fp32" if (c + q) % 2 else "fp64"
                        P.set_precision(prec)
                    elif name in ("channels", "elastic"):
                        prec = "fp32"
                    t = srv.submit(P, b, rtol=RTOL)
                mine.append((name, prec, b, t))
                time.sleep(rnd.random() * 2e-3)
            rnd.shuffle(mine)
            for name, prec, b, t in mine:
                while True:
                    try:
                        x, infos, _ = srv.wait(t, timeout_ms=rnd.choice([-1, 0, 5]))
                        break
                    except bddc.BDDCError as e:
                        if e.code != -5:          # still running: wait again
                            raise
                with lock:
                    records.append((name, prec, b, x, infos))
        except Exception as e:  # noqa: BLE001 - reported by the caller
            errors.append(repr(e))

    host_out = []

    def host_solves():
        try:
            P, wl = probs["host"]
            rng = np.random.default_rng(seed + 100)
            for _ in range(3):
                b = rng.standard_normal((70, wl.n_dof))
                x, infos = P.solve_host(b, rtol=RTOL)
                host_out.append((b, x, infos))
        except Exception as e:  # noqa: BLE001
            errors.append(repr(e))

    th = [threading.Thread(target=client, args=(c,)) for c in range(n_clients)]
    th.append(threading.Thread(target=host_solves))
    for t in th:
        t.start()
    for t in th:
        t.join()
    srv.close()
    return records, host_out, errors


def quiet(bddc, probs, records):
    """The same right-hand sides, one request at a time on a fresh server."""
    srv = bddc.Server(hbm_budget=0, max_slots=1)
    out = []
    for name, prec, b, _, _ in records:
        P, _ = probs[name]
        P.set_precision(prec)
        out.append(srv.wait(srv.submit(P, b, rtol=RTOL)))
    srv.close()
    return out


def check(records, again, host_out):
    """Failures as strings (empty when everything holds)."""
    bad = []
    for (name, prec, b, x, infos), (x2, infos2, _) in zip(records, again):
        xx, xr = np.atleast_2d(x), np.atleast_2d(x2)
        for j, (i1, i2) in enumerate(zip(infos, infos2)):
            if i1["status"] != 0 or not i1["relres_true"] <= RTOL:
                bad.append("%s %s rhs %d: status %d relres_true %g" % (name, prec, j, i1["status"], i1["relres_true"]))
            if abs(i1["iters"] - i2["iters"]) > 1:
                bad.append("%s %s rhs %d: %d vs %d iterations" % (name, prec, j, i1["iters"], i2["iters"]))
            d = np.linalg.norm(xx[j] - xr[j])
            if not d <= 1e-7 * np.linalg.norm(xr[j]):
                bad.append("%s %s rhs %d: |x - x_quiet| = %g of %g" % (name, prec, j, d, np.linalg.norm(xr[j])))
    for b, x, infos in host_out:
        for j, i in enumerate(infos):
            if i["status"] != 0 or not i["relres_true"] <= RTOL or not np.all(np.isfinite(x[j])):
                bad.append("host solve rhs %d: status %d relres_true %g" % (j, i["status"], i["relres_true"]))
    return bad


@pytest.mark.gpu
def test_concurrent_submit_wait_across_problems():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc
    probs = make_problems(bddc)
    try:
        records, host_out, errors = stress(bddc, probs)
        assert not errors, errors
        assert len(records) == 60
        again = quiet(bddc, probs, records)
        bad = check(records, again, host_out)
        assert not bad, bad[:10]
    finally:
        for P, _ in probs.values():
            P.close()
