"""Full-size parity on the 512x512 channel workload (32x32 substructures,
tau = 10), against the oracle's stored results (tests/golden, written by
tests/golden/make_golden.py from oracle/ only).

* n^{st} identical on all 1984 edges, the same edge pairs, the same number
  of coarse DOFs (2253), top eigenvalues within 1e-7 relative;
* one FP64 apply of a seeded vector and the FP64 PCG solution (the same
  iteration count, 27) against the oracle's full vectors, element by
  element: max |z - z_ref| <= 1e-10 max |z_ref| and the norm of the
  difference <= 1e-10 of the oracle's;
* mixed (FP32 / BF16) PCG reaches the true relative residual 1e-8, with the
  FP32 apply within 1e-5 of the FP64 apply.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_0911_5730_gb300 import inputs  # noqa: E402

GDIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GOLD = os.path.join(GDIR, "two_level_channels_512.json")


def _full(kind):
    return np.load(os.path.join(GDIR, "two_level_channels_512_%s.npy" % kind))


def _elementwise(a, ref, tol):
    assert a.shape == ref.shape
    assert np.max(np.abs(a - ref)) <= tol * np.max(np.abs(ref))
    assert np.linalg.norm(a - ref) <= tol * np.linalg.norm(ref)


@pytest.fixture(scope="module")
def prob():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc
    wl = inputs.two_level_channels()
    P = bddc.Problem.from_workload(wl)
    yield wl, P, json.load(open(GOLD))
    P.close()


def test_selection_full_size(prob):
    wl, P, g = prob
    q = P.query(level=1, max_eigs=4)
    assert q["n_dof"] == g["n_dof"]
    assert list(q["n_selected"]) == g["n_sel"][0]
    assert [list(p) for p in q["edge_pairs"]] == g["edge_pairs"][0]
    st = g.get("lam_stride", [1])[0]
    lam = np.array(g["lam_top"][0])
    big = lam > 1e-8 * lam[:, :1]
    assert np.allclose(q["edge_eigs"][::st][big], lam[big], rtol=1e-7)
    assert abs(q["omega_tilde"] - g["omega_tilde"]) <= 1e-7 * g["omega_tilde"]


def test_apply_full_size_fp64(prob):
    wl, P, g = prob
    P.set_precision("fp64")
    r = torch.tensor(inputs.normal_rhs(wl.n_dof, g["apply"]["seed"]), device="cuda")
    z = P.apply(r).cpu().numpy()
    _elementwise(z, _full("z"), 1e-10)
    assert abs(np.linalg.norm(z) - g["apply"]["z_norm"]) <= 1e-10 * g["apply"]["z_norm"]


def test_pcg_full_size_fp64(prob):
    wl, P, g = prob
    P.set_precision("fp64")
    x, info = P.solve(torch.tensor(wl.rhs(), device="cuda"), rtol=1e-8)
    assert info[0]["status"] == 0 and info[0]["iters"] == g["pcg"]["iters"]
    _elementwise(x.cpu().numpy(), _full("x"), 1e-10)
    assert abs(np.linalg.norm(x.cpu().numpy()) - g["x_norm"]) <= 1e-10 * g["x_norm"]
    assert abs(info[0]["kappa_est"] - g["pcg"]["kappa"]) <= 1e-6 * g["pcg"]["kappa"]


def test_mixed_full_size(prob):
    wl, P, g = prob
    r = torch.tensor(inputs.normal_rhs(wl.n_dof, 77), device="cuda")
    P.set_precision("fp64")
    z64 = P.apply(r).cpu().numpy()
    P.set_precision("fp32")
    z32 = P.apply(r).cpu().numpy()
    assert np.linalg.norm(z32 - z64) <= 1e-5 * np.linalg.norm(z64)
    for prec in ("fp32", "bf16"):
        P.set_precision(prec)
        x, info = P.solve(torch.tensor(wl.rhs(), device="cuda"), rtol=1e-8, maxit=300)
        assert info[0]["status"] == 0 and info[0]["relres_true"] <= 1e-8
    P.set_precision("fp64")
