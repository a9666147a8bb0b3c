"""Full-size parity on config 3: 1024x1024 mesh, 128x128 substructures
(H/h = 8) grouped 8x8 into 256 level-2 substructures, log10 k ~ U[0, 6] per
8x8-element block, three-level adaptive BDDC with tau = 10 on both levels,
against the oracle's stored results (tests/golden/three_level_blocks_1024.json,
written by tests/golden/make_golden.py from oracle/ only).

* both levels: the same edges, n^{st} identical on every edge (32512 edges
  on level 1, 480 on level 2), top eigenvalues within 1e-7 (a strided sample
  of the edges on level 1), the same coarse sizes (16129 and 741), omega~;
* one FP64 apply of a seeded vector against the oracle's full vector,
  element by element: max |z - z_ref| <= 1e-10 max |z_ref| and the norm of
  the difference <= 1e-10 of the oracle's (the stated FP64 tolerance);
* FP64 PCG: the same iteration count (37), the full solution element by
  element within 1e-9 and the Lanczos kappa within 1e-5.  After 37 iterations the PCG
  solution of this workload is sensitive to rounding beyond 1e-10: the
  oracle itself, with its preconditioner output perturbed by 1e-14
  (relative, three seeds), moves by 1.1e-10 to 2.0e-10 and its kappa by up
  to 1.5e-6 (also between BLAS thread counts), so 1e-10 would test rounding
  order, not parity;
* the FP32 apply within 1e-5 and the BF16 apply within 1e-2 of the FP64
  apply; FP32 PCG reaches the true relative residual 1e-8.  At this size and
  contrast the BF16 preconditioner is outside its error bound (its PCG stalls
  above 1e-8); the library must say so: BDDC_E_NOCONV with the true residual
  it reached, never OK with a residual above the tolerance.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_0911_5730_gb300 import inputs  # noqa: E402

GDIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GOLD = os.path.join(GDIR, "three_level_blocks_1024.json")


def _full(kind):
    return np.load(os.path.join(GDIR, "three_level_blocks_1024_%s.npy" % kind))


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
    wl = inputs.three_level_blocks()
    P = bddc.Problem.from_workload(wl)
    yield wl, P, json.load(open(GOLD))
    P.close()


@pytest.mark.parametrize("level", [1, 2])
def test_selection_full_size(prob, level):
    wl, P, g = prob
    q = P.query(level=level, max_eigs=4)
    assert q["n_dof"] == g["n_dof"]
    assert list(q["n_selected"]) == g["n_sel"][level - 1]
    assert [list(p) for p in q["edge_pairs"]] == g["edge_pairs"][level - 1]
    st = g["lam_stride"][level - 1]
    lam = np.array(g["lam_top"][level - 1])
    mine = np.asarray(q["edge_eigs"])[::st]
    assert mine.shape == lam.shape
    big = lam > 1e-8 * np.maximum(lam[:, :1], 1e-300)
    assert np.allclose(mine[big], lam[big], rtol=1e-7)
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
    _elementwise(x.cpu().numpy(), _full("x"), 1e-9)
    assert abs(np.linalg.norm(x.cpu().numpy()) - g["x_norm"]) <= 1e-9 * g["x_norm"]
    assert abs(info[0]["kappa_est"] - g["pcg"]["kappa"]) <= 1e-5 * g["pcg"]["kappa"]


def test_mixed_full_size(prob):
    wl, P, g = prob
    r = torch.tensor(inputs.normal_rhs(wl.n_dof, 19), device="cuda")
    P.set_precision("fp64")
    z64 = P.apply(r).cpu().numpy()
    for prec, tol in (("fp32", 1e-5), ("bf16", 1e-2)):
        P.set_precision(prec)
        z = P.apply(r).cpu().numpy()
        assert np.linalg.norm(z - z64) <= tol * np.linalg.norm(z64), prec
        x, info = P.solve(torch.tensor(wl.rhs(), device="cuda"), rtol=1e-8, maxit=500)
        if prec == "fp32":
            assert info[0]["status"] == 0 and info[0]["relres_true"] <= 1e-8, prec
        else:
            assert (info[0]["status"] == 0) == (info[0]["relres_true"] <= 1e-8), info[0]
            assert info[0]["status"] in (0, -4)
