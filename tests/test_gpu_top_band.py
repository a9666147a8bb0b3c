"""The top level as a block-tridiagonal Cholesky factor (the coarse problem of
the last level solved directly, Sec. 2.1), against the CPU oracle's dense
Cholesky of the same A_L.

The setup orders the top-level coarse DOFs by breadth-first level sets of
A_L's graph and merges them into blocks; a coupling between blocks that are
not neighbours would be reported as a setup error, so every passing setup
also checks that the ordering makes A_L block tridiagonal.  Here the dense
inverse is switched off (BDDC_TOP_DENSE_MAX=0) so that every top-level solve
-- one right-hand side and batches -- goes through the factor, and small
block sizes (BDDC_TOP_BMIN) give many blocks even on small meshes.

Tolerances as the FP64 parity tests: 1e-10 per apply and per solution, the
same iteration count.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import bddc as obddc          # noqa: E402
from oracle import pcg as opcg            # noqa: E402
from paper_0911_5730_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc
    return bddc


WL = {
    # 16 x 16 substructures: a top level of several hundred DOFs
    "channels_128_sub8": lambda: inputs.two_level_channels(nx=128, sub=8),
    "unit_c+e": lambda: inputs.two_level_unit(),
    "three_level_64": lambda: inputs.three_level_blocks(nx=64, sub=8, group=4, tau=10.0),
    "voronoi_128_3lev": lambda: inputs.three_level_voronoi(nx=128, cells=8, group=2, levels=3),
    "elastic_64": lambda: inputs.elasticity(nx=64, sub=8, levels=2, constraints="adaptive", tau=3.0),
}
_cache = {}


def _oracle(name):
    if name not in _cache:
        wl = WL[name]()
        _cache[name] = (wl, obddc.build_workload(wl))
    return _cache[name]


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("bmin", [1, 8, 64])
@pytest.mark.parametrize("name", list(WL))
def test_factor_apply_and_solve_match_oracle(lib, name, bmin, monkeypatch):
    monkeypatch.setenv("BDDC_TOP_DENSE_MAX", "0")
    monkeypatch.setenv("BDDC_TOP_BMIN", str(bmin))
    wl, H = _oracle(name)
    P = lib.Problem.from_workload(wl)
    try:
        q = P.query(level=None)
        assert q["top_blocks"] >= 1
        if bmin == 1 and q["n_dof"][-1] > 40:
            assert q["top_blocks"] > 4          # many blocks: the recurrences are exercised
        r = inputs.normal_rhs(wl.n_dof, 3)
        z = P.apply(torch.tensor(r, device="cuda")).cpu().numpy()
        assert _rel(z, H.apply(r)) <= 1e-10
        # a batch of right-hand sides (the batched top solve), ragged width
        R = inputs.normal_rhs(wl.n_dof, 4, 5)
        Z = P.apply(torch.tensor(R, device="cuda")).cpu().numpy()
        for j in range(5):
            assert _rel(Z[j], H.apply(R[j])) <= 1e-10
        b = wl.rhs()
        res = opcg.pcg(H.A, b, H.apply, rtol=1e-8)
        x, info = P.solve(torch.tensor(b, device="cuda"), rtol=1e-8)
        assert info[0]["status"] == 0 and info[0]["iters"] == res.iters
        assert _rel(x.cpu().numpy(), res.x) <= 1e-10
    finally:
        P.close()


def test_unstaged_recurrences_match_oracle(lib, monkeypatch):
    """The recurrence kernels' form for blocks too large to stage in shared
    memory (rows read from global memory), forced on a small problem."""
    monkeypatch.setenv("BDDC_TOP_DENSE_MAX", "0")
    monkeypatch.setenv("BDDC_TOP_BMIN", "8")
    monkeypatch.setenv("BDDC_TOP_STAGED", "0")
    wl, H = _oracle("channels_128_sub8")
    P = lib.Problem.from_workload(wl)
    try:
        r = inputs.normal_rhs(wl.n_dof, 8)
        z = P.apply(torch.tensor(r, device="cuda")).cpu().numpy()
        assert _rel(z, H.apply(r)) <= 1e-10
        R = inputs.normal_rhs(wl.n_dof, 9, 7)
        Z = P.apply(torch.tensor(R, device="cuda")).cpu().numpy()
        for j in range(7):
            assert _rel(Z[j], H.apply(R[j])) <= 1e-10
    finally:
        P.close()


def test_dense_inverse_from_factor_matches_oracle(lib, monkeypatch):
    """With the dense inverse kept (formed by applying the factor to the
    identity), the single right-hand-side apply uses it: same bar."""
    monkeypatch.setenv("BDDC_TOP_BMIN", "8")
    wl, H = _oracle("channels_128_sub8")
    P = lib.Problem.from_workload(wl)
    try:
        assert P.query(level=None)["top_blocks"] > 4
        r = inputs.normal_rhs(wl.n_dof, 6)
        z = P.apply(torch.tensor(r, device="cuda")).cpu().numpy()
        assert _rel(z, H.apply(r)) <= 1e-10
    finally:
        P.close()


def test_batched_forms_agree(lib, monkeypatch):
    """The batched FP64 solve with the factor (BDDC_TOP_FORM=band) and with
    the dense product (BDDC_TOP_FORM=dense; the autotuner picks between them)
    give the oracle's iterations and solutions for 32 right-hand sides."""
    wl, H = _oracle("channels_128_sub8")
    B = inputs.normal_rhs(wl.n_dof, 7, 32)
    ref = [opcg.pcg(H.A, B[j], H.apply, rtol=1e-8) for j in range(0, 32, 8)]
    for form in ("band", "dense"):
        monkeypatch.setenv("BDDC_TOP_FORM", form)
        P = lib.Problem.from_workload(wl)
        try:
            X, infos = P.solve(torch.tensor(B, device="cuda"), rtol=1e-8)
            X = X.cpu().numpy()
            assert (P.query(level=None)["tuned_tile"][2] == 0) == (form == "band")
            for j, rr in zip(range(0, 32, 8), ref):
                assert infos[j]["status"] == 0 and infos[j]["iters"] == rr.iters
                assert _rel(X[j], rr.x) <= 1e-10
        finally:
            P.close()


@pytest.mark.parametrize("variant", ["0", "1", "2", "3", None])
def test_dense_inverse_launch_shapes_match_oracle(lib, variant, monkeypatch):
    """Every launch shape of the single right-hand-side product with the dense
    inverse (BDDC_SYMV_VARIANT; None: the setup's own timing picks one) gives
    the oracle's apply, on a top level whose size is no multiple of the rows
    per block."""
    if variant is None:
        monkeypatch.delenv("BDDC_SYMV_VARIANT", raising=False)
    else:
        monkeypatch.setenv("BDDC_SYMV_VARIANT", variant)
    wl, H = _oracle("unit_c+e")
    P = lib.Problem.from_workload(wl)
    try:
        q = P.query(level=None)
        assert q["tuned_symv"] in (0, 1, 2, 3)
        if variant is not None:
            assert q["tuned_symv"] == int(variant)
        r = inputs.normal_rhs(wl.n_dof, 12)
        z = P.apply(torch.tensor(r, device="cuda")).cpu().numpy()
        assert _rel(z, H.apply(r)) <= 1e-10
    finally:
        P.close()
