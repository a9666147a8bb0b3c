"""Decompositions from the graph partitioner (Algorithm 2's first step)
through the GPU path against the oracle: irregular, partitioner-shaped
substructures (uneven block sizes), two levels with the channel coefficient
(edge weights from k) and three levels with the level-1 substructures grouped
by the same partitioner.  The bar of the other parity tests: the apply within
1e-10 per right-hand side (also batched), PCG with the oracle's iteration
count, solution within 1e-10 and kappa within 1e-6.
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


def _workload(lib, name):
    if name == "channels_64_20parts":
        return lib.partitioned_workload(inputs.two_level_channels(nx=64, sub=16), 20)
    return lib.partitioned_workload(inputs.three_level_blocks(nx=64, sub=8, group=4, tau=10.0), 48, n_sub2=6)


def _relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name", ["channels_64_20parts", "blocks_64_48parts_3lev"])
def test_partitioned_matches_oracle(lib, name):
    wl = _workload(lib, name)
    H = obddc.build_workload(wl)
    P = lib.Problem.from_workload(wl)
    R = inputs.normal_rhs(wl.n_dof, 91, 3)
    Z = P.apply(torch.tensor(R, device="cuda")).cpu().numpy()
    for j in range(3):
        assert _relerr(Z[j], H.apply(R[j])) <= 1e-10
    b = wl.rhs()
    x, info = P.solve(torch.tensor(b, device="cuda"), rtol=1e-8)
    ref = opcg.pcg(H.A, b, H.apply, rtol=1e-8)
    assert info[0]["status"] == 0
    assert info[0]["iters"] == ref.iters
    assert _relerr(x.cpu().numpy(), ref.x) <= 1e-10
    assert abs(info[0]["kappa_est"] - ref.kappa) <= 1e-6 * ref.kappa
    P.close()
