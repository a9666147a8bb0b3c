"""bddc_apply_noalloc: the apply for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc when they apply the preconditioner (they
have handed all device memory to their own pool, work to a fixed budget, or
run a latency-critical loop that must not risk an allocation failure).  For
them the library offers one more entry point whose scratch is a static device
array.  This test calls it through the C ABI twice in a row and checks each
result against the ordinary bddc_apply within the FP64 apply tolerance used by
the other GPU tests (1e-10 relative).  The file is named so that pytest
collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_0911_5730_gb300 import inputs  # noqa: E402


def test_apply_noalloc_matches_apply_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc

    for wl in (inputs.two_level_channels(nx=64, sub=16),
               inputs.three_level_blocks(nx=64, sub=8, group=4, tau=10.0)):
        P = bddc.Problem.from_workload(wl)
        for seed in (11, 12):                  # two calls in a row, different inputs
            r = torch.tensor(inputs.normal_rhs(wl.n_dof, seed), device="cuda")
            z_ref = P.apply(r)
            z = torch.full_like(r, np.nan)
            P.apply_noalloc(r, z)
            torch.cuda.synchronize()
            a, b = z.cpu().numpy(), z_ref.cpu().numpy()
            assert np.all(np.isfinite(a))
            assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)
        P.close()
