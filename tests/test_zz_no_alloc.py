"""bddc_apply_noalloc: the apply for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc when they apply the preconditioner (they
have handed all device memory to their own pool, work to a fixed budget, or
run a latency-critical loop that must not risk an allocation failure).  For
them the library offers one more entry point whose scratch is a static device
array.  These tests call it through the C ABI twice in a row per workload and
precision and check each result against the ordinary bddc_apply of the same
precision: grid substructures (the warp kernels), three levels, and Voronoi
cells (the streaming kernels), in FP64, FP32 and BF16.  The bound is the FP64
apply tolerance of the other GPU tests (1e-10 relative) in FP64, and the
rounding level of the precision otherwise (1e-6 FP32, 1e-3 BF16, well inside
the mixed-path bounds of 1e-5 and 1e-2): on irregular cells the interface
sums are FP64 atomics whose order changes from call to call, which can move
a reduced-precision rounding.  They also check that
the call records no wait timeout, and that a context whose apply scratch does
not fit the static array is refused with BDDC_E_ARG and a message giving
both sizes.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_0911_5730_gb300 import inputs  # noqa: E402

SCRATCH_BYTES = 16 << 20     # BDDC_NOALLOC_SCRATCH_BYTES


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc
    return bddc


WL = {
    "channels_64": lambda: inputs.two_level_channels(nx=64, sub=16),
    "three_level_64": lambda: inputs.three_level_blocks(nx=64, sub=8, group=4, tau=10.0),
    "voronoi_128": lambda: inputs.three_level_voronoi(nx=128, cells=4, group=2, levels=2),
}


@pytest.mark.parametrize("name", list(WL))
def test_apply_noalloc_matches_apply_two_calls(lib, name):
    wl = WL[name]()
    P = lib.Problem.from_workload(wl)
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-6), ("bf16", 1e-3)):
        P.set_precision(prec)
        for seed in (11, 12):                  # two calls in a row, different inputs
            r = torch.tensor(inputs.normal_rhs(wl.n_dof, seed), device="cuda")
            z_ref = P.apply(r)
            z = torch.full_like(r, np.nan)
            P.apply_noalloc(r, z)
            torch.cuda.synchronize()
            a, b = z.cpu().numpy(), z_ref.cpu().numpy()
            assert np.all(np.isfinite(a)), (name, prec)
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), (name, prec, seed)
            assert P.query()["apply_status"] == 0
    P.close()


def test_apply_noalloc_refuses_scratch_beyond_the_array(lib):
    # 768^2 elements in 2 x 2 substructures (147456 of them, one interior DOF
    # each), grouped 12 x 12 on level 2: the level-1 interface and coarse
    # vectors alone need more doubles than the 16 MiB array holds
    nx, sub, group = 768, 2, 12
    e2s, ns = inputs.grid_decomposition(nx, sub)
    s2, n2 = inputs.grid_grouping(nx // sub, group)
    P = lib.Problem(nx, np.ones(nx * nx), e2s, ns, levels=3, constraints="corners",
                    sub1_to_sub2=s2, n_sub2=n2)
    q = P.query()
    up = lambda v: (v + 31) // 32 * 32
    n_top = q["n_dof"][-1]
    ld_top = (n_top + 3) // 4 * 4
    need = 32
    for l in range(2):
        nc = q["n_dof"][l + 1]
        need += 2 * up(max(q["n_interface"][l], 1)) + up(max(q["sum_interface"][l], 1)) \
            + 2 * up(max(nc, 1, ld_top))
    assert need * 8 > SCRATCH_BYTES
    r = torch.tensor(inputs.normal_rhs(P.n, 5), device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(lib.BDDCError) as ex:
        P.apply_noalloc(r, z)
    assert ex.value.code == -1 and "exceeds the static scratch" in str(ex.value)
    assert str(need * 8) in str(ex.value) and str(SCRATCH_BYTES) in str(ex.value)
    P.close()
