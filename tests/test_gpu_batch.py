"""Batched right-hand sides: K <= 32 solved in lockstep by the batch kernels.

The batch path runs the same operators as the single right-hand-side path,
but in other kernels (one lane per right-hand side, interleaved vectors) and
with per-right-hand-side PCG scalars.  It must therefore agree with:
* the oracle and the single right-hand-side GPU apply, to the FP64 apply
  tolerance (1e-10), column by column;
* the FP64 apply within the mixed-path tolerances (1e-5 FP32, 1e-2 BF16);
* the oracle's PCG: the same iteration count and a solution within 1e-10;
  for FP32 and BF16 applies, a true relative residual of 1e-8.
Ragged batch widths (3, and 33 = 32 + 1, two batches) and a zero right-hand
side (converged at the start, x = 0) are covered.
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
    "channels_64": inputs.two_level_channels(nx=64, sub=16),
    "channels_96_ragged": inputs.two_level_channels(nx=96, sub=16, tau=3.0),
    "three_level_64": inputs.three_level_blocks(nx=64, sub=8, group=4, tau=10.0),
}
_cache = {}


def _oracle(name):
    if name not in _cache:
        _cache[name] = obddc.build_workload(WL[name])
    return _cache[name]


def _relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name", list(WL))
def test_batch_apply_matches_single_and_oracle(lib, name):
    wl = WL[name]
    H = _oracle(name)
    P = lib.Problem.from_workload(wl)
    R = inputs.normal_rhs(wl.n_dof, 21, 5)
    Rt = torch.tensor(R, device="cuda")
    Z = P.apply(Rt).cpu().numpy()                      # one call, K = 5
    for j in range(5):
        zs = P.apply(Rt[j].contiguous()).cpu().numpy()   # single right-hand side
        assert _relerr(Z[j], zs) <= 1e-10
        assert _relerr(Z[j], H.apply(R[j])) <= 1e-10
    for prec, tol in (("fp32", 1e-5), ("bf16", 1e-2)):
        P.set_precision(prec)
        Zm = P.apply(Rt).cpu().numpy()
        for j in range(5):
            assert _relerr(Zm[j], Z[j]) <= tol, (prec, j)
    P.close()


@pytest.mark.parametrize("name", list(WL))
def test_batch_pcg_fp64_matches_oracle(lib, name):
    wl = WL[name]
    H = _oracle(name)
    P = lib.Problem.from_workload(wl)
    B = inputs.normal_rhs(wl.n_dof, 31, 3)
    B[1] = 0.0                                          # converged at the start
    X, infos = P.solve(torch.tensor(B, device="cuda"), rtol=1e-8)
    X = X.cpu().numpy()
    assert all(i["batch_width"] == 3 for i in infos)    # the lockstep batch ran
    for j in range(3):
        if j == 1:
            assert np.all(X[j] == 0.0) and infos[j]["iters"] == 0 and infos[j]["status"] == 0
            continue
        ref = opcg.pcg(H.A, B[j], H.apply, rtol=1e-8)
        assert infos[j]["status"] == 0
        assert infos[j]["iters"] == ref.iters, (j, infos[j]["iters"], ref.iters)
        assert _relerr(X[j], ref.x) <= 1e-10
        assert infos[j]["relres_true"] <= 1e-8
        assert abs(infos[j]["kappa_est"] - ref.kappa) <= 1e-6 * ref.kappa
    P.close()


def test_batch_ragged_widths_and_mixed(lib):
    wl = WL["channels_96_ragged"]
    P = lib.Problem.from_workload(wl)
    B = torch.tensor(inputs.normal_rhs(wl.n_dof, 41, 33), device="cuda")   # batches of 32 and 1
    X64, inf64 = P.solve(B)
    assert [i["batch_width"] for i in inf64] == [32] * 32 + [1]
    xs, infs = P.solve(B[32].contiguous())
    assert infs[0]["batch_width"] == 1
    assert inf64[32]["iters"] == infs[0]["iters"]
    assert _relerr(X64[32].cpu().numpy(), xs.cpu().numpy()) <= 1e-10
    x3, inf3 = P.solve(B[:3].contiguous())                                  # K = 3
    for j in range(3):
        assert inf3[j]["iters"] == inf64[j]["iters"]
        assert _relerr(x3[j].cpu().numpy(), X64[j].cpu().numpy()) <= 1e-10
    for prec in ("fp32", "bf16"):
        P.set_precision(prec)
        Xm, infm = P.solve(B)
        for j in range(33):
            assert infm[j]["status"] == 0 and infm[j]["relres_true"] <= 1e-8, (prec, j)
        err = max(_relerr(Xm[j].cpu().numpy(), X64[j].cpu().numpy()) for j in range(33))
        assert err <= 1e-6, (prec, err)
    P.close()


def test_batch_host_buffers(lib):
    wl = WL["channels_64"]
    P = lib.Problem.from_workload(wl)
    B = inputs.normal_rhs(wl.n_dof, 51, 4)
    Xh, infh = P.solve_host(B)
    Xd, infd = P.solve(torch.tensor(B, device="cuda"))
    for j in range(4):
        assert infh[j]["iters"] == infd[j]["iters"]
        # FP64 atomics where three or more substructures meet add in
        # scheduling order, so two runs agree to rounding, not bit for bit
        assert _relerr(Xh[j], Xd[j].cpu().numpy()) <= 1e-12
    P.close()


def _conversion_cases():
    """binary64 values for the narrowing / widening conversions: ties at the
    binary32 rounding point (even and odd last kept bit), just above and below
    them, the overflow edge, the subnormal edge, zeros, infinities, NaN, and
    random bit patterns over the whole range."""
    rng = np.random.default_rng(7)
    bits = []
    for _ in range(2000):
        hi_exp = int(rng.integers(870, 1180))              # around the binary32 normal range
        frac = int(rng.integers(0, 1 << 52))
        sign = int(rng.integers(0, 2))
        base = (sign << 63) | (hi_exp << 52) | (frac & ~((1 << 29) - 1))
        for low in (0, 1, (1 << 28) - 1, 1 << 28, (1 << 28) + 1, (1 << 29) - 1):
            bits.append(base | low)
    edges = [0x47EFFFFFE0000000, 0x47EFFFFFF0000000, 0x47EFFFFFEFFFFFFF,   # FLT_MAX, ties to overflow
             0x3810000000000000, 0x380FFFFFFFFFFFFF, 0x3800000000000000,   # FLT_MIN and below
             0x0, 0x8000000000000000, 0x7FF0000000000000, 0xFFF0000000000000,
             0x7FF8000000000000, 0x3FF0000000000000, 0xBFF0000010000000]
    bits += edges
    bits += [int(v) for v in rng.integers(0, 2**63, 20000, dtype=np.int64)]
    bits += [int(v) | (1 << 63) for v in rng.integers(0, 2**63, 5000, dtype=np.int64)]
    return np.array([b & 0xFFFFFFFFFFFFFFFF for b in bits], dtype=np.uint64).view(np.float64)


def test_integer_conversions_match_hardware(lib):
    vals = torch.tensor(_conversion_cases(), device="cuda")
    assert lib.selftest_convert(vals) == 0


def test_profile_apply_batch(lib):
    wl = WL["channels_64"]
    P = lib.Problem.from_workload(wl)
    R = torch.tensor(inputs.normal_rhs(wl.n_dof, 61, 8), device="cuda")
    ms = P.profile_apply_batch(R, reps=3)
    assert len(ms) == 5 and all(t > 0 for t in ms)       # pre, neumann, top, average, post
    P.close()


def test_autotuned_tiles_reported(lib):
    wl = WL["channels_64"]
    P = lib.Problem.from_workload(wl)
    assert P.query(level=None)["tuned_tile"] == [0, 0, 0]           # not tuned before a batch
    B = torch.tensor(inputs.normal_rhs(wl.n_dof, 71, 4), device="cuda")
    X, infos = P.solve(B)
    t = P.query(level=None)["tuned_tile"]
    # rows per block of the top-level product: 8, 16, 32, or ceil(n / SMs) <= 16
    assert tuple(t[:2]) in {(16, 8), (32, 4), (32, 8), (8, 16)} and (t[2] in (8, 16, 32) or 1 <= t[2] <= 16)
    assert all(i["status"] == 0 for i in infos)
    P.close()


def test_groups_in_flight_match_each_group_alone(lib):
    """70 right-hand sides run as three lockstep groups at once (32, 32 and 6;
    the second and third on their own workspaces and streams); each group's
    results equal the group solved alone: the same iteration counts and
    solutions within 1e-12.  FP64 atomics where three or more substructures
    meet add in scheduling order, so where that moves the stopping test by
    one iteration the two are converged solves one step apart (within
    100 x rtol)."""
    wl = WL["channels_64"]
    P = lib.Problem.from_workload(wl)
    B = torch.tensor(inputs.normal_rhs(wl.n_dof, 81, 70), device="cuda")
    for prec in ("fp64", "fp32"):
        P.set_precision(prec)
        X, infos = P.solve(B)
        assert [i["batch_width"] for i in infos] == [32] * 64 + [6] * 6
        for g0, g1 in ((0, 32), (32, 64), (64, 70)):
            Xg, ig = P.solve(B[g0:g1].contiguous())
            for j in range(g1 - g0):
                d_it = abs(infos[g0 + j]["iters"] - ig[j]["iters"])
                assert d_it <= 1, (prec, g0, j)
                tol = 1e-12 if d_it == 0 else 1e-6
                assert _relerr(X[g0 + j].cpu().numpy(), Xg[j].cpu().numpy()) <= tol
        Xh, ih = P.solve_host(B.cpu().numpy())
        assert _relerr(Xh, X.cpu().numpy()) <= 1e-12
    P.close()


@pytest.mark.parametrize("route", ["staged", "stream"])
@pytest.mark.parametrize("name", ["channels_64", "three_level_64"])
def test_batch_routes_both_match_oracle(lib, monkeypatch, name, route):
    """The autotuner picks, per level and precision, staged or streaming
    Dirichlet kernels and staged or chunked Neumann / averaging kernels where
    both fit; BDDC_ROUTE forces one of them on every level, so both kinds are
    held to the batch bar whatever the tuner picks: FP64 apply within 1e-10
    of the oracle, FP32 / BF16 within 1e-5 / 1e-2 of it, and the reported
    route bits."""
    monkeypatch.setenv("BDDC_ROUTE", route)
    wl = WL[name]
    H = _oracle(name)
    P = lib.Problem.from_workload(wl)
    try:
        R = inputs.normal_rhs(wl.n_dof, 41, 6)
        Rt = torch.tensor(R, device="cuda")
        Z = P.apply(Rt).cpu().numpy()
        for j in range(6):
            assert _relerr(Z[j], H.apply(R[j])) <= 1e-10, j
        routes = P.query(level=None)["tuned_route"]
        if route == "staged":
            assert all(r == 0 for r in routes)
        else:
            assert routes[0] & 0b000010                     # FP64 Neumann chunked on level 1
        for prec, tol in (("fp32", 1e-5), ("bf16", 1e-2)):
            P.set_precision(prec)
            Zm = P.apply(Rt).cpu().numpy()
            for j in range(6):
                assert _relerr(Zm[j], Z[j]) <= tol, (prec, j)
    finally:
        P.close()


@pytest.mark.parametrize("name", ["channels_64", "channels_96_ragged", "three_level_64"])
def test_lane_sweeps_match_oracle(lib, monkeypatch, name):
    """The Dirichlet kernel with a lane per right-hand side (a warp per
    substructure runs both sweeps, the factor streamed through a ring;
    BDDC_DIR_LANE=1), on every level where it fits (blocks of 16 rows on the
    channel problems, 8 on the three-level one) and for both corrections
    (BDDC_TC=0): FP32 applies within 1e-5 and
    BF16 within 1e-2 of the oracle's apply, for a full batch of 32 and a
    ragged one of 5, and the FP32 batched PCG meets the tolerance by its true
    residual with the oracle's iteration count (+-1)."""
    monkeypatch.setenv("BDDC_DIR_LANE", "1")
    monkeypatch.setenv("BDDC_TC", "0")
    wl = WL[name]
    H = _oracle(name)
    P = lib.Problem.from_workload(wl)
    try:
        for K in (32, 5):
            R = inputs.normal_rhs(wl.n_dof, 43 + K, K)
            ref = [H.apply(R[j]) for j in range(K)]
            Rt = torch.tensor(R, device="cuda")
            for prec, tol in (("fp32", 1e-5), ("bf16", 1e-2)):
                P.set_precision(prec)
                Z = P.apply(Rt).cpu().numpy()
                for j in range(K):
                    assert _relerr(Z[j], ref[j]) <= tol, (prec, K, j)
        P.set_precision("fp32")
        b = wl.rhs()
        res = opcg.pcg(H.A, b, H.apply, rtol=1e-8)
        B = np.stack([b] + [inputs.normal_rhs(wl.n_dof, 90 + j) for j in range(7)])
        X, infos = P.solve(torch.tensor(B, device="cuda"), rtol=1e-8)
        assert infos[0]["status"] == 0 and abs(infos[0]["iters"] - res.iters) <= 1
        for i in infos:
            assert i["status"] == 0 and i["relres_true"] <= 1e-8
    finally:
        P.close()
