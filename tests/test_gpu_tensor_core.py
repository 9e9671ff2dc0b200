"""Tensor-core sigma (CCGF_TF32X3: tcgen05 MMAs on TF32-split FP32 operands) against the oracle.

The case is sized so that the ring, ladder and three-body contractions reach the
128-row tensor-core tiles (ov = 48, pair blocks of ~150 rows, several K tiles and a
ragged last tile in M, N and K). Bounds: a single application within 3e-5 relative
of the FP64 oracle (as the FP32 SIMT path: the split keeps ~2^-21 relative per
product, FP32 accumulation), and G refined to tol 1e-10 within 1e-6 max(1, |G|).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2208_07478_gb300 import binding as B
from paper_2208_07478_gb300.synth import make_system
from oracle.kccsd import KEOM

from test_gpu_parity import oracle_gf


@pytest.fixture(scope="module", params=["tuned", "defaults"])
def medium(request):
    """The medium system, with the measured kernel choice (autotuner) on, and off (defaults:
    the tensor cores wherever the shape allows)."""
    B.set_autotune(request.param == "tuned")
    s = make_system((2, 1, 1), 4, 12, 16, seed=11, L_sigma=0.06, t1_sigma=0.01, nomega=2,
                    omega_range=(-0.6, 0.6), eta=0.02)
    h = B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, s.mo_energy, s.L, s.t1, s.t2)
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    yield s, h, ke, request.param
    h.close()
    B.set_autotune(True)


@pytest.mark.parametrize("sector", ["ip", "ea"])
@pytest.mark.parametrize("nvec", [1, 13])
def test_tensor_core_sigma_matches_oracle(medium, sector, nvec):
    s, h, ke, mode = medium
    d = h.dims()
    D = d["dim_ip"] if sector == "ip" else d["dim_ea"]
    rng = np.random.default_rng(17 + nvec)
    fn = B.sigma_ip if sector == "ip" else B.sigma_ea
    sig = ke.sigma_ip if sector == "ip" else ke.sigma_ea
    for K in range(s.nk):
        x = rng.normal(size=(nvec, D)) + 1j * rng.normal(size=(nvec, D))
        xd = torch.from_numpy(x).cuda()
        y_tc, y_32 = torch.zeros_like(xd), torch.zeros_like(xd)
        fn(h, K, xd, y_tc, prec=B.TF32X3)
        fn(h, K, xd, y_32, prec=B.FP32)
        ref = np.stack([sig(K, x[c]) for c in range(nvec)])
        scale = np.abs(ref).max()
        err_tc = np.abs(y_tc.cpu().numpy() - ref).max() / scale
        err_32 = np.abs(y_32.cpu().numpy() - ref).max() / scale
        assert err_tc <= 3e-5, (K, err_tc, err_32)
        if nvec > 1 and mode == "defaults":
            # with 13 columns the ring and ladder GEMMs take the tensor cores: a different
            # arithmetic path from the SIMT FP32 kernels (with one column the IP GEMMs are too
            # narrow and every contraction stays on the SIMT path)
            assert not torch.equal(y_tc, y_32)
        if mode == "tuned":
            # every contraction of the plan has a measured choice: a SIMT tile or a tensor-core kernel
            prof = B.sigma_profile(h, B.IP if sector == "ip" else B.EA, K, xd, y_tc, prec=B.TF32X3)
            kern = [k for _, _, _, k in prof if k != -1]
            assert kern and all(1 <= k % 1000 <= 14 or k in (B.KERNEL_TC_TMA, B.KERNEL_TC_REG, B.KERNEL_TC_BULK, 200) for k in kern), kern


@pytest.mark.parametrize("o,v", [(3, 11), (2, 9)])
def test_tensor_core_odd_sizes(o, v):
    """Odd nvir: A rows of odd length are not TMA-addressable (fallback to the register-fed
    kernel), ragged K tails in every contraction; defaults and tuned kernels both match."""
    s = make_system((3, 1, 1), o, v, 10, seed=13, L_sigma=0.06, t1_sigma=0.01, nomega=0)
    h = B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, s.mo_energy, s.L, s.t1, s.t2)
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    rng = np.random.default_rng(5)
    try:
        for sector in ("ip", "ea"):
            D = h.dims()["dim_ip" if sector == "ip" else "dim_ea"]
            fn = B.sigma_ip if sector == "ip" else B.sigma_ea
            sig = ke.sigma_ip if sector == "ip" else ke.sigma_ea
            for K in range(s.nk):
                x = rng.normal(size=(9, D)) + 1j * rng.normal(size=(9, D))
                y = torch.zeros((9, D), dtype=torch.complex128, device="cuda")
                fn(h, K, torch.from_numpy(x).cuda(), y, prec=B.TF32X3)
                ref = np.stack([sig(K, x[c]) for c in range(9)])
                assert np.abs(y.cpu().numpy() - ref).max() <= 3e-5 * np.abs(ref).max(), (sector, K)
    finally:
        h.close()


def test_tensor_core_refined_greens_function(medium):
    s, h, ke, mode = medium
    G = np.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=np.complex128)
    opt = B.default_options(prec=B.TF32X3, tol=1e-10, restart_m=30, max_iter=5000, max_refine=50)
    status, stats = B.solve_gf(h, B.BOTH, s.omega, s.eta, G, options=opt)
    assert status == B.CCGF_OK
    assert stats["max_rel_residual"] <= 1e-10
    assert stats["lowp_sigma_calls"] > 0
    Gref = oracle_gf(ke, s.omega, s.eta)
    assert np.abs(G - Gref).max() <= 1e-6 * max(1.0, np.abs(Gref).max())


def test_bounded_wait_gives_up_and_context_survives(medium):
    """The tensor-core kernels' wait path: a barrier nothing arrives on times out after its limit,
    the status says so, and the next computation on the same context is still correct."""
    import time
    s, h, ke, mode = medium
    t0 = time.perf_counter()
    st = B.tensor_wait_selftest(50.0)
    dt = time.perf_counter() - t0
    assert st == B.CCGF_ERR_TIMEOUT
    assert dt < 5.0
    D = h.dims()["dim_ea"]
    x = torch.from_numpy(np.random.default_rng(2).normal(size=(3, D)) + 0j).cuda()
    y = torch.zeros_like(x)
    B.sigma_ea(h, 0, x, y, prec=B.TF32X3)
    ref = np.stack([ke.sigma_ea(0, x[c].cpu().numpy()) for c in range(3)])
    assert np.abs(y.cpu().numpy() - ref).max() <= 3e-5 * np.abs(ref).max()
