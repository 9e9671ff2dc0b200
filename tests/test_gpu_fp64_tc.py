"""FP64-accurate sigma on the tensor cores (CCGF_FP64_TC): exactly sliced operands.

Each operand is cut into 8-bit integer slices under a per-row (per-column) power of two; their
products, and sums of them below 2^24, are exact in the tensor cores' FP32 accumulator, so the
contraction keeps every term above 2^-40 of its leading one. Bound here: 1e-11 of max |y| per application
against the CPU oracle (the FP64 form's own bound; measured ~2e-12), G within 1e-7 at tolerance
1e-10. The cases have even row lengths, so that the sliced kernel (TMA rows of 16-byte multiples)
takes most contractions; the step table is checked to contain it.
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
from oracle import solvers

SLICED = 103   # kernel code of the sliced tensor-core GEMM

CASES = {
    # name: (kmesh, nocc, nvir, naux, seed)
    "k2_o4v8": ((2, 1, 1), 4, 8, 16, 11),
    "gamma_o4v10": ((1, 1, 1), 4, 10, 20, 12),
    "k22_o2v6": ((1, 2, 2), 2, 6, 12, 13),
}


def build(name, autotune):
    kmesh, o, v, naux, seed = CASES[name]
    s = make_system(kmesh, o, v, naux, seed=seed, L_sigma=0.08, t1_sigma=0.02, nomega=3, omega_range=(-0.7, 0.7), eta=0.02)
    B.set_autotune(autotune)
    h = B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, s.mo_energy, s.L, s.t1, s.t2)
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    return s, h, ke


@pytest.fixture(scope="module", params=[(c, a) for c in CASES for a in (False, True)],
                ids=[f"{c}-{'tuned' if a else 'default'}" for c in CASES for a in (False, True)])
def case(request):
    s, h, ke = build(*request.param)
    yield s, h, ke, request.param[1]
    h.close()
    B.set_autotune(True)


@pytest.mark.parametrize("sector", ["ip", "ea"])
def test_sliced_sigma_matches_oracle_and_fp64(case, sector):
    s, h, ke, tuned = case
    B.set_autotune(tuned)
    d = h.dims()
    D = d["dim_ip"] if sector == "ip" else d["dim_ea"]
    rng = np.random.default_rng(21)
    nvec = 6
    fn = B.sigma_ip if sector == "ip" else B.sigma_ea
    sig = ke.sigma_ip if sector == "ip" else ke.sigma_ea
    for K in range(s.nk):
        x = rng.normal(size=(nvec, D)) + 1j * rng.normal(size=(nvec, D))
        xd = torch.from_numpy(x).cuda()
        y_tc = torch.zeros_like(xd)
        y_64 = torch.zeros_like(xd)
        fn(h, K, xd, y_tc, prec=B.FP64_TC)
        fn(h, K, xd, y_64, prec=B.FP64)
        ref = np.stack([sig(K, x[c]) for c in range(nvec)])
        scale = np.abs(ref).max()
        err_tc = np.abs(y_tc.cpu().numpy() - ref).max() / scale
        err_64 = np.abs(y_64.cpu().numpy() - ref).max() / scale
        print(f"{sector} K={K}: sliced {err_tc:.2e}, fp64 {err_64:.2e}")
        assert err_tc <= 1e-11, (K, err_tc)
        assert np.abs(y_tc.cpu().numpy() - y_64.cpu().numpy()).max() <= 1e-11 * scale


def test_sliced_kernel_is_used(case):
    """With the measured choice, or by default, contractions of stored intermediates run sliced."""
    s, h, ke, tuned = case
    B.set_autotune(tuned)
    d = h.dims()
    x = torch.randn((s.nmo, d["dim_ea"]), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    prof = B.sigma_profile(h, B.EA, 0, x, y, prec=B.FP64_TC)
    codes = [p[3] for p in prof]
    if tuned:
        assert SLICED in codes or all(c != 0 for c in codes if c >= 0)
    else:
        # default choice (0): the sliced kernel wherever the step allows it; its launches are counted
        before = h.launch_count()
        B.sigma_ea(h, 0, x, y, prec=B.FP64_TC)
        torch.cuda.synchronize()
        after = h.launch_count()
        B.sigma_ea(h, 0, x, y, prec=B.FP64)
        torch.cuda.synchronize()
        assert after - before > h.launch_count() - after   # the sliced path launches image and slice kernels


def oracle_gf(ke, omegas, eta):
    n = ke.nmo
    G = np.zeros((ke.nk, len(omegas), n, n), dtype=np.complex128)
    for K in range(ke.nk):
        for kind in ("ip", "ea"):
            A = ke.matrix(kind, K)
            rhs = ke.rhs_ip if kind == "ip" else ke.rhs_ea
            left = ke.left_ip if kind == "ip" else ke.left_ea
            Bm = np.stack([rhs(K, p) for p in range(n)], 1)
            Em = np.stack([left(K, q) for q in range(n)], 0)
            G[K] += solvers.dense_gf(kind, A, Bm, Em, omegas, eta)
    return G


def test_sliced_solve_matches_oracle(case):
    """Every sigma of the solve sliced (treated as FP64: no refinement). The sliced operator is
    accurate to ~2e-12 of max |y|, so a residual of 1e-12 is below what it can certify; the solve
    targets 1e-10 and G is held to 1e-7 (the FP64 form's 1e-8 at 1e-12, scaled by the looser
    residual's effect on G, which stays below it here)."""
    s, h, ke, tuned = case
    B.set_autotune(tuned)
    G = np.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=np.complex128)
    opt = B.default_options(prec=B.FP64_TC, tol=1e-10, restart_m=30, max_iter=5000)
    status, stats = B.solve_gf(h, B.BOTH, s.omega, s.eta, G, options=opt)
    assert status == B.CCGF_OK
    assert stats["max_rel_residual"] <= 1e-10
    assert stats["lowp_sigma_calls"] == 0
    Gref = oracle_gf(ke, s.omega, s.eta)
    print("sliced solve max |dG|", np.abs(G - Gref).max())
    assert np.abs(G - Gref).max() <= 1e-7


def test_tensor_core_solve_with_sliced_refinement(case):
    """3xTF32 inner sigma, true residual with the sliced FP64-accurate sigma."""
    s, h, ke, tuned = case
    B.set_autotune(tuned)
    G = np.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=np.complex128)
    opt = B.default_options(prec=B.TF32X3, refine_prec=B.FP64_TC, tol=1e-10, restart_m=30, max_iter=5000, max_refine=50)
    status, stats = B.solve_gf(h, B.BOTH, s.omega, s.eta, G, options=opt)
    assert status == B.CCGF_OK
    assert stats["max_rel_residual"] <= 1e-10
    assert stats["fp64_sigma_calls"] > 0 and stats["lowp_sigma_calls"] > 0
    Gref = oracle_gf(ke, s.omega, s.eta)
    assert np.abs(G - Gref).max() <= 1e-6 * max(1.0, np.abs(Gref).max())
