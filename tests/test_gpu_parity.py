"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

FP64 form: element-wise bounds 1e-11 relative for single sigma applications and
the right-hand / left vectors (pure FP64 contractions, only the summation order
differs), 1e-8 absolute on G at solver tolerance 1e-12 (the workload's bound for
the plain form). FP32 inner sigma: bound 3e-5 relative per application (FP32
rounding of ~10^3-term complex sums).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2208_07478_gb300 import binding as B
from paper_2208_07478_gb300.synth import make_system, make_workload
from oracle.kccsd import KEOM, KMesh
from oracle import solvers

from oracle_cases import symmetric_lambda2

CASES = {
    # name: (kmesh, nocc, nvir, naux, seed, t1_sigma, random_lambda)
    "gamma_o3v5": ((1, 1, 1), 3, 5, 8, 1, 0.02, False),
    "k2_o2v3_lambda": ((2, 1, 1), 2, 3, 6, 2, 0.02, True),
    "k3_o1v4": ((3, 1, 1), 1, 4, 5, 3, 0.02, True),
    "k22_o2v3": ((1, 2, 2), 2, 3, 6, 4, 0.01, False),
}


def build_case(name, mode="stored"):
    """mode: 'stored' keeps every H_bar block; 'direct' forms the W_vvvo r1 term, the EA singles'
    (2<am|ef> - <am|fe>) term and the ladder's T2 part from the density-fitting factors."""
    kmesh, o, v, naux, seed, t1s, rl = CASES[name]
    s = make_system(kmesh, o, v, naux, seed=seed, L_sigma=0.08, t1_sigma=t1s, nomega=3,
                    omega_range=(-0.7, 0.7), eta=0.02)
    l1 = l2 = None
    if rl:
        rng = np.random.default_rng(seed + 7)
        l1 = 0.05 * (rng.normal(size=s.t1.shape) + 1j * rng.normal(size=s.t1.shape))
        l2 = symmetric_lambda2(KMesh(kmesh), 0.05 * (rng.normal(size=s.t2.shape) + 1j * rng.normal(size=s.t2.shape)))
    opt = B.default_options(direct_terms=1 if mode == "stored" else 2)
    h = B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, s.mo_energy, s.L, s.t1, s.t2, l1, l2, options=opt)
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L, l1=l1, l2=l2)
    return s, h, ke


@pytest.fixture(scope="module", params=[(c, m) for c in CASES for m in ("stored", "direct")],
                ids=[f"{c}-{m}" for c in CASES for m in ("stored", "direct")])
def case(request):
    s, h, ke = build_case(*request.param)
    yield s, h, ke
    h.close()


def _rand(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


@pytest.mark.parametrize("sector", ["ip", "ea"])
@pytest.mark.parametrize("prec", [B.FP64, B.FP32])
def test_sigma_matches_oracle(case, sector, prec):
    s, h, ke = case
    d = h.dims()
    D = d["dim_ip"] if sector == "ip" else d["dim_ea"]
    rng = np.random.default_rng(5)
    nvec = 7
    for K in range(s.nk):
        x = _rand(rng, (nvec, D))
        xd = torch.from_numpy(x).cuda()
        yd = torch.zeros_like(xd)
        (B.sigma_ip if sector == "ip" else B.sigma_ea)(h, K, xd, yd, prec=prec)
        y = yd.cpu().numpy()
        sig = ke.sigma_ip if sector == "ip" else ke.sigma_ea
        ref = np.stack([sig(K, x[c]) for c in range(nvec)])
        scale = np.abs(ref).max()
        tol = 1e-11 if prec == B.FP64 else 3e-5
        assert np.abs(y - ref).max() <= tol * scale, (K, np.abs(y - ref).max() / scale)


@pytest.mark.parametrize("sector", ["ip", "ea"])
def test_rhs_and_left_match_oracle(case, sector):
    s, h, ke = case
    d = h.dims()
    D = d["dim_ip"] if sector == "ip" else d["dim_ea"]
    sec = B.IP if sector == "ip" else B.EA
    for K in range(s.nk):
        for p in range(s.nmo):
            out = torch.zeros(D, dtype=torch.complex128, device="cuda")
            B.rhs(h, sec, K, p, out)
            ref = ke.rhs_ip(K, p) if sector == "ip" else ke.rhs_ea(K, p)
            np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-13, rtol=1e-12)
            B.left(h, sec, K, p, out)
            ref = ke.left_ip(K, p) if sector == "ip" else ke.left_ea(K, p)
            np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-13, rtol=1e-12)


def oracle_gf(ke, omegas, eta, sectors=("ip", "ea")):
    n = ke.nmo
    G = np.zeros((ke.nk, len(omegas), n, n), dtype=np.complex128)
    for K in range(ke.nk):
        for kind in sectors:
            A = ke.matrix(kind, K)
            if kind == "ip":
                Bm = np.stack([ke.rhs_ip(K, p) for p in range(n)], 1)
                Em = np.stack([ke.left_ip(K, q) for q in range(n)], 0)
            else:
                Bm = np.stack([ke.rhs_ea(K, p) for p in range(n)], 1)
                Em = np.stack([ke.left_ea(K, q) for q in range(n)], 0)
            G[K] += solvers.dense_gf(kind, A, Bm, Em, omegas, eta)
    return G


@pytest.mark.parametrize("chunk", [1, 3])
def test_greens_function_fp64(case, chunk):
    s, h, ke = case
    G = np.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=np.complex128)
    opt = B.default_options(tol=1e-12, restart_m=30, max_iter=5000, omega_chunk=chunk)
    status, stats = B.solve_gf(h, B.BOTH, s.omega, s.eta, G, options=opt)
    assert status == B.CCGF_OK
    assert stats["max_rel_residual"] <= 1e-12
    Gref = oracle_gf(ke, s.omega, s.eta)
    assert np.abs(G - Gref).max() <= 1e-8


def test_greens_function_fp32_refined(case):
    """FP32 inner sigma + FP64 true residuals reach the same tolerance and the same G."""
    s, h, ke = case
    G = np.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=np.complex128)
    opt = B.default_options(prec=B.FP32, tol=1e-10, restart_m=30, max_iter=5000, max_refine=50)
    status, stats = B.solve_gf(h, B.BOTH, s.omega, s.eta, G, options=opt)
    assert status == B.CCGF_OK
    assert stats["max_rel_residual"] <= 1e-10
    assert stats["lowp_sigma_calls"] > 0
    Gref = oracle_gf(ke, s.omega, s.eta)
    assert np.abs(G - Gref).max() <= 1e-6 * max(1.0, np.abs(Gref).max())


def test_sector_split(case):
    """IP-only plus EA-only equals both (G = G+ + G-)."""
    s, h, ke = case
    opt = B.default_options(tol=1e-12)
    Gs = []
    for sec in (B.IP, B.EA, B.BOTH):
        G = np.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=np.complex128)
        B.solve_gf(h, sec, s.omega, s.eta, G, options=opt)
        Gs.append(G)
    assert np.abs(Gs[0] + Gs[1] - Gs[2]).max() < 1e-10
