"""GPU edge cases: degenerate sizes, the Hartree-Fock limit, ragged frequency chunks,
iteration caps, non-finite inputs and invalid arguments (all through the C ABI)."""
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


def _build(s, **kw):
    return B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, s.mo_energy, s.L, s.t1, s.t2, **kw)


def test_hartree_fock_limit_closed_form():
    """No two-electron integrals and T = Lambda = 0: G_pp = 1/(w - e_p -+ i eta) (Eq. 1 for a determinant)."""
    s = make_system((2, 1, 1), 2, 3, 4, seed=5, L_sigma=0.0, t1_sigma=0.0, nomega=4, omega_range=(-1.2, 1.2), eta=0.03)
    s.t2[:] = 0.0
    h = _build(s)
    G = np.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=np.complex128)
    B.solve_gf(h, B.BOTH, s.omega, s.eta, G, options=B.default_options(tol=1e-13))
    h.close()
    for K in range(s.nk):
        for w, om in enumerate(s.omega):
            e = s.mo_energy[K]
            ref = np.diag([1.0 / (om - e[p] - 1j * s.eta) if p < s.nocc else 1.0 / (om - e[p] + 1j * s.eta)
                           for p in range(s.nmo)])
            np.testing.assert_allclose(G[K, w], ref, atol=1e-12)


@pytest.mark.parametrize("o,v", [(1, 1), (3, 1), (1, 2)])
def test_degenerate_sizes(o, v):
    s = make_system((2, 1, 1), o, v, 3, seed=7, L_sigma=0.1, t1_sigma=0.02, nomega=2, omega_range=(-0.5, 0.5), eta=0.02)
    h = _build(s)
    G = np.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=np.complex128)
    st, _ = B.solve_gf(h, B.BOTH, s.omega, s.eta, G, options=B.default_options(tol=1e-12))
    h.close()
    assert st == B.CCGF_OK
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    assert np.abs(G - oracle_gf(ke, s.omega, s.eta)).max() <= 1e-8


def test_single_vector_and_ragged_chunks():
    s = make_system((3, 1, 1), 1, 3, 4, seed=9, L_sigma=0.08, t1_sigma=0.02, nomega=4, omega_range=(-0.6, 0.6), eta=0.02)
    h = _build(s)
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    D = h.dims()["dim_ea"]
    x = np.random.default_rng(1).normal(size=(1, D)) + 0j
    y = torch.zeros((1, D), dtype=torch.complex128, device="cuda")
    B.sigma_ea(h, 2, torch.from_numpy(x).cuda(), y)
    ref = ke.sigma_ea(2, x[0])
    assert np.abs(y.cpu().numpy()[0] - ref).max() <= 1e-11 * np.abs(ref).max()
    G = np.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=np.complex128)
    B.solve_gf(h, B.BOTH, s.omega, s.eta, G, options=B.default_options(tol=1e-12, omega_chunk=3))   # chunks 3 + 1
    h.close()
    assert np.abs(G - oracle_gf(ke, s.omega, s.eta)).max() <= 1e-8


def test_iteration_cap_reports_not_converged_and_writes_g():
    s = make_system((1, 1, 1), 2, 4, 6, seed=3, L_sigma=0.1, t1_sigma=0.0, nomega=1, omega_range=(-0.4, -0.4), eta=0.01)
    h = _build(s)
    G = np.full((1, 1, s.nmo, s.nmo), np.nan, dtype=np.complex128)
    st, stats = B.solve_gf(h, B.BOTH, s.omega, s.eta, G, options=B.default_options(tol=1e-14, max_iter=1, max_refine=1))
    h.close()
    assert st == B.CCGF_NOT_CONVERGED
    assert np.isfinite(G).all()
    assert stats["max_rel_residual"] > 1e-14


def test_non_finite_input_is_refused():
    s = make_system((1, 1, 1), 2, 3, 4, seed=2, nomega=0)
    s.t2[0, 0, 0, 0, 0, 0, 0] = np.nan
    with pytest.raises(B.CCGFError) as e:
        _build(s)
    assert e.value.status == B.CCGF_ERR_NAN


def test_invalid_arguments():
    s = make_system((2, 1, 1), 1, 2, 3, seed=2, nomega=0)
    h = _build(s)
    D = h.dims()["dim_ip"]
    x = torch.zeros((2, D), dtype=torch.complex128, device="cuda")
    for K in (-1, 2):
        with pytest.raises(B.CCGFError) as e:
            B.sigma_ip(h, K, x, x.clone())
        assert e.value.status == B.CCGF_ERR_INVALID_ARG
    G = np.zeros((2, 1, 3, 3), dtype=np.complex128)
    with pytest.raises(B.CCGFError):
        B.solve_gf(h, B.BOTH, [], 0.01, G)                       # no frequencies
    with pytest.raises(B.CCGFError):
        B.solve_gf(h, B.BOTH, [0.1], 0.0, G)                     # eta must be positive
    with pytest.raises(B.CCGFError):
        B.solve_gf(h, B.BOTH, [np.inf], 0.01, G)                 # non-finite frequency
    for sec in (0, 4):
        with pytest.raises(B.CCGFError):
            B.solve_gf(h, sec, [0.1], 0.01, G)
    h.close()
