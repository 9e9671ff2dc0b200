"""Spectral function / density of states (Eq. 10) on the GPU against the oracle's definition.

The kernel is compared with oracle.spectral.dos on random G arrays (both conventions) to 1e-13, and
on the G of a GPU solve (IP and EA parts solved separately) of a small system whose oracle G comes
from dense LU: the DOS agrees to 1e-8 (the G tolerance of the plain form).
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
from oracle.spectral import dos as oracle_dos


def test_dos_kernel_matches_definition():
    rng = np.random.default_rng(3)
    nk, nw, n = 3, 17, 7
    Gp = rng.normal(size=(nk, nw, n, n)) + 1j * rng.normal(size=(nk, nw, n, n))
    Gm = rng.normal(size=(nk, nw, n, n)) + 1j * rng.normal(size=(nk, nw, n, n))
    gp, gm = torch.from_numpy(Gp).cuda(), torch.from_numpy(Gm).cuda()
    d = torch.zeros((nk, nw), dtype=torch.float64, device="cuda")
    tot = torch.zeros(nw, dtype=torch.float64, device="cuda")
    B.spectral_function(gp, d, dos_total=tot)
    torch.cuda.synchronize()
    np.testing.assert_allclose(d.cpu().numpy(), oracle_dos(Gp), atol=1e-13)
    np.testing.assert_allclose(tot.cpu().numpy(), oracle_dos(Gp).mean(axis=0), atol=1e-13)
    B.spectral_function(gp, d, G_minus=gm)
    torch.cuda.synchronize()
    np.testing.assert_allclose(d.cpu().numpy(), oracle_dos(Gp, Gm), atol=1e-13)


def test_dos_of_a_solve_matches_oracle():
    s = make_system((2, 1, 1), 2, 4, 8, seed=13, L_sigma=0.05, t1_sigma=0.01, nomega=9, omega_range=(-1.2, 1.2), eta=0.02)
    h = B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, s.mo_energy, s.L, s.t1, s.t2)
    parts = {}
    for sec in (B.IP, B.EA):
        G = torch.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=torch.complex128, device="cuda")
        st, _ = B.solve_gf(h, sec, s.omega, s.eta, G, options=B.default_options(tol=1e-12), on_device=True)
        assert st == B.CCGF_OK
        parts[sec] = G
    d = torch.zeros((s.nk, len(s.omega)), dtype=torch.float64, device="cuda")
    B.spectral_function(parts[B.EA], d, G_minus=parts[B.IP])
    torch.cuda.synchronize()
    h.close()
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    ref = {}
    for kind in ("ip", "ea"):
        G = np.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=np.complex128)
        for K in range(s.nk):
            A = ke.matrix(kind, K)
            Bm = np.stack([(ke.rhs_ip if kind == "ip" else ke.rhs_ea)(K, p) for p in range(s.nmo)], 1)
            Em = np.stack([(ke.left_ip if kind == "ip" else ke.left_ea)(K, q) for q in range(s.nmo)], 0)
            G[K] = solvers.dense_gf(kind, A, Bm, Em, s.omega, s.eta)
        ref[kind] = G
    np.testing.assert_allclose(d.cpu().numpy(), oracle_dos(ref["ea"], ref["ip"]), atol=1e-8)
