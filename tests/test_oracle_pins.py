"""Pins of the CPU oracle against definitions, closed forms and exact theory.

Chain of evidence (no stored value comes from the CUDA path):
  FCI (exact Eq. 1, no cluster operators)
    -> brute-force CCGF of Eqs. 4-9 (Fock space), exact for 2-electron IP / 2-hole EA
    -> spin-orbital EOM-CCSD equations (all blocks, RHS, left vectors, G)
    -> spin-adapted k-point EOM-CCSD (via the supercell, and directly vs brute force)
  plus the Hartree-Fock-limit closed form and three independent linear solvers.
"""
import numpy as np
import pytest

from oracle.fockspace import (BruteForceCCGF, hf_core_hamiltonian, fci_greens_function,
                              cluster_amplitudes_from_state, lambda_amplitudes_from_state,
                              expm_apply)
from oracle.spinorb import SpinOrbitalEOM
from oracle.supercell import supercell_system
from oracle.kccsd import KEOM, KMesh
from oracle import solvers
from paper_2208_07478_gb300.synth import make_system

from oracle_cases import random_molecule, symmetric_lambda2

OMEGAS = np.array([-1.3, -0.45, 0.2, 0.9])
ETA = 0.05


def keom_gf(ke, omegas, eta, sectors=("ip", "ea")):
    """G[K, w, p, q] from the k-point oracle by dense LU solves."""
    n = ke.nmo
    G = np.zeros((ke.nk, len(omegas), n, n), dtype=np.complex128)
    for K in range(ke.nk):
        for kind in sectors:
            A = ke.matrix(kind, K)
            if kind == "ip":
                B = np.stack([ke.rhs_ip(K, p) for p in range(n)], 1)
                E = np.stack([ke.left_ip(K, q) for q in range(n)], 0)
            else:
                B = np.stack([ke.rhs_ea(K, p) for p in range(n)], 1)
                E = np.stack([ke.left_ea(K, q) for q in range(n)], 0)
            G[K] += solvers.dense_gf(kind, A, B, E, omegas, eta)
    return G


# ---------------------------------------------------------------- HF limit
def test_hf_limit_closed_form():
    """T = Lambda = 0 and no two-electron integrals: G_pp = 1/(w - e_p -+ i eta), Eq. 1 with a determinant."""
    s = make_system((2, 1, 1), 2, 3, 4, seed=5, L_sigma=0.0, t1_sigma=0.0, nomega=0)
    z1 = np.zeros_like(s.t1)
    z2 = np.zeros_like(s.t2)
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, z1, z2, L=s.L, l1=z1, l2=z2)
    G = keom_gf(ke, OMEGAS, ETA)
    for K in range(s.nk):
        e = s.mo_energy[K]
        for w, om in enumerate(OMEGAS):
            ref = np.zeros((s.nmo, s.nmo), dtype=complex)
            for p in range(s.nmo):
                ref[p, p] = 1.0 / (om - e[p] - 1j * ETA) if p < s.nocc else 1.0 / (om - e[p] + 1j * ETA)
            np.testing.assert_allclose(G[K, w], ref, atol=1e-13)


# ---------------------------------------------------------------- FCI exactness
def _fci_case(nocc, nvir, seed):
    m = random_molecule(nocc, nvir, seed, t1_sigma=0.0, lam=False)
    f, g = m["f"], m["g"]
    h = hf_core_hamiltonian(f, g, nocc)
    Gp, Gm, E0, psi, fs, H = fci_greens_function(h, g, nocc, OMEGAS, ETA)
    t1, t2 = cluster_amplitudes_from_state(fs, nocc, psi)
    T = fs.cluster_T(nocc, t1, t2)
    ref, s0 = fs.reference(nocc)
    c = psi / psi[s0]
    assert np.abs(expm_apply(T, ref) - c).max() < 1e-12      # CCSD represents the state exactly
    left = psi.conj() / np.vdot(psi, c)
    l1, l2, row = lambda_amplitudes_from_state(fs, nocc, T, left)
    return dict(f=f, g=g, h=h, Gp=Gp, Gm=Gm, E0=E0, t1=t1, t2=t2, l1=l1, l2=l2, row=row)


@pytest.mark.parametrize("nvir", [1, 3])
def test_fci_exact_ip_two_electrons(nvir):
    """Two electrons: 1h + 2h1p spans every N-1 state, so CC G- equals the exact G- of Eq. 1."""
    c = _fci_case(1, nvir, seed=10 + nvir)
    bf = BruteForceCCGF(c["h"], c["g"], 1, c["t1"], c["t2"], c["l1"], c["l2"])
    assert abs(bf.Ecc - c["E0"]) < 1e-12
    assert np.abs(bf.bra - c["row"]).max() < 1e-12
    G_bf = bf.greens_function(OMEGAS, ETA, sectors=("ip",))
    np.testing.assert_allclose(G_bf, c["Gm"], atol=1e-11)
    # the spin-adapted k-point oracle at nk = 1 with the same T and Lambda
    eps = np.real(np.diag(c["f"]))[None, :]
    ke = KEOM((1, 1, 1), 1, eps, c["t1"][None], c["t2"][None, None, None], g=c["g"][None, None, None],
              l1=c["l1"][None], l2=c["l2"][None, None, None])
    G_k = keom_gf(ke, OMEGAS, ETA, sectors=("ip",))[0]
    np.testing.assert_allclose(G_k, c["Gm"], atol=1e-11)


@pytest.mark.parametrize("nocc", [1, 3])
def test_fci_exact_ea_two_holes(nocc):
    """One virtual orbital: 1p + 2p1h spans every N+1 state, so CC G+ equals the exact G+ of Eq. 1."""
    c = _fci_case(nocc, 1, seed=20 + nocc)
    bf = BruteForceCCGF(c["h"], c["g"], nocc, c["t1"], c["t2"], c["l1"], c["l2"])
    G_bf = bf.greens_function(OMEGAS, ETA, sectors=("ea",))
    np.testing.assert_allclose(G_bf, c["Gp"], atol=1e-11)
    eps = np.real(np.diag(c["f"]))[None, :]
    ke = KEOM((1, 1, 1), nocc, eps, c["t1"][None], c["t2"][None, None, None], g=c["g"][None, None, None],
              l1=c["l1"][None], l2=c["l2"][None, None, None])
    G_k = keom_gf(ke, OMEGAS, ETA, sectors=("ea",))[0]
    np.testing.assert_allclose(G_k, c["Gp"], atol=1e-11)


def test_fci_not_exact_where_ansatz_truncates():
    """Two electrons in >1 virtual: EA needs 3p2h, so CC G+ must differ from exact (the pin has teeth)."""
    c = _fci_case(1, 3, seed=13)
    bf = BruteForceCCGF(c["h"], c["g"], 1, c["t1"], c["t2"], c["l1"], c["l2"])
    G_bf = bf.greens_function(OMEGAS, ETA, sectors=("ea",))
    assert np.abs(G_bf - c["Gp"]).max() > 1e-4


# ---------------------------------------------------------------- spin-orbital equations
@pytest.mark.parametrize("nocc,nvir,hermitian,seed", [(2, 2, False, 1), (2, 2, True, 2), (1, 3, False, 3), (3, 2, True, 4)])
def test_spinorbital_equations_vs_bruteforce(nocc, nvir, hermitian, seed):
    """Every block of A, every b and e, and G against the operator definition (random T1, Lambda)."""
    m = random_molecule(nocc, nvir, seed, hermitian=hermitian, fock_offdiag=0.0 if hermitian else 0.05)
    h = hf_core_hamiltonian(m["f"], m["g"], nocc)
    bf = BruteForceCCGF(h, m["g"], nocc, m["t1"], m["t2"], m["l1"], m["l2"])
    so = SpinOrbitalEOM(m["f"], m["g"], nocc, m["t1"], m["t2"], m["l1"], m["l2"])
    n = nocc + nvir
    for kind in ("ip", "ea"):
        A1, basis = bf.eom_matrix(kind)
        A2 = so.matrix(kind)
        np.testing.assert_allclose(A2, A1, atol=1e-12)
        pack = so.pack_ip if kind == "ip" else so.pack_ea
        for p in range(n):
            for s in (0, 1):
                P = 2 * p + s
                b2 = pack(*(so.rhs_ip(P) if kind == "ip" else so.rhs_ea(P)))
                e2 = pack(*(so.left_ip(P) if kind == "ip" else so.left_ea(P)))
                np.testing.assert_allclose(b2, bf.rhs(kind, basis, p, s), atol=1e-13)
                np.testing.assert_allclose(e2, bf.left(kind, basis, p, s), atol=1e-13)
    np.testing.assert_allclose(so.greens_function(OMEGAS, ETA), bf.greens_function(OMEGAS, ETA), atol=1e-11)


# ---------------------------------------------------------------- k-point, spin-adapted
@pytest.mark.parametrize("kmesh,o,v,seed", [((1, 1, 1), 2, 3, 1), ((2, 1, 1), 1, 2, 4), ((3, 1, 1), 1, 2, 5), ((1, 2, 2), 1, 1, 6)])
def test_kpoint_vs_supercell(kmesh, o, v, seed):
    """k-point G equals the k-diagonal blocks of the supercell G; k-off-diagonal blocks vanish (Eq. 9)."""
    s = make_system(kmesh, o, v, 4, seed=seed, L_sigma=0.2, t1_sigma=0.1, nomega=0)
    km = KMesh(kmesh)
    rng = np.random.default_rng(seed + 100)
    l1 = 0.1 * (rng.normal(size=s.t1.shape) + 1j * rng.normal(size=s.t1.shape))
    l2 = symmetric_lambda2(km, 0.1 * (rng.normal(size=s.t2.shape) + 1j * rng.normal(size=s.t2.shape)))
    sc = supercell_system(kmesh, o, s.mo_energy, s.L, s.t1, s.t2, l1, l2)
    so = SpinOrbitalEOM(sc["f"], sc["g"], sc["nocc"], sc["t1"], sc["t2"], sc["l1"], sc["l2"])
    Gsc = so.greens_function(OMEGAS, ETA)
    ke = KEOM(kmesh, o, s.mo_energy, s.t1, s.t2, L=s.L, l1=l1, l2=l2)
    Gk = keom_gf(ke, OMEGAS, ETA)
    for K in range(s.nk):
        idx = sc["sc"][K]
        np.testing.assert_allclose(Gk[K], Gsc[:, idx][:, :, idx], atol=1e-11)
        for K2 in range(s.nk):
            if K2 != K:
                assert np.abs(Gsc[:, idx][:, :, sc["sc"][K2]]).max() < 1e-14


def test_kpoint_vs_bruteforce_direct():
    """k-point oracle against the operator definition on a 2-point mesh (12 spin-orbitals)."""
    kmesh, o, v = (2, 1, 1), 1, 2
    s = make_system(kmesh, o, v, 3, seed=8, L_sigma=0.2, t1_sigma=0.1, nomega=0)
    sc = supercell_system(kmesh, o, s.mo_energy, s.L, s.t1, s.t2)
    h = hf_core_hamiltonian(sc["f"], sc["g"], sc["nocc"])
    bf = BruteForceCCGF(h, sc["g"], sc["nocc"], sc["t1"], sc["t2"], sc["l1"], sc["l2"])
    Gbf = bf.greens_function(OMEGAS, ETA)
    ke = KEOM(kmesh, o, s.mo_energy, s.t1, s.t2, L=s.L)
    Gk = keom_gf(ke, OMEGAS, ETA)
    for K in range(s.nk):
        idx = sc["sc"][K]
        np.testing.assert_allclose(Gk[K], Gbf[:, idx][:, :, idx], atol=1e-11)


def test_planted_sign_error_is_caught(monkeypatch):
    """Flip the sign of the IP three-body term in the oracle: the brute-force pin must fail."""
    m = random_molecule(2, 2, 2)
    h = hf_core_hamiltonian(m["f"], m["g"], 2)
    bf = BruteForceCCGF(h, m["g"], 2, m["t1"], m["t2"], m["l1"], m["l2"])
    A1, _ = bf.eom_matrix("ip")
    orig = SpinOrbitalEOM.sigma_ip

    def planted(self, r1, r2):
        s1, s2 = orig(self, r1, r2)
        return s1, s2 - np.einsum("mnef,mnf,ijae->ija", self.v_oovv, r2, self.t2)

    monkeypatch.setattr(SpinOrbitalEOM, "sigma_ip", planted)
    so = SpinOrbitalEOM(m["f"], m["g"], 2, m["t1"], m["t2"], m["l1"], m["l2"])
    assert np.abs(so.matrix("ip") - A1).max() > 1e-3


# ---------------------------------------------------------------- solvers
def test_solvers_agree_dense_lehmann_gmres():
    """LU, eigen-decomposition (Lehmann sum) and restarted GMRES give the same G (config-1 shape, few w)."""
    s = make_system((1, 1, 1), 4, 12, 48, seed=0, L_sigma=0.05, t1_sigma=0.0, nomega=0)
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    n = s.nmo
    om = np.array([-0.7, 0.1])
    for kind in ("ip", "ea"):
        A = ke.matrix(kind, 0)
        if kind == "ip":
            B = np.stack([ke.rhs_ip(0, p) for p in range(n)], 1)
            E = np.stack([ke.left_ip(0, q) for q in range(n)], 0)
        else:
            B = np.stack([ke.rhs_ea(0, p) for p in range(n)], 1)
            E = np.stack([ke.left_ea(0, q) for q in range(n)], 0)
        Gd = solvers.dense_gf(kind, A, B, E, om, 0.01)
        Gl = solvers.lehmann_gf(kind, A, B, E, om, 0.01)
        np.testing.assert_allclose(Gl, Gd, atol=1e-9)
        for w, o_ in enumerate(om):
            M = solvers.shift_matrix(kind, o_, 0.01, A)
            for p in (0, 5, n - 1):
                x, it, res = solvers.gmres(lambda y: M @ y, B[:, p], tol=1e-12, restart=30)
                assert res <= 1e-12
                g = E @ x
                ref = Gd[w, p, :] if kind == "ip" else Gd[w, :, p]
                np.testing.assert_allclose(g, ref, atol=1e-9)


def test_high_frequency_moment_expansion():
    """Far from every pole: G- = sum_k (-1)^k e.A^k b / (w - i eta)^(k+1) (Neumann series of Eq. 6)."""
    s = make_system((1, 1, 1), 2, 4, 8, seed=3, L_sigma=0.05, t1_sigma=0.01, nomega=0)
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    A = ke.matrix("ip", 0)
    om = 60.0
    b = ke.rhs_ip(0, 3)
    e = ke.left_ip(0, 1)
    z = om - 1j * ETA
    series, v = 0.0, b.copy()
    for k in range(40):
        series += (-1) ** k * (e @ v) / z ** (k + 1)
        v = A @ v
    exact = solvers.dense_gf("ip", A, b[:, None], e[None, :], [om], ETA)[0, 0, 0]
    assert abs(series - exact) < 1e-13


# ---------------------------------------------------------------- element-wise oracle for large systems
@pytest.mark.parametrize("kmesh,o,v,seed", [((2, 1, 1), 2, 3, 31), ((1, 2, 2), 1, 3, 32), ((3, 1, 1), 2, 2, 33)])
def test_rows_oracle_equals_full_oracle(kmesh, o, v, seed):
    """oracle.rows.KRows (per-element H_bar from the density-fitting factors) reproduces every element
    of KEOM's sigma vectors (which forms every integral and H_bar block), both sectors, all K."""
    from oracle.rows import KRows
    s = make_system(kmesh, o, v, 5, seed=seed, L_sigma=0.1, t1_sigma=0.05, nomega=0)
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    kr = KRows(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, s.L)
    rng = np.random.default_rng(seed)
    for K in range(s.nk):
        for kind in ("ip", "ea"):
            D = ke.ip_dim() if kind == "ip" else ke.ea_dim()
            x = rng.normal(size=D) + 1j * rng.normal(size=D)
            full = (ke.sigma_ip if kind == "ip" else ke.sigma_ea)(K, x)
            rows = (kr.sigma_ip_elements if kind == "ip" else kr.sigma_ea_elements)(K, x, range(D))
            np.testing.assert_allclose(rows, full, atol=1e-12 * np.abs(full).max())


def test_rows_oracle_vectors_equal_full_oracle():
    from oracle.rows import KRows
    s = make_system((2, 1, 1), 2, 3, 5, seed=34, L_sigma=0.1, t1_sigma=0.05, nomega=0)
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    kr = KRows(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, s.L)
    for K in range(s.nk):
        for p in range(s.nmo):
            np.testing.assert_allclose(kr.rhs("ip", K, p), ke.rhs_ip(K, p), atol=1e-15)
            np.testing.assert_allclose(kr.rhs("ea", K, p), ke.rhs_ea(K, p), atol=1e-15)
            np.testing.assert_allclose(kr.left("ip", K, p), ke.left_ip(K, p), atol=1e-15)
            np.testing.assert_allclose(kr.left("ea", K, p), ke.left_ea(K, p), atol=1e-15)


def test_dos_hartree_fock_lorentzians_and_sum_rule():
    """HF limit: G_pp = 1/(w - e_p -+ i eta), so the retarded-convention DOS is a sum of Lorentzians
    eta / pi / ((w - e_p)^2 + eta^2) (one per orbital); on a wide fine grid it integrates to nmo."""
    from oracle.spectral import dos
    s = make_system((2, 1, 1), 2, 3, 4, seed=5, L_sigma=0.0, t1_sigma=0.0, nomega=0)
    z1, z2 = np.zeros_like(s.t1), np.zeros_like(s.t2)
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, z1, z2, L=s.L, l1=z1, l2=z2)
    eta = 0.05
    w = np.linspace(-40.0, 40.0, 16001)
    Gp = keom_gf(ke, w, eta, sectors=("ea",))
    Gm = keom_gf(ke, w, eta, sectors=("ip",))
    d = dos(Gp, Gm)
    for K in range(s.nk):
        ref = sum(eta / np.pi / ((w - e) ** 2 + eta ** 2) for e in s.mo_energy[K])
        np.testing.assert_allclose(d[K], ref, rtol=1e-10, atol=1e-12)
        integral = float(np.sum(0.5 * (d[K][1:] + d[K][:-1]) * np.diff(w)))
        assert abs(integral - s.nmo) < 2e-3 * s.nmo
    # the time-ordered trace alone is negative at the occupied levels
    d_to = dos(Gp + Gm)
    i_occ = np.argmin(np.abs(w - s.mo_energy[0, 0]))
    assert d_to[0, i_occ] < 0 < d[0, i_occ]


def test_self_energy_algebra_limits():
    """Eqs. 12-14: equal GW and CC active-space G give back G_GW; a full active space (V unitary)
    gives back the coupled-cluster G (rotated by V); Dyson form cross-check."""
    from oracle.selfenergy import cc_gw
    rng = np.random.default_rng(8)
    nk, nw, n, m = 2, 3, 6, 3
    c = lambda *sh: rng.normal(size=sh) + 1j * rng.normal(size=sh)
    Ggw = c(nk, nw, n, n) + 4 * np.eye(n)
    Q, _ = np.linalg.qr(c(n, n))
    V = np.stack([Q[:, :m]] * nk)
    Gcas = c(nk, nw, m, m) + 3 * np.eye(m)
    np.testing.assert_allclose(cc_gw(V, Ggw, Gcas, Gcas), Ggw, atol=1e-12)
    Vfull = np.stack([Q] * nk)
    Gcc = c(nk, nw, n, n) + 3 * np.eye(n)
    Ggw_cas = np.einsum('kia,kwij,kjb->kwab', Vfull.conj(), Ggw, Vfull)      # GW in the rotated basis
    out = cc_gw(Vfull, Ggw, Ggw_cas, Gcc)
    np.testing.assert_allclose(out, np.einsum('kia,kwab,kjb->kwij', Vfull, Gcc, Vfull.conj()), atol=1e-11)


def test_mor_reproduces_model_frequencies_and_converges():
    """MOR frequency interpolation: exact (up to rounding) at the model frequencies (Galerkin with the
    solution in the subspace), and equal to the full G everywhere once the model frequencies span the
    space the right-hand sides reach; with a few model points it interpolates a smooth G closely."""
    from oracle.mor import mor_gf
    s = make_system((2, 1, 1), 2, 3, 5, seed=41, L_sigma=0.05, t1_sigma=0.02, nomega=0)
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    eta = 0.05
    grid = np.linspace(-1.0, 1.0, 41)
    for kind in ("ip", "ea"):
        A = ke.matrix(kind, 0)
        n = s.nmo
        Bm = np.stack([(ke.rhs_ip if kind == "ip" else ke.rhs_ea)(0, p) for p in range(n)], 1)
        Em = np.stack([(ke.left_ip if kind == "ip" else ke.left_ea)(0, q) for q in range(n)], 0)
        full = solvers.dense_gf(kind, A, Bm, Em, grid, eta)
        wm = grid[::10]
        G, r = mor_gf(kind, A, Bm, Em, wm, grid, eta, rel_tol=1e-10)
        np.testing.assert_allclose(G[::10], full[::10], atol=1e-9 * np.abs(full).max())
        np.testing.assert_allclose(G, full, atol=1e-6 * np.abs(full).max())     # 5 model points, smooth G
        # enough model points to span every state the right-hand sides reach: exact on the whole grid
        D = A.shape[0]
        many = np.linspace(-3.0, 3.0, int(np.ceil(D / n)) + 4)
        G2, r2 = mor_gf(kind, A, Bm, Em, many, grid, eta, rel_tol=1e-10)
        assert r < r2 <= D
        np.testing.assert_allclose(G2, full, atol=1e-9 * np.abs(full).max())
