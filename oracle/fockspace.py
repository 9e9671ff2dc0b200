"""Second-quantised brute force for the CC Green's function (tiny systems).

Test infrastructure only (see the package docstring).

Everything here follows the definitions literally, with operators as sparse
matrices on the full Fock space of n spin-orbitals (2**n determinants):

* the Hamiltonian H = sum h_pq E_pq + 1/2 sum (pq|rs) (E_pq E_rs - d_qr E_ps)
  with E_pq = sum_s a+_{p s} a_{q s}; h = f - (2J - K) so that the Fock matrix
  of the reference determinant is f (canonical HF orbitals);
* the CC ground state e^T |Phi0> (Eq. 2) with closed-shell
  T = sum t_ia E_ai + 1/2 sum t_ijab E_ai E_bj;
* the CC bra <Phi0|(1 + Lambda) e^-T (Eq. 3) with
  Lambda = sum l_ia E_ia + 1/2 sum l_ijab E_ia E_jb;
* similarity-transformed operators a_bar = e^-T a e^T, H_bar = e^-T H e^T (Eq. 5);
* the EOM spaces 1h + 2h1p and 1p + 2p1h (Eq. 8) as determinant lists;
* the projected shifted systems of Eq. 6 and the contractions of Eq. 7 / Eq. 9.

The EOM operator is the commutator (connected) form
A[mu, nu] = <mu| [H_bar, R_nu] |Phi0>, which equals <mu|(H_bar - E)|nu> whenever
T solves the CCSD equations (then <lambda|H_bar|Phi0> = 0 for singles and
doubles) and stays well defined for amplitudes that are not CCSD solutions.
``literal=True`` builds <mu|H_bar - E_cc|nu> instead, for exact-T tests.

Spin-orbital index = 2*P + s (s = 0 alpha, 1 beta); spatial orbitals P are
ordered occupied first. Only practical up to ~14 spin-orbitals.
"""
import itertools
import numpy as np
import scipy.sparse as sp


class FockSpace:
    def __init__(self, nspatial):
        self.nspatial = nspatial
        self.n = 2 * nspatial
        self.dim = 1 << self.n
        states = np.arange(self.dim, dtype=np.int64)
        self.nelec = np.bitwise_count(states).astype(np.int64)
        self.ann = []
        for P in range(self.n):
            occ = (states >> P) & 1
            cols = states[occ == 1]
            rows = cols ^ (1 << P)
            below = np.bitwise_count(cols & ((1 << P) - 1)).astype(np.int64)
            vals = np.where(below % 2 == 0, 1.0, -1.0)
            self.ann.append(sp.csr_matrix((vals, (rows, cols)), shape=(self.dim, self.dim)))
        self.cre = [a.T.tocsr() for a in self.ann]
        self._E = {}

    def so(self, p, s):
        return 2 * p + s

    def a(self, p, s=0):
        return self.ann[self.so(p, s)]

    def ad(self, p, s=0):
        return self.cre[self.so(p, s)]

    def E(self, p, q):
        """Spin-summed excitation operator E_pq = sum_s a+_{ps} a_{qs}."""
        key = (p, q)
        if key not in self._E:
            self._E[key] = (self.cre[2 * p] @ self.ann[2 * q] + self.cre[2 * p + 1] @ self.ann[2 * q + 1]).tocsr()
        return self._E[key]

    def one_body(self, h, tol=0.0):
        n = self.nspatial
        out = sp.csr_matrix((self.dim, self.dim), dtype=np.complex128)
        for p in range(n):
            for q in range(n):
                if abs(h[p, q]) > tol:
                    out = out + h[p, q] * self.E(p, q)
        return out.tocsr()

    def hamiltonian(self, h, g):
        """H = sum h_pq E_pq + 1/2 sum (pq|rs)(E_pq E_rs - d_qr E_ps)."""
        n = self.nspatial
        H = self.one_body(h)
        corr = np.einsum('pqqs->ps', g)
        H = H - 0.5 * self.one_body(corr)
        for p in range(n):
            for q in range(n):
                Fpq = self.one_body(g[p, q])
                if Fpq.nnz:
                    H = H + 0.5 * (self.E(p, q) @ Fpq)
        return H.tocsr()

    def reference(self, nocc):
        """|Phi0>: the lowest nocc spatial orbitals doubly occupied."""
        s = 0
        for p in range(nocc):
            s |= (1 << (2 * p)) | (1 << (2 * p + 1))
        v = np.zeros(self.dim, dtype=np.complex128)
        v[s] = 1.0
        return v, s

    def cluster_T(self, nocc, t1, t2):
        """T = sum t1[i,a] E_ai + 1/2 sum t2[i,j,a,b] E_ai E_bj (a, b virtual indices)."""
        no, nv = t1.shape
        T = sp.csr_matrix((self.dim, self.dim), dtype=np.complex128)
        for i in range(no):
            for a in range(nv):
                if t1[i, a] != 0:
                    T = T + t1[i, a] * self.E(nocc + a, i)
        for i, j, a, b in itertools.product(range(no), range(no), range(nv), range(nv)):
            if t2[i, j, a, b] != 0:
                T = T + 0.5 * t2[i, j, a, b] * (self.E(nocc + a, i) @ self.E(nocc + b, j))
        return T.tocsr()

    def cluster_Lambda(self, nocc, l1, l2):
        """Lambda = sum l1[i,a] E_ia + 1/2 sum l2[i,j,a,b] E_ia E_jb."""
        no, nv = l1.shape
        Lm = sp.csr_matrix((self.dim, self.dim), dtype=np.complex128)
        for i in range(no):
            for a in range(nv):
                if l1[i, a] != 0:
                    Lm = Lm + l1[i, a] * self.E(i, nocc + a)
        for i, j, a, b in itertools.product(range(no), range(no), range(nv), range(nv)):
            if l2[i, j, a, b] != 0:
                Lm = Lm + 0.5 * l2[i, j, a, b] * (self.E(i, nocc + a) @ self.E(j, nocc + b))
        return Lm.tocsr()


def expm_apply(X, v, sign=1.0, maxorder=64):
    """e^{sign X} v for a nilpotent X (finite series)."""
    out = v.copy()
    term = v.copy()
    for k in range(1, maxorder):
        term = (sign / k) * (X @ term)
        if not np.any(term):
            return out
        out = out + term
    raise RuntimeError("cluster operator is not nilpotent within maxorder")


def eom_basis(fs, nocc, kind):
    """Determinant basis of the EOM space (Eq. 8).

    IP: a_I |Phi0>, then a+_A a_J a_I |Phi0> (I < J).
    EA: a+_A |Phi0>, then a+_A a+_B a_J |Phi0> (A < B).
    Returns a list of (operator, vector) pairs; each vector is +-1 on one
    determinant, the operator maps |Phi0> onto it.
    """
    ref, _ = fs.reference(nocc)
    occ = [fs.so(p, s) for p in range(nocc) for s in (0, 1)]
    vir = [fs.so(p, s) for p in range(nocc, fs.nspatial) for s in (0, 1)]
    ops = []
    if kind == "ip":
        for I in occ:
            ops.append(fs.ann[I])
        for I, J in itertools.combinations(occ, 2):
            for A in vir:
                ops.append(fs.cre[A] @ fs.ann[J] @ fs.ann[I])
    elif kind == "ea":
        for A in vir:
            ops.append(fs.cre[A])
        for A, B in itertools.combinations(vir, 2):
            for J in occ:
                ops.append(fs.cre[A] @ fs.cre[B] @ fs.ann[J])
    else:
        raise ValueError(kind)
    basis = []
    for R in ops:
        v = R @ ref
        basis.append((R.tocsr(), v))
    return basis


def _project(basis, w):
    """Components <mu|w> over the basis determinants (basis vectors are real +-1 unit vectors)."""
    return np.array([np.vdot(v, w) for _, v in basis])


class BruteForceCCGF:
    """CCGF of Eqs. 4-9 by explicit operators on the Fock space."""

    def __init__(self, h, g, nocc, t1, t2, l1, l2, literal=False):
        n = h.shape[0]
        self.fs = FockSpace(n)
        self.nocc = nocc
        self.H = self.fs.hamiltonian(h, g)
        self.T = self.fs.cluster_T(nocc, t1, t2)
        self.Lam = self.fs.cluster_Lambda(nocc, l1, l2)
        self.ref, self.ref_state = self.fs.reference(nocc)
        self.literal = literal
        # H_bar |Phi0> and E_cc = <Phi0|H_bar|Phi0>
        self.Hbar0 = self.hbar_apply(self.ref)
        self.Ecc = self.Hbar0[self.ref_state]
        # bra <Phi0|(1+Lambda) as a row vector (no conjugation)
        self.bra = self.ref + self.Lam.T @ self.ref

    def hbar_apply(self, v):
        return expm_apply(self.T, self.H @ expm_apply(self.T, v, +1.0), -1.0)

    def abar(self, op, v):
        """e^-T op e^T v."""
        return expm_apply(self.T, op @ expm_apply(self.T, v, +1.0), -1.0)

    def bra_abar(self, op):
        """Row vector of <Phi0|(1+Lambda) e^-T op e^T (acting to the right)."""
        row = self.bra
        row = expm_apply(self.T.T, row, -1.0)       # row @ e^-T
        row = op.T @ row                               # row @ op
        row = expm_apply(self.T.T, row, +1.0)        # row @ e^T
        return row

    def eom_matrix(self, kind):
        basis = eom_basis(self.fs, self.nocc, kind)
        D = len(basis)
        A = np.zeros((D, D), dtype=np.complex128)
        for nu, (R, v) in enumerate(basis):
            w = self.hbar_apply(v)
            if self.literal:
                w = w - self.Ecc * v
            else:
                w = w - R @ self.Hbar0
            A[:, nu] = _project(basis, w)
        return A, basis

    def rhs(self, kind, basis, p, s=0):
        """b = P e^-T a_p e^T |Phi0> (IP) or P e^-T a+_q e^T |Phi0> (EA)."""
        op = self.fs.a(p, s) if kind == "ip" else self.fs.ad(p, s)
        return _project(basis, self.abar(op, self.ref))

    def left(self, kind, basis, q, s=0):
        """e[mu] = <Phi0|(1+Lambda) e^-T a+_q e^T|mu> (IP) or <..|a_p ..|mu> (EA)."""
        op = self.fs.ad(q, s) if kind == "ip" else self.fs.a(q, s)
        row = self.bra_abar(op)
        return np.array([row @ v for _, v in basis])

    def greens_function(self, omegas, eta, sectors=("ip", "ea"), spin=0):
        """G[w, p, q] = G+ + G- over spatial orbitals (alpha spin), Eq. 4 / Eq. 9."""
        n = self.fs.nspatial
        G = np.zeros((len(omegas), n, n), dtype=np.complex128)
        for kind in sectors:
            A, basis = self.eom_matrix(kind)
            D = A.shape[0]
            B = np.stack([self.rhs(kind, basis, p, spin) for p in range(n)], axis=1)     # [D, p]
            Lf = np.stack([self.left(kind, basis, q, spin) for q in range(n)], axis=0)   # [q, D]
            for w, om in enumerate(omegas):
                if kind == "ip":
                    X = np.linalg.solve((om - 1j * eta) * np.eye(D) + A, B)   # X[:, p]
                    G[w] += (Lf @ X).T                                           # G-[p,q] = e_q . X_p
                else:
                    Y = np.linalg.solve((om + 1j * eta) * np.eye(D) - A, B)   # Y[:, q]
                    G[w] += Lf @ Y                                               # G+[p,q] = e_p . Y_q
        return G


def fci_greens_function(h, g, nocc, omegas, eta, state="max_overlap"):
    """Exact G of Eq. 1 from the Hamiltonian alone (no cluster operators).

    The N-electron state is the eigenvector with the largest overlap with the
    reference determinant. G-[p,q] = <Psi|a+_q (w + H - E - i eta)^-1 a_p|Psi>,
    G+[p,q] = <Psi|a_p (w - H + E + i eta)^-1 a+_q|Psi>, alpha spin.
    Returns (G_plus, G_minus, E0, Psi, fock_space, H).
    """
    n = h.shape[0]
    fs = FockSpace(n)
    H = fs.hamiltonian(h, g)
    nel = 2 * nocc
    idx = np.nonzero(fs.nelec == nel)[0]
    Hn = H[idx][:, idx].toarray()
    ev, U = np.linalg.eig(Hn) if not np.allclose(Hn, Hn.conj().T) else np.linalg.eigh(Hn)
    _, s0 = fs.reference(nocc)
    pos0 = int(np.nonzero(idx == s0)[0][0])
    m = int(np.argmax(np.abs(U[pos0]))) if state == "max_overlap" else int(np.argmin(ev.real))
    E0 = ev[m]
    psi = np.zeros(fs.dim, dtype=np.complex128)
    psi[idx] = U[:, m]
    psi /= np.linalg.norm(psi)
    Gm = np.zeros((len(omegas), n, n), dtype=np.complex128)
    Gp = np.zeros_like(Gm)
    im = np.nonzero(fs.nelec == nel - 1)[0]
    ipl = np.nonzero(fs.nelec == nel + 1)[0]
    Hm = H[im][:, im].toarray()
    Hp = H[ipl][:, ipl].toarray()
    ap = [(fs.a(p) @ psi)[im] for p in range(n)]
    adq = [(fs.ad(q) @ psi)[ipl] for q in range(n)]
    for w, om in enumerate(omegas):
        Mm = (om - 1j * eta - E0) * np.eye(len(im)) + Hm
        Mp = (om + 1j * eta + E0) * np.eye(len(ipl)) - Hp
        Xm = np.linalg.solve(Mm, np.stack(ap, axis=1))
        Xp = np.linalg.solve(Mp, np.stack(adq, axis=1))
        Am = np.stack(ap, axis=1)
        Ap = np.stack(adq, axis=1)
        # G-[p,q] = (a_q psi)^H X_p ; G+[p,q] = (a+_p psi)^H Xp_q
        Gm[w] = (Am.conj().T @ Xm).T
        Gp[w] = Ap.conj().T @ Xp
    return Gp, Gm, E0, psi, fs, H


def hf_core_hamiltonian(f, g, nocc):
    """h = f - (2J - K) over the occupied orbitals, so that the reference Fock matrix is f."""
    J = np.einsum('pqii->pq', g[:, :, :nocc, :nocc])
    K = np.einsum('piiq->pq', g[:, :nocc, :nocc, :])
    return f - 2.0 * J + K


def cluster_amplitudes_from_state(fs, nocc, psi):
    """Closed-shell T1, T2 with e^T|Phi0> = psi / <Phi0|psi> through doubles.

    t1[i,a] is the coefficient of E_ai|Phi0>'s alpha determinant; t2 follows
    from the alpha-beta doubles minus the disconnected t1*t1 part.
    """
    ref, s0 = fs.reference(nocc)
    c = psi / psi[s0]
    n = fs.nspatial
    nv = n - nocc
    t1 = np.zeros((nocc, nv), dtype=np.complex128)
    t2 = np.zeros((nocc, nocc, nv, nv), dtype=np.complex128)
    for i in range(nocc):
        for a in range(nv):
            v = fs.ad(nocc + a, 0) @ (fs.a(i, 0) @ ref)
            t1[i, a] = np.vdot(v, c)
    for i, j, a, b in itertools.product(range(nocc), range(nocc), range(nv), range(nv)):
        v = fs.ad(nocc + a, 0) @ (fs.ad(nocc + b, 1) @ (fs.a(j, 1) @ (fs.a(i, 0) @ ref)))
        t2[i, j, a, b] = np.vdot(v, c) - t1[i, a] * t1[j, b]
    return t1, t2


def lambda_amplitudes_from_state(fs, nocc, T, psi_left_row):
    """Closed-shell Lambda1, Lambda2 with <Phi0|(1+Lambda) = <L| e^T through doubles.

    ``psi_left_row`` is the left state as a row vector normalised so that
    <L|e^T|Phi0> = 1. Coefficients are read off the alpha singles and the
    alpha-beta doubles; the caller checks the full identity.
    """
    ref, s0 = fs.reference(nocc)
    row = expm_apply(T.T, psi_left_row, +1.0)     # <L| e^T
    n = fs.nspatial
    nv = n - nocc
    l1 = np.zeros((nocc, nv), dtype=np.complex128)
    l2 = np.zeros((nocc, nocc, nv, nv), dtype=np.complex128)
    for i in range(nocc):
        for a in range(nv):
            v = fs.ad(nocc + a, 0) @ (fs.a(i, 0) @ ref)
            l1[i, a] = row @ v
    for i, j, a, b in itertools.product(range(nocc), range(nocc), range(nv), range(nv)):
        v = fs.ad(nocc + a, 0) @ (fs.ad(nocc + b, 1) @ (fs.a(j, 1) @ (fs.a(i, 0) @ ref)))
        l2[i, j, a, b] = row @ v
    return l1, l2, row
