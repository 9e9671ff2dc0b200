"""Spin-orbital EOM-IP/EA-CCSD for a molecule (or a k-point supercell).

Test infrastructure only (see the package docstring).

The EOM spaces are those of Eq. 8 (1h + 2h1p, 1p + 2p1h); the operator is the
connected similarity-transformed Hamiltonian of Eq. 5 restricted to them.
T1 enters through the similarity transformation of the Hamiltonian alone:
e^-T1 a+_p e^T1 = sum_r a+_r X_rp and e^-T1 a_q e^T1 = sum_s Y_qs a_s with
X = 1 - t and Y = 1 + t (t[a,i] = t1[i,a]), so H_bar = e^-T2 H~ e^T2 where H~
carries the dressed one- and two-electron integrals. The blocks of H_bar below
are then the T1 = 0 expressions in the dressed integrals.

Spin-orbital index = 2*p + s, occupied spin-orbitals first within each block;
R_IP = sum r1[I] a_I + 1/2 sum r2[I,J,A] a+_A a_J a_I,
R_EA = sum r1[A] a+_A + 1/2 sum r2[J,A,B] a+_A a+_B a_J,
r2 antisymmetric in its pair. v[P,Q,R,S] = <PQ||RS> (dressed).
"""
import numpy as np


def dress(f, g, t1, nocc):
    """T1-dressed Fock matrix and ERIs (spatial, closed shell).

    h = f - (2J - K) is the core Hamiltonian that makes f the reference Fock
    matrix; the dressed Fock matrix is h~ + 2J~ - K~ over the occupied orbitals.
    """
    n = f.shape[0]
    nv = n - nocc
    t = np.zeros((n, n), dtype=np.complex128)
    t[nocc:, :nocc] = t1.T
    X = np.eye(n) - t
    Y = np.eye(n) + t
    J = np.einsum('pqii->pq', g[:, :, :nocc, :nocc])
    K = np.einsum('piiq->pq', g[:, :nocc, :nocc, :])
    h = f - 2.0 * J + K
    hd = X @ h @ Y
    gd = np.einsum('Pp,pqrs,qQ,Rr,sS->PQRS', X, g, Y, X, Y, optimize=True)
    Jd = np.einsum('pqii->pq', gd[:, :, :nocc, :nocc])
    Kd = np.einsum('piiq->pq', gd[:, :nocc, :nocc, :])
    fd = hd + 2.0 * Jd - Kd
    return fd, gd, X, Y


def spin_blocks(fd, gd, nocc):
    """Spin-orbital Fock matrix and antisymmetrised <PQ||RS> from spatial arrays."""
    n = fd.shape[0]
    ns = 2 * n
    # spin-orbital ordering: occupied (2*i+s), then virtual (2*(nocc + a)+s)
    spat = np.arange(ns) // 2
    spin = np.arange(ns) % 2
    F = fd[np.ix_(spat, spat)] * (spin[:, None] == spin[None, :])
    same = (spin[:, None] == spin[None, :])
    chem = gd[np.ix_(spat, spat, spat, spat)] * same[:, :, None, None] * same[None, None, :, :]
    phys = chem.transpose(0, 2, 1, 3)          # <PQ|RS> = (PR|QS)
    v = phys - phys.transpose(0, 1, 3, 2)
    return F, v


def t2_spinorb(t2, nocc_sp):
    """t_{IJ}^{AB} from closed-shell t2[i,j,a,b] (alpha-beta amplitude)."""
    no, _, nv, _ = t2.shape
    O, V = 2 * no, 2 * nv
    so = np.arange(O) % 2
    sv = np.arange(V) % 2
    io = np.arange(O) // 2
    iv = np.arange(V) // 2
    T = t2[np.ix_(io, io, iv, iv)]
    Tx = t2[np.ix_(io, io, iv, iv)].transpose(0, 1, 3, 2)   # t[i,j,b,a]
    d1 = (so[:, None, None, None] == sv[None, None, :, None]) & (so[None, :, None, None] == sv[None, None, None, :])
    d2 = (so[:, None, None, None] == sv[None, None, None, :]) & (so[None, :, None, None] == sv[None, None, :, None])
    return T * d1 - Tx * d2


def t1_spinorb(t1):
    no, nv = t1.shape
    so = np.arange(2 * no) % 2
    sv = np.arange(2 * nv) % 2
    return t1[np.ix_(np.arange(2 * no) // 2, np.arange(2 * nv) // 2)] * (so[:, None] == sv[None, :])


class SpinOrbitalEOM:
    def __init__(self, f, g, nocc, t1, t2, l1, l2):
        """f, g: spatial Fock (diag of reference) and chemist ERIs; nocc spatial."""
        self.nocc_sp = nocc
        fd, gd, X, Y = dress(f, g, t1, nocc)
        F, v = spin_blocks(fd, gd, nocc)
        O = 2 * nocc
        self.O = O
        self.V = F.shape[0] - O
        o, w = slice(0, O), slice(O, None)
        self.f_oo, self.f_ov, self.f_vv = F[o, o], F[o, w], F[w, w]
        self.v = v
        self.t2 = t2_spinorb(t2, nocc)
        self.t1 = t1_spinorb(t1)
        self.l1 = t1_spinorb(l1)
        self.l2 = t2_spinorb(l2, nocc)     # l2[I,J,A,B] = lambda_{AB}^{IJ}
        self._intermediates(o, w)

    def _intermediates(self, o, w):
        v, t = self.v, self.t2
        self.v_oovv = v[o, o, w, w]
        self.Foo = self.f_oo + 0.5 * np.einsum('mnef,inef->mi', v[o, o, w, w], t)
        self.Fvv = self.f_vv - 0.5 * np.einsum('mnef,mnaf->ae', v[o, o, w, w], t)
        self.Fov = self.f_ov.copy()
        self.Woooo = v[o, o, o, o] + 0.5 * np.einsum('mnef,ijef->mnij', v[o, o, w, w], t)
        self.Wvvvv = v[w, w, w, w] + 0.5 * np.einsum('mnef,mnab->abef', v[o, o, w, w], t)
        self.Wovvo = v[o, w, w, o] - np.einsum('mnef,jnfb->mbej', v[o, o, w, w], t)
        self.Wooov = v[o, o, o, w].copy()
        self.Wvovv = v[w, o, w, w].copy()
        tmp = np.einsum('mnie,jnbe->mbij', v[o, o, o, w], t)
        self.Wovoo = (v[o, w, o, o] + 0.5 * np.einsum('mbef,ijef->mbij', v[o, w, w, w], t)
                      - np.einsum('me,ijbe->mbij', self.Fov, t) + tmp - tmp.transpose(0, 1, 3, 2))
        tmp = np.einsum('mbef,miaf->abei', v[o, w, w, w], t)
        self.Wvvvo = (v[w, w, w, o] + 0.5 * np.einsum('mnei,mnab->abei', v[o, o, w, o], t)
                      - np.einsum('me,miab->abei', self.Fov, t) - tmp + tmp.transpose(1, 0, 2, 3))

    # ---------------- IP -----------------
    def sigma_ip(self, r1, r2):
        s1 = (-np.einsum('mi,m->i', self.Foo, r1)
              + np.einsum('me,ime->i', self.Fov, r2)
              - 0.5 * np.einsum('mnie,mne->i', self.Wooov, r2))
        s2 = -np.einsum('maij,m->ija', self.Wovoo, r1)
        s2 += np.einsum('ae,ije->ija', self.Fvv, r2)
        tmp = np.einsum('mi,mja->ija', self.Foo, r2)
        s2 -= tmp - tmp.transpose(1, 0, 2)
        s2 += 0.5 * np.einsum('mnij,mna->ija', self.Woooo, r2)
        tmp = np.einsum('maei,mje->ija', self.Wovvo, r2)
        s2 += tmp - tmp.transpose(1, 0, 2)
        s2 += 0.5 * np.einsum("mnef,mnf,ijae->ija", self.v_oovv, r2, self.t2)
        return s1, s2

    def rhs_ip(self, p):
        """b for a_p (spin-orbital p over occ then vir)."""
        O, V = self.O, self.V
        r1 = np.zeros(O, dtype=np.complex128)
        r2 = np.zeros((O, O, V), dtype=np.complex128)
        if p < O:
            r1[p] = 1.0
        else:
            a = p - O
            r1 += self.t1[:, a]
            r2 += self.t2[:, :, a, :]
        return r1, r2

    def left_ip(self, q):
        """e for a+_q: e[mu] = <0|(1+L) e^-T a+_q e^T|mu>."""
        O, V = self.O, self.V

        def e_occ(k):
            e1 = np.zeros(O, dtype=np.complex128)
            e1[k] = 1.0
            e1 -= 0.5 * np.einsum('lcd,cdil->i', self.t2[k], self.l2.transpose(2, 3, 0, 1))
            e2 = np.zeros((O, O, V), dtype=np.complex128)
            e2[k, :, :] += self.l1
            e2[:, k, :] -= self.l1
            return e1, e2

        def e_vir(c):
            e1 = self.l1[:, c].copy()
            e2 = self.l2[:, :, c, :].copy()
            return e1, e2

        if q < O:
            e1, e2 = e_occ(q)
            for c in range(V):
                if self.t1[q, c] != 0:
                    f1, f2 = e_vir(c)
                    e1 = e1 - self.t1[q, c] * f1
                    e2 = e2 - self.t1[q, c] * f2
            return e1, e2
        return e_vir(q - O)

    # ---------------- EA -----------------
    def sigma_ea(self, r1, r2):
        s1 = (np.einsum('ae,e->a', self.Fvv, r1)
              + np.einsum('me,mae->a', self.Fov, r2)
              + 0.5 * np.einsum('amef,mef->a', self.Wvovv, r2))
        s2 = np.einsum('abej,e->jab', self.Wvvvo, r1)
        tmp = np.einsum('ae,jeb->jab', self.Fvv, r2)
        s2 += tmp - tmp.transpose(0, 2, 1)
        s2 -= np.einsum('mj,mab->jab', self.Foo, r2)
        tmp = np.einsum('mbej,mae->jab', self.Wovvo, r2)
        s2 += tmp - tmp.transpose(0, 2, 1)
        s2 += 0.5 * np.einsum('abef,jef->jab', self.Wvvvv, r2)
        s2 -= 0.5 * np.einsum('mnef,nef,mjab->jab', self.v_oovv, r2, self.t2)
        return s1, s2

    def rhs_ea(self, q):
        """b for a+_q."""
        O, V = self.O, self.V
        r1 = np.zeros(V, dtype=np.complex128)
        r2 = np.zeros((O, V, V), dtype=np.complex128)
        if q >= O:
            r1[q - O] = 1.0
        else:
            k = q
            r1 -= self.t1[k, :]
            r2 += self.t2[:, k, :, :]
        return r1, r2

    def left_ea(self, p):
        """e for a_p: e[mu] = <0|(1+L) e^-T a_p e^T|mu>."""
        O, V = self.O, self.V

        def e_occ(i):
            e1 = -self.l1[i, :].copy()
            e2 = self.l2[:, i, :, :].copy()
            return e1, e2

        def e_vir(c):
            e1 = np.zeros(V, dtype=np.complex128)
            e1[c] = 1.0
            e1 += 0.5 * np.einsum('kld,klda->a', self.t2[:, :, c, :], self.l2)
            e2 = np.zeros((O, V, V), dtype=np.complex128)
            e2[:, c, :] += self.l1
            e2[:, :, c] -= self.l1
            return e1, e2

        if p < O:
            return e_occ(p)
        c = p - O
        e1, e2 = e_vir(c)
        for k in range(O):
            if self.t1[k, c] != 0:
                f1, f2 = e_occ(k)
                e1 = e1 + self.t1[k, c] * f1
                e2 = e2 + self.t1[k, c] * f2
        return e1, e2

    # ------------- packing into the determinant order of the brute force -------------
    def pack_ip(self, r1, r2):
        O = self.O
        out = [r1]
        for I in range(O):
            for J in range(I + 1, O):
                out.append(r2[I, J, :])
        return np.concatenate(out)

    def unpack_ip(self, x):
        O, V = self.O, self.V
        r1 = x[:O].copy()
        r2 = np.zeros((O, O, V), dtype=np.complex128)
        pos = O
        for I in range(O):
            for J in range(I + 1, O):
                r2[I, J] = x[pos:pos + V]
                r2[J, I] = -x[pos:pos + V]
                pos += V
        return r1, r2

    def pack_ea(self, r1, r2):
        V = self.V
        out = [r1]
        for A in range(V):
            for B in range(A + 1, V):
                out.append(r2[:, A, B])
        return np.concatenate(out)

    def unpack_ea(self, x):
        O, V = self.O, self.V
        r1 = x[:V].copy()
        r2 = np.zeros((O, V, V), dtype=np.complex128)
        pos = V
        for A in range(V):
            for B in range(A + 1, V):
                r2[:, A, B] = x[pos:pos + O]
                r2[:, B, A] = -x[pos:pos + O]
                pos += O
        return r1, r2

    def matrix(self, kind):
        """Dense EOM matrix in packed determinant order (for tests and tiny solves)."""
        if kind == "ip":
            O, V = self.O, self.V
            D = O + O * (O - 1) // 2 * V
            unpack, sig, pack = self.unpack_ip, self.sigma_ip, self.pack_ip
        else:
            O, V = self.O, self.V
            D = V + V * (V - 1) // 2 * O
            unpack, sig, pack = self.unpack_ea, self.sigma_ea, self.pack_ea
        A = np.zeros((D, D), dtype=np.complex128)
        for j in range(D):
            e = np.zeros(D, dtype=np.complex128)
            e[j] = 1.0
            A[:, j] = pack(*sig(*unpack(e)))
        return A

    def greens_function(self, omegas, eta, sectors=("ip", "ea")):
        """G[w,p,q] over spatial orbitals (alpha spin), dense solves (Eq. 6-7)."""
        nsp = (self.O + self.V) // 2
        G = np.zeros((len(omegas), nsp, nsp), dtype=np.complex128)
        alpha = [2 * p for p in range(nsp)]   # spin-orbital index of p alpha in occ-then-vir order
        for kind in sectors:
            A = self.matrix(kind)
            D = A.shape[0]
            if kind == "ip":
                B = np.stack([self.pack_ip(*self.rhs_ip(P)) for P in alpha], axis=1)
                E = np.stack([self.pack_ip(*self.left_ip(P)) for P in alpha], axis=0)
            else:
                B = np.stack([self.pack_ea(*self.rhs_ea(P)) for P in alpha], axis=1)
                E = np.stack([self.pack_ea(*self.left_ea(P)) for P in alpha], axis=0)
            for w, om in enumerate(omegas):
                if kind == "ip":
                    X = np.linalg.solve((om - 1j * eta) * np.eye(D) + A, B)
                    G[w] += (E @ X).T
                else:
                    Y = np.linalg.solve((om + 1j * eta) * np.eye(D) - A, B)
                    G[w] += E @ Y
        return G
