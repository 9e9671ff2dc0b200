"""Spin-adapted closed-shell k-point EOM-IP/EA-CCSD Green's function (CPU, FP64).

Test infrastructure only (see the package docstring).

Problem statement: given orbital energies, density-fitted integrals
(p k1 q k2 | r k3 s k4) = sum_Q L[k1,k2,Q,p,q] L[k3,k4,Q,r,s] (zero unless
k1 + k3 = k2 + k4), T1/T2 and Lambda1/Lambda2 (Lambda = conj(T) by default,
the approximation of the paper's implementation section), return the k-point
CCGF G_pq(k, w) = G+ + G- of Eq. 9 with the EOM-CCSD ansatz of Eq. 8.

Formulation (derived from the spin-orbital equations of ``spinorb`` by
inserting the closed-shell spin structure; pinned against them):

* IP vector at total momentum K: r1[i] (k_i = K) and r2[ki,kj][i,j,a] with
  k_a = ki + kj - K, the amplitude of (a+_{a s} a_{j s}) a_{i alpha} summed over s.
* EA vector at K: r1[a] (k_a = K) and r2[kj,ka][j,a,b] with k_b = K + kj - ka,
  the amplitude of a+_{a alpha} (a+_{b s} a_{j s}) summed over s.
* T1 is folded into the integrals (T1 dressing); the H_bar blocks are the
  T2-only expressions in the dressed integrals.
* Sigma = connected (commutator) EOM operator; RHS b_p = P a_bar_p |Phi0>,
  left vectors e_q = <Phi0|(1+Lambda) a_bar+_q |mu> contracted with the
  spin-adapted amplitudes (Eq. 6-7).

Index conventions: k-point tensors carry three k labels, the fourth follows
from momentum conservation. Chemist ERIs g[k1,k2,k3][p,q,r,s] with
k4 = k1 - k2 + k3; t2[ki,kj,ka][i,j,a,b] with kb = ki + kj - ka; physicist
blocks W[kp,kq,kr][p,q,r,s] with ks = kp + kq - kr.
"""
import numpy as np


class KMesh:
    def __init__(self, kmesh):
        self.kmesh = tuple(int(x) for x in kmesh)
        n1, n2, n3 = self.kmesh
        self.nk = n1 * n2 * n3
        vec = [(k // (n2 * n3), (k // n3) % n2, k % n3) for k in range(self.nk)]
        idx = {v: i for i, v in enumerate(vec)}
        self.add = np.zeros((self.nk, self.nk), dtype=np.int64)
        self.sub = np.zeros((self.nk, self.nk), dtype=np.int64)
        for a in range(self.nk):
            for b in range(self.nk):
                va, vb = vec[a], vec[b]
                self.add[a, b] = idx[tuple((va[d] + vb[d]) % self.kmesh[d] for d in range(3))]
                self.sub[a, b] = idx[tuple((va[d] - vb[d]) % self.kmesh[d] for d in range(3))]

    def c(self, k1, k2, k3):
        """k1 - k2 + k3."""
        return self.add[self.sub[k1, k2], k3]


def eris_from_df(km, L):
    """g[k1,k2,k3] = sum_Q L[k1,k2,Q] (x) L[k3,k4,Q], k4 = k1 - k2 + k3."""
    nk = km.nk
    nmo = L.shape[-1]
    g = np.zeros((nk, nk, nk, nmo, nmo, nmo, nmo), dtype=np.complex128)
    for k1 in range(nk):
        for k2 in range(nk):
            for k3 in range(nk):
                k4 = km.c(k1, k2, k3)
                g[k1, k2, k3] = np.einsum('Qpq,Qrs->pqrs', L[k1, k2], L[k3, k4], optimize=True)
    return g


class KEOM:
    """Spin-adapted k-point EOM-IP/EA-CCSD operator, right-hand sides and left vectors."""

    def __init__(self, kmesh, nocc, mo_energy, t1, t2, L=None, g=None, l1=None, l2=None):
        self.km = KMesh(kmesh)
        nk = self.km.nk
        self.nk = nk
        self.nocc = o = nocc
        self.nmo = n = mo_energy.shape[1]
        self.nvir = v = n - o
        self.t1 = t1
        self.t2 = t2
        self.l1 = t1.conj() if l1 is None else l1
        self.l2 = t2.conj() if l2 is None else l2
        if g is None:
            g = eris_from_df(self.km, L)
        self._dress(mo_energy, g)
        self._intermediates()

    # ----------------------------------------------------------------- dressing
    def _dress(self, mo_energy, g):
        km, nk, o, n = self.km, self.nk, self.nocc, self.nmo
        # X = 1 - t, Y = 1 + t with t[a,i] = t1[i,a] (k-diagonal)
        X = np.zeros((nk, n, n), dtype=np.complex128)
        Y = np.zeros((nk, n, n), dtype=np.complex128)
        for k in range(nk):
            X[k] = np.eye(n)
            Y[k] = np.eye(n)
            X[k][o:, :o] = -self.t1[k].T
            Y[k][o:, :o] = self.t1[k].T
        # core Hamiltonian h = f - (2J - K) (occupied over all k), then dress it
        f = np.zeros((nk, n, n), dtype=np.complex128)
        for k in range(nk):
            f[k] = np.diag(mo_energy[k])
        h = f.copy()
        for k in range(nk):
            for kj in range(nk):
                # J: (p k q k | j kj j kj), K: (p k j kj | j kj q k)
                h[k] -= 2.0 * np.einsum('pqjj->pq', g[k, k, kj][:, :, :o, :o], optimize=True)
                h[k] += np.einsum('pjjq->pq', g[k, kj, kj][:, :o, :o, :], optimize=True)
        gd = np.zeros_like(g)
        for k1 in range(nk):
            for k2 in range(nk):
                for k3 in range(nk):
                    k4 = km.c(k1, k2, k3)
                    gd[k1, k2, k3] = np.einsum('Pp,pqrs,qQ,Rr,sS->PQRS', X[k1], g[k1, k2, k3],
                                               Y[k2], X[k3], Y[k4], optimize=True)
        fd = np.zeros_like(f)
        for k in range(nk):
            fd[k] = X[k] @ h[k] @ Y[k]
            for kj in range(nk):
                fd[k] += 2.0 * np.einsum('pqjj->pq', gd[k, k, kj][:, :, :o, :o], optimize=True)
                fd[k] -= np.einsum('pjjq->pq', gd[k, kj, kj][:, :o, :o, :], optimize=True)
        self.g = gd
        self.f = fd

    def phys(self, kp, kq, kr):
        """<p kp, q kq | r kr, s ks> = (p r | q s) block, ks = kp + kq - kr."""
        return self.g[kp, kr, kq].transpose(0, 2, 1, 3)

    # ------------------------------------------------------------ intermediates
    def _intermediates(self):
        km, nk, o = self.km, self.nk, self.nocc
        O, V = slice(0, o), slice(o, None)
        t = self.t2
        P = self.phys
        fo = [self.f[k][O, O] for k in range(nk)]
        fv = [self.f[k][V, V] for k in range(nk)]
        fov = [self.f[k][O, V] for k in range(nk)]
        self.Fov = fov
        Foo, Fvv = [], []
        for k in range(nk):
            acc = fo[k].copy()
            for kn in range(nk):
                for ke in range(nk):
                    kf = km.c(k, ke, kn)
                    mnef = P(k, kn, ke)[O, O, V, V]
                    mnfe = P(k, kn, kf)[O, O, V, V].transpose(0, 1, 3, 2)
                    acc += np.einsum('mnef,inef->mi', 2 * mnef - mnfe, t[k, kn, ke], optimize=True)
            Foo.append(acc)
            acc = fv[k].copy()
            for kmm in range(nk):
                for kn in range(nk):
                    kf = km.c(kmm, k, kn)
                    ke = k
                    mnef = P(kmm, kn, ke)[O, O, V, V]
                    mnfe = P(kmm, kn, kf)[O, O, V, V].transpose(0, 1, 3, 2)
                    acc -= np.einsum('mnef,mnaf->ae', 2 * mnef - mnfe, t[kmm, kn, k], optimize=True)
            Fvv.append(acc)
        self.Foo, self.Fvv = Foo, Fvv

        sh = lambda *s: np.zeros((nk, nk, nk) + s, dtype=np.complex128)
        v = self.nvir
        Woooo, Wvvvv = sh(o, o, o, o), sh(v, v, v, v)
        Wovvo, Wovov = sh(o, v, v, o), sh(o, v, o, v)
        Wooov, Wvovv = sh(o, o, o, v), sh(v, o, v, v)
        Wovoo, Wvvvo = sh(o, v, o, o), sh(v, v, v, o)
        for k1 in range(nk):
            for k2 in range(nk):
                for k3 in range(nk):
                    k4 = km.c(k1, k3, k2)  # k1 + k2 - k3
                    # Woooo[km,kn,ki][m,n,i,j]
                    w = P(k1, k2, k3)[O, O, O, O].copy()
                    for ke in range(nk):
                        kf = km.c(k1, ke, k2)
                        w += np.einsum('mnef,ijef->mnij', P(k1, k2, ke)[O, O, V, V], t[k3, k4, ke], optimize=True)
                    Woooo[k1, k2, k3] = w
                    # Wvvvv[ka,kb,ke][a,b,e,f]
                    w = P(k1, k2, k3)[V, V, V, V].copy()
                    for kmm in range(nk):
                        kn = km.c(k1, kmm, k2)
                        w += np.einsum('mnef,mnab->abef', P(kmm, kn, k3)[O, O, V, V], t[kmm, kn, k1], optimize=True)
                    Wvvvv[k1, k2, k3] = w
                    # Wovvo[km,kb,ke][m,b,e,j], kj = km + kb - ke
                    kmm, kb, ke, kj = k1, k2, k3, k4
                    w = P(kmm, kb, ke)[O, V, V, O].copy()
                    for kn in range(nk):
                        kf = km.c(kmm, ke, kn)
                        mnef = P(kmm, kn, ke)[O, O, V, V]
                        mnfe = P(kmm, kn, kf)[O, O, V, V].transpose(0, 1, 3, 2)
                        w += np.einsum('mnef,jnbf->mbej', 2 * mnef - mnfe, t[kj, kn, kb], optimize=True)
                        w -= np.einsum('mnef,jnfb->mbej', mnef, t[kj, kn, kf], optimize=True)
                    Wovvo[k1, k2, k3] = w
                    # Wovov[km,kb,kj][m,b,j,e], ke = km + kb - kj
                    kmm, kb, kj, ke = k1, k2, k3, k4
                    w = P(kmm, kb, kj)[O, V, O, V].copy()
                    for kn in range(nk):
                        kf = km.c(kmm, ke, kn)
                        mnfe = P(kmm, kn, kf)[O, O, V, V]
                        w -= np.einsum('mnfe,jnfb->mbje', mnfe, t[kj, kn, kf], optimize=True)
                    Wovov[k1, k2, k3] = w
                    Wooov[k1, k2, k3] = P(k1, k2, k3)[O, O, O, V]
                    Wvovv[k1, k2, k3] = P(k1, k2, k3)[V, O, V, V]
                    # Wovoo[km,kb,ki][m,b,i,j], kj = km + kb - ki
                    kmm, kb, ki, kj = k1, k2, k3, k4
                    w = P(kmm, kb, ki)[O, V, O, O].copy()
                    for ke in range(nk):
                        w += np.einsum('mbef,ijef->mbij', P(kmm, kb, ke)[O, V, V, V], t[ki, kj, ke], optimize=True)
                    w += np.einsum('me,ijeb->mbij', fov[kmm], t[ki, kj, kmm], optimize=True)
                    for kn in range(nk):
                        ke = km.c(kmm, ki, kn)
                        mnie = P(kmm, kn, ki)[O, O, O, V]
                        mnei = P(kmm, kn, ke)[O, O, V, O].transpose(0, 1, 3, 2)
                        w += np.einsum('mnie,jnbe->mbij', 2 * mnie - mnei, t[kj, kn, kb], optimize=True)
                        w -= np.einsum('mnie,jneb->mbij', mnie, t[kj, kn, ke], optimize=True)
                        ke2 = km.c(kmm, kj, kn)
                        w -= np.einsum('mnej,ineb->mbij', P(kmm, kn, ke2)[O, O, V, O], t[ki, kn, ke2], optimize=True)
                    Wovoo[k1, k2, k3] = w
                    # Wvvvo[ka,kb,ke][a,b,e,j], kj = ka + kb - ke
                    ka, kb, ke, kj = k1, k2, k3, k4
                    w = P(ka, kb, ke)[V, V, V, O].copy()
                    for kmm in range(nk):
                        kn = km.c(ka, kmm, kb)
                        w += np.einsum('mnej,mnab->abej', P(kmm, kn, ke)[O, O, V, O], t[kmm, kn, ka], optimize=True)
                    w -= np.einsum('me,mjab->abej', fov[ke], t[ke, kj, ka], optimize=True)
                    for kmm in range(nk):
                        kf = km.c(kmm, ka, kj)
                        w -= np.einsum('mbef,mjaf->abej', P(kmm, kb, ke)[O, V, V, V], t[kmm, kj, ka], optimize=True)
                        kf2 = km.c(kmm, ke, ka)
                        maef = P(kmm, ka, ke)[O, V, V, V]
                        mafe = P(kmm, ka, kf2)[O, V, V, V].transpose(0, 1, 3, 2)
                        w += np.einsum('maef,mjfb->abej', 2 * mafe - maef, t[kmm, kj, kf2], optimize=True)
                        w -= np.einsum('maef,mjbf->abej', mafe, t[kmm, kj, kb], optimize=True)
                    Wvvvo[k1, k2, k3] = w
        self.Woooo, self.Wvvvv = Woooo, Wvvvv
        self.Wovvo, self.Wovov = Wovvo, Wovov
        self.Wooov, self.Wvovv = Wooov, Wvovv
        self.Wovoo, self.Wvvvo = Wovoo, Wvvvo

    # ---------------------------------------------------------------- vectors
    def ip_dim(self):
        return self.nocc + self.nk * self.nk * self.nocc * self.nocc * self.nvir

    def ea_dim(self):
        return self.nvir + self.nk * self.nk * self.nocc * self.nvir * self.nvir

    def ip_unpack(self, x):
        o, v, nk = self.nocc, self.nvir, self.nk
        return x[:o], x[o:].reshape(nk, nk, o, o, v)

    def ea_unpack(self, x):
        o, v, nk = self.nocc, self.nvir, self.nk
        return x[:v], x[v:].reshape(nk, nk, o, v, v)

    @staticmethod
    def pack(r1, r2):
        return np.concatenate([r1.ravel(), r2.ravel()])

    # ---------------------------------------------------------------- IP sigma
    def sigma_ip(self, K, x):
        km, nk, o = self.km, self.nk, self.nocc
        O, V = slice(0, o), slice(o, None)
        P, t = self.phys, self.t2
        r1, r2 = self.ip_unpack(x)
        s1 = -self.Foo[K].T @ r1
        for kmm in range(nk):
            s1 += np.einsum('me,ime->i', self.Fov[kmm], 2 * r2[K, kmm] - r2[kmm, K].transpose(1, 0, 2), optimize=True)
            for kn in range(nk):
                ke = km.c(kmm, K, kn)
                mnie = P(kmm, kn, K)[O, O, O, V]
                mnei = P(kmm, kn, ke)[O, O, V, O].transpose(0, 1, 3, 2)
                s1 -= np.einsum('mnie,mne->i', 2 * mnie - mnei, r2[kmm, kn], optimize=True)
        s2 = np.zeros_like(r2)
        # three-body intermediate X[e], k_e = K
        X = np.zeros(self.nvir, dtype=np.complex128)
        for kmm in range(nk):
            for kn in range(nk):
                kf = km.c(kmm, K, kn)
                mnef = P(kmm, kn, K)[O, O, V, V]
                mnfe = P(kmm, kn, kf)[O, O, V, V].transpose(0, 1, 3, 2)
                X += np.einsum('mnef,mnf->e', 2 * mnef - mnfe, r2[kmm, kn], optimize=True)
        for ki in range(nk):
            for kj in range(nk):
                ka = km.c(ki, K, kj)
                acc = -np.einsum('maij,m->ija', self.Wovoo[K, ka, ki], r1, optimize=True)
                acc += np.einsum('ae,ije->ija', self.Fvv[ka], r2[ki, kj], optimize=True)
                acc -= np.einsum('mi,mja->ija', self.Foo[ki], r2[ki, kj], optimize=True)
                acc -= np.einsum('mj,ima->ija', self.Foo[kj], r2[ki, kj], optimize=True)
                for kmm in range(nk):
                    kn = km.c(ki, kmm, kj)
                    acc += np.einsum('mnij,mna->ija', self.Woooo[kmm, kn, ki], r2[kmm, kn], optimize=True)
                    acc -= np.einsum('maie,mje->ija', self.Wovov[kmm, ka, ki], r2[kmm, kj], optimize=True)
                    ke = km.c(ki, K, kmm)
                    acc += np.einsum('maej,ime->ija', self.Wovvo[kmm, ka, ke],
                                     2 * r2[ki, kmm] - r2[kmm, ki].transpose(1, 0, 2), optimize=True)
                    acc -= np.einsum('maje,ime->ija', self.Wovov[kmm, ka, kj], r2[ki, kmm], optimize=True)
                acc -= np.einsum('e,ijea->ija', X, t[ki, kj, K], optimize=True)
                s2[ki, kj] = acc
        return self.pack(s1, s2)

    # ---------------------------------------------------------------- EA sigma
    def sigma_ea(self, K, x):
        km, nk, o = self.km, self.nk, self.nocc
        O, V = slice(0, o), slice(o, None)
        P, t = self.phys, self.t2
        r1, r2 = self.ea_unpack(x)
        s1 = self.Fvv[K] @ r1
        for kmm in range(nk):
            s1 += np.einsum('me,mae->a', self.Fov[kmm], 2 * r2[kmm, K] - r2[kmm, kmm].transpose(0, 2, 1), optimize=True)
            for ke in range(nk):
                kf = km.c(K, ke, kmm)
                amef = P(K, kmm, ke)[V, O, V, V]
                amfe = P(K, kmm, kf)[V, O, V, V].transpose(0, 1, 3, 2)
                s1 += np.einsum('amef,mef->a', 2 * amef - amfe, r2[kmm, ke], optimize=True)
        Y = np.zeros(self.nocc, dtype=np.complex128)
        for kn in range(nk):
            for ke in range(nk):
                kf = km.c(K, ke, kn)
                mnef = P(K, kn, ke)[O, O, V, V]
                mnfe = P(K, kn, kf)[O, O, V, V].transpose(0, 1, 3, 2)
                Y += np.einsum('mnef,nef->m', 2 * mnef - mnfe, r2[kn, ke], optimize=True)
        s2 = np.zeros_like(r2)
        for kj in range(nk):
            for ka in range(nk):
                kb = km.c(K, ka, kj)
                acc = np.einsum('abej,e->jab', self.Wvvvo[ka, kb, K], r1, optimize=True)
                acc += np.einsum('ae,jeb->jab', self.Fvv[ka], r2[kj, ka], optimize=True)
                acc += np.einsum('be,jae->jab', self.Fvv[kb], r2[kj, ka], optimize=True)
                acc -= np.einsum('mj,mab->jab', self.Foo[kj], r2[kj, ka], optimize=True)
                for kmm in range(nk):
                    ke = km.c(K, ka, kmm)
                    acc += np.einsum('mbej,mae->jab', self.Wovvo[kmm, kb, ke],
                                     2 * r2[kmm, ka] - r2[kmm, ke].transpose(0, 2, 1), optimize=True)
                    acc -= np.einsum('mbje,mae->jab', self.Wovov[kmm, kb, kj], r2[kmm, ka], optimize=True)
                    ke2 = km.c(kmm, kj, ka)
                    acc -= np.einsum('maje,meb->jab', self.Wovov[kmm, ka, kj], r2[kmm, ke2], optimize=True)
                for ke in range(nk):
                    acc += np.einsum('abef,jef->jab', self.Wvvvv[ka, kb, ke], r2[kj, ke], optimize=True)
                acc -= np.einsum('m,mjab->jab', Y, t[K, kj, ka], optimize=True)
                s2[kj, ka] = acc
        return self.pack(s1, s2)

    # ------------------------------------------------------ RHS / left vectors
    def rhs_ip(self, K, p):
        o, v, nk = self.nocc, self.nvir, self.nk
        r1 = np.zeros(o, dtype=np.complex128)
        r2 = np.zeros((nk, nk, o, o, v), dtype=np.complex128)
        if p < o:
            r1[p] = 1.0
        else:
            a = p - o
            r1 += self.t1[K][:, a]
            for kk in range(nk):
                for kl in range(nk):
                    r2[kk, kl] = self.t2[kk, kl, K][:, :, a, :]
        return self.pack(r1, r2)

    def left_ip(self, K, q):
        km, o, v, nk = self.km, self.nocc, self.nvir, self.nk
        t, l1, l2, t1 = self.t2, self.l1, self.l2, self.t1
        e1 = np.zeros(o, dtype=np.complex128)
        e2 = np.zeros((nk, nk, o, o, v), dtype=np.complex128)

        def vir_part(c, scale, e1, e2):
            e1 += scale * l1[K][:, c]
            for ki in range(nk):
                for kj in range(nk):
                    ka = km.c(ki, K, kj)
                    e2[ki, kj] += scale * (2 * l2[ki, kj, K][:, :, c, :] - l2[ki, kj, ka][:, :, :, c])

        if q < o:
            k = q
            e1[k] = 1.0
            for kl in range(nk):
                for kc in range(nk):
                    kd = km.c(K, kc, kl)
                    tt = 2 * t[K, kl, kc][k] - t[K, kl, kd][k].transpose(0, 2, 1)
                    e1 -= np.einsum('lcd,ilcd->i', tt, l2[K, kl, kc], optimize=True)
            for kj in range(nk):
                e2[K, kj][k, :, :] += 2 * l1[kj]
            for ki in range(nk):
                e2[ki, K][:, k, :] -= l1[ki]
            for c in range(v):
                vir_part(c, -t1[K][k, c], e1, e2)
        else:
            vir_part(q - o, 1.0, e1, e2)
        return self.pack(e1, e2)

    def rhs_ea(self, K, q):
        o, v, nk = self.nocc, self.nvir, self.nk
        r1 = np.zeros(v, dtype=np.complex128)
        r2 = np.zeros((nk, nk, o, v, v), dtype=np.complex128)
        if q >= o:
            r1[q - o] = 1.0
        else:
            k = q
            r1 -= self.t1[K][k, :]
            for kl in range(nk):
                for kc in range(nk):
                    r2[kl, kc] = -self.t2[K, kl, kc][k]
        return self.pack(r1, r2)

    def left_ea(self, K, p):
        km, o, v, nk = self.km, self.nocc, self.nvir, self.nk
        t, l1, l2, t1 = self.t2, self.l1, self.l2, self.t1
        e1 = np.zeros(v, dtype=np.complex128)
        e2 = np.zeros((nk, nk, o, v, v), dtype=np.complex128)

        def occ_part(i, scale, e1, e2):
            e1 -= scale * l1[K][i, :]
            for kj in range(nk):
                for ka in range(nk):
                    e2[kj, ka] += scale * (l2[kj, K, ka][:, i, :, :] - 2 * l2[K, kj, ka][i])

        if p < o:
            occ_part(p, 1.0, e1, e2)
        else:
            c = p - o
            e1[c] = 1.0
            for kk in range(nk):
                for kl in range(nk):
                    kd = km.c(kk, K, kl)
                    ll = 2 * l2[kk, kl, K] - l2[kl, kk, K].transpose(1, 0, 2, 3)
                    e1 -= np.einsum('kld,klad->a', t[kk, kl, K][:, :, c, :], ll, optimize=True)
            for kj in range(nk):
                # k_a = K term, then k_b = K term (k_a = kj)
                e2[kj, K][:, c, :] += 2 * l1[kj]
                e2[kj, kj][:, :, c] -= l1[kj]
            for k in range(o):
                occ_part(k, t1[K][k, c], e1, e2)
        return self.pack(e1, e2)

    # ---------------------------------------------------------- dense matrices
    def matrix(self, kind, K):
        D = self.ip_dim() if kind == "ip" else self.ea_dim()
        sig = self.sigma_ip if kind == "ip" else self.sigma_ea
        A = np.zeros((D, D), dtype=np.complex128)
        for j in range(D):
            e = np.zeros(D, dtype=np.complex128)
            e[j] = 1.0
            A[:, j] = sig(K, e)
        return A

    def diagonal(self, kind, K):
        """Exact diagonal of the EOM matrix (by unit vectors; tiny systems only)."""
        return np.diag(self.matrix(kind, K)).copy()


def diag_estimate(ke, kind, K):
    """One-body part of diag(A) at total momentum K (a preconditioner; it does not change the solution).

    IP: r1[i] -> -Foo_ii,  r2[ki,kj][i,j,a] -> Fvv_aa - Foo_ii - Foo_jj;
    EA: r1[a] -> Fvv_aa,   r2[kj,ka][j,a,b] -> Fvv_aa + Fvv_bb - Foo_jj.
    """
    km, nk, o, v = ke.km, ke.nk, ke.nocc, ke.nvir
    foo = [np.real(np.diag(ke.Foo[k])) for k in range(nk)]
    fvv = [np.real(np.diag(ke.Fvv[k])) for k in range(nk)]
    if kind == "ip":
        d2 = np.zeros((nk, nk, o, o, v))
        for ki in range(nk):
            for kj in range(nk):
                ka = km.c(ki, K, kj)
                d2[ki, kj] = fvv[ka][None, None, :] - foo[ki][:, None, None] - foo[kj][None, :, None]
        return np.concatenate([-foo[K], d2.ravel()])
    d2 = np.zeros((nk, nk, o, v, v))
    for kj in range(nk):
        for ka in range(nk):
            kb = km.c(K, ka, kj)
            d2[kj, ka] = fvv[ka][None, :, None] + fvv[kb][None, None, :] - foo[kj][:, None, None]
    return np.concatenate([fvv[K], d2.ravel()])
