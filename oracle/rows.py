"""Selected elements of the EOM-IP/EA-CCSD sigma vectors for systems too large for ``kccsd``.

Test infrastructure only (see the package docstring).

``KEOM`` forms every integral block and every H_bar block, which at a 3x3x3 mesh with 30
virtuals per k (or a 2x2x2 mesh with 18 / 60) would take hundreds of GB. ``KRows`` evaluates the
same operator (the spin-adapted sigma of ``kccsd``, Eq. 8 spaces, H_bar of Eq. 5 in the T1-dressed
integrals) one output element at a time: every H_bar element an output needs is formed from its
definition with the integrals <p q|r s> = (p r|q s) = sum_Q L~[kp,kr,Q][p,r] L~[kq,ks,Q][q,s]
taken from the dressed density-fitting factors. The only stored four-index quantity is the
<m n|e f> block (nk^3 o^2 v^2), an integral block by definition. The formulas are those of
``kccsd.KEOM._intermediates`` / ``sigma_ip`` / ``sigma_ea`` restricted to the requested output
indices; ``tests/test_oracle_pins.py`` checks element by element that both give the same numbers.
"""
import numpy as np

from oracle.kccsd import KMesh


class KRows:
    def __init__(self, kmesh, nocc, mo_energy, t1, t2, L, l1=None, l2=None):
        self.km = km = KMesh(kmesh)
        self.nk = nk = km.nk
        self.nocc = o = nocc
        self.nmo = n = mo_energy.shape[1]
        self.nvir = n - o
        self.t1, self.t2 = t1, t2
        self._l1, self._l2 = l1, l2
        O, V = slice(0, o), slice(o, None)
        # dressing X = 1 - t, Y = 1 + t (t[a,i] = t1[i,a]) applied to the factors: L~ = X L Y
        X = np.zeros((nk, n, n), dtype=np.complex128)
        Y = np.zeros((nk, n, n), dtype=np.complex128)
        for k in range(nk):
            X[k] = np.eye(n)
            Y[k] = np.eye(n)
            X[k][o:, :o] = -t1[k].T
            Y[k][o:, :o] = t1[k].T
        Ld = np.zeros_like(L)
        for k1 in range(nk):
            for k2 in range(nk):
                Ld[k1, k2] = np.einsum('Pp,Qpq,qR->QPR', X[k1], L[k1, k2], Y[k2], optimize=True)
        self.Ld = Ld
        # core Hamiltonian h = f - (2J - K) over the occupied orbitals of every k, from the bare factors
        f = np.zeros((nk, n, n), dtype=np.complex128)
        for k in range(nk):
            f[k] = np.diag(mo_energy[k])
        h = f.copy()
        for k in range(nk):
            for kj in range(nk):
                h[k] -= 2.0 * np.einsum('Qpq,Qjj->pq', L[k, k], L[kj, kj][:, :o, :o], optimize=True)
                h[k] += np.einsum('Qpj,Qjq->pq', L[k, kj][:, :, :o], L[kj, k][:, :o, :], optimize=True)
        fd = np.zeros_like(f)
        for k in range(nk):
            fd[k] = X[k] @ h[k] @ Y[k]
            for kj in range(nk):
                fd[k] += 2.0 * np.einsum('Qpq,Qjj->pq', Ld[k, k], Ld[kj, kj][:, :o, :o], optimize=True)
                fd[k] -= np.einsum('Qpj,Qjq->pq', Ld[k, kj][:, :, :o], Ld[kj, k][:, :o, :], optimize=True)
        self.fov = [fd[k][O, V] for k in range(nk)]
        # <m n|e f> [km][kn][ke], kf = km + kn - ke
        oovv = np.zeros((nk, nk, nk, o, o, self.nvir, self.nvir), dtype=np.complex128)
        for kmm in range(nk):
            for kn in range(nk):
                for ke in range(nk):
                    kf = km.c(kmm, ke, kn)
                    oovv[kmm, kn, ke] = np.einsum('Qme,Qnf->mnef', Ld[kmm, ke][:, O, V], Ld[kn, kf][:, O, V], optimize=True)
        self.oovv = oovv
        t = t2
        self.Foo, self.Fvv = [], []
        for k in range(nk):
            acc = fd[k][O, O].copy()
            for kn in range(nk):
                for ke in range(nk):
                    kf = km.c(k, ke, kn)
                    acc += np.einsum('mnef,inef->mi', 2 * oovv[k, kn, ke] - oovv[k, kn, kf].transpose(0, 1, 3, 2), t[k, kn, ke],
                                     optimize=True)
            self.Foo.append(acc)
            acc = fd[k][V, V].copy()
            for kmm in range(nk):
                for kn in range(nk):
                    kf = km.c(kmm, k, kn)
                    acc -= np.einsum('mnef,mnaf->ae', 2 * oovv[kmm, kn, k] - oovv[kmm, kn, kf].transpose(0, 1, 3, 2),
                                     t[kmm, kn, k], optimize=True)
            self.Fvv.append(acc)

    # ---------------------------------------------------------------- integrals
    def P(self, kp, kq, kr, p, q, r, s):
        """<p kp, q kq | r kr, s ks> for the index ranges / lists p, q, r, s (ks = kp + kq - kr)."""
        ks = self.km.c(kp, kr, kq)
        A = self.Ld[kp, kr][:, p][:, :, r]
        B = self.Ld[kq, ks][:, q][:, :, s]
        return np.einsum('Qpr,Qqs->pqrs', A, B, optimize=True)

    def _ix(self, part, idx=None):
        o = self.nocc
        if part == 'o':
            return np.arange(o) if idx is None else np.atleast_1d(idx)
        return (o + np.arange(self.nvir)) if idx is None else o + np.atleast_1d(idx)

    def g(self, kp, kq, kr, pp, qq, rr, ss):
        """<p q|r s> with each index given as ('o'|'v', None for the whole range or an index)."""
        return self.P(kp, kq, kr, self._ix(*pp), self._ix(*qq), self._ix(*rr), self._ix(*ss))

    # ---------------------------------------------------------------- H_bar slices
    def Wvvvv(self, ka, kb, ke, a, b):
        """W[ka,kb,ke][a,b,:,:] = <ab|ef> + sum_{km,m,n} <mn|ef> t[km,kn,ka][m,n,a,b]."""
        km_, t = self.km, self.t2
        w = self.g(ka, kb, ke, ('v', a), ('v', b), ('v', None), ('v', None))[0, 0]
        for kmm in range(self.nk):
            kn = km_.c(ka, kmm, kb)
            w = w + np.einsum('mnef,mn->ef', self.oovv[kmm, kn, ke], t[kmm, kn, ka][:, :, a, b], optimize=True)
        return w

    def Wovvo(self, kmm, kb, ke, b, j):
        """W[km,kb,ke][:, b, :, j] (kj = km + kb - ke)."""
        km_, t, nk = self.km, self.t2, self.nk
        kj = km_.c(kmm, ke, kb)
        w = self.g(kmm, kb, ke, ('o', None), ('v', b), ('v', None), ('o', j))[:, 0, :, 0]
        for kn in range(nk):
            kf = km_.c(kmm, ke, kn)
            mnef = self.oovv[kmm, kn, ke]
            mnfe = self.oovv[kmm, kn, kf].transpose(0, 1, 3, 2)
            w = w + np.einsum('mnef,nf->me', 2 * mnef - mnfe, t[kj, kn, kb][j, :, b, :], optimize=True)
            w = w - np.einsum('mnef,nf->me', mnef, t[kj, kn, kf][j, :, :, b], optimize=True)
        return w

    def Wovov(self, kmm, kb, kj, b, j):
        """W[km,kb,kj][:, b, j, :] (ke = km + kb - kj)."""
        km_, t, nk = self.km, self.t2, self.nk
        ke = km_.c(kmm, kj, kb)
        w = self.g(kmm, kb, kj, ('o', None), ('v', b), ('o', j), ('v', None))[:, 0, 0, :]
        for kn in range(nk):
            kf = km_.c(kmm, ke, kn)
            w = w - np.einsum('mnfe,nf->me', self.oovv[kmm, kn, kf], t[kj, kn, kf][j, :, :, b], optimize=True)
        return w

    def Wvvvo(self, ka, kb, ke, a, b, j):
        """W[ka,kb,ke][a, b, :, j] (kj = ka + kb - ke)."""
        km_, t, nk = self.km, self.t2, self.nk
        kj = km_.c(ka, ke, kb)
        w = self.g(ka, kb, ke, ('v', a), ('v', b), ('v', None), ('o', j))[0, 0, :, 0]
        for kmm in range(nk):
            kn = km_.c(ka, kmm, kb)
            w = w + np.einsum('mne,mn->e', self.g(kmm, kn, ke, ('o', None), ('o', None), ('v', None), ('o', j))[:, :, :, 0],
                              t[kmm, kn, ka][:, :, a, b], optimize=True)
        w = w - np.einsum('me,m->e', self.fov[ke], t[ke, kj, ka][:, j, a, b], optimize=True)
        for kmm in range(nk):
            w = w - np.einsum('mef,mf->e', self.g(kmm, kb, ke, ('o', None), ('v', b), ('v', None), ('v', None))[:, 0],
                              t[kmm, kj, ka][:, j, a, :], optimize=True)
            kf2 = km_.c(kmm, ke, ka)
            maef = self.g(kmm, ka, ke, ('o', None), ('v', a), ('v', None), ('v', None))[:, 0]
            mafe = self.g(kmm, ka, kf2, ('o', None), ('v', a), ('v', None), ('v', None))[:, 0].transpose(0, 2, 1)
            w = w + np.einsum('mef,mf->e', 2 * mafe - maef, t[kmm, kj, kf2][:, j, :, b], optimize=True)
            w = w - np.einsum('mef,mf->e', mafe, t[kmm, kj, kb][:, j, b, :], optimize=True)
        return w

    def Woooo(self, kmm, kn, ki, i, j):
        """W[km,kn,ki][:, :, i, j] (kj = km + kn - ki)."""
        km_, t, nk = self.km, self.t2, self.nk
        kj = km_.c(kmm, ki, kn)
        w = self.g(kmm, kn, ki, ('o', None), ('o', None), ('o', i), ('o', j))[:, :, 0, 0]
        for ke in range(nk):
            w = w + np.einsum('mnef,ef->mn', self.oovv[kmm, kn, ke], t[ki, kj, ke][i, j], optimize=True)
        return w

    def Wovoo(self, kmm, kb, ki, b, i, j):
        """W[km,kb,ki][:, b, i, j] (kj = km + kb - ki)."""
        km_, t, nk, o = self.km, self.t2, self.nk, self.nocc
        kj = km_.c(kmm, ki, kb)
        w = self.g(kmm, kb, ki, ('o', None), ('v', b), ('o', i), ('o', j))[:, 0, 0, 0]
        for ke in range(nk):
            w = w + np.einsum('mef,ef->m', self.g(kmm, kb, ke, ('o', None), ('v', b), ('v', None), ('v', None))[:, 0],
                              t[ki, kj, ke][i, j], optimize=True)
        w = w + np.einsum('me,e->m', self.fov[kmm], t[ki, kj, kmm][i, j, :, b], optimize=True)
        for kn in range(nk):
            ke = km_.c(kmm, ki, kn)
            mnie = self.g(kmm, kn, ki, ('o', None), ('o', None), ('o', i), ('v', None))[:, :, 0, :]
            mnei = self.g(kmm, kn, ke, ('o', None), ('o', None), ('v', None), ('o', i))[:, :, :, 0]
            w = w + np.einsum('mne,ne->m', 2 * mnie - mnei, t[kj, kn, kb][j, :, b, :], optimize=True)
            w = w - np.einsum('mne,ne->m', mnie, t[kj, kn, ke][j, :, :, b], optimize=True)
            ke2 = km_.c(kmm, kj, kn)
            w = w - np.einsum('mne,ne->m', self.g(kmm, kn, ke2, ('o', None), ('o', None), ('v', None), ('o', j))[:, :, :, 0],
                              t[ki, kn, ke2][i, :, :, b], optimize=True)
        return w

    # ---------------------------------------------------------------- vectors
    def ea_unpack(self, x):
        o, v, nk = self.nocc, self.nvir, self.nk
        return x[:v], x[v:].reshape(nk, nk, o, v, v)

    def ip_unpack(self, x):
        o, v, nk = self.nocc, self.nvir, self.nk
        return x[:o], x[o:].reshape(nk, nk, o, o, v)

    def ea_index(self, mu):
        """(kj, ka, j, a, b) of EA vector element mu >= nvir."""
        o, v, nk = self.nocc, self.nvir, self.nk
        return np.unravel_index(mu - v, (nk, nk, o, v, v))

    def ip_index(self, mu):
        o, v, nk = self.nocc, self.nvir, self.nk
        return np.unravel_index(mu - o, (nk, nk, o, o, v))

    def sigma_ea_elements(self, K, x, mus):
        """(A_EA x)[mu] for the listed mu (Eq. 8 addition part, the formulas of kccsd.sigma_ea)."""
        km_, nk, t = self.km, self.nk, self.t2
        r1, r2 = self.ea_unpack(x)
        out = []
        Ym = None
        for mu in mus:
            mu = int(mu)
            if mu < self.nvir:
                a = mu
                val = self.Fvv[K][a] @ r1
                for kmm in range(nk):
                    val += np.einsum('me,me->', self.fov[kmm], 2 * r2[kmm, K][:, a, :] - r2[kmm, kmm][:, :, a], optimize=True)
                    for ke in range(nk):
                        kf = km_.c(K, ke, kmm)
                        amef = self.g(K, kmm, ke, ('v', a), ('o', None), ('v', None), ('v', None))[0]
                        amfe = self.g(K, kmm, kf, ('v', a), ('o', None), ('v', None), ('v', None))[0].transpose(0, 2, 1)
                        val += np.einsum('mef,mef->', 2 * amef - amfe, r2[kmm, ke], optimize=True)
                out.append(val)
                continue
            kj, ka, j, a, b = (int(z) for z in self.ea_index(mu))
            kb = km_.c(K, ka, kj)
            val = self.Wvvvo(ka, kb, K, a, b, j) @ r1
            val += self.Fvv[ka][a] @ r2[kj, ka][j, :, b]
            val += self.Fvv[kb][b] @ r2[kj, ka][j, a, :]
            val -= self.Foo[kj][:, j] @ r2[kj, ka][:, a, b]
            for kmm in range(nk):
                ke = km_.c(K, ka, kmm)
                val += np.einsum('me,me->', self.Wovvo(kmm, kb, ke, b, j), 2 * r2[kmm, ka][:, a, :] - r2[kmm, ke][:, :, a])
                val -= np.einsum('me,me->', self.Wovov(kmm, kb, kj, b, j), r2[kmm, ka][:, a, :])
                ke2 = km_.c(kmm, kj, ka)
                val -= np.einsum('me,me->', self.Wovov(kmm, ka, kj, a, j), r2[kmm, ke2][:, :, b])
            for ke in range(nk):
                val += np.einsum('ef,ef->', self.Wvvvv(ka, kb, ke, a, b), r2[kj, ke][j])
            if Ym is None:
                Ym = np.zeros(self.nocc, dtype=np.complex128)
                for kn in range(nk):
                    for ke in range(nk):
                        kf = km_.c(K, ke, kn)
                        mnef = self.oovv[K, kn, ke]
                        mnfe = self.oovv[K, kn, kf].transpose(0, 1, 3, 2)
                        Ym += np.einsum('mnef,nef->m', 2 * mnef - mnfe, r2[kn, ke], optimize=True)
            val -= Ym @ t[K, kj, ka][:, j, a, b]
            out.append(val)
        return np.array(out)

    def sigma_ip_elements(self, K, x, mus):
        """(A_IP x)[mu] for the listed mu (Eq. 8 removal part, the formulas of kccsd.sigma_ip)."""
        km_, nk, t = self.km, self.nk, self.t2
        r1, r2 = self.ip_unpack(x)
        out = []
        Xe = None
        for mu in mus:
            mu = int(mu)
            if mu < self.nocc:
                i = mu
                val = -self.Foo[K][:, i] @ r1
                for kmm in range(nk):
                    val += np.einsum('me,me->', self.fov[kmm], 2 * r2[K, kmm][i] - r2[kmm, K][:, i, :], optimize=True)
                    for kn in range(nk):
                        ke = km_.c(kmm, K, kn)
                        mnie = self.g(kmm, kn, K, ('o', None), ('o', None), ('o', i), ('v', None))[:, :, 0, :]
                        mnei = self.g(kmm, kn, ke, ('o', None), ('o', None), ('v', None), ('o', i))[:, :, :, 0]
                        val -= np.einsum('mne,mne->', 2 * mnie - mnei, r2[kmm, kn], optimize=True)
                out.append(val)
                continue
            ki, kj, i, j, a = (int(z) for z in self.ip_index(mu))
            ka = km_.c(ki, K, kj)
            val = -self.Wovoo(K, ka, ki, a, i, j) @ r1
            val += self.Fvv[ka][a] @ r2[ki, kj][i, j, :]
            val -= self.Foo[ki][:, i] @ r2[ki, kj][:, j, a]
            val -= self.Foo[kj][:, j] @ r2[ki, kj][i, :, a]
            for kmm in range(nk):
                kn = km_.c(ki, kmm, kj)
                val += np.einsum('mn,mn->', self.Woooo(kmm, kn, ki, i, j), r2[kmm, kn][:, :, a])
                val -= np.einsum('me,me->', self.Wovov(kmm, ka, ki, a, i), r2[kmm, kj][:, j, :])
                ke = km_.c(ki, K, kmm)
                val += np.einsum('me,me->', self.Wovvo(kmm, ka, ke, a, j), 2 * r2[ki, kmm][i] - r2[kmm, ki][:, i, :])
                val -= np.einsum('me,me->', self.Wovov(kmm, ka, kj, a, j), r2[ki, kmm][i])
            if Xe is None:
                Xe = np.zeros(self.nvir, dtype=np.complex128)
                for kmm in range(nk):
                    for kn in range(nk):
                        kf = km_.c(kmm, K, kn)
                        mnef = self.oovv[kmm, kn, K]
                        mnfe = self.oovv[kmm, kn, kf].transpose(0, 1, 3, 2)
                        Xe += np.einsum('mnef,mnf->e', 2 * mnef - mnfe, r2[kmm, kn], optimize=True)
            val -= Xe @ t[ki, kj, K][i, j, :, a]
            out.append(val)
        return np.array(out)

    # ---------------------------------------------------------------- right-hand sides, left vectors
    # b and e of Eqs. 6-7 need only the amplitudes: the KEOM methods apply as they stand.
    @property
    def l1(self):
        return self.t1.conj() if self._l1 is None else self._l1

    @property
    def l2(self):
        return self.t2.conj() if self._l2 is None else self._l2

    @staticmethod
    def pack(r1, r2):
        return np.concatenate([r1.ravel(), r2.ravel()])

    def rhs(self, kind, K, p):
        from oracle.kccsd import KEOM
        return (KEOM.rhs_ip if kind == "ip" else KEOM.rhs_ea)(self, K, p)

    def left(self, kind, K, p):
        from oracle.kccsd import KEOM
        return (KEOM.left_ip if kind == "ip" else KEOM.left_ea)(self, K, p)
