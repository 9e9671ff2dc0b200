"""k-point system -> supercell ("molecular") arrays.

Test infrastructure only (see the package docstring).

The supercell orbitals are ordered occupied first: occupied (k, i) has index
k*nocc + i, virtual (k, a) has index nk*nocc + k*nvir + a. Momentum
conservation (Eq. 9 and the integral definition of the workloads) appears as
explicit zero blocks.
"""
import numpy as np


def _kvec(kmesh, k):
    n1, n2, n3 = kmesh
    return (k // (n2 * n3), (k // n3) % n2, k % n3)


def _kidx(kmesh, v):
    n1, n2, n3 = kmesh
    return ((v[0] % n1) * n2 + (v[1] % n2)) * n3 + (v[2] % n3)


def k_conserved(kmesh, k1, k2, k3, k4):
    """True when k1 - k2 + k3 - k4 = 0 on the mesh."""
    a, b, c, d = (_kvec(kmesh, k) for k in (k1, k2, k3, k4))
    return all((a[x] - b[x] + c[x] - d[x]) % kmesh[x] == 0 for x in range(3))


def k_combine(kmesh, k1, k2, k3):
    """Index of k1 - k2 + k3 on the mesh."""
    a, b, c = (_kvec(kmesh, k) for k in (k1, k2, k3))
    return _kidx(kmesh, tuple(a[x] - b[x] + c[x] for x in range(3)))


def orbital_index(nk, nocc, nvir):
    """sc[k, p] = supercell index of orbital p (occupied first) at k."""
    sc = np.zeros((nk, nocc + nvir), dtype=np.int64)
    for k in range(nk):
        for i in range(nocc):
            sc[k, i] = k * nocc + i
        for a in range(nvir):
            sc[k, nocc + a] = nk * nocc + k * nvir + a
    return sc


def supercell_system(kmesh, nocc, mo_energy, L, t1, t2, l1=None, l2=None):
    """Return dict with f, g, t1, t2, l1, l2 over the supercell orbitals.

    g[P,Q,R,S] = sum_Q L[k1,k2,Q,p,q] L[k3,k4,Q,r,s] when k1+k3 = k2+k4 (else 0).
    t2[I,J,A,B] = t[ki,kj,ka][i,j,a,b] placed at the momentum-allowed blocks.
    """
    kmesh = tuple(kmesh)
    nk, _, naux, nmo, _ = L.shape
    nvir = nmo - nocc
    n = nk * nmo
    sc = orbital_index(nk, nocc, nvir)
    g = np.zeros((n, n, n, n), dtype=np.complex128)
    for k1 in range(nk):
        for k2 in range(nk):
            for k3 in range(nk):
                for k4 in range(nk):
                    if not k_conserved(kmesh, k1, k2, k3, k4):
                        continue
                    blk = np.einsum('Qpq,Qrs->pqrs', L[k1, k2], L[k3, k4])
                    g[np.ix_(sc[k1], sc[k2], sc[k3], sc[k4])] = blk
    f = np.zeros((n, n), dtype=np.complex128)
    for k in range(nk):
        f[sc[k], sc[k]] = mo_energy[k]
    no, nv = nk * nocc, nk * nvir
    T1 = np.zeros((no, nv), dtype=np.complex128)
    T2 = np.zeros((no, no, nv, nv), dtype=np.complex128)
    L1 = np.zeros((no, nv), dtype=np.complex128)
    L2 = np.zeros((no, no, nv, nv), dtype=np.complex128)
    if l1 is None:
        l1 = t1.conj()
    if l2 is None:
        l2 = t2.conj()
    oi = sc[:, :nocc]
    va = sc[:, nocc:] - no
    for k in range(nk):
        T1[np.ix_(oi[k], va[k])] = t1[k]
        L1[np.ix_(oi[k], va[k])] = l1[k]
    for ki in range(nk):
        for kj in range(nk):
            for ka in range(nk):
                kb = k_combine(kmesh, ki, ka, kj)  # ki - ka + kj
                T2[np.ix_(oi[ki], oi[kj], va[ka], va[kb])] = t2[ki, kj, ka]
                L2[np.ix_(oi[ki], oi[kj], va[ka], va[kb])] = l2[ki, kj, ka]
    return dict(f=f, g=g, t1=T1, t2=T2, l1=L1, l2=L2, nocc=no, nvir=nv, sc=sc)
