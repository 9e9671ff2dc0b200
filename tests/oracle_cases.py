"""Small systems shared by the oracle tests (data only)."""
import numpy as np


def random_molecule(nocc, nvir, seed, hermitian=True, t1_sigma=0.1, lam=True, fock_offdiag=0.0, naux=6, scale=0.2):
    """Random f (diagonal unless fock_offdiag), DF-built ERIs, T1/T2, Lambda1/Lambda2."""
    rng = np.random.default_rng(seed)
    n = nocc + nvir
    c = lambda shape, s: rng.normal(0, s, shape) + 1j * rng.normal(0, s, shape)
    f = np.diag(np.concatenate([rng.uniform(-1, -0.3, nocc), rng.uniform(0.1, 2, nvir)])).astype(complex)
    if fock_offdiag:
        f = f + c((n, n), fock_offdiag)
    L = c((naux, n, n), scale)
    if hermitian:
        L = L + L.conj().transpose(0, 2, 1)
        g = np.einsum('Qpq,Qrs->pqrs', L, L)
    else:
        L2 = c((naux, n, n), scale)
        g = np.einsum('Qpq,Qrs->pqrs', L, L2)
        g = g + g.transpose(2, 3, 0, 1)
    t1 = c((nocc, nvir), t1_sigma) if t1_sigma else np.zeros((nocc, nvir), complex)
    t2 = c((nocc, nocc, nvir, nvir), 0.1)
    t2 = t2 + t2.transpose(1, 0, 3, 2)
    l1 = c((nocc, nvir), 0.1) if lam else np.zeros((nocc, nvir), complex)
    l2 = c((nocc, nocc, nvir, nvir), 0.1)
    l2 = l2 + l2.transpose(1, 0, 3, 2)
    return dict(f=f, g=g, t1=t1, t2=t2, l1=l1, l2=l2, nocc=nocc)


def symmetric_lambda2(km, l2):
    """Impose l2[ki,kj,ka][i,j,a,b] = l2[kj,ki,kb][j,i,b,a] (closed-shell pair symmetry)."""
    nk = l2.shape[0]
    out = np.zeros_like(l2)
    for ki in range(nk):
        for kj in range(nk):
            for ka in range(nk):
                kb = km.c(ki, ka, kj)
                out[ki, kj, ka] = l2[ki, kj, ka] + l2[kj, ki, kb].transpose(1, 0, 3, 2)
    return out
