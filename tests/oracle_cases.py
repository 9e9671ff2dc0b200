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


def oracle_column(ke, kind, K, p, omega, eta, tol=1e-12, restart=60):
    """One right-hand side solved by the oracle's GMRES; returns (G row (IP) / column (EA), iterations)."""
    from oracle.kccsd import diag_estimate
    from oracle import solvers
    z = omega - 1j * eta if kind == "ip" else omega + 1j * eta
    sg = 1.0 if kind == "ip" else -1.0
    d = diag_estimate(ke, kind, K)
    sig = ke.sigma_ip if kind == "ip" else ke.sigma_ea
    b = ke.rhs_ip(K, p) if kind == "ip" else ke.rhs_ea(K, p)
    x, it, res = solvers.gmres(lambda v: z * v + sg * sig(K, v), b, tol=tol, restart=restart,
                               precond=lambda v: v / (z + sg * d))
    assert res <= tol, res
    n = ke.nmo
    E = [ke.left_ip(K, q) if kind == "ip" else ke.left_ea(K, q) for q in range(n)]
    return np.array([e @ x for e in E]), it


def locate_pole(ke, kind, K, p, omega0, eta, steps=4):
    """Real frequency of the pole of G_pp(w) nearest omega0, from the oracle alone.

    Near a simple pole G_pp(w) = c / (w - w* +- i eta) + (smooth), so 1 / G_pp is close to linear
    in w; secant steps on 1 / G_pp move w to the real point where the linear model is smallest.
    Returns (w*, |G_pp(w*)|).
    """
    def inv_g(w):
        col, _ = oracle_column(ke, kind, K, p, w, eta, tol=1e-11)
        return 1.0 / col[p]
    w1, w2 = omega0, omega0 + 4 * eta
    f1, f2 = inv_g(w1), inv_g(w2)
    for _ in range(steps):
        alpha = (f2 - f1) / (w2 - w1)
        w3 = w2 - float(np.real(f2 * np.conj(alpha))) / float(abs(alpha) ** 2)
        w1, f1 = w2, f2
        w2, f2 = w3, inv_g(w3)
        if abs(w2 - w1) < 1e-3 * eta:
            break
    return w2, float(1.0 / abs(f2))
