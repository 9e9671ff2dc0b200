"""Solutions of the shifted EOM systems (Eq. 6) and the G contraction (Eq. 7, Eq. 9).

Test infrastructure only (see the package docstring).

Sector conventions (time-ordered G, read literally from Eq. 1 / Eq. 4 / Eq. 6):
  IP (removal):  (w - i eta + A_IP) X_p = b_p,   G-[p,q] = e_q . X_p
  EA (addition): (w + i eta - A_EA) Y_q = b_q,   G+[p,q] = e_p . Y_q
The contraction is bilinear (no complex conjugation).

Three independent ways to the same numbers:
* ``dense_gf``    LU solves on the explicit matrix (tiny / small systems);
* ``lehmann_gf``  sum over the eigenpairs of A (right eigenvectors R_n, left
                  eigenvectors L_n with L_n R_m = delta): G-[p,q] =
                  sum_n (e_q R_n)(L_n b_p) / (w - i eta + W_n), and likewise G+;
* ``gmres``       restarted GMRES (Arnoldi with modified Gram-Schmidt, Givens
                  rotations), the Krylov method the hot path uses, here in FP64.
"""
import numpy as np


def shift_matrix(kind, omega, eta, A):
    D = A.shape[0]
    if kind == "ip":
        return (omega - 1j * eta) * np.eye(D) + A
    return (omega + 1j * eta) * np.eye(D) - A


def dense_gf(kind, A, B, E, omegas, eta):
    """B[:, p] right-hand sides, E[q, :] left vectors; returns G[w, p, q] for the sector."""
    G = np.zeros((len(omegas), B.shape[1], E.shape[0]), dtype=np.complex128)
    for w, om in enumerate(omegas):
        X = np.linalg.solve(shift_matrix(kind, om, eta, A), B)
        if kind == "ip":
            G[w] = (E @ X).T
        else:
            G[w] = E @ X
    return G


def lehmann_gf(kind, A, B, E, omegas, eta):
    wn, R = np.linalg.eig(A)
    Linv = np.linalg.inv(R)           # rows are the left eigenvectors, Linv @ R = 1
    ER = E @ R                        # [q, n]
    LB = Linv @ B                     # [n, p]
    G = np.zeros((len(omegas), B.shape[1], E.shape[0]), dtype=np.complex128)
    for w, om in enumerate(omegas):
        if kind == "ip":
            den = om - 1j * eta + wn
            G[w] = (ER @ (LB / den[:, None])).T
        else:
            den = om + 1j * eta - wn
            G[w] = ER @ (LB / den[:, None])
    return G


def gmres(apply_op, b, tol=1e-12, restart=50, max_iter=20000, x0=None, precond=None):
    """Right-preconditioned restarted GMRES for M x = b.

    apply_op(x) returns M x; precond(v) returns P^-1 v (identity if None).
    Stops when ||b - M x|| <= tol ||b|| (recomputed at every restart).
    Returns (x, iterations, relative residual).
    """
    nb = np.linalg.norm(b)
    D = b.shape[0]
    if nb == 0.0:
        return np.zeros_like(b), 0, 0.0
    x = np.zeros(D, dtype=np.complex128) if x0 is None else x0.astype(np.complex128).copy()
    Pinv = (lambda v: v) if precond is None else precond
    it = 0
    r = b - apply_op(x)
    beta = np.linalg.norm(r)
    while beta > tol * nb and it < max_iter:
        m = restart
        V = np.zeros((m + 1, D), dtype=np.complex128)
        Z = np.zeros((m, D), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        V[0] = r / beta
        g[0] = beta
        j_done = 0
        for j in range(m):
            Z[j] = Pinv(V[j])
            w = apply_op(Z[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                a, bb = H[i, j], H[i + 1, j]
                H[i, j] = np.conj(cs[i]) * a + np.conj(sn[i]) * bb
                H[i + 1, j] = -sn[i] * a + cs[i] * bb
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[j] = a / den if den != 0 else 1.0
            sn[j] = bb / den if den != 0 else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            j_done = j + 1
            if abs(g[j + 1]) <= tol * nb * 0.5 or it >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + y @ Z[:j_done]
        r = b - apply_op(x)
        beta = np.linalg.norm(r)
    return x, it, beta / nb
