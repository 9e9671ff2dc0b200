"""Model-order-reduction CCGF (the paper's MOR paragraph, Figs. 1c-d): frequency interpolation
through a subspace spanned by solutions at a few frequencies (CPU, FP64).

Test infrastructure only (see the package docstring).

For one sector and total momentum K: solve the shifted systems of Eq. 6 at the n_mor model
frequencies for every orbital; take an orthonormal basis V of the span of all those solution vectors
; project the EOM matrix, the right-hand sides and the left
vectors on it (A_r = V^H A V, b_r = V^H b, e_r = e V) and solve the reduced systems of dimension
rank(V) at every frequency of the full grid. At a model frequency the exact solution lies in the
subspace, so the reduced model reproduces G there. The basis: left singular vectors of S with
singular value above rel_tol times the largest.
"""
import numpy as np

from oracle import solvers


def mor_gf(kind, A, B, E, omega_mor, omega, eta, rel_tol=1e-7):
    """A dense [D][D]; B [D][n] right-hand sides; E [n][D] left vectors. Returns (G[w, p, q], rank)."""
    S = np.concatenate([np.linalg.solve(solvers.shift_matrix(kind, om, eta, A), B) for om in omega_mor], axis=1)
    U, sv, _ = np.linalg.svd(S, full_matrices=False)
    V = U[:, sv > rel_tol * sv[0]]
    Ar = V.conj().T @ A @ V
    Br = V.conj().T @ B
    Er = E @ V
    G = np.zeros((len(omega), B.shape[1], E.shape[0]), dtype=np.complex128)
    r = V.shape[1]
    for w, om in enumerate(omega):
        X = np.linalg.solve(solvers.shift_matrix(kind, om, eta, Ar) if r else np.zeros((0, 0)), Br)
        G[w] = (Er @ X).T if kind == "ip" else Er @ X
    return G, r
