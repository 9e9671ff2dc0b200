"""Active-space self-energy correction (Eqs. 12-14) on the CPU, FP64, by explicit inverses.

Test infrastructure only (see the package docstring).

For every k and frequency: Sigma_CAS = G_GW,CAS^-1 - G_CC,CAS^-1 (Eq. 12), Sigma_full = V Sigma_CAS V^+
(Eq. 13), G_CC+GW = [G_GW,full^-1 - Sigma_full]^-1 (Eq. 14); V holds the natural-orbital coefficients
of the active orbitals (columns) in the full orbital basis.
"""
import numpy as np


def cc_gw(V, G_gw, G_gw_cas, G_cc_cas):
    nk, nw = G_gw.shape[:2]
    out = np.zeros_like(G_gw)
    for k in range(nk):
        for w in range(nw):
            sig_cas = np.linalg.inv(G_gw_cas[k, w]) - np.linalg.inv(G_cc_cas[k, w])
            sig = V[k] @ sig_cas @ V[k].conj().T
            out[k, w] = np.linalg.inv(np.linalg.inv(G_gw[k, w]) - sig)
    return out
