"""Spectral function and density of states (Eq. 10) from a Green's function (CPU, FP64).

Test infrastructure only (see the package docstring).

A(k, w) = -(1/pi) Im G(k, w); its trace over the orbitals is the density of states at k. For the
time-ordered G of Eq. 9 the removal part has the opposite sign of the imaginary part at its poles;
given the two parts separately, the retarded convention -(1/pi) Im G+ + (1/pi) Im G- makes both
sides positive.
"""
import numpy as np


def dos(G, G_minus=None):
    """G [nk][nomega][n][n] -> dos [nk][nomega]."""
    tr = np.trace(G, axis1=2, axis2=3)
    out = -tr.imag / np.pi
    if G_minus is not None:
        out = out + np.trace(G_minus, axis1=2, axis2=3).imag / np.pi
    return out
