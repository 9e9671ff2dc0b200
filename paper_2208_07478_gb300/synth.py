"""Seeded synthetic inputs for the periodic CCGF path.

This module only draws random numbers and lays them out; it holds none of the
Green's-function arithmetic. Both the CUDA path (through the tests and the
benchmark) and the CPU oracle consume its output, so they see the same system.

What one "system" holds, and the layouts used at the C ABI:

* ``kmesh``       (n1, n2, n3); k index = (k1*n2 + k2)*n3 + k3, addition modulo
                  each mesh dimension.
* ``mo_energy``   float64 [nk][nmo]: occupied first, then virtual, sorted within
                  each block. The reference Fock matrix is diag(mo_energy) at
                  every k (canonical Hartree-Fock orbitals).
* ``L``           complex128 [nk][nk][naux][nmo][nmo]: density-fitting factors,
                  (p k1 q k2 | r k3 s k4) = sum_Q L[k1,k2,Q,p,q] L[k3,k4,Q,r,s]
                  when k1 + k3 = k2 + k4, zero otherwise. L[k2,k1,Q] is the
                  conjugate transpose of L[k1,k2,Q] so that the Hamiltonian is
                  Hermitian; at a one-point mesh L is real.
* ``t1``          complex128 [nk][nocc][nvir]: T1 amplitudes t[k][i][a].
* ``t2``          complex128 [nk][nk][nk][nocc][nocc][nvir][nvir]:
                  t[ki,kj,ka][i,j,a,b] with kb = ki + kj - ka, the closed-shell
                  amplitude of the alpha-beta pair (i alpha, j beta -> a alpha,
                  b beta).
* ``omega``       float64 grid, inclusive endpoints (Hartree); ``eta`` broadening.

Draw order (numpy PCG64 ``default_rng(seed)``): orbital energies (per k:
occupied, then virtual), then L blocks (pairs k1 <= k2 in row-major order,
per pair the real parts then the imaginary parts), then T1 (real parts, then
imaginary parts). T2 holds MP2 amplitudes of the drawn integrals,
t[ki,kj,ka][i,j,a,b] = (a i | b j) / (e_i + e_j - e_a - e_b), the first-order
amplitudes of the recipe the workloads name; it draws no random numbers.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


@dataclass
class System:
    kmesh: tuple
    nocc: int
    nvir: int
    naux: int
    mo_energy: np.ndarray
    L: np.ndarray
    t1: np.ndarray
    t2: np.ndarray
    omega: np.ndarray = field(default_factory=lambda: np.zeros(0))
    eta: float = 0.01
    name: str = ""

    @property
    def nk(self) -> int:
        return int(np.prod(self.kmesh))

    @property
    def nmo(self) -> int:
        return self.nocc + self.nvir


def kindex(kmesh, kv):
    n1, n2, n3 = kmesh
    return ((kv[0] % n1) * n2 + (kv[1] % n2)) * n3 + (kv[2] % n3)


def kvector(kmesh, k):
    n1, n2, n3 = kmesh
    return (k // (n2 * n3), (k // n3) % n2, k % n3)


def kadd_table(kmesh):
    """kadd[k1][k2] = index of k1 + k2 on the mesh."""
    nk = int(np.prod(kmesh))
    tab = np.zeros((nk, nk), dtype=np.int32)
    for a in range(nk):
        va = kvector(kmesh, a)
        for b in range(nk):
            vb = kvector(kmesh, b)
            tab[a, b] = kindex(kmesh, tuple(va[d] + vb[d] for d in range(3)))
    return tab


def kneg_table(kmesh):
    nk = int(np.prod(kmesh))
    return np.array([kindex(kmesh, tuple(-x for x in kvector(kmesh, k))) for k in range(nk)], dtype=np.int32)


def _complex_normal(rng, shape, sigma):
    # |z| has standard deviation sigma: real and imaginary parts each sigma/sqrt(2).
    s = sigma / np.sqrt(2.0)
    re = rng.normal(0.0, s, size=shape)
    im = rng.normal(0.0, s, size=shape)
    return re + 1j * im


def draw_mo_energy(rng, nk, nocc, nvir, occ_range, vir_range, occ_cluster=None):
    e = np.zeros((nk, nocc + nvir))
    for k in range(nk):
        if occ_cluster is None:
            eo = rng.uniform(occ_range[0], occ_range[1], size=nocc)
        else:
            ncl, lo, hi = occ_cluster
            eo = np.concatenate([rng.uniform(lo, hi, size=ncl),
                                 rng.uniform(occ_range[0], occ_range[1], size=nocc - ncl)])
        ev = rng.uniform(vir_range[0], vir_range[1], size=nvir)
        e[k, :nocc] = np.sort(eo)
        e[k, nocc:] = np.sort(ev)
    return e


def draw_L(rng, nk, naux, nmo, sigma):
    L = np.zeros((nk, nk, naux, nmo, nmo), dtype=np.complex128)
    if nk == 1:
        # Gamma-only: real orbitals, L[Q] real symmetric with entries of std sigma.
        a = rng.normal(0.0, sigma, size=(naux, nmo, nmo))
        L[0, 0] = (a + a.transpose(0, 2, 1)) / np.sqrt(2.0)
        idx = np.arange(nmo)
        L[0, 0][:, idx, idx] = a[:, idx, idx]
        return L
    for k1 in range(nk):
        for k2 in range(k1, nk):
            z = _complex_normal(rng, (naux, nmo, nmo), sigma)
            if k1 == k2:
                # Hermitian per Q: off-diagonal entries keep std sigma, diagonal real.
                h = (z + z.conj().transpose(0, 2, 1)) / np.sqrt(2.0)
                idx = np.arange(nmo)
                h[:, idx, idx] = z[:, idx, idx].real * np.sqrt(2.0)
                L[k1, k1] = h
            else:
                L[k1, k2] = z
                L[k2, k1] = z.conj().transpose(0, 2, 1)
    return L


def mp2_t2(kmesh, nocc, mo_energy, L):
    """First-order (MP2) doubles of the drawn integrals, layout t[ki,kj,ka][i,j,a,b]."""
    nk = int(np.prod(kmesh))
    kadd = kadd_table(kmesh)
    kneg = kneg_table(kmesh)
    nvir = mo_energy.shape[1] - nocc
    o, v = slice(0, nocc), slice(nocc, None)
    t2 = np.zeros((nk, nk, nk, nocc, nocc, nvir, nvir), dtype=np.complex128)
    kas = np.arange(nk)
    for ki in range(nk):
        for kj in range(nk):
            # all ka at once; kb = ki + kj - ka, so (a ka, i ki | b kb, j kj) conserves momentum
            kbs = kadd[kadd[ki, kj], kneg[kas]]
            ai = L[kas, ki][:, :, v, o]            # [ka][Q][a][i]
            bj = L[kbs, kj][:, :, v, o]            # [ka][Q][b][j]
            nq = ai.shape[1]
            # sum over Q as one batched matrix product: [ka][(a,i)][Q] @ [ka][Q][(b,j)]
            num = np.matmul(ai.reshape(nk, nq, nvir * nocc).transpose(0, 2, 1), bj.reshape(nk, nq, nvir * nocc))
            num = num.reshape(nk, nvir, nocc, nvir, nocc).transpose(0, 2, 4, 1, 3)
            eo_i = mo_energy[ki, :nocc]
            eo_j = mo_energy[kj, :nocc]
            ev_a = mo_energy[kas, nocc:]           # [ka][a]
            ev_b = mo_energy[kbs, nocc:]           # [ka][b]
            den = (eo_i[None, :, None, None, None] + eo_j[None, None, :, None, None]
                   - ev_a[:, None, None, :, None] - ev_b[:, None, None, None, :])
            t2[ki, kj] = num / den
    return t2


def make_system(kmesh, nocc, nvir, naux, *, seed, L_sigma=0.05, t1_sigma=0.0,
                occ_range=(-1.0, -0.3), vir_range=(0.1, 2.0), occ_cluster=None,
                nomega=16, omega_range=(-1.0, 1.0), eta=0.01, name="") -> System:
    kmesh = tuple(int(x) for x in kmesh)
    nk = int(np.prod(kmesh))
    nmo = nocc + nvir
    rng = np.random.default_rng(seed)
    e = draw_mo_energy(rng, nk, nocc, nvir, occ_range, vir_range, occ_cluster)
    L = draw_L(rng, nk, naux, nmo, L_sigma)
    if t1_sigma > 0.0:
        if nk == 1:
            t1 = rng.normal(0.0, t1_sigma, size=(nk, nocc, nvir)).astype(np.complex128)
        else:
            t1 = _complex_normal(rng, (nk, nocc, nvir), t1_sigma)
    else:
        t1 = np.zeros((nk, nocc, nvir), dtype=np.complex128)
    t2 = mp2_t2(kmesh, nocc, e, L)
    omega = np.linspace(omega_range[0], omega_range[1], nomega) if nomega > 0 else np.zeros(0)
    return System(kmesh, nocc, nvir, naux, e, L, t1, t2, omega, eta, name)


# The five workloads, by the shapes of the paper's Si / ZnO calculations.
WORKLOADS = {
    "gamma_ip_o4v12": dict(kmesh=(1, 1, 1), nocc=4, nvir=12, naux=48, seed=0, L_sigma=0.05,
                           t1_sigma=0.0, nomega=16, omega_range=(-1.0, 1.0), eta=0.01,
                           sectors="ip", tol=1e-10),
    "si_k222_o4v22": dict(kmesh=(2, 2, 2), nocc=4, nvir=22, naux=96, seed=1, L_sigma=0.05,
                          t1_sigma=0.01, nomega=64, omega_range=(-0.8, 0.8), eta=0.005,
                          sectors="ipea", tol=1e-6),
    "si_k333_o4v30": dict(kmesh=(3, 3, 3), nocc=4, nvir=30, naux=96, seed=2, L_sigma=0.05,
                          t1_sigma=0.01, nomega=128, omega_range=(-0.8, 0.8), eta=0.005,
                          sectors="ipea", tol=1e-6),
    "zno_k222_o18v60": dict(kmesh=(2, 2, 2), nocc=18, nvir=60, naux=240, seed=3, L_sigma=0.03,
                            t1_sigma=0.01, nomega=96, omega_range=(-0.8, 0.8), eta=0.005,
                            occ_range=(-1.5, -0.2), vir_range=(0.05, 3.0),
                            occ_cluster=(10, -0.75, -0.65), sectors="ipea", tol=1e-6),
}


def make_workload(name, **override) -> System:
    cfg = dict(WORKLOADS[name])
    cfg.update(override)
    cfg.pop("sectors", None)
    cfg.pop("tol", None)
    return make_system(name=name, **cfg)


def random_vectors(rng_seed, shape, scale=1.0):
    rng = np.random.default_rng(rng_seed)
    return _complex_normal(rng, shape, scale)
