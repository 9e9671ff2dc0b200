"""The seeded input generator (CPU): determinism, the structure its layouts promise, and the
MP2 amplitudes recomputed element by element from the drawn integrals."""
import numpy as np

from paper_2208_07478_gb300.synth import make_system, kadd_table, kneg_table


def _system(seed=4):
    return make_system((2, 1, 1), 2, 3, 5, seed=seed, L_sigma=0.05, t1_sigma=0.01, nomega=3,
                       omega_range=(-0.5, 0.5), eta=0.01)


def test_same_seed_same_system_other_seed_differs():
    a, b, c = _system(4), _system(4), _system(5)
    for x, y in ((a.L, b.L), (a.t1, b.t1), (a.t2, b.t2), (a.mo_energy, b.mo_energy)):
        assert np.array_equal(x, y)
    assert not np.allclose(a.L, c.L)


def test_orbital_energies_sorted_occupied_below_virtual():
    s = _system()
    for k in range(s.nk):
        e = s.mo_energy[k]
        assert np.all(np.diff(e[:s.nocc]) >= 0) and np.all(np.diff(e[s.nocc:]) >= 0)
        assert e[:s.nocc].max() < 0 < e[s.nocc:].min()
    assert np.allclose(s.omega, np.linspace(-0.5, 0.5, 3))


def test_factors_are_hermitian_across_momentum_pairs():
    s = _system()
    for k1 in range(s.nk):
        for k2 in range(s.nk):
            assert np.allclose(s.L[k2, k1], np.conj(np.transpose(s.L[k1, k2], (0, 2, 1))))
    g = make_system((1, 1, 1), 2, 3, 4, seed=1, nomega=0)
    assert np.all(g.L.imag == 0)


def test_momentum_tables_are_a_group():
    kmesh = (2, 3, 1)
    add, neg = kadd_table(kmesh), kneg_table(kmesh)
    nk = 6
    for a in range(nk):
        assert add[a, neg[a]] == 0
        for b in range(nk):
            assert add[a, b] == add[b, a]
            for c in range(nk):
                assert add[add[a, b], c] == add[a, add[b, c]]


def test_mp2_amplitudes_from_the_integrals():
    s = _system()
    o, add, neg = s.nocc, kadd_table(s.kmesh), kneg_table(s.kmesh)
    e = s.mo_energy
    for ki in range(s.nk):
        for kj in range(s.nk):
            for ka in range(s.nk):
                kb = add[add[ki, kj], neg[ka]]
                for i in range(o):
                    for j in range(o):
                        for a in range(s.nvir):
                            for b in range(s.nvir):
                                eri = np.sum(s.L[ka, ki, :, o + a, i] * s.L[kb, kj, :, o + b, j])
                                den = e[ki, i] + e[kj, j] - e[ka, o + a] - e[kb, o + b]
                                assert np.isclose(s.t2[ki, kj, ka, i, j, a, b], eri / den, rtol=1e-12, atol=1e-15)
