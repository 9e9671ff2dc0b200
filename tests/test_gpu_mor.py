"""Model-order-reduction CCGF (the paper's MOR frequency interpolation) on the GPU.

A 2x1x1 mesh (nocc 2, nvir 4) with five model frequencies over a 41-point grid, both sectors:
  - at the model frequencies the reduced model reproduces the full G (Galerkin projection with the
    solutions in the subspace): |dG| <= 1e-7 max |G| against the oracle's dense LU;
  - on the whole grid the GPU reduced model equals the oracle's reduced model (oracle.mor, same
    model frequencies and rank rule) to 1e-7 max |G|;
  - and interpolates the full G (smooth between the model points) to 1e-4 max |G|.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2208_07478_gb300 import binding as B
from paper_2208_07478_gb300.synth import make_system
from oracle.kccsd import KEOM
from oracle import solvers
from oracle.mor import mor_gf


def test_mor_matches_oracle_and_full_solve():
    s = make_system((2, 1, 1), 2, 4, 8, seed=17, L_sigma=0.05, t1_sigma=0.01, nomega=41, omega_range=(-1.0, 1.0), eta=0.05)
    h = B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, s.mo_energy, s.L, s.t1, s.t2)
    wm = s.omega[::10]
    G = np.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=np.complex128)
    st, stats = B.solve_gf_mor(h, B.BOTH, wm, s.omega, s.eta, G, options=B.default_options(tol=1e-12, restart_m=40))
    assert st == B.CCGF_OK
    h.close()
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    full = np.zeros_like(G)
    red = np.zeros_like(G)
    for K in range(s.nk):
        for kind in ("ip", "ea"):
            A = ke.matrix(kind, K)
            Bm = np.stack([(ke.rhs_ip if kind == "ip" else ke.rhs_ea)(K, p) for p in range(s.nmo)], 1)
            Em = np.stack([(ke.left_ip if kind == "ip" else ke.left_ea)(K, q) for q in range(s.nmo)], 0)
            full[K] += solvers.dense_gf(kind, A, Bm, Em, s.omega, s.eta)
            red[K] += mor_gf(kind, A, Bm, Em, wm, s.omega, s.eta)[0]
    scale = np.abs(full).max()
    print(f"reduced dimension {stats['columns_per_batch']}; max |dG| vs oracle MOR {np.abs(G - red).max() / scale:.2e}, "
          f"at model points {np.abs(G[:, ::10] - full[:, ::10]).max() / scale:.2e}, vs full {np.abs(G - full).max() / scale:.2e}")
    assert np.abs(G[:, ::10] - full[:, ::10]).max() <= 1e-7 * scale
    assert np.abs(G - red).max() <= 1e-7 * scale
    assert np.abs(G - full).max() <= 1e-4 * scale
