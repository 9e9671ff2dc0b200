"""The largest workloads on one GPU, element by element against the oracle.

  si_k333_o4v30:   3x3x3 mesh, nocc 4, nvir 30, Naux 96 (Si-like band-structure mesh)
  zno_k222_o18v60: 2x2x2 mesh, nocc 18, nvir 60, Naux 240 (ZnO-like)

At these sizes the build stores no O(nk^3 o v^3) block (the W_vvvo r1 term, the EA singles'
(2<am|ef> - <am|fe>) term and the ladder's T2 part come from the density-fitting factors in every
sigma), and the oracle cannot form the operator: it evaluates sampled output elements one by one
(oracle.rows.KRows, pinned element by element to the full oracle on small meshes). Checked:
  - right-hand sides b and left vectors e of sampled orbitals (all elements, 1e-12);
  - sampled rows of y = A x (IP and EA, two k-points, rows of every k-block class and the singles):
    FP64 1e-11 relative to max |y|; FP32 and 3xTF32 forms 3e-5 relative (the low-precision
    kernels run on FP64-stored blocks where the device holds no FP32 copy);
  - a solve of HOMO and LUMO at k = 0 and one frequency to relative residual 1e-6 in the plain
    and the chosen form: both converge (FP64-recomputed residuals) and their G rows / columns agree
    within 1e-6 max(1, |G|).
"""
import gc

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2208_07478_gb300 import binding as B
from paper_2208_07478_gb300.synth import make_workload
from oracle.rows import KRows

WORKLOADS = ["si_k333_o4v30", "zno_k222_o18v60"]


@pytest.fixture(scope="module", params=WORKLOADS)
def big(request):
    s = make_workload(request.param)
    torch.cuda.empty_cache()
    h = B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, s.mo_energy, s.L, s.t1, s.t2)
    kr = KRows(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, s.L)
    yield s, h, kr
    h.close()
    del kr
    gc.collect()
    torch.cuda.empty_cache()


def sample_rows(kr, kind, D, rng, count=24):
    n1 = kr.nocc if kind == "ip" else kr.nvir
    rows = list(rng.choice(n1, size=min(3, n1), replace=False))
    rows += list(n1 + rng.choice(D - n1, size=count, replace=False))
    return sorted(int(r) for r in rows)


@pytest.mark.parametrize("kind", ["ip", "ea"])
def test_vectors_match_oracle(big, kind):
    s, h, kr = big
    d = h.dims()
    D = d["dim_ip"] if kind == "ip" else d["dim_ea"]
    sec = B.IP if kind == "ip" else B.EA
    out = torch.zeros(D, dtype=torch.complex128, device="cuda")
    for K in (0, s.nk - 1):
        for p in (s.nocc - 1, s.nocc):
            B.rhs(h, sec, K, p, out)
            np.testing.assert_allclose(out.cpu().numpy(), kr.rhs(kind, K, p), atol=1e-12)
            B.left(h, sec, K, p, out)
            np.testing.assert_allclose(out.cpu().numpy(), kr.left(kind, K, p), atol=1e-12)


@pytest.mark.parametrize("kind", ["ip", "ea"])
def test_sigma_rows_match_oracle(big, kind):
    s, h, kr = big
    d = h.dims()
    D = d["dim_ip"] if kind == "ip" else d["dim_ea"]
    rng = np.random.default_rng(7)
    nvec = 2
    for K in (0, s.nk // 2):
        x = rng.normal(size=(nvec, D)) + 1j * rng.normal(size=(nvec, D))
        xd = torch.from_numpy(x).cuda()
        rows = sample_rows(kr, kind, D, rng)
        ref = np.stack([(kr.sigma_ip_elements if kind == "ip" else kr.sigma_ea_elements)(K, x[c], rows)
                        for c in range(nvec)])
        for prec, tol in ((B.FP64, 1e-11), (B.FP32, 3e-5), (B.TF32X3, 3e-5)):
            yd = torch.zeros_like(xd)
            (B.sigma_ip if kind == "ip" else B.sigma_ea)(h, K, xd, yd, prec=prec)
            y = yd.cpu().numpy()
            scale = np.abs(y).max()
            err = np.abs(y[:, rows] - ref).max() / scale
            print(f"{s.name} {kind} K={K} prec {prec}: max |dy| / max |y| = {err:.2e} over {len(rows)} rows")
            assert err <= tol, (prec, err)
        del xd, yd
        torch.cuda.empty_cache()


def test_slice_solve_plain_and_chosen(big):
    s, h, kr = big
    om = [float(s.omega[len(s.omega) // 2])]
    Gs = {}
    for prec in (B.FP64, B.TF32X3):
        G = np.zeros((s.nk, 1, s.nmo, s.nmo), dtype=np.complex128)
        opt = B.default_options(prec=prec, tol=1e-6, restart_m=30, max_iter=4000, max_refine=40, kpoint=0,
                                orbital_first=s.nocc - 1, orbital_count=2)
        st, stats = B.solve_gf(h, B.BOTH, om, s.eta, G, options=opt)
        assert st == B.CCGF_OK
        assert stats["max_rel_residual"] <= 1e-6
        assert stats["rhs_solved"] == 4
        print(f"{s.name} prec {prec}: {stats['inner_iterations']} iterations, restart {stats['restart_used']}, "
              f"{stats['columns_per_batch']} columns per batch, {stats['total_ms'] / 1e3:.1f} s")
        Gs[prec] = G[0, 0]
    for p in (s.nocc - 1, s.nocc):
        for g in (Gs[B.FP64][p, :], Gs[B.FP64][:, p]):
            assert np.abs(g).max() > 0
    d = np.abs(Gs[B.TF32X3] - Gs[B.FP64])
    assert (d / np.maximum(1.0, np.abs(Gs[B.FP64]))).max() <= 1e-6
