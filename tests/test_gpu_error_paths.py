"""Error paths free what they allocated (failures made on the host, no GPU fault).

ccgf_inject_alloc_failure makes the library's n-th next device allocation report out of
memory. A solve that fails that way part-way (after its Krylov basis, right-hand sides and
other per-sector buffers were allocated) must return CCGF_ERR_OOM and leave the device's free
memory where it was; the handle must stay usable and give the same G afterwards. The same
for a build that fails after its intermediates were partly formed.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2208_07478_gb300 import binding as B
from paper_2208_07478_gb300.synth import make_system

SLACK = 64 << 20     # allocation granularity and driver bookkeeping


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.fixture(scope="module")
def system():
    return make_system((2, 1, 1), 2, 6, 10, seed=21, L_sigma=0.05, t1_sigma=0.01, nomega=3,
                       omega_range=(-0.6, 0.6), eta=0.02)


def test_solve_failing_midway_frees_its_buffers(system):
    s = system
    h = B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, s.mo_energy, s.L, s.t1, s.t2)
    opt = B.default_options(tol=1e-10, restart_m=30, max_iter=4000)
    G0 = np.zeros((s.nk, len(s.omega), s.nmo, s.nmo), dtype=np.complex128)
    st, _ = B.solve_gf(h, B.BOTH, s.omega, s.eta, G0, options=opt)
    assert st == B.CCGF_OK
    before = free_bytes()
    for after in (2, 9, 20, 31):
        B.inject_alloc_failure(after)
        G = np.zeros_like(G0)
        try:
            with pytest.raises(B.CCGFError) as e:
                B.solve_gf(h, B.BOTH, s.omega, s.eta, G, options=opt)
            assert e.value.status == B.CCGF_ERR_OOM
        finally:
            B.inject_alloc_failure(-1)
        assert free_bytes() >= before - SLACK, after
    G = np.zeros_like(G0)
    st, _ = B.solve_gf(h, B.BOTH, s.omega, s.eta, G, options=opt)
    assert st == B.CCGF_OK
    assert np.abs(G - G0).max() <= 1e-12 * max(1.0, np.abs(G0).max())
    h.close()


def test_build_failing_midway_frees_its_buffers(system):
    s = system
    before = free_bytes()
    for after in (5, 15, 30):
        B.inject_alloc_failure(after)
        try:
            with pytest.raises(B.CCGFError) as e:
                B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, s.mo_energy, s.L, s.t1, s.t2)
            assert e.value.status == B.CCGF_ERR_OOM
        finally:
            B.inject_alloc_failure(-1)
        assert free_bytes() >= before - SLACK, after
