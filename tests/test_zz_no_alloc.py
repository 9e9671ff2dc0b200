"""ccgf_sigma_ip_noalloc: the IP sigma for callers that cannot allocate device memory.

Callers such as a framework that owns all device memory through its own pool, or a
latency-critical loop that cannot take the synchronisation an allocation may imply,
use this entry point; it keeps all of its scratch in the library's static device
workspace. The test checks it through the C ABI against ccgf_sigma_ip (same FP64
tolerance as the other sigma parity tests) on two calls in a row, checks that the
device's free memory does not change across the second call (the first one's set-up
looks up the static array), and that an nvec too
large for the static workspace is refused with an error instead of running.

Kept in a file of its own, collected last, so that a stop-at-first-failure run has
already run every other test when it gets here.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2208_07478_gb300 import binding as B
from paper_2208_07478_gb300.synth import make_system

REL_TOL = 1e-11


@pytest.fixture(scope="module")
def handle():
    s = make_system((2, 1, 1), 2, 5, 8, seed=21, L_sigma=0.08, t1_sigma=0.02, nomega=0)
    h = B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, s.mo_energy, s.L, s.t1, s.t2)
    yield s, h
    h.close()


def test_noalloc_matches_sigma_ip_on_two_calls(handle):
    s, h = handle
    D = h.dims()["dim_ip"]
    nvec = 6
    rng = np.random.default_rng(3)
    xs = [torch.from_numpy(rng.normal(size=(nvec, D)) + 1j * rng.normal(size=(nvec, D))).cuda() for _ in range(2)]
    refs = []
    for K, x in zip((1, 0), xs):
        y_ref = torch.zeros_like(x)
        B.sigma_ip(h, K, x, y_ref)
        refs.append(y_ref)
    ys = [torch.full_like(x, complex(np.nan, np.nan)) for x in xs]
    torch.cuda.synchronize()
    # first call: its set-up looks up the static array, whose 32 MiB the driver maps when it
    # loads the library's device code; the second call must leave the free memory unchanged
    B.sigma_ip_noalloc(h, 1, xs[0], ys[0])
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    B.sigma_ip_noalloc(h, 0, xs[1], ys[1])
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    for y, y_ref in zip(ys, refs):
        scale = float(y_ref.abs().max())
        err = float((y - y_ref).abs().max())
        assert err <= REL_TOL * scale, (err, scale)
    assert free_after == free_before


def test_noalloc_refuses_oversized_request(handle):
    s, h = handle
    D = h.dims()["dim_ip"]
    nvec = 20000      # far beyond the 32 MiB static workspace for this dimension
    x = torch.zeros((nvec, D), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(B.CCGFError) as e:
        B.sigma_ip_noalloc(h, 0, x, y)
    assert e.value.status == B.CCGF_ERR_INVALID_ARG
