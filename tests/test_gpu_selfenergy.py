"""Active-space self-energy correction (Eqs. 12-14) on the GPU against the oracle's explicit inverses.

Random well-conditioned Green's-function-like matrices (complex, nmo 26 / nact 14 as the Si
(8e, 14o)-type active spaces, and nmo 78 as the ZnO-like orbital count) for several (k, w): the
kernel's G_CC+GW agrees with oracle.selfenergy.cc_gw to 1e-11 relative; equal GW and CC active-space
G give back G_GW; a singular input is refused with CCGF_ERR_INVALID_ARG.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2208_07478_gb300 import binding as B
from oracle.selfenergy import cc_gw


def inputs(nk, nw, n, m, seed):
    rng = np.random.default_rng(seed)
    c = lambda *sh: rng.normal(size=sh) + 1j * rng.normal(size=sh)
    Ggw = 0.2 * c(nk, nw, n, n) + (2.0 + 0.1j) * np.eye(n)
    V = np.stack([np.linalg.qr(c(n, n))[0][:, :m] for _ in range(nk)])
    Ggw_cas = 0.2 * c(nk, nw, m, m) + (1.5 - 0.2j) * np.eye(m)
    Gcc_cas = 0.2 * c(nk, nw, m, m) + (1.7 + 0.3j) * np.eye(m)
    return V, Ggw, Ggw_cas, Gcc_cas


@pytest.mark.parametrize("nk,nw,n,m", [(2, 5, 26, 14), (1, 3, 78, 30), (3, 2, 8, 8)])
def test_self_energy_matches_oracle(nk, nw, n, m):
    V, Ggw, Ggw_cas, Gcc_cas = inputs(nk, nw, n, m, seed=n + m)
    ref = cc_gw(V, Ggw, Ggw_cas, Gcc_cas)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.zeros_like(d(Ggw))
    B.self_energy_correction(d(V), d(Ggw), d(Ggw_cas), d(Gcc_cas), out)
    torch.cuda.synchronize()
    err = np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 1e-11, err
    # no correction when the two active-space G agree
    B.self_energy_correction(d(V), d(Ggw), d(Ggw_cas), d(Ggw_cas), out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - Ggw).max() <= 1e-11 * np.abs(Ggw).max()


def test_singular_input_is_refused():
    V, Ggw, Ggw_cas, Gcc_cas = inputs(1, 1, 6, 3, seed=1)
    Gcc_cas[0, 0] = 0.0
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.zeros_like(d(Ggw))
    with pytest.raises(B.CCGFError) as e:
        B.self_energy_correction(d(V), d(Ggw), d(Ggw_cas), d(Gcc_cas), out)
    assert e.value.status == B.CCGF_ERR_INVALID_ARG
