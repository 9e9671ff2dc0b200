"""One sigma application (or one solve) on a configurable synthetic system, for profilers.

    python -m paper_2208_07478_gb300.profile_case --kmesh 2 2 2 --nocc 4 --nvir 16 --sector ea --prec fp64
    python -m paper_2208_07478_gb300.profile_case --workload si_k222_o4v22 --solve --prec tf32x3

Builds the similarity-transformed Hamiltonian blocks, then applies the EA (or
IP) sigma of momentum 0 to nvec random vectors (after one warm-up call that
builds and tunes the plan), once more inside the NVTX range "profiled", and
prints the per-step device times and kernel choices of a profiled call.
With --solve: one warm-up solve and one solve inside "profiled" of all k-points
and orbitals at the middle frequency of the workload's grid (rel. residual 1e-6),
then the solver's statistics (sigma, vector-step and refinement times).
"""
import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kmesh", type=int, nargs=3, default=[2, 2, 2])
    ap.add_argument("--nocc", type=int, default=4)
    ap.add_argument("--nvir", type=int, default=16)
    ap.add_argument("--naux", type=int, default=64)
    ap.add_argument("--nvec", type=int, default=0, help="default: nocc + nvir")
    ap.add_argument("--sector", default="ea", choices=["ip", "ea"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "tf32x3", "fp64_tc"])
    ap.add_argument("--refine", default="fp64", choices=["fp64", "fp64_tc"], help="--solve: true-residual sigma")
    ap.add_argument("--calls", type=int, default=1)
    ap.add_argument("--workload", default=None, help="a named synthetic workload (replaces the shape options)")
    ap.add_argument("--solve", action="store_true", help="profile solve_gf instead of one sigma call")
    a = ap.parse_args()
    import torch
    from paper_2208_07478_gb300 import binding as B
    from paper_2208_07478_gb300.synth import make_system, make_workload
    if a.workload:
        s = make_workload(a.workload)
    else:
        s = make_system(tuple(a.kmesh), a.nocc, a.nvir, a.naux, seed=1, L_sigma=0.05, t1_sigma=0.01, nomega=0)
    h = B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, s.mo_energy, s.L, s.t1, s.t2)
    prec = {"fp64": B.FP64, "fp32": B.FP32, "tf32x3": B.TF32X3, "fp64_tc": B.FP64_TC}[a.prec]
    if a.solve:
        G = torch.zeros((s.nk, 1, s.nmo, s.nmo), dtype=torch.complex128, device="cuda")
        om = s.omega[[len(s.omega) // 2]] if len(s.omega) else np.zeros(1)
        opt = B.default_options(prec=prec, tol=1e-6, restart_m=40, max_iter=4000, max_refine=40,
                                refine_prec=B.FP64_TC if a.refine == "fp64_tc" else B.FP64)
        B.solve_gf(h, B.BOTH, om, s.eta, G, options=opt, on_device=True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled")
        status, st = B.solve_gf(h, B.BOTH, om, s.eta, G, options=opt, on_device=True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        keys = ("inner_iterations", "fp64_sigma_calls", "lowp_sigma_calls", "max_rel_residual", "sigma_ms", "refine_ms",
                "vector_ms", "vector_bytes", "vector_flops", "total_ms", "kernel_launches", "columns_per_batch")
        print({k: st[k] for k in keys}, "status", status)
        h.close()
        return
    d = h.dims()
    D = d["dim_ea"] if a.sector == "ea" else d["dim_ip"]
    nvec = a.nvec or s.nmo
    x = torch.randn((nvec, D), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    fn = B.sigma_ea if a.sector == "ea" else B.sigma_ip
    fn(h, 0, x, y, prec=prec)
    for _ in range(a.calls):
        fn(h, 0, x, y, prec=prec)
    torch.cuda.synchronize()
    # one call inside an NVTX range, for captures restricted to it (ncu --nvtx --nvtx-include "profiled/")
    torch.cuda.nvtx.range_push("profiled")
    fn(h, 0, x, y, prec=prec)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    prof = B.sigma_profile(h, B.EA if a.sector == "ea" else B.IP, 0, x, y, prec=prec)
    for name, ms, fl, kern in prof:
        print(f"{name:20s} {ms:9.3f} ms  {fl / 1e9:10.3f} GFLOP  {fl / max(ms, 1e-9) / 1e9:8.3f} TFLOP/s  kernel {kern}")
    h.close()


if __name__ == "__main__":
    main()
