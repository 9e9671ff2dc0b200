"""Benchmark of the periodic CCGF hot path on GB300.

Workload (default): the Si-like 3x3x3 k-mesh system (nk = 27, nocc = 4, nvir = 30 per k,
Naux = 96, 128 frequencies in [-0.8, 0.8] Ha, eta = 0.005 Ha), synthetic seeded inputs. One step
= one (k-point, frequency) pair: the removal (IP) and addition (EA) shifted systems of all 34
orbitals are solved by batched GMRES to relative residual 1e-6 and contracted into G_pq(k, w)
(34^2 = 1156 complex elements per step); successive steps take successive (k, w) pairs. The
build of the similarity-transformed Hamiltonian blocks is timed apart (a one-time cost).
`value` there is the chosen form: inner sigma on the tensor cores (3xTF32) inside refinement
whose true residual is computed in FP64; the plain FP64 form is timed on an equal-work slice.

--workload si_k222_o4v22: the Si 2x2x2 shape (nk = 8, nocc = 4, nvir = 22, 64 frequencies);
one step = one frequency for all 8 k-points. `value` there is the plain FP64 form (every step in
FP64), the chosen form (true residual from the FP64-accurate sliced tensor-core sigma) is timed
on the same steps beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference] [--workload NAME]

Under torchrun every rank solves its own (k, w) points (no data-path collective); rank 0
prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G_pq(k,ω) elements/s at rel. residual 1e-6; sigma TFLOP/s vs GB300 peak"
WORKLOAD = "si_k333_o4v30"
TOL = 1e-6
# FP64 SIMT peak: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (the nominal 1.25 TFLOP/s of the part)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# dense TF32 tensor peak: the measured bf16 GEMM burst figure x the nominal TF32/BF16 ratio (1.1/2.25);
# the 3xTF32 split issues three real MMAs on the 2x2 real embedding of every complex multiply-add
# (24 real flop per 8 algorithmic flop), so its ceiling in algorithmic flop/s is a third of that
TF32_NOMINAL_RATIO = 1.1 / 2.25


KERNEL_NAMES = {100: "tc_zgemm_tma_kernel", 101: "tc_zgemm_kernel", 102: "tc_zgemm_bulk_kernel", 103: "tc_zgemm_oz_kernel",
                200: "zgemm_smallm_kernel",
                300: "tc_zgemm_kernel<FP64-stored A>", 301: "tgemm_kernel<float, FP64-stored A>", 400: "tgemm_kernel"}
# the SIMT launcher's tile candidates in its order: per-thread rows, columns of complex outputs,
# thread rows of the CTA
SIMT_TILES = [(4, 4, 16), (3, 4, 16), (2, 4, 16), (4, 3, 16), (4, 2, 16), (4, 7, 16), (3, 7, 16), (2, 7, 16),
              (2, 2, 16), (1, 4, 16), (1, 7, 16), (1, 2, 16), (11, 2, 8), (3, 2, 8)]


def kernel_name(code, dtype):
    """Name of the kernel behind a plan step's choice code (ccgf_sigma_step_kernel)."""
    if code in KERNEL_NAMES:
        return KERNEL_NAMES[code]
    if code <= 0:
        return f"zgemm_kernel<{dtype}>"
    tm, tn, ty = SIMT_TILES[code % 1000 - 1]
    return f"zgemm_kernel<{dtype}, {tm}, {tn}, {ty}>" + (f" split-K {code // 1000}" if code >= 1000 else "")


def gemm_kernel_sha():
    """sha256 of the SIMT GEMM kernel's source (the template definition in kernels.cu): a stored
    DRAM-traffic figure is used only while the kernel it was measured on is unchanged."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_2208_07478_gb300", "csrc", "kernels.cu")).read()
    start = src.index("template <typename R, int TM, int TN, int TY = 16>\n__global__")
    end = src.index("\n}\n", start) + 3
    return hashlib.sha256(src[start:end].encode()).hexdigest()


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: the workload's, about a minute of timed work)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-chosen", action="store_true", help="skip the chosen-form measurement")
    ap.add_argument("--chosen-prec", default="tf32x3", choices=["tf32x3", "fp32"],
                    help="inner sigma of the chosen form: tensor cores (3xTF32) or FP32 SIMT")
    ap.add_argument("--refine", default="auto", choices=["auto", "fp64", "fp64_tc"],
                    help="true residual of the chosen form: FP64 SIMT sigma, or the FP64-accurate sliced tensor-core "
                         "sigma (auto: the workload's setting)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed
def dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("CCGF_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg, device=None):
    if pg is not None:
        if device is not None:
            pg.barrier(device_ids=[device])
        else:
            pg.barrier()


def max_over_ranks(pg, x, device=None):
    """Largest value over the ranks (device None: a CPU tensor, for the gloo backend)."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def omega_index(rank, world, step, nomega):
    """Frequency point of (rank, step): a rank-strided walk over the grid, so ranks never share a point."""
    return (rank + world * step) % nomega


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm
# Per workload: the form its configuration names (`value`), and the right-hand sides of one step.
#   all_k: one frequency, every k-point and orbital (nk * nmo^2 G elements per step)
#   one_k: one (k-point, frequency) pair, every orbital (nmo^2 G elements per step), for meshes where a
#          step over all k would take minutes
PROFILE = {
    # refine: the chosen form's true-residual sigma. The sliced FP64-accurate tensor-core sigma where
    # its copies of the intermediates fit; on the 3x3x3 and ZnO-like meshes the ladder's would not,
    # the other sliced copies then only take memory from the batch, and FP64 SIMT is used
    # steps: the default number of timed steps (about a minute of timed work)
    "gamma_ip_o4v12": dict(form="fp64", per_step="all_k", sectors="ip", refine="fp64_tc", steps=4),
    "si_k222_o4v22": dict(form="fp64", per_step="all_k", sectors="ipea", refine="fp64_tc", steps=4),
    "si_k333_o4v30": dict(form="tf32x3", per_step="one_k", sectors="ipea", refine="fp64", steps=1),
    "zno_k222_o18v60": dict(form="tf32x3", per_step="one_k", sectors="ipea", refine="fp64", steps=1),
}


def step_point(rank, world, step, nk, nomega, per_step):
    """(k-point or -1 for all, frequency index) of a step: a rank-strided walk, ranks never share a point."""
    idx = rank + world * step
    if per_step == "all_k":
        return -1, idx % nomega
    return idx % nk, (nomega // 2 + idx // nk) % nomega


def vector_roofline(solver):
    """Roofline of the Arnoldi vector steps (shift, CGS2, norm, normalisation): HBM bytes and FP64
    flops against their peaks; the bound is the resource whose minimum time is longer."""
    vms = solver.get("vector_ms") or 0.0
    if vms <= 0:
        return {"gbs": None}
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    t_hbm = solver["vector_bytes"] / (hbm * 1e9)
    t_alu = solver["vector_flops"] / (FP64_PEAK_TFLOPS * 1e12)
    bound = "hbm" if t_hbm >= t_alu else "alu"
    t_min = max(t_hbm, t_alu)
    return {"gbs": solver["vector_gbs"], "frac_of_hbm": round(solver["vector_gbs"] / hbm, 4),
            "tflops_fp64": solver["vector_tflops"], "frac_of_fp64": round(solver["vector_tflops"] / FP64_PEAK_TFLOPS, 4),
            "bound": bound, "frac_of_bound": round(t_min / (vms / 1e3), 4),
            "peak_basis": "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs, of measured); FP64 SIMT "
                          "152 x 2 DFMA x 2 x 2.07 GHz (derived, of nominal)",
            "what": "shift, CGS2 dots and updates, norm, normalisation after every sigma: 16 (4J + 12) D nv bytes and "
                    "(32 J + 14) D nv FP64 flops per Arnoldi step over CUDA-event time"}


def gpu_arm(args):
    import torch
    from paper_2208_07478_gb300 import binding as B
    from paper_2208_07478_gb300.synth import make_workload

    rank, world, local, pg = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    prof_cfg = PROFILE[args.workload]
    if args.refine == "auto":
        args.refine = prof_cfg["refine"]
    s = make_workload(args.workload)
    nk, N = s.nk, s.nmo
    nomega = len(s.omega)
    sectors = B.IP if prof_cfg["sectors"] == "ip" else B.BOTH
    per_step = prof_cfg["per_step"]
    elems_per_step = (nk if per_step == "all_k" else 1) * N * N
    form_prec = {"fp64": B.FP64, "tf32x3": B.TF32X3, "fp32": B.FP32}
    vprec = form_prec[prof_cfg["form"]]
    oprec = B.TF32X3 if vprec == B.FP64 else B.FP64
    if args.chosen_prec == "fp32":
        vprec = B.FP32 if vprec != B.FP64 else vprec
        oprec = B.FP32 if oprec != B.FP64 else oprec

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    Gd = torch.zeros((nk, 1, N, N), dtype=torch.complex128, device=dev)

    def options(prec, K=-1, orbitals=None):
        kw = dict(prec=prec, tol=TOL, restart_m=40, max_iter=4000, max_refine=40, kpoint=K,
                  refine_prec=B.FP64_TC if args.refine == "fp64_tc" else B.FP64)
        if orbitals is not None:
            kw.update(orbital_first=orbitals[0], orbital_count=orbitals[1])
        return B.default_options(**kw)

    def run_step(h, prec, step, keep=None, orbitals=None, point=None):
        K, w = point if point is not None else step_point(rank, world, step, nk, nomega, per_step)
        status, st = B.solve_gf(h, sectors, s.omega[[w]], s.eta, Gd, options=options(prec, K, orbitals), on_device=True,
                                stream=stream)
        if status != B.CCGF_OK:
            raise RuntimeError(f"solve did not converge (status {status})")
        if keep is not None:
            keep.append(Gd.clone())
        return st

    # build (timed on its own: a one-time cost amortised over the whole frequency grid)
    dL, dt1, dt2, deps = to_dev(s.L), to_dev(s.t1), to_dev(s.t2), to_dev(s.mo_energy)
    torch.cuda.synchronize()
    eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eb0.record(stream)
    h = B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, deps, dL, dt1, dt2, on_device=True, stream=stream)
    eb1.record(stream)
    torch.cuda.synchronize()
    build_ms = eb0.elapsed_time(eb1)
    del dL, dt1, dt2, deps
    torch.cuda.empty_cache()

    def timed(prec, first, keep=None):
        """W warm-up steps (plans, autotuning, low-precision copies), then K timed steps between
        synchronised barriers; returns (ms, stats, launches in the timed region)."""
        for k in range(args.warmup):
            run_step(h, prec, first + k)
        torch.cuda.synchronize()
        barrier(pg, local)
        torch.cuda.synchronize()
        l0 = h.launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        torch.cuda.nvtx.range_push("timed")     # for profiler captures restricted to the timed region
        st = [run_step(h, prec, first + args.warmup + k, keep) for k in range(args.steps)]
        torch.cuda.nvtx.range_pop()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(pg, local)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), st, h.launch_count() - l0

    def solver_summary(st):
        vms = sum(float(x["vector_ms"]) for x in st)
        vbytes = sum(float(x["vector_bytes"]) for x in st)
        return {"inner_iterations": sum(int(x["inner_iterations"]) for x in st),
                "fp64_sigma_calls": sum(int(x["fp64_sigma_calls"]) for x in st),
                "lowp_sigma_calls": sum(int(x["lowp_sigma_calls"]) for x in st),
                "max_rel_residual": max(float(x["max_rel_residual"]) for x in st),
                "restart_used": max(int(x["restart_used"]) for x in st),
                "columns_per_batch": max(int(x["columns_per_batch"]) for x in st),
                "sigma_ms": round(sum(float(x["sigma_ms"]) for x in st), 2),
                "vector_ms": round(vms, 2),
                "refine_ms": round(sum(float(x["refine_ms"]) for x in st), 2),
                "vector_gbs": round(vbytes / (vms / 1e3) / 1e9, 1) if vms > 0 else None,
                "vector_tflops": (round(sum(float(x["vector_flops"]) for x in st) / (vms / 1e3) / 1e12, 4)
                                  if vms > 0 else None),
                "vector_bytes": vbytes, "vector_flops": sum(float(x["vector_flops"]) for x in st)}

    def sigma_roofline(prec):
        """Live per-step timing of one EA sigma (k = 0, nmo vectors) in form prec: the dominant kernel."""
        D = h.dims()["dim_ea"]
        x = torch.randn((N, D), dtype=torch.complex128, device=dev)
        y = torch.empty_like(x)
        B.sigma_profile(h, B.EA, 0, x, y, prec=prec, stream=stream)          # plan + warm-up
        prof = B.sigma_profile(h, B.EA, 0, x, y, prec=prec, stream=stream)
        del x, y
        torch.cuda.empty_cache()
        sig_ms = sum(p[1] for p in prof)
        sig_fl = sum(p[2] for p in prof)
        top = max(prof, key=lambda p: p[1])
        achieved = top[2] / (top[1] / 1e3) / 1e12
        dtype = "double" if prec in (B.FP64, B.FP64_TC) else "float"
        if prec == B.FP64 or (prec == B.FP64_TC and top[3] != 103):
            roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                    "peak_basis": "FP64 SIMT: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz (derived, of nominal)"}
        else:
            # 3xTF32: three TF32 products per complex multiply-add; sliced FP64: fifteen
            nprod = 15 if prec == B.FP64_TC else 3
            bf16 = measured_peaks().get("bf16_tflops")
            peak = (bf16 or 1900.0) * TF32_NOMINAL_RATIO / nprod
            roof = {"bound": "tensor", "achieved": round(achieved, 3), "peak": round(peak, 1), "unit": "TFLOP/s",
                    "peak_basis": ("measured bf16 burst %.0f TFLOP/s x nominal TF32/BF16 1.1/2.25 / %d MMAs per product (%s)"
                                   % (bf16 or 1900.0, nprod, "of measured" if bf16 else "of fallback"))}
        roof.update({"kernel": f"{kernel_name(top[3], dtype)} ({top[0]})", "frac": round(achieved / roof["peak"], 4),
                     "traffic": None, "launch_ms": round(top[1], 4), "algorithmic_flops_per_launch": top[2]})
        tfile = os.path.join(ROOT, "profiles", "roofline_traffic.json")
        if prec == B.FP64 and os.path.exists(tfile):
            try:
                tinfo = json.load(open(tfile))
                same = (tinfo.get("kernel_source_sha256") == gemm_kernel_sha() and tinfo.get("kernel") == kernel_name(top[3], dtype)
                        and tinfo.get("kernel_step") == top[0] and tinfo.get("precision") == "fp64"
                        and tinfo.get("workload") == args.workload)
                if same:
                    roof["traffic"] = tinfo.get("dram_bytes_per_launch")
                    roof["traffic_source"] = tinfo.get("source")
            except (OSError, ValueError):
                pass
        sig = {"precision": {B.FP64: "fp64", B.FP32: "fp32", B.TF32X3: "tf32x3", B.FP64_TC: "fp64_tc"}[prec], "sector": "ea", "nvec": N,
               "ms": round(sig_ms, 3), "tflops": round(sig_fl / (sig_ms / 1e3) / 1e12, 4)}
        return roof, sig

    clocks = ClockSampler(local)
    clocks.start()
    Gv = []
    ms_v, st_v, launches = timed(vprec, 0, Gv)
    clk = clocks.stop()
    ms_v = max_over_ranks(pg, ms_v, dev)
    value = world * args.steps * elems_per_step / (ms_v / 1e3)
    roof, sig = sigma_roofline(vprec)
    roof_inner = sig_inner = None
    if vprec != B.FP64:
        # the dominant kernel of a refined form sits in whichever sigma took more of the timed region
        inner_ms = sum(float(x["sigma_ms"]) for x in st_v)
        refine_ms = sum(float(x["refine_ms"]) for x in st_v)
        if refine_ms > inner_ms:
            roof_inner, sig_inner = roof, sig
            roof, sig = sigma_roofline(B.FP64_TC if args.refine == "fp64_tc" else B.FP64)
            roof["dominant"] = (f"true-residual sigma: {refine_ms / 1e3:.1f} s of the timed region against "
                                f"{inner_ms / 1e3:.1f} s of inner sigma")
    total_elems = nk * nomega * N * N
    step_s = ms_v / 1e3 / args.steps
    steps_grid = total_elems / elems_per_step
    form_names = {B.FP64: "plain fp64 (every step in FP64)",
                  B.TF32X3: ("chosen: tensor-core sigma (tcgen05 kind::tf32, operands split hi+lo, 3 MMAs, FP32 accumulate) "
                             "inside FP64 refinement (FP64 Krylov basis; true residual with the "
                             + ("FP64-accurate sliced tensor-core sigma, exact 8-bit slices, error ~2^-41 of n max|a| max|b|, "
                                "FP64 SIMT where the sliced copy does not fit)" if args.refine == "fp64_tc" else "FP64 SIMT sigma)")),
                  B.FP32: "chosen: FP32 SIMT sigma inside FP64 refinement"}
    out = {"metric": METRIC, "value": round(value, 3), "unit": "G elements/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_v / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 (complex128)" if vprec == B.FP64 else "f32 sigma (complex64, 3xTF32) + f64 refinement",
           "data": f"synthetic (seeded; shapes of the {args.workload} workload)",
           "config": {"workload": args.workload, "kmesh": list(s.kmesh), "nocc": s.nocc, "nvir": s.nvir,
                      "naux": s.naux, "eta": s.eta, "omega_grid": [float(s.omega[0]), float(s.omega[-1]), nomega],
                      "step": ("one frequency, all k-points and orbitals" if per_step == "all_k"
                               else "one (k-point, frequency) pair, all orbitals"),
                      "g_elements_per_step": elems_per_step, "sectors": prof_cfg["sectors"], "tol": TOL,
                      "form": form_names[vprec],
                      "timed": "K steps (the build is timed separately, below)",
                      "l2": "inputs larger than L2 (intermediates and Krylov basis of several GB)",
                      "parallelism": f"replicas x{world} (frequency / k-point batches sharded)"},
           "build": {"ms": round(build_ms, 1),
                     "value_with_build_amortised_over_grid": round(total_elems / (build_ms / 1e3 + steps_grid * step_s), 3),
                     "what": f"build + {steps_grid:.0f} steps of this kind cover all nk x nomega x nmo^2 = {total_elems} G elements"},
           "roofline": roof, "sigma": sig, "gpu_launches": launches, "clocks": clk,
           **({"roofline_inner_sigma": roof_inner, "inner_sigma": sig_inner} if roof_inner else {}),
           "solver": solver_summary(st_v)}
    out["vector_steps"] = vector_roofline(out["solver"])
    for key in ("vector_bytes", "vector_flops"):
        out["solver"].pop(key, None)

    if not args.no_chosen:
        other = {}
        if per_step == "all_k":
            # the other form on the same steps
            Go = []
            ms_o, st_o, _ = timed(oprec, 0, Go)
            ms_o = max_over_ranks(pg, ms_o, dev)
            v_o = world * args.steps * elems_per_step / (ms_o / 1e3)
            other = {"value": round(v_o, 3), "unit": "G elements/s", "ms_per_step": round(ms_o / args.steps, 3),
                     "same_steps_as_value": True, "solver": solver_summary(st_o)}
            ga, gb = (torch.stack(Gv) if vprec == B.FP64 else torch.stack(Go)), (torch.stack(Go) if vprec == B.FP64 else torch.stack(Gv))
            t_fp64, t_low = (ms_v, ms_o) if vprec == B.FP64 else (ms_o, ms_v)
        else:
            # equal work: both forms on one slice (k = 0, four orbitals around the gap, one frequency)
            orbs = (max(0, s.nocc - 2), min(4, N))
            point = (0, nomega // 2)
            Gs = {}
            times = {}
            for prec in (vprec, oprec):
                run_step(h, prec, 0, orbitals=orbs, point=point)                 # warm-up (plans, tuning)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                keep = []
                e0.record(stream)
                st_o = run_step(h, prec, 0, keep=keep, orbitals=orbs, point=point)
                e1.record(stream)
                torch.cuda.synchronize()
                times[prec] = e0.elapsed_time(e1)
                Gs[prec] = keep[0]
            other = {"slice": f"k=0, orbitals {orbs[0]}..{orbs[0] + orbs[1] - 1}, w={float(s.omega[point[1]]):.4f}, both sectors",
                     "ms_value_form": round(times[vprec], 1), "ms_other_form": round(times[oprec], 1),
                     "projected_value": round(value * times[vprec] / times[oprec], 3),
                     "what": "the other form timed on an equal-work slice (1 warm-up + 1 timed run each); projected_value "
                             "scales `value` by the slice time ratio"}
            ga, gb = Gs[B.FP64][None], Gs[vprec if vprec != B.FP64 else oprec][None]
            t_fp64, t_low = times[B.FP64], times[vprec if vprec != B.FP64 else oprec]
        other["form"] = form_names[oprec]
        ga, gb = ga.cpu().numpy(), gb.cpu().numpy()
        mask = np.abs(ga) > 0
        dg = np.abs(gb - ga)[mask]
        rel = dg / np.maximum(1.0, np.abs(ga)[mask])
        out["other_form"] = other
        out["chosen_vs_plain_fp64"] = {
            "speedup": round(t_fp64 / t_low, 3),
            "elements": int(dg.size), "max_abs_dG": float(dg.max()), "max_rel_dG": float(rel.max()),
            "rel_dG_quantiles_50_90_99": [float(q) for q in np.quantile(rel, [0.5, 0.9, 0.99])],
            "max_abs_G": float(np.abs(ga).max()),
            "what": "|G_chosen - G_fp64| / max(1, |G_fp64|) per element, both at rel. residual 1e-6"}

    if not args.no_e2e:
        # end to end through the public API with host buffers: H2D of the inputs from pinned memory,
        # build, one step, D2H of G, inside the timed region
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hL, ht1, ht2, heps = pin(s.L), pin(s.t1), pin(s.t2), pin(s.mo_energy)
        Gh = torch.zeros((nk, 1, N, N), dtype=torch.complex128).pin_memory()
        h_in = sum(int(t.numel() * t.element_size()) for t in (hL, ht1, ht2, heps))
        h.close()
        torch.cuda.empty_cache()
        K, w = step_point(rank, world, args.warmup + args.steps, nk, nomega, per_step)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        he = B.build_intermediates(s.kmesh, s.nocc, s.nvir, s.naux, heps, hL, ht1, ht2, stream=stream)
        e2e_status, e2e_st = B.solve_gf(he, sectors, s.omega[[w]], s.eta, Gh, options=options(vprec, K), stream=stream)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        he.close()
        if e2e_status != B.CCGF_OK:
            raise RuntimeError(f"end-to-end solve did not converge (status {e2e_status})")
        te = max_over_ranks(pg, te, dev)
        out["e2e"] = {"value": round(world * elems_per_step / te, 3), "unit": "G elements/s",
                      "h2d_bytes_per_step": h_in, "d2h_bytes_per_step": int(Gh.numel() * Gh.element_size()),
                      "max_rel_residual": float(e2e_st["max_rel_residual"]),
                      "what": "build_intermediates from pinned host arrays + solve_gf of one step with G to host "
                              "(the build, a one-time cost, is inside this region)"}
    else:
        h.close()

    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(s, args.workload, per_step)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()


# ----------------------------------------------------------------------------- oracle (CPU) arm
def oracle_build(s):
    from oracle.kccsd import KEOM
    t0 = time.perf_counter()
    ke = KEOM(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, L=s.L)
    return ke, time.perf_counter() - t0


def oracle_sample(s, ke, omega, samples):
    """GMRES (same tolerance, the oracle's own diagonal preconditioner) of the IP and EA right-hand
    sides of each sampled (K, orbital) at one frequency; returns the per-right-hand-side times."""
    from oracle.kccsd import diag_estimate
    from oracle import solvers
    om = float(omega)
    t_ip, t_ea = [], []
    for K, p in samples:
        for kind in ("ip", "ea"):
            z = om - 1j * s.eta if kind == "ip" else om + 1j * s.eta
            sgn = 1.0 if kind == "ip" else -1.0
            d = diag_estimate(ke, kind, K)
            sig = ke.sigma_ip if kind == "ip" else ke.sigma_ea
            b = ke.rhs_ip(K, p) if kind == "ip" else ke.rhs_ea(K, p)
            t1 = time.perf_counter()
            solvers.gmres(lambda x: z * x + sgn * sig(K, x), b, tol=TOL, restart=40,
                          precond=lambda v: v / (z + sgn * d))
            (t_ip if kind == "ip" else t_ea).append(time.perf_counter() - t1)
    return t_ip, t_ea


def oracle_rate(s, t_build, t_ip, t_ea):
    """G elements/s of a step (nk * nmo right-hand sides per sector) with the build amortised over the grid."""
    nrhs = s.nk * s.nmo
    t_step = nrhs * (float(np.mean(t_ip)) + float(np.mean(t_ea))) + t_build / len(s.omega)
    return s.nk * s.nmo * s.nmo / t_step, t_step


def baseline_samples(s):
    """(K, orbital) pairs the CPU baseline solves: HOMO and LUMO at the first and last k-point."""
    ks = sorted({0, s.nk - 1})
    return [(K, p) for K in ks for p in (s.nocc - 1, s.nocc)]


def rows_oracle_build(s):
    from oracle.rows import KRows
    t0 = time.perf_counter()
    kr = KRows(s.kmesh, s.nocc, s.mo_energy, s.t1, s.t2, s.L)
    return kr, time.perf_counter() - t0


def rows_oracle_time(s, kr, rows_per_sector, seed):
    """Seconds per output row of one IP and one EA sigma at k = 0 (sampled rows): {kind: (s per row, D)}."""
    rng = np.random.default_rng(seed)
    per_row = {}
    for kind in ("ip", "ea"):
        n1 = s.nocc if kind == "ip" else s.nvir
        D = n1 + s.nk * s.nk * s.nocc * s.nvir * (s.nocc if kind == "ip" else s.nvir)
        x = rng.normal(size=D) + 1j * rng.normal(size=D)
        rows = n1 + rng.choice(D - n1, size=rows_per_sector, replace=False)
        t1 = time.perf_counter()
        (kr.sigma_ip_elements if kind == "ip" else kr.sigma_ea_elements)(0, x, rows)
        per_row[kind] = ((time.perf_counter() - t1) / rows_per_sector, D)
    return per_row


def rows_oracle_sample(s, rows_per_sector=4, seed=3):
    """The element-wise oracle (the only one that fits the large meshes): its build, then sampled
    output rows of one IP and one EA sigma at k = 0; returns (build s, {kind: (s per row, D)})."""
    kr, t_build = rows_oracle_build(s)
    return t_build, rows_oracle_time(s, kr, rows_per_sector, seed)


SIGMA_PER_RHS = 10   # sigma applications per right-hand side assumed for the element-wise oracle's estimate


def rows_oracle_rate(s, t_build, per_row):
    """G elements/s of a one-(k, w) step: nmo right-hand sides per sector, each needing SIGMA_PER_RHS full
    sigma applications of D rows, plus the build amortised over the grid."""
    t_step = sum(s.nmo * SIGMA_PER_RHS * D * t for t, D in per_row.values()) + t_build / (s.nk * len(s.omega))
    return s.nmo * s.nmo / t_step, t_step


def cpu_baseline(s, workload, per_step):
    """The CPU oracle as it stands, timed on the host cores on a bounded sample of one step."""
    t0 = time.perf_counter()
    if per_step == "all_k":
        ke, t_build = oracle_build(s)
        samples = baseline_samples(s)
        t_ip, t_ea = oracle_sample(s, ke, s.omega[0], samples)
        v, t_step = oracle_rate(s, t_build, t_ip, t_ea)
        sample = (f"oracle build {t_build:.1f} s (amortised over {len(s.omega)} frequencies) + GMRES to rel. "
                  f"residual {TOL:g} of {len(t_ip)} IP (mean {np.mean(t_ip):.2f} s) and {len(t_ea)} EA (mean "
                  f"{np.mean(t_ea):.2f} s) right-hand sides (K, orbital) = {samples} at w={float(s.omega[0]):.4f}, "
                  f"extrapolated to the step's {s.nk * s.nmo} + {s.nk * s.nmo} right-hand sides "
                  f"({t_step:.0f} s per step); numpy, default BLAS threads")
        measured = round(float(np.sum(t_ip) + np.sum(t_ea)), 1)
    else:
        t_build, per_row = rows_oracle_sample(s)
        v, t_step = rows_oracle_rate(s, t_build, per_row)
        sample = (f"element-wise oracle (the full oracle would need the ~{16 * s.nk ** 3 * s.nmo ** 4 / 1e9:.0f} GB "
                  f"integral tensor): build {t_build:.1f} s, then sampled sigma rows at k=0 "
                  f"(IP {per_row['ip'][0]:.3f} s / row of {per_row['ip'][1]}, EA {per_row['ea'][0]:.3f} s / row of "
                  f"{per_row['ea'][1]}); one step = {s.nmo} right-hand sides per sector x {SIGMA_PER_RHS} sigma "
                  f"applications of all rows (assumed), = {t_step:.3g} s; numpy, default BLAS threads")
        measured = round(sum(4 * t for t, _ in per_row.values()), 1)
    return {"value": float(f"{v:.4g}"), "unit": "G elements/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": sample, "seconds_measured": round(time.perf_counter() - t0, 1), "solve_seconds_measured": measured}


def reference_arm(args):
    """The oracle as the reference arm, on the same workload: build once, then per step a bounded
    sample of that step's work, rate extrapolated per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2208_07478_gb300.synth import make_workload
    s = make_workload(args.workload)
    per_step = PROFILE[args.workload]["per_step"]
    t_all = time.perf_counter()
    rates, steps_ms, measured = [], [], []
    if per_step == "all_k":
        ke, t_build = oracle_build(s)
        samples = baseline_samples(s)
        for k in range(args.warmup + args.steps):
            t_ip, t_ea = oracle_sample(s, ke, s.omega[k % len(s.omega)], [samples[k % len(samples)]])
            v, t_step = oracle_rate(s, t_build, t_ip, t_ea)
            if k >= args.warmup:
                rates.append(v)
                steps_ms.append(t_step * 1e3)
                measured.append(float(np.sum(t_ip) + np.sum(t_ea)))
        sample = (f"oracle build {t_build:.1f} s amortised over {len(s.omega)} frequencies; per step GMRES to rel. "
                  f"residual {TOL:g} of 1 IP + 1 EA right-hand side, (K, orbital) cycling over {samples}, "
                  f"extrapolated to the step's {s.nk * s.nmo} + {s.nk * s.nmo} right-hand sides")
    else:
        kr, t_build = rows_oracle_build(s)
        for k in range(args.warmup + args.steps):
            t1 = time.perf_counter()
            per_row = rows_oracle_time(s, kr, 2, seed=k)
            v, t_step = rows_oracle_rate(s, t_build, per_row)
            if k >= args.warmup:
                rates.append(v)
                steps_ms.append(t_step * 1e3)
                measured.append(time.perf_counter() - t1)
        sample = (f"element-wise oracle: build {t_build:.1f} s, sampled sigma rows (IP {per_row['ip'][0]:.3f} s, EA "
                  f"{per_row['ea'][0]:.3f} s per row); a step = {s.nmo} right-hand sides per sector x {SIGMA_PER_RHS} "
                  f"full sigma applications (assumed)")
    v = float(np.mean(rates))
    out = {"metric": METRIC, "value": float(f"{v:.4g}"), "unit": "G elements/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(float(np.mean(steps_ms)), 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (complex128)",
           "data": f"synthetic (seeded; shapes of the {args.workload} workload)", "impl": "reference",
           "config": {"workload": args.workload, "kmesh": list(s.kmesh), "nocc": s.nocc, "nvir": s.nvir,
                      "naux": s.naux, "eta": s.eta, "sectors": "ip+ea", "tol": TOL},
           "cpu_baseline": {"value": float(f"{v:.4g}"), "unit": "G elements/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": float(f"{v:.4g}"), "unit": "G elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "ms_per_step_is": "extrapolated from the measured sample below",
           "measured": {"build_s": round(t_build, 1), "solve_s_per_timed_step": [round(x, 2) for x in measured],
                        "total_s": round(time.perf_counter() - t_all, 1)},
           "seconds": round(time.perf_counter() - t_all, 1)}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.steps is None:
        args.steps = PROFILE[args.workload]["steps"]
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
