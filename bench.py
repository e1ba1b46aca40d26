#!/usr/bin/env python3
"""Throughput of the batched CMA-ES generation loop on GB300.

Workload (default): the IPOP-CMA-ES configuration on the rotated Rastrigin,
n = 100, lambda0 = 17 with population levels 17 * 2^k for k = 0..9 (lambda up
to 8704), laid out as the paper's K-Distributed strategy (§3.2.3): the ten
levels run side by side as one batch of ten searches, each restarting at its
own size when a stop test fires. One step = one generation of every search =
17391 candidates sampled, evaluated and used in the update (rank,
recombination, paths, step size, rank-one + rank-mu covariance update), plus
the lazy FP64 eigendecomposition when due (every generation here) and the
stop tests. Inputs are seeded synthetic instances (no BBOB data).

Prints one JSON line (rank 0). Timing: W warm-up generations, then K timed
generations, each bracketed by CUDA events on the launch stream, with a
256 MiB write between timed generations to flush L2. Per-phase device times
come from CUDA events the engine records on the same stream.

--impl reference times the FP64 CPU oracle on this host's cores on the same
workload (test infrastructure; it is the method's plain restatement).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "candidates/sec sampled+evaluated+updated; mixed vs plain FP64 GPU; % roofline"
UNIT = "candidates/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["engine", "reference"], default="engine")
    ap.add_argument("--precision", choices=["fp64", "tf32", "bf16"], default="tf32",
                    help="headline path; the other two are measured beside it")
    ap.add_argument("--headline-only", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    from paper_2409_11765_gb300 import dist as D
    return D.env()


def workload():
    from paper_2409_11765_gb300 import workloads as W
    return W.rastrigin_n100_ipop(concurrent=True)


def workload_config(wl, precision):
    s0 = wl.searches[0]
    return {"workload": wl.name, "searches": len(wl.searches), "n": s0.n,
            "lambdas": [s.lam for s in wl.searches],
            "candidates_per_step": wl.candidates_per_generation,
            "objective": "rotated Rastrigin (seeded Haar Q, x* ~ U[-4,4]^n)",
            "layout": "K-Distributed: levels lambda=17*2^k, k=0..9, one batch",
            "precision": precision,
            "gemms": {"fp64": "FP64 CUDA cores", "tf32": "tcgen05 kind::tf32 (objective, rank-mu: 3-term split)",
                      "bf16": "tcgen05 kind::f16 bf16 (objective, rank-mu: 3-term split)"}[precision],
            "eig": "FP64 warm-started Jacobi, every generation (lazy rule gives 1)",
            "l2": "256 MiB write between timed generations", "seed": 20240918}


# ----------------------------- CPU oracle ----------------------------------
def oracle_searches(wl):
    from oracle import cmaes
    sts, probs = [], []
    for s in wl.searches:
        sts.append(cmaes.State(s.n, s.lam, s.sigma0, s.x0.copy(), s.sigma0))
        p = s.problem
        probs.append(cmaes.Problem(p.kind, p.xstar, p.Q, p.lamdiag))
    opts = cmaes.Options(f_target=wl.f_target, box_lo=wl.box_lo, box_hi=wl.box_hi,
                         max_restarts=wl.max_restarts if wl.max_restarts < 255 else 10 ** 9,
                         ipop_double=wl.ipop_double)
    return sts, probs, opts


def oracle_step(sts, probs, opts):
    from oracle import cmaes
    from paper_2409_11765_gb300 import workloads as W
    cand = 0
    for i, (st, pr) in enumerate(zip(sts, probs)):
        if not st.done:
            cand += st.lam
            cmaes.generation(st, W.SEED, i, pr, opts)
    return cand


def cpu_baseline(wl, seconds):
    """The oracle as it stands, on this host's cores, for a bounded sample of
    generations of the same batch."""
    sts, probs, opts = oracle_searches(wl)
    t0 = time.perf_counter()
    cand = 0
    gens = 0
    while True:
        cand += oracle_step(sts, probs, opts)
        gens += 1
        el = time.perf_counter() - t0
        if el >= seconds and gens >= 2:
            break
    return {"value": cand / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d generations of the full 10-search batch (%d candidates) in %.1f s; "
                      "numpy FP64, BLAS threads = host cores" % (gens, cand, el)}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    wl = workload()
    sts, probs, opts = oracle_searches(wl)
    for _ in range(args.warmup):
        oracle_step(sts, probs, opts)
    t0 = time.perf_counter()
    cand = 0
    for _ in range(args.steps):
        cand += oracle_step(sts, probs, opts)
    el = time.perf_counter() - t0
    value = cand / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(wl, "fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": "%d timed generations of the full batch" % args.steps},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------- clocks -------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index),
                                       "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------ GPU engine ----------------------------------
def eig_flops(n, decompositions):
    """Algorithmic FP64 flops of the eigendecompositions: per decomposition of
    an n x n C warm-started from the previous basis, 4 n^3 for B^T C B, 9 n^3
    per Jacobi sweep with s = 2 sweeps (a warm start needs one to three) and
    2 n^3 for the basis update B V: 24 n^3. The figure is the problem's, not
    the engine's: its refined route spends its FP64 flops on dense products
    and its sweeps in FP32 (cmaes_eig_stats reports what actually ran)."""
    return (4.0 + 9.0 * 2 + 2.0) * n ** 3 * decompositions


# DRAM bytes of the eigendecomposition phase per generation (ncu dram__bytes_read.sum +
# dram__bytes_write.sum over its kernels, one warm generation of the headline workload, one
# capture). Valid only for the engine sources it was
# measured on: any change to them makes the roofline's traffic null until it is measured again.
EIG_TRAFFIC = {"bytes": 36944896, "sources_sha256_16": "6040ce6c27b78da5"}


def engine_sources_sha():
    """Hash of the engine's CUDA/C++ sources with comments and blank lines
    removed: a change to the code voids the recorded traffic, a change to a
    comment does not."""
    import glob
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2409_11765_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "*.cu"))) + sorted(glob.glob(os.path.join(csrc, "*.cuh"))) \
        + sorted(glob.glob(os.path.join(csrc, "*.h")))
    # string and character literals are kept whole so that "//" inside them is not a comment
    token = re.compile(r'"(?:\\.|[^"\\\n])*"|\'(?:\\.|[^\'\\\n])*\'|//[^\n]*|/\*.*?\*/', re.S)
    h = hashlib.sha256()
    for f in files:
        text = open(f, encoding="utf-8").read()
        code = token.sub(lambda m: m.group(0) if m.group(0)[0] in "\"'" else " ", text)
        lines = [ln.rstrip() for ln in code.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


PREC = {"fp64": 0, "tf32": 1, "bf16": 2}
DTYPE = {"fp64": "f64", "tf32": "tf32+f64", "bf16": "bf16+f64"}


def phase_flops(wl, prec_name, eig):
    """Algorithmic work per step of each phase (flops), for the roofline."""
    n = wl.searches[0].n
    count = len(wl.searches)
    lam_sum = wl.candidates_per_generation
    mu_sum = sum(s.lam // 2 for s in wl.searches)
    split = 1 if prec_name == "fp64" else 3   # split operands: three products
    return {
        "sample": 2.0 * lam_sum * n * n,
        "objective": 2.0 * lam_sum * n * n * split,
        "cov": (1.0 * mu_sum * n * (n + 1)) * split + 3.0 * count * n * n,
        "eig": eig,
        "update": 2.0 * count * n * n + 4.0 * mu_sum * n,
        "stop": 0.0,
    }


def measure(args, prec_name, world, rank, dist, want_clocks):
    import torch
    import paper_2409_11765_gb300 as eng
    wl = workload()
    count = len(wl.searches)
    opt = eng.cmaes_default_options(precision=PREC[prec_name], f_target=wl.f_target,
                                    box_lo=wl.box_lo, box_hi=wl.box_hi, max_restarts=255,
                                    ipop_double=0)
    ns = [s.n for s in wl.searches]
    from paper_2409_11765_gb300 import dist as D
    h = eng.cmaes_create_batch(ns, [s.lam for s in wl.searches], [s.x0 for s in wl.searches],
                               [s.sigma0 for s in wl.searches], D.rank_seed(20240918, rank), opt)
    try:
        for i, s in enumerate(wl.searches):
            p = s.problem
            eng.cmaes_set_problem(h, i, p.kind, p.Q, p.lamdiag, p.xstar)
        # a dedicated stream: the engine launches on it and the CUDA events
        # that time the steps are recorded on it
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        sptr = stream.cuda_stream
        flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
        for _ in range(args.warmup):
            eng.cmaes_step_batch(h, 1, sptr)
        torch.cuda.synchronize()
        eig0 = [eng.cmaes_eig_stats(h, i) for i in range(count)]
        eng.cmaes_phase_times(h, reset=True)
        eng.cmaes_set_profiling(h, True)
        launches0 = eng.cmaes_kernel_launches(h)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        sampler = None
        if want_clocks:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES")
            local = int(os.environ.get("LOCAL_RANK", "0"))
            gpu_index = vis.split(",")[local] if vis else str(local)
            sampler = ClockSampler(gpu_index)
            time.sleep(0.3)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k & 255)
            starts[k].record(stream)
            eng.cmaes_step_batch(h, 1, sptr)
            ends[k].record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clocks = sampler.stop() if sampler else None
        launches = eng.cmaes_kernel_launches(h) - launches0
        eng.cmaes_set_profiling(h, False)
        phase_ms, _ = eng.cmaes_phase_times(h, reset=True)
        total_ms = D.max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(starts, ends)), dist,
                                    device="cuda")
        eig1 = [eng.cmaes_eig_stats(h, i) for i in range(count)]
        dec = sum(b["decompositions"] - a["decompositions"] for a, b in zip(eig0, eig1))
        rot = sum(b["rotations"] - a["rotations"] for a, b in zip(eig0, eig1))
        swp = sum(b["sweeps"] - a["sweeps"] for a, b in zip(eig0, eig1))
        swp32 = sum(b["sweeps32"] - a["sweeps32"] for a, b in zip(eig0, eig1))
        torch.cuda.set_stream(torch.cuda.default_stream())
        # e2e through the public API: one generation and a host read of every
        # search's best point and value, synchronised each step
        e2e_t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            eng.cmaes_step_batch(h, 1)
            for i in range(count):
                eng.cmaes_best(h, i, ns[i])
        e2e_el = time.perf_counter() - e2e_t0
    finally:
        eng.cmaes_destroy(h)
    cand = wl.candidates_per_generation
    n = ns[0]
    flops = phase_flops(wl, prec_name, eig_flops(n, dec) / args.steps)
    return {
        "value": D.whole_job_rate(cand, args.steps, world, total_ms),
        "ms_per_step": total_ms / args.steps,
        "phases_ms_per_step": {k: v / args.steps for k, v in phase_ms.items()},
        "phase_flops_per_step": flops,
        "gpu_launches": int(launches),
        "eig_work": {"decompositions": dec, "sweeps": swp, "rotations": rot, "sweeps_fp32": swp32},
        "e2e": {"value": cand * args.e2e_steps * world / e2e_el, "unit": UNIT,
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": sum(8 * m + 8 for m in ns)},
        "clocks": clocks,
    }


def run_engine(args):
    import torch
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import paper_2409_11765_gb300 as eng
    from paper_2409_11765_gb300 import _build
    if rank == 0 or world == 1:
        _build.build()
    if dist is not None:
        dist.barrier()

    head = args.precision
    runs = {head: measure(args, head, world, rank, dist, want_clocks=True)}
    for other in ("fp64", "tf32", "bf16"):
        if other != head and not args.headline_only:
            runs[other] = measure(args, other, world, rank, dist, want_clocks=False)
    r = runs[head]

    # roofline of the dominant phase of the headline run
    fp64_peak = eng.probe_fma_tflops(64)
    import json as _json
    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    dom = max(r["phases_ms_per_step"], key=r["phases_ms_per_step"].get)
    dom_ms = r["phases_ms_per_step"][dom]
    achieved = r["phase_flops_per_step"][dom] / (dom_ms * 1e-3) / 1e12
    if dom in ("eig", "update", "stop") or head == "fp64":
        bound, peak, src = "alu", fp64_peak, "FP64 DFMA probe measured live on this GPU"
    else:
        bf16 = peaks.get("bf16_tflops", 1908.7)
        peak = bf16 * (0.5 if head == "tf32" else 1.0)
        bound, src = "tensor", ("MEASURED_PEAKS.json bf16 x nominal tf32/bf16 ratio 0.5"
                                if head == "tf32" else "MEASURED_PEAKS.json bf16")
    traffic = None
    if dom == "eig" and head != "fp64" and engine_sources_sha() == EIG_TRAFFIC["sources_sha256_16"]:
        traffic = EIG_TRAFFIC["bytes"]
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": dom, "peak_source": src,
                "algorithmic_flops_per_step": r["phase_flops_per_step"][dom]}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    wl = workload()
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[head], "data": "synthetic", "config": workload_config(wl, head),
            "roofline": roofline, "e2e": r["e2e"], "gpu_launches": r["gpu_launches"],
            "clocks": r["clocks"], "phases_ms_per_step": r["phases_ms_per_step"],
            "eig_ms_per_step": r["phases_ms_per_step"]["eig"], "eig_work": r["eig_work"]}
    for other, o in runs.items():
        if other != head:
            line[other + "_path"] = {"value": o["value"], "ms_per_step": o["ms_per_step"],
                                     "phases_ms_per_step": o["phases_ms_per_step"],
                                     "eig_work": o["eig_work"]}
    if "fp64_path" in line:
        line["mixed_over_fp64"] = r["value"] / line["fp64_path"]["value"]
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_engine(args)


if __name__ == "__main__":
    main()
