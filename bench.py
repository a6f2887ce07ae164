"""Benchmark: image-pair subtractions/s at 4096^2 through the GB300 SFFT path.

One step = one whole image pair through the hot path (build the system,
solve it, subtract) on device-resident inputs.  The headline runs the
serving path (sfft_submit: --depth pairs in flight, their systems solved
--batch at a time in one launch); the one-pair-at-a-time path
(sfft_run_pair) is reported beside it, with its per-pair latency.  Default workload: the
4096^2 float32 wide-field pair (20000 sources, w=8, D_K=D_B=2, constant
photometric ratio, 1735 unknowns), mixed precision.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: independent pairs per rank (replicas, weak scaling, no
collective on the data path); value = all pairs / max time over ranks.
The reference arm times the FP64 CPU oracle on the host cores.
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "image-pair subtractions/s at 4096^2 (build + solve + subtract)"
UNIT = "pairs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pair4096")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stages", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 single-pair comparison")
    ap.add_argument("--no-bspline", action="store_true", help="skip the B-spline basis measurement")
    ap.add_argument("--mode", default="full", choices=["full", "pair"],
                    help="pair: only warmup + steps pairs through sfft_run_pair (for profiler captures)")
    ap.add_argument("--depth", type=int, default=8, help="pairs in flight in the serving path (1..8)")
    ap.add_argument("--batch", type=int, default=8, help="systems solved per launch in the serving path")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in launch shapes (for launch lists without the tuning replays)")
    ap.add_argument("--solve-grid", type=int, default=0,
                    help="blocks of the cooperative solve (0: two per SM in FP32, one in FP64)")
    ap.add_argument("--sector-solve", default="batched", choices=["batched", "single"],
                    help="sectors64: solve the sectors' systems eight per launch, or one per pair")
    ap.add_argument("--no-masked", action="store_true", help="skip the transient-masked pair measurement")
    ap.add_argument("--no-solve-batch", action="store_true", help="skip the batched-solve measurement")
    ap.add_argument("--solve-tc", action="store_true",
                    help="pair mode: the solve's tile products on the tensor cores (for profiler captures)")
    ap.add_argument("--no-sectors", action="store_true", help="skip the 64-sector batch measurement")
    ap.add_argument("--no-stream", action="store_true", help="skip the loaded serving-stream measurement")
    ap.add_argument("--oracle-sample", type=int, default=0,
                    help=argparse.SUPPRESS)  # child process: time the oracle on a crop, print JSON
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(vals, world, device=None):
    """Element-wise maximum of `vals` over all ranks (the slowest rank sets the
    time of a replicated run); a no-op for one rank."""
    if world <= 1:
        return list(vals)
    import torch
    t = torch.tensor(list(vals), dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def pairs_per_second(world, steps, total_ms):
    """Whole-job throughput of a replicated run: every rank processes `steps`
    pairs, and the job takes as long as its slowest rank."""
    return world * steps / (total_ms / 1e3)


def workload_config(spec, precision):
    f = spec.fit
    return {"workload": f"{spec.name}: {spec.n0}x{spec.n1} {spec.dtype} pair, {spec.n_src} sources, "
                        f"w={f.w0}, D_K={f.dk}, D_B={f.db}, const_phot_ratio={f.const_phot_ratio}",
            "image": [spec.n0, spec.n1], "w": f.w0, "dk": f.dk, "db": f.db,
            "const_phot_ratio": f.const_phot_ratio, "precision": precision,
            "l2": "not flushed: each step touches ~1.3 GB (inputs 134 MB + workspace), > 129 MB L2; "
                  "two input pairs alternate"}


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample: central crop with the same fit parameters)

def oracle_sample(R, S, spec, crop):
    import numpy as np
    import oracle
    n0, n1 = spec.n0, spec.n1
    c0, c1 = (n0 - crop) // 2, (n1 - crop) // 2
    Rc = np.ascontiguousarray(R[c0:c0 + crop, c1:c1 + crop], dtype=np.float64)
    Sc = np.ascontiguousarray(S[c0:c0 + crop, c1:c1 + crop], dtype=np.float64)
    f = spec.fit
    cfg = oracle.OracleConfig(crop, crop, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio)
    t0 = time.perf_counter()
    M, rhs = oracle.build_system(Rc, Sc, cfg)
    t1 = time.perf_counter()
    x = oracle.cholesky_solve(M, rhs)
    t2 = time.perf_counter()
    oracle.subtract(Rc, Sc, x, cfg)
    t3 = time.perf_counter()
    scale = (n0 * n1) / float(crop * crop)
    # lag sums and the stencil scale with the pixel count; the n x n solve does not
    full = scale * ((t1 - t0) + (t3 - t2)) + (t2 - t1)
    return {"t_build": t1 - t0, "t_solve": t2 - t1, "t_sub": t3 - t2, "scale": scale, "t_pair": full,
            "crop": crop, "threads": oracle.threads()}


def oracle_sample_child(crop, workload, threads):
    """The same sample in a child process with `threads` OpenMP threads (the
    oracle's thread count is fixed when its library loads)."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(crop),
                        "--workload", workload], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(f"oracle sample failed: {r.stderr[-400:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_sample(args):
    import synth
    spec = synth.SPECS[args.workload]
    R, S = synth.make_pair(spec, seed=100)
    print(json.dumps(oracle_sample(R, S, spec, args.oracle_sample)), flush=True)


def cpu_leg(smp):
    """Measured times of one oracle sample and the full-pair model built from them."""
    return {"crop": f"{smp['crop']}^2", "threads": smp["threads"],
            "t_build_s": round(smp["t_build"], 3), "t_solve_s": round(smp["t_solve"], 3),
            "t_sub_s": round(smp["t_sub"], 3),
            "t_pair_model_s": round(smp["t_pair"], 2),
            "model": f"build and subtract times x{smp['scale']:.0f} (pixel count of the full pair), "
                     "solve time as measured (same n)"}


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.proc = None
        self.bus_id = bus_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# per-stage algorithmic bytes (compulsory reads + writes of each stage's kernels)

def stage_bytes(spec, n):
    f = spec.fit
    P = spec.n0 * spec.n1
    H = (spec.n1 // 2 + 1) * spec.n0
    c = 8                                  # FP32 complex
    b = 4 if spec.dtype == "float32" else 8
    nk = (f.dk + 1) * (f.dk + 2) // 2
    nimg = nk + 1
    # stage-1 rows of the Omega and Theta products (Lambda is evaluated in
    # closed form for the polynomial basis, outside the gather)
    nrows = (nk * (nk + 1) // 2) * (4 * f.w0 + 1) + nk * (2 * f.w0 + 1)
    h1c = spec.n1 // 2 + 1
    return {
        "rows": 2 * P * b + (f.dk + 2) * H * c,
        "cols": (f.dk + 2) * H * c + nimg * H * c,
        "gather": nimg * H * c + nrows * h1c * c,
        "lags": nrows * h1c * c + n * n * 8,
        "solve": 2 * n * n * 8,
        "subtract": (f.dk + 2) * H * c + 2 * H * c + P * b,
    }


def stage_flops(spec, n):
    """Arithmetic of each stage in FP32 operations (an FMA counts 2)."""
    import math
    f = spec.fit
    n0, n1 = spec.n0, spec.n1
    h1c = n1 // 2 + 1
    nk = (f.dk + 1) * (f.dk + 2) // 2
    nimg = nk + 1
    na = min(64, n0)
    units = h1c * (n0 // na)
    n_om = nk * (nk + 1) // 2
    n_other = nk  # Theta; Lambda is in closed form for the polynomial basis (not in the gather)
    # per pair and residue class: products, two 8-point DFTs, twiddles, compensated outer sums
    per_unit = lambda lags: na * 6 + 2 * 60 * (na // 8) + 7 * 6 * (na // 8) + lags * 18
    nfft_rows = (f.dk + 3) // 2
    return {
        "rows": n0 * nfft_rows * 5 * n1 * math.log2(n1) + 60 * n0 * n1,
        "cols": h1c * nimg * 5 * n0 * math.log2(n0),
        "gather": units * (n_om * per_unit(4 * f.w0 + 1) + n_other * per_unit(2 * f.w0 + 1)),
        "lags": 0.0,
        "solve": n ** 3 / 3.0,
        "subtract": h1c * n0 * nk * (2 * f.w0 + 1) * 8 + (n0 // 2) * 5 * n1 * math.log2(n1),
    }


def fp32_peak_tflops(sm_mhz):
    """CUDA-core FP32 peak: 152 SMs x 128 lanes x 2 (FMA) x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def pair_alg_bytes(spec):
    """Bytes the method itself must move per pair: read R, S once, write and read
    each forward spectrum once, read the R and S spectra again, write D."""
    f = spec.fit
    P = spec.n0 * spec.n1
    H = (spec.n1 // 2 + 1) * spec.n0
    b = 4 if spec.dtype == "float32" else 8
    nk = (f.dk + 1) * (f.dk + 2) // 2
    nb = (f.db + 1) * (f.db + 2) // 2
    return 3 * b * P + 2 * b * H * (3 * (nk + 1) + nb)


def load_traffic(kernel):
    """DRAM bytes (read + write) per launch of `kernel` from its committed ncu
    summary profiles/<kernel>_pair4096_mixed.md, used only while the hash of
    the kernel's source recorded there matches the source as it is now."""
    import re
    path = os.path.join(ROOT, "profiles", f"{kernel}_pair4096_mixed.md")
    try:
        with open(path) as fh:
            text = fh.read()
    except OSError:
        return None
    m_hash = re.search(r"kernel source hash: `([0-9a-f]+)`", text)
    m_rd = re.search(r"\| DRAM bytes read \| ([0-9.]+) Mbyte", text)
    m_wr = re.search(r"\| DRAM bytes written \| ([0-9.]+) Mbyte", text)
    if not (m_hash and m_rd and m_wr) or m_hash.group(1) != kernel_source_hash(kernel):
        return None
    return int(round((float(m_rd.group(1)) + float(m_wr.group(1))) * 1e6))


def kernel_source_hash(kernel):
    """Hash of a kernel's own text in csrc (from its template line to the
    closing brace at column 0) plus the headers it includes."""
    csrc = os.path.join(ROOT, "paper_2109_09334_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        if not name.endswith(".cu"):
            continue
        with open(os.path.join(csrc, name)) as fh:
            text = fh.read()
        i = text.find(f" {kernel}(")
        if i < 0:
            continue
        start = text.rfind("\ntemplate", 0, i)
        start = start + 1 if start >= 0 else text.rfind("\n", 0, i) + 1
        end = text.find("\n}\n", i)
        h.update(text[start:end].encode())
    for name in ("common.cuh", "fft.cuh", "fft16.cuh"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs"), "measured"
    except (OSError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch
    import synth
    from paper_2109_09334_gb300 import SfftPlan, binding

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    dev = torch.device("cuda", local)
    spec = synth.SPECS[args.workload]
    f = spec.fit
    # two distinct input pairs per rank (seeded by rank) alternate between steps
    made = [synth.make_pair(spec, seed=100 + 2 * rank + k, return_transients=True) for k in range(2)]
    pairs = [(R, S) for R, S, _ in made]
    plan = SfftPlan(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio, dtype=spec.dtype,
                    precision=args.precision)
    stream = plan.stream
    dev_pairs = [(torch.from_numpy(R).to(dev), torch.from_numpy(S).to(dev)) for R, S in pairs]
    D = torch.empty((spec.n0, spec.n1), dtype=dev_pairs[0][0].dtype, device=dev)
    x = torch.empty(plan.n, dtype=torch.float64, device=dev)
    info = torch.zeros(24, dtype=torch.uint8, device=dev)

    def step(k):
        Rt, St = dev_pairs[k & 1]
        binding.sfft_run_pair(plan.handle, Rt, St, None, None, None, x, info, D, stream)

    # launch shapes picked by timing (kept for the server's plans below)
    tuning = binding.sfft_plan_tuning(plan.handle) if args.no_autotune else plan.autotune(*dev_pairs[0])
    if args.solve_grid:  # set by hand; the server's slots (created below) start with it
        tuning["solve_grid"] = args.solve_grid
        binding.sfft_plan_set_tuning(plan.handle, tuning)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    from paper_2109_09334_gb300 import info_from_bytes
    inf = info_from_bytes(info.cpu().numpy())
    if inf["status"] != 0:
        raise RuntimeError(f"solve status {inf}")

    bus = None
    try:
        props = torch.cuda.get_device_properties(dev)
        bus = "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except Exception:
        bus = None
    sampler = ClockSampler(bus)

    # serving path: args.depth pairs in flight; outputs alternate between two buffer sets
    from paper_2109_09334_gb300 import SfftServer
    srv = SfftServer(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio, dtype=spec.dtype,
                     precision=args.precision, depth=args.depth, batch=args.batch)
    cur = torch.cuda.current_stream(dev)
    outs = [(torch.empty_like(D), torch.empty_like(x), torch.zeros_like(info)) for _ in range(2)]

    def submit(k):
        Rt, St = dev_pairs[k & 1]
        Dk, xk, ik = outs[k & 1]
        return srv.submit(Rt, St, diff=Dk, x=xk, info=ik, stream=cur)[0]

    for k in range(args.warmup):
        t = submit(k)
    srv.wait(t)
    for _, _, ik in outs:
        inf_s = info_from_bytes(ik.cpu().numpy())
        if inf_s["status"] != 0:
            raise RuntimeError(f"solve status {inf_s}")

    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    launches0 = binding.sfft_plan_launch_count(plan.handle)
    slaunch0 = srv.launch_count
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.25)
    # sequential: one pair at a time on one stream (per-pair latency)
    evs[0].record(stream)
    for k in range(args.steps):
        step(k)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    # serving: the timed region is ordered on `cur` before the first and after the last request
    es0, es1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    es0.record(cur)
    for k in range(args.steps):
        t = submit(k)
    srv.stream_wait(t, cur)
    es1.record(cur)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    srv.wait(t)
    launches = srv.launch_count - slaunch0
    seq_launches = binding.sfft_plan_launch_count(plan.handle) - launches0
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    seq_ms = evs[0].elapsed_time(evs[-1])
    total_ms = es0.elapsed_time(es1)
    total_ms, seq_ms = max_over_ranks([total_ms, seq_ms], world, dev)
    value = pairs_per_second(world, args.steps, total_ms)
    ms_step = total_ms / args.steps
    P = spec.n0 * spec.n1

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
              "data": "synthetic (seeded star fields shaped like the paper's wide-field pairs)",
              "config": workload_config(spec, args.precision), "gpu_launches": int(launches),
              "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                         "reasons": clocks["reasons"], "samples": clocks["samples"]},
              "mpix_per_s": value * P / 1e6,
              "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99)),
                             "note": "one pair alone (sfft_run_pair), device-timed per step"},
              "serving": {"api": "sfft_submit", "depth": args.depth, "batch": args.batch, "ms_per_pair": ms_step},
              "tuning": tuning,
              "sequential": {"api": "sfft_run_pair", "value": world * args.steps / (seq_ms / 1e3),
                             "ms_per_pair": seq_ms / args.steps, "gpu_launches": int(seq_launches)},
              "solve": inf}

    # per-stage times: replay each stage of the last pair with events on the plan's stream
    if not args.no_stages:
        reps = 20
        stage_ms = {}
        for sid, name in enumerate(binding.STAGE_NAMES):
            binding.sfft_replay_stage(plan.handle, sid, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                binding.sfft_replay_stage(plan.handle, sid, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            stage_ms[name] = e0.elapsed_time(e1) / reps
        # restore a consistent state for the e2e run
        step(0)
        torch.cuda.synchronize()
        # noise decorrelation of the last pair's difference image (App. C), a
        # post-process outside the step: time per call
        Ddc = torch.empty_like(D)
        plan.decorrelate(x, D, spec.sigma, spec.sigma, 0.0, 0.0, out=Ddc)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(10):
            plan.decorrelate(x, D, spec.sigma, spec.sigma, 0.0, 0.0, out=Ddc)
        e1.record(stream)
        torch.cuda.synchronize()
        result["decorrelation_ms"] = e0.elapsed_time(e1) / 10
        # the co-added form (Eq. 21-24 in full): 4 science and 4 reference
        # exposures with 7x7 homogenisation kernels (Gaussian blurs, sum 1/4)
        gy = torch.arange(-3, 4, dtype=torch.float64, device=dev)
        gk = torch.exp(-(gy[:, None] ** 2 + gy[None, :] ** 2) / (2 * 1.2 ** 2))
        Gk = (gk / gk.sum() / 4).expand(4, 7, 7).contiguous()
        sig = [spec.sigma] * 4
        plan.decorrelate_coadd(x, D, Gk, sig, Gk, sig, 0.0, 0.0, out=Ddc)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(10):
            plan.decorrelate_coadd(x, D, Gk, sig, Gk, sig, 0.0, 0.0, out=Ddc)
        e1.record(stream)
        torch.cuda.synchronize()
        result["decorrelation_coadd_ms"] = e0.elapsed_time(e1) / 10
        result["decorrelation_coadd_config"] = "4 science + 4 reference exposures, 7x7 homogenisation kernels"
        step(0)
        torch.cuda.synchronize()
        sb = stage_bytes(spec, plan.n)
        peak, peak_kind = measured_peaks()
        # shares of the serving path's time per pair: the solve runs `batch`
        # systems per launch, so its share per pair is what the other stages
        # leave of the measured time per pair
        per_pair = {k: v for k, v in stage_ms.items() if k != "solve"}
        per_pair["solve"] = max(ms_step - sum(per_pair.values()), 0.0)
        top = max(per_pair, key=per_pair.get)
        tot = sum(per_pair.values())
        # the solve with its tile products on the tensor cores (tcgen05, 3xTF32)
        # against the built-in CUDA-core tiles, one system per launch
        shapes = binding.sfft_plan_tuning(plan.handle)
        solve_var = {}
        for name, tcv in (("cuda_cores", 0), ("tensor_cores", 2)):
            binding.sfft_plan_set_tuning(plan.handle, dict(shapes, solve_tensor_cores=tcv))
            step(0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(10):
                binding.sfft_replay_stage(plan.handle, binding.SFFT_STAGE_SOLVE, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            solve_var[name] = {"ms": round(e0.elapsed_time(e1) / 10, 4),
                               "solve": info_from_bytes(info.cpu().numpy())}
        binding.sfft_plan_set_tuning(plan.handle, shapes)
        step(0)
        torch.cuda.synchronize()
        result["solve_tile_products_ms"] = solve_var
        result["stages_ms"] = {k: round(v, 4) for k, v in stage_ms.items()}
        result["stages_note"] = ("each stage replayed alone on one plan; 'solve' is one system per launch, "
                                 "the serving path solves `batch` per launch")
        result["serving_share"] = {k: round(v / tot, 3) for k, v in per_pair.items()}
        kern = {"rows": "k_rows", "cols": "k_cols", "gather": "k_gather", "lags": "k_stage2",
                "solve": "k_solve_coop", "subtract": "k_sub_cols + k_rows_inv"}[top]
        sf = stage_flops(spec, plan.n)
        clk = clocks["sm_max_mhz"] or 2070.0
        alu_peak = fp32_peak_tflops(clk)
        t_s = stage_ms[top] / 1e3
        single = kern.startswith("k_") and " " not in kern
        # the FFT, gather and subtraction passes are classed HBM-bound: the
        # roofline is the algorithmic bytes of the stage (compulsory reads and
        # writes) over its time, against the measured copy bandwidth
        ach = sb[top] / t_s / 1e9
        result["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                              "frac": ach / peak, "traffic": load_traffic(kern) if single else None,
                              "kernel": kern, "stage": top, "alg_bytes_per_launch": sb[top],
                              "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json)"}
        # beside it, the same stage against the FP32 CUDA-core peak, counting
        # the operations of this implementation (not an algorithmic minimum)
        ach_alu = sf[top] / t_s / 1e12
        result["roofline_alu"] = {"bound": "alu", "achieved": ach_alu, "peak": alu_peak, "unit": "TFLOP/s",
                                  "frac": ach_alu / alu_peak, "kernel": kern, "flops_per_launch": sf[top],
                                  "flops_source": "this implementation's own operation count of the stage",
                                  "peak_source": f"FP32 CUDA-core peak 152 SM x 128 lanes x 2 x {clk:.0f} MHz"}
        result["stages_hbm_frac"] = {k: round(sb[k] / (stage_ms[k] / 1e3) / 1e9 / peak, 3)
                                     for k in ("rows", "cols", "gather", "subtract") if stage_ms.get(k)}
        ba = pair_alg_bytes(spec)
        result["pair_roofline"] = {"alg_bytes_per_pair": ba, "achieved_GBs": ba / (ms_step / 1e3) / 1e9,
                                   "frac": ba / (ms_step / 1e3) / 1e9 / peak}

    # end to end through the serving API with host requests: pinned host buffers, the
    # host->device copies of each pair's inputs and the device->host copies of its
    # difference image, coefficients and status inside the timed region
    if not args.no_e2e:
        pin = [(torch.from_numpy(R).pin_memory(), torch.from_numpy(S).pin_memory()) for R, S in pairs]
        hout = [(torch.empty((spec.n0, spec.n1), dtype=pin[0][0].dtype).pin_memory(),
                 torch.empty(plan.n, dtype=torch.float64).pin_memory(),
                 torch.zeros(24, dtype=torch.uint8).pin_memory()) for _ in range(args.depth + 1)]

        def submit_host(k):
            Rh, Sh = pin[k & 1]
            Dh, xh, ih = hout[k % len(hout)]
            return srv.submit(Rh, Sh, diff=Dh, x=xh, info=ih)[0]

        # a request's host outputs are reused only after it has completed
        def run_host(count):
            tickets = []
            for k in range(count):
                if k >= len(hout):
                    srv.wait(tickets[k - len(hout)])
                tickets.append(submit_host(k))
            srv.wait(tickets[-1])

        run_host(3)
        ke = max(3, min(args.steps, 50))
        # host wall clock: the median of three runs, so that one disturbed by
        # other work on the host does not stand for the path
        runs = []
        for _ in range(3):
            if world > 1:
                torch.distributed.barrier()
            t0 = time.perf_counter()
            run_host(ke)
            runs.append(time.perf_counter() - t0)
        te = sorted(runs)[1]
        te = max_over_ranks([te], world, dev)[0]
        inf_h = info_from_bytes(hout[(ke - 1) % len(hout)][2].numpy())
        if inf_h["status"] != 0:
            raise RuntimeError(f"host-request solve status {inf_h}")
        Rh = pin[0][0]
        bi = Rh.numel() * Rh.element_size() * 2
        bo = Rh.numel() * Rh.element_size() + plan.n * 8 + 24
        result["e2e"] = {"value": world * ke / te, "unit": UNIT, "h2d_bytes_per_step": bi,
                         "d2h_bytes_per_step": bo, "steps": ke, "api": "sfft_submit (host requests)",
                         "clock": "host wall clock, submit of the first to completion of the last; "
                                  "median of three runs",
                         "runs_pairs_per_s": [round(world * ke / r, 1) for r in runs]}

    # the solve of `batch` built systems in one launch (sfft_solve_batch), with
    # 32- and 64-wide Cholesky panels: the serving path's solve step alone
    if not args.no_solve_batch and world == 1:
        from paper_2109_09334_gb300 import SfftPlan as _Plan
        nb = args.batch
        bplans = [_Plan(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio, dtype=spec.dtype,
                        precision=args.precision) for _ in range(nb)]
        systems = []
        for k, bp in enumerate(bplans):
            _, _, _, Mk, rk = bp.run_pair(*dev_pairs[k & 1], keep_system=True)
            systems.append((Mk, rk))
        xb = [torch.empty(bp.n, dtype=torch.float64, device=dev) for bp in bplans]
        ib = [torch.zeros(24, dtype=torch.uint8, device=dev) for _ in bplans]
        sb_out = {}
        for panel in (32, 64):
            for bp in bplans:
                bp.solve_panel = panel

            def solve_all():
                binding.sfft_solve_batch([bp.handle for bp in bplans], [s[0] for s in systems],
                                         [s[1] for s in systems], xb, ib, stream)

            for _ in range(2):
                solve_all()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(10):
                solve_all()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 10
            st = [info_from_bytes(i.cpu().numpy()) for i in ib]
            if any(s["status"] != 0 for s in st):
                raise RuntimeError(f"batched solve status {st}")
            sb_out[str(panel)] = {"ms_per_launch": round(ms, 4), "ms_per_system": round(ms / nb, 4),
                                  "iters": [s["iters"] for s in st]}
        result["solve_batch"] = {"api": "sfft_solve_batch", "systems": nb, "n": plan.n, "panels": sb_out}
        for bp in bplans:
            bp.close()

    # the plain FP64 GPU path (FP64 FFTs, products, sums, Cholesky), one pair
    # at a time on the same inputs, and how far the headline path's difference
    # image is from it (in units of the noise sigma)
    if not args.no_fp64 and args.precision == "mixed":
        p64 = SfftPlan(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio, dtype=spec.dtype,
                       precision="fp64")
        s64 = p64.stream
        D64 = torch.empty_like(D)
        x64 = torch.empty_like(x)
        i64 = torch.zeros_like(info)
        for k in range(2):
            binding.sfft_run_pair(p64.handle, dev_pairs[k & 1][0], dev_pairs[k & 1][1], None, None, None, x64, i64,
                                  D64, s64)
        k64 = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s64)
        for k in range(k64):
            binding.sfft_run_pair(p64.handle, dev_pairs[k & 1][0], dev_pairs[k & 1][1], None, None, None, x64, i64,
                                  D64, s64)
        e1.record(s64)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / k64
        # both paths on pair 0
        binding.sfft_run_pair(p64.handle, dev_pairs[0][0], dev_pairs[0][1], None, None, None, x64, i64, D64, s64)
        step(0)
        torch.cuda.synchronize()
        dd = float(torch.sqrt(torch.mean((D.double() - D64.double()) ** 2)).item())
        result["fp64_single_pair"] = {"value": world * 1e3 / t64, "unit": UNIT, "ms_per_pair": t64, "steps": k64,
                                      "solve": info_from_bytes(i64.cpu().numpy()),
                                      "rms_diff_vs_headline_sigma": dd / spec.sigma,
                                      "note": "plain FP64 path, sfft_run_pair, same inputs; D of the mixed path "
                                              "compared with it on pair 0"}
        p64.close()

    # the same pairs with the B-spline basis of Eq. 7-9 (piecewise-linear
    # kernel variation with one interior knot, quadratic background with one
    # interior knot), one pair at a time, with its stage times
    if not args.no_bspline:
        spl = (1, 1, 2, 1)
        pb = SfftPlan(spec.n0, spec.n1, f.w0, f.w1, 0, 0, f.const_phot_ratio, dtype=spec.dtype,
                      precision=args.precision, spline=spl)
        sb = pb.stream
        Db = torch.empty_like(D)
        xb = torch.empty(pb.n, dtype=torch.float64, device=dev)
        ib = torch.zeros_like(info)
        for k in range(2):
            binding.sfft_run_pair(pb.handle, dev_pairs[k & 1][0], dev_pairs[k & 1][1], None, None, None, xb, ib,
                                  Db, sb)
        kb = 10
        l0 = binding.sfft_plan_launch_count(pb.handle)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(sb)
        for k in range(kb):
            binding.sfft_run_pair(pb.handle, dev_pairs[k & 1][0], dev_pairs[k & 1][1], None, None, None, xb, ib,
                                  Db, sb)
        e1.record(sb)
        torch.cuda.synchronize()
        tb = e0.elapsed_time(e1) / kb
        lb = binding.sfft_plan_launch_count(pb.handle) - l0
        bst = {}
        for st, name in enumerate(binding.STAGE_NAMES):
            for _ in range(2):
                binding.sfft_replay_stage(pb.handle, st, sb)
            e0.record(sb)
            for _ in range(5):
                binding.sfft_replay_stage(pb.handle, st, sb)
            e1.record(sb)
            torch.cuda.synchronize()
            bst[name] = round(e0.elapsed_time(e1) / 5, 4)
        result["bspline"] = {"value": world * 1e3 / tb, "unit": UNIT, "ms_per_pair": tb, "steps": kb,
                             "gpu_launches": int(lb), "n": pb.n,
                             "basis": {"kernel_degree": spl[0], "kernel_interior_knots": spl[1],
                                       "background_degree": spl[2], "background_interior_knots": spl[3]},
                             "stages_ms": bst, "solve": info_from_bytes(ib.cpu().numpy()),
                             "api": "sfft_run_pair, one pair at a time, same inputs as the headline"}
        pb.close()

    # the two-step process of Sec. 3 on the same pairs: the build with the
    # transients masked (squares of half-width 14 px zeroed), the subtraction
    # unmasked; one pair at a time
    if not args.no_masked and spec.n_transients:
        masks = [torch.from_numpy(synth.transient_mask((spec.n0, spec.n1), tp, half=14)).to(dev)
                 for _, _, tp in made]
        Dm = torch.empty_like(D)
        xm = torch.empty_like(x)
        im = torch.zeros_like(info)

        def step_masked(k):
            binding.sfft_run_pair(plan.handle, dev_pairs[k & 1][0], dev_pairs[k & 1][1], masks[k & 1], None, None,
                                  xm, im, Dm, stream)

        for k in range(2):
            step_masked(k)
        km = 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(km):
            step_masked(k)
        e1.record(stream)
        torch.cuda.synchronize()
        tm = e0.elapsed_time(e1) / km
        result["masked"] = {"value": world * 1e3 / tm, "unit": UNIT, "ms_per_pair": tm, "steps": km,
                            "masked_pixels": int(sum(int((m == 0).sum().item()) for m in masks) // len(masks)),
                            "solve": info_from_bytes(im.cpu().numpy()),
                            "api": "sfft_run_pair with a mask: build on the masked pair (50 transients, "
                                   "squares of half-width 14 px), subtraction on the unmasked pair"}

    if not args.no_sectors:
        result["sectors64"] = measure_sectors(args, dev, world, rank)
    if not args.no_stream:
        result["stream"] = measure_stream_load(args, dev, rank)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle as it stands, on the host cores: all cores on the central
        # 1024^2 crop, one core on the central 384^2 crop (child processes,
        # since the thread count is fixed when the oracle loads)
        crop_all = 1024 if spec.n0 >= 2048 else spec.n0
        crop_one = 384 if spec.n0 >= 768 else spec.n0
        smp = oracle_sample_child(crop_all, args.workload, os.cpu_count() or 1)
        one = oracle_sample_child(crop_one, args.workload, 1)
        result["cpu_baseline"] = {"value": 1.0 / smp["t_pair"], "unit": UNIT, "cores": smp["threads"],
                                  "kind": "oracle",
                                  "sample": f"FP64 oracle build + Cholesky + subtract of one pair on the central "
                                            f"{crop_all}^2 crop with the same fit (n={plan.n}), measured; value "
                                            f"= modelled full pair (build and subtract x{smp['scale']:.0f} by "
                                            f"pixel count, solve as measured)",
                                  "t_sample_s": round(smp["t_build"] + smp["t_solve"] + smp["t_sub"], 2),
                                  "all_cores": cpu_leg(smp),
                                  "single_thread": dict(cpu_leg(one), value=1.0 / one["t_pair"], unit=UNIT)}
    srv.close()
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle
    import synth
    spec = synth.SPECS[args.workload]
    R, S = synth.make_pair(spec, seed=100)
    crop = 256 if spec.n0 >= 512 else spec.n0
    for _ in range(args.warmup):
        oracle_sample(R, S, spec, crop)
    models, walls = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        smp = oracle_sample(R, S, spec, crop)
        models.append(smp["t_pair"])
        walls.append(smp["t_build"] + smp["t_solve"] + smp["t_sub"])
    wall = time.perf_counter() - t0
    t = float(np.mean(models))
    value = 1.0 / t
    sample = (f"each step: FP64 oracle build + Cholesky + subtract of the central {crop}^2 crop with the same "
              f"fit, measured (ms_per_step); value = the modelled full pair: build and subtract time "
              f"x{spec.n0 * spec.n1 // (crop * crop)} by pixel count, solve time as measured")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(spec, "fp64 oracle"),
           "t_pair_model_ms": t * 1e3, "t_sample_ms": float(np.mean(walls)) * 1e3,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def crop_field(n_field, fit, seed):
    """One seeded wide field of the sector recipe (one source per 500 px^2,
    the PSF/sky family of the 4096^2 pair), to cut uneven sectors from."""
    import synth
    spec = synth.sector(n_field, fit, name=f"field{n_field}")
    return synth.make_pair(spec, seed=seed)


def measure_sectors(args, dev, world, rank):
    """Batched uneven sectors: 64 square pairs, n uniform in [512, 2048], fit
    drawn per sector, processed as one batch captured by the library into a
    CUDA graph (sfft_batch_create, solve grouping autotuned) and replayed as
    one launch (sfft_batch_launch).  Checks the replay against the pairs run
    one at a time (bit for bit) and times both."""
    import numpy as np
    import torch
    import synth
    from paper_2109_09334_gb300 import SfftBatch, SfftPlan, binding, info_from_bytes

    specs = synth.draw_sectors(64, seed=4 + rank)
    R, S = crop_field(4096, synth.FitParams(8, 8, 2, 2, True), seed=40 + rank)
    rng = np.random.default_rng(7 + rank)
    work = []
    for sp in specs:
        n = sp.n0
        x0, y0 = (int(v) for v in rng.integers(0, 4096 - n + 1, size=2))
        f = sp.fit
        plan = SfftPlan(n, n, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio, dtype="float32", precision=args.precision)
        # systems solved several per launch: 64-wide Cholesky panels
        plan.solve_panel = 64 if args.sector_solve == "batched" else 32
        Rt = torch.from_numpy(np.ascontiguousarray(R[x0:x0 + n, y0:y0 + n])).to(dev)
        St = torch.from_numpy(np.ascontiguousarray(S[x0:x0 + n, y0:y0 + n])).to(dev)
        work.append((plan, Rt, St, n, f))
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    group = {"batched": 0, "single": 1}[args.sector_solve]
    batch = SfftBatch([w[0] for w in work], [w[1] for w in work], [w[2] for w in work], solve_group=group)
    binfo = batch.info_dict
    K = max(1, min(args.steps, 20))

    def timed(fn):
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    graph_ms = timed(lambda: batch.launch(stream))
    got = [d.clone() for d in batch.D]
    bad = [k for k, i in enumerate(batch.info) if info_from_bytes(i.cpu().numpy())["status"] != 0]
    if bad:
        raise RuntimeError(f"solve failed on sectors {bad}")
    # one pair at a time (sfft_run_pair), the same inputs: the reference for
    # the batch's results and the eager comparison
    Dk = [torch.empty_like(w[1]) for w in work]
    xk = [torch.empty(w[0].n, dtype=torch.float64, device=dev) for w in work]
    ik = [torch.zeros(24, dtype=torch.uint8, device=dev) for w in work]

    def run_seq():
        for k, (plan, Rt, St, n, f) in enumerate(work):
            binding.sfft_run_pair(plan.handle, Rt, St, None, None, None, xk[k], ik[k], Dk[k], stream)

    # the check on the batch's panel width, then one at a time timed with the
    # width that is fastest for a single system (32)
    run_seq()
    torch.cuda.synchronize()
    if not all(torch.equal(a, b) for a, b in zip(got, Dk)):
        raise RuntimeError("graph-captured batch differs from the pairs run one at a time")
    panel = work[0][0].solve_panel
    for w in work:
        w[0].solve_panel = 32
    seq_ms = timed(run_seq)
    batch.close()
    ms, seq_ms = max_over_ranks([graph_ms, seq_ms], world, dev)
    npix = sum(w[3] * w[3] for w in work)
    out = {"value": world * len(work) * 1e3 / ms, "unit": "pairs/s", "ms_per_batch": ms, "steps": K,
           "mpix_per_s": world * npix / (ms * 1e3), "gpu_launches_per_batch": binfo["launches"],
           "api": "sfft_batch_create (library-captured CUDA graph) + sfft_batch_launch",
           "solve_group": binfo["solve_group"], "solve_group_tuning_ms": binfo["tune_ms"],
           "solve_panel": panel,
           "one_at_a_time": {"value": world * len(work) * 1e3 / seq_ms, "ms_per_batch": seq_ms,
                             "api": "sfft_run_pair per sector", "solve_panel": 32},
           "sizes": [w[3] for w in work], "fits": [[w[4].w0, w[4].dk, w[4].db] for w in work],
           "check": "every difference image bitwise equal to sfft_run_pair's (same panel width)"}
    for w in work:
        w[0].close()
    return out


def run_sectors(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    dev = torch.device("cuda", local)
    r = measure_sectors(args, dev, world, rank)
    out = {"metric": "pairs/s over a batch of 64 uneven sectors (512..2048 px, fit drawn per sector)",
           "value": r["value"], "unit": "pairs/s", "n_gpus": world, "steps": r["steps"],
           "warmup": args.warmup, "ms_per_step": r["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
           "data": "synthetic sectors cut from one seeded field (one source per 500 px^2)",
           "config": {"workload": "sectors64", "sizes": r["sizes"], "fits": r["fits"], "precision": args.precision,
                      "solve": args.sector_solve},
           "gpu_launches": int(r["gpu_launches_per_batch"] * r["steps"]), "sectors64": r}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_stream(args):
    """Serving stream: host requests of mixed sizes (1024..4096) and fits
    arriving as a Poisson process at 20 pairs/s, through the pool (plans and
    spectra kept on the device, admission under a 180 GB budget); reports
    the arrival-to-completion latency percentiles and the throughput."""
    import threading
    import numpy as np
    import torch
    import synth
    from paper_2109_09334_gb300 import SfftPool, info_from_bytes

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    R, S = crop_field(4096, synth.FitParams(8, 8, 2, 2, True), seed=50 + rank)
    rng = np.random.default_rng(9 + rank)
    count = max(8, min(args.steps, 200))
    reqs = []
    for k in range(count):
        n = int(rng.integers(1024, 4097))
        w, dk, db = int(rng.integers(4, 9)), int(rng.integers(0, 3)), int(rng.integers(0, 3))
        x0, y0 = (int(v) for v in rng.integers(0, 4096 - n + 1, size=2))
        Rh = torch.from_numpy(np.ascontiguousarray(R[x0:x0 + n, y0:y0 + n])).pin_memory()
        Sh = torch.from_numpy(np.ascontiguousarray(S[x0:x0 + n, y0:y0 + n])).pin_memory()
        reqs.append((Rh, Sh, (w, w, dk, db, True), n))
    gaps = rng.exponential(1.0 / 20.0, size=count)
    arrive = np.cumsum(gaps) - gaps[0]
    pool = SfftPool(180 << 30, depth=1, batch=1)
    done_at = [None] * count
    tickets = [None] * count
    ready = threading.Semaphore(0)

    def waiter():
        for k in range(count):
            ready.acquire()
            pool.wait(tickets[k][0])
            done_at[k] = time.perf_counter()

    th = threading.Thread(target=waiter)
    th.start()
    t0 = time.perf_counter()
    for k, (Rh, Sh, fit, n) in enumerate(reqs):
        delay = t0 + arrive[k] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        got = pool.submit(Rh, Sh, *fit, precision=args.precision)
        while got is None:  # not admitted yet: wait for the oldest pending request
            time.sleep(0.001)
            got = pool.submit(Rh, Sh, *fit, precision=args.precision)
        tickets[k] = got
        ready.release()
    th.join()
    lat = np.array([done_at[k] - (t0 + arrive[k]) for k in range(count)]) * 1e3
    span = max(done_at) - t0
    bad = [k for k in range(count) if info_from_bytes(tickets[k][3].numpy())["status"] != 0]
    used, lanes = pool.usage
    pool.close()
    out = {"metric": "serving stream: pairs/s and arrival-to-completion latency (Poisson 20 pairs/s, 1024..4096 px)",
           "value": world * count / span, "unit": "pairs/s", "n_gpus": world, "steps": count, "warmup": 0,
           "ms_per_step": span * 1e3 / count, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if args.precision == "mixed" else "f64",
           "data": "synthetic sectors cut from one seeded field, host requests (pinned)",
           "config": {"workload": "stream", "rate_per_s": 20, "sizes": [r[3] for r in reqs], "budget_gb": 180},
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max())},
           "note": "each size is new, so every request also builds its plan (tables, workspace) inside its latency",
           "failed": bad, "pool_end": {"bytes": used, "lanes": lanes}}
    if rank == 0:
        print(json.dumps(out), flush=True)


def measure_stream_load(args, dev, rank, rates=(100.0, 300.0, 600.0), count=240, nconf=8):
    """The serving stream under load: host requests (pinned) drawn from
    `nconf` sector configurations (square n uniform in [1024, 4096], w in
    4..8, D_K and D_B in 0..2, all drawn once, as a survey's sectors come in a
    few shapes), cut from one seeded 4096^2 field, arriving as a Poisson
    process at each rate in `rates`, through the pool (one lane per
    configuration, depth 4, batch 2, eager flushing, 180 GB budget).  The lanes are warmed
    (plans built) before the timed streams.  A waiter thread waits for the
    tickets in submission order; a request's latency is arrival to the end of
    its wait.  Requests of one configuration that arrive together share a
    solve launch; the lanes' builds, solves and copies overlap on the GPU."""
    import threading
    import numpy as np
    import torch
    import synth
    from paper_2109_09334_gb300 import SfftPool, info_from_bytes

    R, S = crop_field(4096, synth.FitParams(8, 8, 2, 2, True), seed=60 + rank)
    rng = np.random.default_rng(11 + rank)
    confs = []
    for _ in range(nconf):
        n = int(rng.integers(1024, 4097))
        w, dk, db = int(rng.integers(4, 9)), int(rng.integers(0, 3)), int(rng.integers(0, 3))
        x0, y0 = (int(v) for v in rng.integers(0, 4096 - n + 1, size=2))
        Rh = torch.from_numpy(np.ascontiguousarray(R[x0:x0 + n, y0:y0 + n])).pin_memory()
        Sh = torch.from_numpy(np.ascontiguousarray(S[x0:x0 + n, y0:y0 + n])).pin_memory()
        confs.append((Rh, Sh, (w, w, dk, db, True), n))
    pool = SfftPool(180 << 30, depth=4, batch=2, eager=True)
    # outputs: a ring of pinned buffers per configuration, reused only after
    # the request that used them has completed
    ring = 12
    outs = [[(torch.empty((n, n), dtype=torch.float32).pin_memory(),) for _ in range(ring)] for *_, n in confs]

    def submit(ci, slot):
        Rh, Sh, fit, n = confs[ci]
        while True:
            got = pool.submit(Rh, Sh, *fit, precision=args.precision, diff=outs[ci][slot][0])
            if got is not None:
                return got
            time.sleep(0.0005)  # not admitted yet

    for ci in range(nconf):  # warm the lanes
        t = submit(ci, 0)
        pool.wait(t[0])
    legs = []
    for rate in rates:
        pick = rng.integers(0, nconf, size=count)
        gaps = rng.exponential(1.0 / rate, size=count)
        arrive = np.cumsum(gaps) - gaps[0]
        done_at = [None] * count
        tickets = [None] * count
        ready = threading.Semaphore(0)
        used = [[] for _ in range(nconf)]  # request indices per configuration (ring reuse)

        def waiter():
            for k in range(count):
                ready.acquire()
                pool.wait(tickets[k][0])
                done_at[k] = time.perf_counter()

        th = threading.Thread(target=waiter)
        th.start()
        t0 = time.perf_counter()
        for k in range(count):
            delay = t0 + arrive[k] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ci = int(pick[k])
            if len(used[ci]) >= ring:  # the output buffer of this slot must be free
                prev = used[ci][-ring]
                while done_at[prev] is None:
                    time.sleep(0.0002)
            tickets[k] = submit(ci, len(used[ci]) % ring)
            used[ci].append(k)
            ready.release()
        th.join()
        lat = np.array([done_at[k] - (t0 + arrive[k]) for k in range(count)]) * 1e3
        span = max(done_at) - t0
        bad = [k for k in range(count) if info_from_bytes(tickets[k][3].numpy())["status"] != 0]
        npix = sum(confs[int(c)][3] ** 2 for c in pick)
        legs.append({"rate_per_s": rate, "requests": count, "pairs_per_s": count / span,
                     "mpix_per_s": npix / span / 1e6,
                     "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                    "max": float(lat.max())}, "failed": bad})
    used_bytes, lanes = pool.usage
    pool.close()
    return {"api": "sfft_pool_submit / sfft_pool_wait (host requests, pinned)", "depth": 4, "batch": 2,
            "policy": "eager flush (sfft_pool_set_eager): a batch starts when its lane is idle",
            "budget_gb": 180, "configurations": [[c[3], *c[2][:1], c[2][2], c[2][3]] for c in confs],
            "configuration_fields": ["n", "w", "dk", "db"], "lanes_warmed": True, "legs": legs,
            "pool_end": {"bytes": used_bytes, "lanes": lanes}}


def run_pairs_only(args):
    """warmup + steps pairs of the workload through sfft_run_pair on one plan
    and one stream, nothing else (the command the ncu captures profile)."""
    import torch
    import synth
    from paper_2109_09334_gb300 import SfftPlan, info_from_bytes
    spec = synth.SPECS[args.workload]
    f = spec.fit
    R, S = synth.make_pair(spec, seed=100)
    plan = SfftPlan(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio, dtype=spec.dtype,
                    precision=args.precision)
    Rt, St = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    if args.solve_tc:
        from paper_2109_09334_gb300 import binding
        binding.sfft_plan_set_tuning(plan.handle, dict(binding.sfft_plan_tuning(plan.handle), solve_tensor_cores=2))
    for _ in range(args.warmup + args.steps):
        D, x, info, _, _ = plan.run_pair(Rt, St)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "pair", "workload": spec.name, "pairs": args.warmup + args.steps,
                      "solve": info_from_bytes(info.cpu().numpy())}), flush=True)
    plan.close()


def main():
    args = parse()
    if args.oracle_sample:
        run_oracle_sample(args)
    elif args.mode == "pair":
        run_pairs_only(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "sectors64":
        run_sectors(args)
    elif args.workload == "stream":
        run_stream(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
