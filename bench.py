"""Benchmark: the CR solver's hot path on the Planck-143-shaped workload
(HEALPix Nside 2048, lmax 3000, 7.3' beam, RMS log-uniform in [10, 60] uK,
|b| < 10 deg galactic cut plus 3000 holes of 5').

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
(the reference arm) on a bounded sample of the same workload.

Step: one application of A = S^-1 + B Y^T N^-1 Y B (one SHT pair plus the
diagonals) in FP64, inputs resident in HBM.  Multi-GPU runs are independent
replicas (the workload does not shard across GPUs).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s/realization to <1uK max-pixel err, Nside 2048 (mixed vs FP64); SHT pairs/s"
WORKLOAD = "nside2048_lmax3000"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([s.strip() for s in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx = max(mx, float(s[1]))
                for n, v in zip(names, s[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# FP64 FMA-pipe peak of this GB300 pool, measured with an FMA-loop probe
# (152 SMs, independent DFMA chains, CUDA events): 1.19 TFLOP/s.
FP64_FMA_PEAK_TFLOPS = 1.19


def algorithmic_sht_flops(nside, lmax):
    """Algorithmic flops of one synthesis or adjoint synthesis: ring pairs x
    coefficients x 8 (recurrence ~4, accumulation ~4), no polar skipping."""
    npairs = 2 * nside
    nlm = (lmax + 1) * (lmax + 2) // 2
    return npairs * nlm * 8.0


def cpu_baseline(cfg, seconds_budget=15.0):
    """The oracle (plain FP64 direct SHT, as it stands) timed on this host's
    cores on a bounded sample of rings of the same grid; scaled to SHT pairs/s
    of the full grid."""
    import numpy as np

    from oracle import geometry, sht

    nside, lmax = cfg["nside"], cfg["lmax"]
    g = geometry.healpix_grid(nside)
    rng = np.random.default_rng(0)
    a = rng.normal(size=sht.n_lm(lmax)) + 1j * rng.normal(size=sht.n_lm(lmax))
    a[: lmax + 1] = a[: lmax + 1].real
    y = rng.normal(size=g["npix"])
    nr = 16
    spent = 0.0
    done_rings = 0
    t_total = 0.0
    while spent < seconds_budget and done_rings < g["nring"]:
        rings = np.linspace(0, g["nring"] - 1, nr).astype(np.int64)
        t0 = time.perf_counter()
        sht.synth(a, lmax, g, rings=rings)
        sht.adjoint(y, lmax, g, rings=rings)
        dt = time.perf_counter() - t0
        spent += dt
        t_total += dt
        done_rings += nr
        nr *= 2
    per_pair = t_total / done_rings * g["nring"]
    return {"value": 1.0 / per_pair, "unit": "SHT pairs/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d rings (synthesis + adjoint, direct Legendre + direct DFT) of the Nside %d / lmax %d "
                      "grid, scaled to all %d rings" % (done_rings, nside, lmax, g["nring"])}


def run_reference(args, rank, world):
    from paper_1308_5299_gb300 import synthetic

    if rank != 0:
        return
    cfg = synthetic.CONFIGS[args.workload]
    steps = []
    base = None
    for i in range(args.warmup + args.steps):
        b = cpu_baseline(cfg, seconds_budget=8.0)
        if i >= args.warmup:
            steps.append(1.0 / b["value"])
            base = b
    sec = statistics.median(steps)
    v = 1.0 / sec
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "SHT pairs/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "nside": cfg["nside"], "lmax": cfg["lmax"]},
           "cpu_baseline": dict(base, value=v),
           "e2e": {"value": v, "unit": "SHT pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    import __graft_entry__
    from paper_1308_5299_gb300 import binding, synthetic

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
        __graft_entry__.build()

    cfg, cl, bl, ninv = synthetic.problem_inputs(args.workload)
    nside, lmax = cfg["nside"], cfg["lmax"]
    stream = torch.cuda.current_stream(dev)
    plan = binding.Plan(lmax, nside=nside, cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev), stream=stream)
    nlm = binding.n_lm(lmax)
    x = torch.from_numpy(synthetic.draw_prior(cl, index=rank)).to(dev)
    y = torch.empty_like(x)

    def step():
        plan.apply_A(x, y)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.set_timing(True)  # per-stage CUDA events on the plan's stream
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    stages = plan.timing()
    plan.set_timing(False)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * 1e3 / ms  # SHT pairs per second over all replicas
    dom = "legendre_synth"
    synth_ms = stages[dom][0] / stages[dom][1]
    flops = algorithmic_sht_flops(nside, lmax)
    launches = sum(v[1] for v in stages.values())

    # end to end through the C ABI with host buffers
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xd = xh.to(dev, non_blocking=True)
        plan.apply_A(xd, y)
        yh.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps

    if rank != 0:
        return
    peaks = measured_peaks()
    clocks = clk.summary()
    out = {
        "metric": METRIC, "value": value, "unit": "SHT pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "nside": nside, "lmax": lmax, "step": "apply_A (one SHT pair) FP64",
                   "l2": "inputs larger than L2 (x 72 MB, N^-1 403 MB, phase 393 MB per step)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": world / e2e_s, "unit": "SHT pairs/s", "h2d_bytes_per_step": int(xh.numel() * 16),
                "d2h_bytes_per_step": int(yh.numel() * 16)},
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
        "roofline": {"bound": "alu", "kernel": "legendre_synth (FP64 recurrence + accumulation)",
                     "achieved": flops / (synth_ms * 1e-3) / 1e12, "peak": FP64_FMA_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": flops / (synth_ms * 1e-3) / 1e12 / FP64_FMA_PEAK_TFLOPS,
                     "traffic": None, "peak_source": "measured FP64 FMA-loop probe",
                     "synth_ms": synth_ms, "algorithmic_gflop": flops / 1e9},
        "clocks": clocks,
        "gpu_launches": int(launches),
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
