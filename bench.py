"""Benchmark: the CR solver's hot path on the Planck-143-shaped workload
(HEALPix Nside 2048, lmax 3000, 7.3' beam, RMS log-uniform in [10, 60] uK,
|b| < 10 deg galactic cut plus 3000 holes of 5').

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
(the reference arm) on a bounded sample of the same workload.

Step: one constrained realization, i.e. CR-Solve of b = A x_true (the
paper's synthetic protocol) with FP32 W-cycles inside FP64 iterative
refinement, run for the fixed number of cycles that reaches a max-pixel error
below 1 uK (found before the timed region).  The plan (levels, smoothers,
dense bottom) is built once outside the timed region and reported as
precompute time.  The plain FP64 solve and the SHT-pair rates are reported
beside it.  Multi-GPU runs are independent replicas (the workload does not
shard across GPUs).
"""
import argparse
import hashlib
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
    ap.add_argument("--no-cg", action="store_true", help="skip the CG comparison on the Nside 256 workload")
    ap.add_argument("--no-df", action="store_true", help="skip the double-float outer-residual variant")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched mixed-resolution measurement")
    ap.add_argument("--schwarz", action="store_true",
                    help="also time the realization with the additive Schwarz pixel smoother (about a minute)")
    ap.add_argument("--no-graph", action="store_true", help="time the solves launched directly, not as a CUDA graph")
    ap.add_argument("--ref-cycles", type=int, default=2,
                    help="cycles per realization priced by the reference arm (the GPU arm's measured count)")
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


def gl_noise_grid(nside, lmax_h):
    """Gauss-Legendre grid the library uses for a level's inverse-noise term
    (auto rule): 2 lmax_h + 1 rings, nphi the power of two >= 4 lmax_h + 1,
    when that is at most 3/5 of the observation grid's rings; else None."""
    if 5 * (2 * lmax_h + 1) > 3 * (4 * nside - 1):
        return None
    nphi = 2
    while nphi < 4 * lmax_h + 1:
        nphi *= 2
    return (2 * lmax_h + 1, nphi)


def realization_pairs(nside, lmax, levels, cycles):
    """SHT pairs (one synthesis + one adjoint) of one realization: `cycles`
    CR-Cycles from zero (Fig. code:mg; n_rec 1 at the top, the table's n_rec
    below; the top smoother is diagonal, the bottom dense) and the FP64
    residual before every cycle but the first.  levels: list of (nside_h,
    lmax_h, n_rec, noise) with noise None (observation grid) or (ntheta,
    nphi).  Returns {grid key: pairs}, keys ("healpix", nside, L) or
    ("gl", ntheta, nphi, L)."""
    from collections import Counter

    def a_key(h):
        if h == 0:
            return ("healpix", nside, lmax)
        nh, lh, _, noise = levels[h - 1]
        return ("healpix", nside, lh) if noise is None else ("gl", noise[0], noise[1], lh)

    def cycle(h, start):
        if h == len(levels) + 1:
            return Counter()
        c = Counter()
        sm = None if h == 0 else ("healpix", levels[h - 1][0], levels[h - 1][1])
        if start != "zero":
            c[a_key(h)] += 1
        if sm:
            c[sm] += 1
        c[a_key(h)] += 1
        nrec = 1 if h == 0 else levels[h - 1][2]
        for i in range(nrec):
            c += cycle(h + 1, "zero" if i == 0 else "gen")
        c[a_key(h)] += 1
        if sm:
            c[sm] += 1
        return c

    tot = Counter()
    for _ in range(cycles):
        tot += cycle(0, "zero")
    tot[("healpix", nside, lmax)] += cycles - 1
    return dict(tot)


def oracle_pair_seconds(key, nring_sample=32):
    """The oracle's time for one synthesis + adjoint on the full grid of
    `key`, from its time on evenly spaced sample rings (scaled by rings)."""
    import numpy as np

    from oracle import geometry, sht

    if key[0] == "healpix":
        g = geometry.healpix_grid(key[1])
    else:
        g = geometry.gl_grid(key[1], key[2])
    L = key[-1]
    nr = min(nring_sample, g["nring"])
    idx = np.unique(np.linspace(0, g["nring"] - 1, nr).astype(np.int64))
    nphi = g["nphi"][idx]
    sub = dict(kind=g["kind"], z=g["z"][idx], sth=g["sth"][idx], nphi=nphi,
               off=np.concatenate([[0], np.cumsum(nphi)[:-1]]).astype(np.int64), phi0=g["phi0"][idx],
               wgt=g["wgt"][idx], npix=int(nphi.sum()), nring=len(idx))
    rng = np.random.default_rng(0)
    a = rng.normal(size=sht.n_lm(L)) + 1j * rng.normal(size=sht.n_lm(L))
    a[: L + 1] = a[: L + 1].real
    y = rng.normal(size=sub["npix"])
    t0 = time.perf_counter()
    sht.synth(a, L, sub)
    sht.adjoint(y, L, sub)
    dt = time.perf_counter() - t0
    return dt * g["nring"] / len(idx), len(idx)


def oracle_levels(nside, lmax):
    """The level table (with the noise grid of each level) the library builds
    by default, from the oracle's level-table rule."""
    from oracle import multilevel

    t = multilevel.level_table(nside, lmax)
    return [(lv["nside_h"], lv["lmax_h"], lv["n_rec"], gl_noise_grid(nside, lv["lmax_h"])) for lv in t["levels"]]


def oracle_full_pair_seconds(nside, lmax):
    """The oracle's wall time for one synthesis + adjoint over the whole
    observation grid (every ring), and for one application of A there --
    the full-size SHT pair, not a ring sample."""
    import numpy as np

    from oracle import geometry, operators, sht
    from paper_1308_5299_gb300 import synthetic

    g = geometry.healpix_grid(nside)
    rng = np.random.default_rng(0)
    a = rng.normal(size=sht.n_lm(lmax)) + 1j * rng.normal(size=sht.n_lm(lmax))
    a[: lmax + 1] = a[: lmax + 1].real
    t0 = time.perf_counter()
    mp = sht.synth(a, lmax, g)
    sht.adjoint(mp, lmax, g)
    pair = time.perf_counter() - t0
    name = "nside%d_lmax%d" % (nside, lmax)
    apply_s = None
    if name in synthetic.CONFIGS:
        _, cl, bl, ninv = synthetic.problem_inputs(name)
        prob = operators.Problem(lmax, cl, bl, ninv, g)
        t1 = time.perf_counter()
        operators.apply_A(prob, a)
        apply_s = time.perf_counter() - t1
    return pair, apply_s


def cpu_baseline(nside, lmax, levels, cycles, full=True):
    """The oracle (plain FP64 direct SHT, C + OpenMP, as it stands) priced on
    one realization: the SHT pairs the realization needs, each at the
    oracle's time for that (grid, band limit).  The observation grid at the
    full band limit -- most of the cost -- is timed over the whole grid (one
    full-size pair and one application of A); the other grids on a sample of
    rings scaled by ring count.  The pixel smoothers' triangular solves and
    the dense bottom solves are not counted, so this is a lower bound."""
    pairs = realization_pairs(nside, lmax, levels, cycles)
    total, rings = 0.0, 0
    top = ("healpix", nside, lmax)
    full_pair = apply_s = sampled_top = None
    if full and top in pairs:
        full_pair, apply_s = oracle_full_pair_seconds(nside, lmax)
    for key, n in pairs.items():
        t, nr = oracle_pair_seconds(key)
        if key == top:
            sampled_top = t
            if full_pair is not None:
                t, nr = full_pair, 4 * nside - 1
        total += n * t
        rings += nr
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": total, "unit": "s/realization", "cores": cores, "kind": "oracle",
           "sample": "%d SHT pairs of one %d-cycle realization at Nside %d / lmax %d over %d (grid, lmax) "
                     "combinations: the observation grid at lmax %s, the others from sample rings scaled to "
                     "full grids (%d rings timed); smoother and bottom solves excluded: lower bound"
                     % (sum(pairs.values()), cycles, nside, lmax, len(pairs),
                        "timed over the full grid" if full_pair is not None else "from sample rings", rings)}
    if full_pair is not None:
        out["full_grid_pair_s"] = full_pair
        out["full_grid_apply_A_s"] = apply_s
        out["sampled_estimate_of_that_pair_s"] = sampled_top
        out["pairs_per_cycle"] = {"_".join(str(x) for x in k): v / cycles for k, v in pairs.items()}
    return out


def oracle_cg_baseline(iterations, workload="nside256_lmax767", k=3):
    """The oracle's own diagonal-preconditioned CG (plain FP64 direct SHTs on
    the host cores) on the Nside 256 workload: k iterations timed and priced
    at the GPU CG's iteration count (the whole solve would take hours).
    Part of the CPU baseline."""
    import numpy as np

    from oracle import geometry, operators, solvers
    from paper_1308_5299_gb300 import synthetic

    cfg, cl, bl, ninv = synthetic.problem_inputs(workload)
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, bl, ninv, g)
    l = prob.l
    with np.errstate(divide="ignore"):
        sinv = np.where(prob.active, 1.0 / np.where(prob.active, cl[l], 1.0), 0.0)
    dg = sinv + bl[l] ** 2 * operators.diag_inv_noise_dm0(prob)
    pc = np.where(prob.active & (dg > 0), 1.0 / np.where(dg > 0, dg, 1.0), 0.0)
    b = operators.apply_A(prob, prob.clean(synthetic.draw_prior(cl, index=7)))
    t0 = time.perf_counter()
    solvers.pcg(lambda v: operators.apply_A(prob, v), b, pc, prob.lmax, tol=0.0, maxiter=k)
    per_it = (time.perf_counter() - t0) / k
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"workload": workload, "s_per_iteration": per_it, "iterations_timed": k, "cores": cores,
            "iterations": iterations, "s_extrapolated": per_it * iterations if iterations else None}


def run_reference(args, rank, world):
    """The reference arm: the oracle on the machine's host cores.  Once, the
    full-size observation-grid SHT pair and A (a minute or so); then every
    step times the oracle's pairs on sample rings of every (grid, band limit)
    of a realization and prices the realization with them, the observation
    grid at lmax taken from the full-size timing.  value is that
    extrapolated time per realization; ms_per_step is the wall time of one
    step's sampling (what was actually timed)."""
    from paper_1308_5299_gb300 import synthetic

    if rank != 0:
        return
    cfg = synthetic.CONFIGS[args.workload]
    nside, lmax = cfg["nside"], cfg["lmax"]
    levels = oracle_levels(nside, lmax)
    cycles = args.ref_cycles
    t_full = time.perf_counter()
    full_pair, apply_s = oracle_full_pair_seconds(nside, lmax)
    t_full = time.perf_counter() - t_full
    pairs = realization_pairs(nside, lmax, levels, cycles)
    top = ("healpix", nside, lmax)
    steps, walls = [], []
    rings = 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        total, rings = 0.0, 0
        for key, n in pairs.items():
            t, nr = oracle_pair_seconds(key)
            if key == top:
                t, nr = full_pair, 4 * nside - 1
            total += n * t
            rings += nr
        if i >= args.warmup:
            steps.append(total)
            walls.append(time.perf_counter() - t0)
    v = statistics.median(steps)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s/realization", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(walls) * 1e3,
           "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "nside": nside, "lmax": lmax,
                      "step": "one realization: CR-Solve of b = A x_true, FP32 W-cycles under FP64 refinement, "
                              "fixed cycle count reaching < 1 uK max-pixel error (found before the timed region)",
                      "cycles": cycles, "levels": [lv[0] for lv in levels],
                      "value_is": "extrapolated: the realization's SHT pairs priced at the oracle's measured "
                                  "pair times (observation grid at lmax timed over the full grid once, %.1f s; "
                                  "other grids from sample rings each step); smoother and bottom solves not "
                                  "counted (lower bound)" % t_full,
                      "ms_per_step_is": "wall time of one step's ring sampling"},
           "cpu_baseline": {"value": v, "unit": "s/realization", "cores": cores, "kind": "oracle",
                            "full_grid_pair_s": full_pair, "full_grid_apply_A_s": apply_s,
                            "sample": "full-grid observation pair (Nside %d, lmax %d) plus %d sample rings of the "
                                      "other %d (grid, lmax) combinations per step" % (nside, lmax, rings - (4 * nside - 1),
                                                                                     len(pairs) - 1)},
           "e2e": {"value": v, "unit": "s/realization", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def max_pixel_error(plan, x, x_true, npix, dev):
    """max_i |Y (x - x_true)|_i over the observation grid (uK)."""
    import torch
    m = torch.empty(npix, dtype=torch.float64, device=dev)
    plan.sht_synth(x - x_true, m)
    return float(m.abs().max())


# Nominal FMA-pipe rates (152 SMs at 2070 MHz): FP32 128 FMA lanes per SM ->
# 80.5 TFLOP/s; FP64 the part's 1.25 TFLOP/s.  The roofline uses the rates
# measured live by the library's FMA probe (cr_probe_fma_peak) and falls back
# to these only if the probe cannot run.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 1.25

# stages that time a sequence of kernels rather than one kernel
COMPOSITE = {"outer_residual"}

# ncu DRAM traffic per launch of the dominant kernels, read from the profile
# summaries committed under profiles/ (a line "traffic_bytes_per_launch: N"
# beside the kernel's name and template arguments)
TRAFFIC_FILES = {"legendre_adjoint_f64": "legendre_adjoint_f64_dram_nside2048_lmax3000.txt"}


def profile_traffic(stage):
    fn = TRAFFIC_FILES.get(stage)
    if not fn:
        return None, None
    path = os.path.join(ROOT, "profiles", fn)
    try:
        vals = {}
        for line in open(path):
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        sha = vals.get("source_sha256")
        src = os.path.join(ROOT, "paper_1308_5299_gb300", "csrc", "legendre.cu")
        if sha and hashlib.sha256(open(src, "rb").read()).hexdigest() != sha:
            return None, vals.get("kernel") + " (counters taken on an earlier source: traffic withheld)"
        return float(vals["traffic_bytes_per_launch"]), vals.get("kernel")
    except (OSError, KeyError, ValueError):
        return None, None


def live_peaks(binding):
    """FMA-pipe peaks measured now on this GPU (TFLOP/s)."""
    out = {}
    for k in ("f32", "f32x2", "f64"):
        try:
            out[k] = binding.fma_peak(k)
        except Exception:  # noqa: BLE001 -- report what could be measured
            out[k] = None
    return out


def roofline_of(stages, exec_work, steps, peaks_live):
    """Roofline of the kernel stage with the largest share of the timed
    region.  Legendre stages are bound by the FMA pipe of their precision:
    achieved = the flops of the terms the kernel evaluates (8 per ring pair
    and (l, m) past the start tables) per launch over the launch's CUDA-event
    time, against the FMA rate measured live on this GPU; the dense count of
    every ring pair and (l, m) is reported beside it.  Ring-FFT stages and
    the pixel smoother: algorithmic bytes against the measured HBM copy
    bandwidth."""
    peaks = measured_peaks()
    kern = {k: v for k, v in stages.items() if k not in COMPOSITE and "." not in k}
    dom = max(kern, key=lambda k: kern[k][0])
    ms, n, work = kern[dom]
    wex = exec_work.get(dom, 0.0)
    traffic, traffic_kernel = profile_traffic(dom)
    base = {"kernel": dom, "ms_per_step": ms / steps, "launches_per_step": n / steps,
            "algorithmic_work_per_launch": (wex or work) / max(n, 1), "traffic": traffic}
    if traffic_kernel:
        base["traffic_kernel"] = traffic_kernel
    if dom.startswith("legendre") and work > 0:
        f64 = dom.endswith("_f64")
        live = peaks_live.get("f64" if f64 else "f32")
        peak = live if live else (FP64_PEAK_TFLOPS if f64 else FP32_PEAK_TFLOPS)
        src = ("measured live: FMA-chain probe on this GPU (cr_probe_fma_peak)" if live else
               "nominal: 152 SMs x 2070 MHz x FMA lanes x 2")
        ach_dense = work / (ms * 1e-3) / 1e12
        ach = (wex if wex > 0 else work) / (ms * 1e-3) / 1e12
        return dict(base, bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                    frac_executed=ach / peak, achieved_dense=ach_dense, frac_dense=ach_dense / peak,
                    work_note="achieved counts the terms the kernel evaluates (past the 2^-60 start of every "
                              "(m, ring pair)); achieved_dense counts every ring pair and (l, m)",
                    peak_source=src)
    if work > 0:
        peak = peaks.get("hbm_gbs", 6778.0)
        ach = work / (ms * 1e-3) / 1e9
        return dict(base, bound="hbm", achieved=ach, peak=peak, unit="GB/s", frac=ach / peak,
                    peak_source="MEASURED_PEAKS.json hbm_gbs (measured)")
    return dict(base, bound="alu", achieved=None, peak=None, unit=None, frac=None)


def schwarz_variant(binding, synthetic, dev, stream, args, cfg, cl, bl, ninv, x_true, npix):
    """The same realization with the additive Schwarz (block Jacobi over
    tiles) pixel smoother instead of the multicolour block ICC(0): fewest
    cycles to < 1 uK (stationary mixed, or mixed PCG when it needs fewer),
    time per realization (CUDA events; stationary solves replayed from a
    graph), error, and the smoother's share."""
    import torch

    plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                        stream=stream, levels="default", smoother="schwarz")
    b = torch.empty_like(x_true)
    plan.apply_A(x_true, b)
    x = torch.empty_like(b)

    def fewest(mode, cap):
        for c in range(1, cap + 1):
            plan.solve(b, x, eps=0.0, max_cycles=c, mode=mode | binding.CR_FIXED, check=False)
            if max_pixel_error(plan, x, x_true, npix, dev) < 1.0:
                return c
        return None

    c_st = fewest(binding.CR_MIXED, 16)
    c_pcg = fewest(binding.CR_MIXED | binding.CR_PCG, c_st - 1 if c_st else 16)
    if c_st is None and c_pcg is None:
        return {"converged_within": 16, "note": "no cycle count up to 16 reached 1 uK"}
    pcg = c_pcg is not None
    cyc = c_pcg if pcg else c_st
    mode = binding.CR_MIXED | (binding.CR_PCG if pcg else 0)
    graph = None if (pcg or args.no_graph) else binding.Batch([plan], [x], [b], cyc, binding.CR_MIXED)

    def step():
        if graph is not None:
            graph.run()
        else:
            plan.solve(b, x, eps=0.0, max_cycles=cyc, mode=mode | binding.CR_FIXED, check=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3 / args.steps
    err = max_pixel_error(plan, x, x_true, npix, dev)
    if graph is not None:
        graph.close()
    plan.set_timing(True)
    plan.solve(b, x, eps=0.0, max_cycles=cyc, mode=mode | binding.CR_FIXED, check=False)
    torch.cuda.synchronize()
    sm = {k: v[0] for k, v in plan.timing().items() if k.startswith("pixel_smoother")}
    plan.set_timing(False)
    del plan
    torch.cuda.synchronize()
    return {"cycles": cyc, "pcg": pcg, "stationary_cycles": c_st, "s_per_realization": sec,
            "max_pixel_error_uK": err, "pixel_smoother_ms": sm.get("pixel_smoother"),
            "note": "additive Schwarz without overlap: one parallel tile-inverse pass per smoothing step"}


def df_variant(binding, synthetic, dev, stream, args, cfg, cl, bl, ninv, x_true, npix):
    """Mixed-precision realization with the outer residual's FP64 Legendre
    stages in double-float arithmetic: cycles to < 1 uK, time per
    realization (CUDA events, same protocol as the headline), error."""
    import torch

    plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                        stream=stream, levels="default", fp64_df=True)
    b = torch.empty_like(x_true)
    plan.apply_A(x_true, b)
    x = torch.empty_like(b)
    mode = binding.CR_MIXED | binding.CR_FIXED
    cyc = 1
    for cyc in range(1, 13):
        plan.solve(b, x, eps=0.0, max_cycles=cyc, mode=mode, check=False)
        if max_pixel_error(plan, x, x_true, npix, dev) < 1.0:
            break
    graph = None if args.no_graph else binding.Batch([plan], [x], [b], cyc, binding.CR_MIXED)

    def step():
        if graph is not None:
            graph.run()
        else:
            plan.solve(b, x, eps=0.0, max_cycles=cyc, mode=mode, check=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) * 1e-3 / args.steps
    err = max_pixel_error(plan, x, x_true, npix, dev)
    if graph is not None:
        graph.close()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    y = torch.empty_like(b)
    a0.record(stream)
    plan.apply_A(x_true, y)
    a1.record(stream)
    torch.cuda.synchronize()
    del plan
    torch.cuda.synchronize()
    return {"s_per_realization": s, "cycles": cyc, "max_pixel_error_uK": err,
            "apply_A_f64_df_s": a0.elapsed_time(a1) * 1e-3,
            "note": "outer residual with FP64 Legendre stages in double-float (FP32-pair, error-free transforms)"}


def fewest_cycles(solve_with, worst_error, start, cap):
    """Fewest fixed cycle counts c <= cap for which solve_with(c) leaves every
    right-hand side below 1 uK (worst_error()), searched from `start` (a
    neighbouring form's count): down while c - 1 still passes, else up.
    None when cap cycles do not reach it."""
    c = max(1, min(start, cap))
    solve_with(c)
    if worst_error() < 1.0:
        while c > 1:
            solve_with(c - 1)
            if worst_error() >= 1.0:
                break
            c -= 1
        solve_with(c)  # leave the solution of the chosen count behind
        return c
    while c < cap:
        c += 1
        solve_with(c)
        if worst_error() < 1.0:
            return c
    return None


def batch_measurement(binding, synthetic, dev, args, nrhs=16):
    """Batched mixed-resolution realizations: nrhs right-hand sides at
    Nside 1024 / lmax 2047 and nrhs at Nside 512 / lmax 1023, mixed-precision
    fixed-count CR-Solves captured into one CUDA graph and replayed with one
    launch; the cycle count is the fewest reaching < 1 uK max-pixel error on
    every right-hand side.  Reports realizations/s for the graph and for the
    same solves launched directly, and every realization's error."""
    import numpy as np
    import torch

    st = torch.cuda.Stream(dev)
    with torch.cuda.stream(st):
        plans, xs, bs, xts, npx = [], [], [], [], []
        for k, name in enumerate(["nside1024_lmax2047", "nside512_lmax1023"]):
            cfg, cl, bl, ninv = synthetic.problem_inputs(name)
            plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                                stream=st, levels="default", autotune=True)
            xt = torch.from_numpy(np.stack([synthetic.draw_prior(cl, index=100 * (k + 1) + j)
                                            for j in range(nrhs)])).to(dev)
            b = torch.empty_like(xt)
            plan.apply_A(xt, b)
            plans.append(plan)
            xs.append(torch.zeros_like(b))
            bs.append(b)
            xts.append(xt)
            npx.append(12 * cfg["nside"] ** 2)

        def errors():
            out = []
            for plan, x, xt, n in zip(plans, xs, xts, npx):
                for j in range(x.shape[0]):
                    out.append(max_pixel_error(plan, x[j], xt[j], n, dev))
            return out

        total = sum(x.shape[0] for x in xs)

        def variant(mode, start=3):
            # fewest fixed cycles reaching < 1 uK on every right-hand side,
            # then the same solves launched directly and from one graph
            def solve_with(c):
                for plan, x, b in zip(plans, xs, bs):
                    plan.solve(b, x, eps=0.0, max_cycles=c, mode=mode | binding.CR_FIXED, check=False)

            cycles = fewest_cycles(solve_with, lambda: max(errors()), start, 12)
            if cycles is None:
                return {"converged_within": 12, "max_pixel_error_uK": max(errors()),
                        "graph_realizations_per_s": 0.0}

            def direct():
                for plan, x, b in zip(plans, xs, bs):
                    plan.solve(b, x, eps=0.0, max_cycles=cycles, mode=mode | binding.CR_FIXED, check=False)

            direct()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            direct()
            torch.cuda.synchronize()
            t_direct = time.perf_counter() - t0
            graph = binding.Batch(plans, xs, bs, cycles, mode)
            graph.run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 2
            e0.record(st)
            for _ in range(reps):
                graph.run()
            e1.record(st)
            torch.cuda.synchronize()
            t_graph = e0.elapsed_time(e1) * 1e-3 / reps
            errs = errors()
            out = {"cycles": cycles, "graph_nodes": graph.nodes(),
                   "graph_realizations_per_s": total / t_graph, "graph_s": t_graph,
                   "direct_realizations_per_s": total / t_direct, "direct_s": t_direct,
                   "max_pixel_error_uK": {"max": max(errs), "median": float(np.median(errs))}}
            graph.close()
            return out

        fp32 = variant(binding.CR_MIXED)
        c0 = fp32.get("cycles", 3)
        tc = variant(binding.CR_MIXED | binding.CR_TC_CYCLES, c0)
        tc_split = variant(binding.CR_MIXED | binding.CR_TC_CYCLES | binding.CR_TC_SPLIT, c0)
        tc_top = variant(binding.CR_MIXED | binding.CR_TC_CYCLES | binding.CR_TC_TOP_F32, c0)
        # batched synthesis of the 16 Nside 1024 solutions: Legendre
        # contraction on the tensor cores vs 16 FP32 syntheses
        p0, x0 = plans[0], xs[0]
        x32 = x0.to(torch.complex64)
        maps = torch.empty((x32.shape[0], npx[0]), dtype=torch.float32, device=dev)
        p0.sht_synth(x32, maps, tensor_cores=True)
        torch.cuda.synchronize()
        t0, t1, t2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        t0.record(st)
        p0.sht_synth(x32, maps, tensor_cores=True)
        t1.record(st)
        for j in range(x32.shape[0]):
            p0.sht_synth(x32[j], maps[j])
        t2.record(st)
        torch.cuda.synchronize()
        tc_ms, f32_ms = t0.elapsed_time(t1), t1.elapsed_time(t2)
        # the system matrix on the same 16 vectors: both Legendre stages on
        # the tensor cores vs 16 FP32 applications; accuracy against FP64
        y32 = torch.empty_like(x32)
        p0.apply_A(x32, y32, tensor_cores=True)
        torch.cuda.synchronize()
        t0.record(st)
        p0.apply_A(x32, y32, tensor_cores=True)
        t1.record(st)
        yf = torch.empty_like(x32)
        for j in range(x32.shape[0]):
            p0.apply_A(x32[j], yf[j])
        t2.record(st)
        torch.cuda.synchronize()
        atc_ms, af32_ms = t0.elapsed_time(t1), t1.elapsed_time(t2)
        y64 = torch.empty_like(x0)
        p0.apply_A(x0, y64)
        torch.cuda.synchronize()
        rel_tc = float(torch.linalg.vector_norm(y32.to(torch.complex128) - y64) / torch.linalg.vector_norm(y64))
        rel_f32 = float(torch.linalg.vector_norm(yf.to(torch.complex128) - y64) / torch.linalg.vector_norm(y64))
        del y32, yf, y64
    forms = {"fp32_cycles": fp32, "tensor_core_cycles": tc, "tensor_core_cycles_split": tc_split,
             "tensor_core_cycles_fp32_top": tc_top}
    best = max(forms, key=lambda k: forms[k]["graph_realizations_per_s"])
    return {"workload": "%d x (Nside 1024, lmax 2047) + %d x (Nside 512, lmax 1023)" % (nrhs, nrhs),
            "realizations": total,
            "realizations_per_s": forms[best]["graph_realizations_per_s"],
            "form": best,
            "tensor_core_cycles_fp32_top": dict(tc_top, note="CR_TC_CYCLES | CR_TC_TOP_F32: pixel levels batched on "
                                                            "tcgen05, top-level residuals per right-hand side on the "
                                                            "FP32 CUDA cores"),
            "tensor_core_cycles_split": dict(tc_split, note="CR_MIXED | CR_TC_CYCLES | CR_TC_SPLIT: the "
                                                            "tensor-core cycles with hi + lo BF16 operands "
                                                            "(three MMAs per step)"),
            "tensor_core_cycles": dict(tc, note="CR_MIXED | CR_TC_CYCLES: FP32 cycles of 16 right-hand sides "
                                                "together, every Legendre stage on tcgen05 (BF16 in, FP32 "
                                                "accumulation); FP64 outer residual per right-hand side"),
            "fp32_cycles": dict(fp32, note="CR_MIXED: FP32 CUDA-core cycles per right-hand side"),
            "synthesis_16rhs_nside1024": {"tensor_core_ms": tc_ms, "fp32_ms": f32_ms,
                                          "note": "Legendre contraction on tcgen05 (BF16 in, FP32 accumulation) "
                                                  "vs the FP32 CUDA-core kernels; ring FFTs included in both"},
            "apply_A_16rhs_nside1024": {"tensor_core_ms": atc_ms, "fp32_ms": af32_ms,
                                        "rel_l2_vs_f64": {"tensor_core": rel_tc, "fp32": rel_f32},
                                        "note": "A = S^-1 + B Y^T N^-1 Y B, both Legendre stages on tcgen05 "
                                                "vs the FP32 CUDA-core kernels"}}


def batch_nside2048(binding, synthetic, dev, args, nrhs=16):
    """Batched Planck-shaped realizations: nrhs right-hand sides b = A x_true
    at Nside 2048 / lmax 3000 solved together in one CUDA graph, for the
    per-right-hand-side FP32 cycles (CR_MIXED) and the tensor-core cycles
    with split (hi + lo) BF16 operands (16 right-hand sides per contraction);
    every form with the fewest fixed cycles reaching < 1 uK max-pixel error on
    every right-hand side.  Reports seconds per realization (graph replay /
    nrhs), cycles, and the per-right-hand-side errors.  The plain-BF16 cycles
    are measured on the Nside 1024 / 512 batch only: at this size their
    inexact preconditioner needs many more cycles."""
    import numpy as np
    import torch

    st = torch.cuda.Stream(dev)
    out = {"workload": "%d x (Nside 2048, lmax 3000)" % nrhs, "realizations": nrhs}
    with torch.cuda.stream(st):
        cfg, cl, bl, ninv = synthetic.problem_inputs("nside2048_lmax3000")
        npix = 12 * cfg["nside"] ** 2
        plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                            stream=st, levels="default", autotune=True)
        xt = torch.from_numpy(np.stack([synthetic.draw_prior(cl, index=300 + j) for j in range(nrhs)])).to(dev)
        b = torch.empty_like(xt)
        plan.apply_A(xt, b)
        x = torch.zeros_like(b)

        def errors():
            return [max_pixel_error(plan, x[j], xt[j], npix, dev) for j in range(nrhs)]

        start = 2
        for name, mode in (("fp32_cycles", binding.CR_MIXED),
                           ("tensor_core_cycles_split", binding.CR_MIXED | binding.CR_TC_CYCLES | binding.CR_TC_SPLIT)):
            def solve_with(c, mode=mode):
                plan.solve(b, x, eps=0.0, max_cycles=c, mode=mode | binding.CR_FIXED, check=False)

            cycles = fewest_cycles(solve_with, lambda: max(errors()), start, 6)
            if cycles is None:
                out[name] = {"converged_within": 6, "max_pixel_error_uK": max(errors())}
                continue
            start = cycles
            graph = binding.Batch([plan], [x], [b], cycles, mode)
            graph.run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            graph.run()
            e1.record(st)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) * 1e-3
            errs = errors()
            out[name] = {"cycles": cycles, "graph_s": t, "s_per_realization": t / nrhs,
                         "graph_nodes": graph.nodes(),
                         "max_pixel_error_uK": {"max": max(errs), "median": float(np.median(errs))}}
            graph.close()
        del plan, xt, b, x
        torch.cuda.synchronize()
    forms = [k for k in ("fp32_cycles", "tensor_core_cycles_split") if "s_per_realization" in out.get(k, {})]
    if forms:
        best = min(forms, key=lambda k: out[k]["s_per_realization"])
        out["form"] = best
        out["s_per_realization"] = out[best]["s_per_realization"]
    return out


def cg_comparison(binding, synthetic, dev, stream, workload="nside256_lmax767"):
    """The multi-level solver against diagonal-preconditioned CG (the method
    the paper compares against) on the Nside 256 workload: iterations and
    GPU time to a 1e-6 relative residual r^T S^-1 r / b^T S^-1 b < 1e-12."""
    import torch

    cfg, cl, bl, ninv = synthetic.problem_inputs(workload)
    plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                        stream=stream, levels="default")
    x_true = torch.from_numpy(synthetic.draw_prior(cl, index=7)).to(dev)
    b = torch.empty_like(x_true)
    plan.apply_A(x_true, b)
    x = torch.empty_like(b)
    out = {"workload": workload, "stop": "relative residual 1e-6 (r^T S^-1 r < 1e-12 b^T S^-1 b)"}
    for name, mode, cap in [("multilevel_f64", binding.CR_F64 | binding.CR_PCG, 400),
                            ("multilevel_mixed", binding.CR_MIXED | binding.CR_PCG, 400),
                            ("cg_diag_f64", binding.CR_F64 | binding.CR_CG, 20000)]:
        plan.solve(b, x, eps=1e-12, max_cycles=cap, mode=mode, check=False)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cyc, rel, hist, rc = plan.solve(b, x, eps=1e-12, max_cycles=cap, mode=mode, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"iterations": int(cyc[0]), "relres": float(rel[0]), "s": e0.elapsed_time(e1) * 1e-3,
                     "converged": rc == 0}
    return out


def whole_job(t_local, world, dev=None):
    """Timing across replicas: the MAX over ranks of the per-step time
    t_local, and the whole job's time per realization -- every rank solves
    its own realization each step, so `world` realizations finish per step.
    Returns (t_max, t_max / world).  One rank: (t_local, t_local)."""
    t = float(t_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        v = torch.tensor([t], dtype=torch.float64, device=dev if dev is not None else "cpu")
        dist.all_reduce(v, op=dist.ReduceOp.MAX)
        t = float(v.item())
    return t, t / world


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
    npix = 12 * nside * nside
    peaks_live = live_peaks(binding)
    # a created stream (the legacy default stream cannot be captured into a graph)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    torch.cuda.synchronize()
    # precompute in the paper's two parts (Section 5): the plan structure
    # and the observation-dependent terms, then the C_l-dependent part; a
    # second C_l update (same active set) times what a new C_l costs alone
    ninv_d = torch.from_numpy(ninv).to(dev)
    t0 = time.perf_counter()
    plan = binding.Plan(lmax, nside=nside, cl=cl, bl=bl, ninv=ninv_d, stream=stream, levels="default",
                        defer_precompute=True)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    plan.update_cl(cl)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    plan.update_cl(cl)
    torch.cuda.synchronize()
    precompute_s = t2 - t0
    precompute_split = {"structure_s": t1 - t0, "first_numeric_s": t2 - t1,
                        "cl_update_s": time.perf_counter() - t2}
    del ninv_d
    # Legendre autotuner: ring-block choice per grid, band limit, precision
    t3 = time.perf_counter()
    table = plan.autotune()
    autotune = {"s": time.perf_counter() - t3,
                "observation_grid": {"%s_%s" % (t["precision"], t["stage"]):
                                     ({"pairs_per_thread": t["pairs_per_thread"], "m_tile": t["m_tile"]}
                                      if "pairs_per_thread" in t else {"variant": t["variant"]})
                                     for t in table if t["nring"] == 4 * nside - 1 and t["lmax"] == lmax},
                "m_tile_2_chosen": sum(1 for t in table if t.get("m_tile") == 2),
                "entries": len(table)}
    x_true = torch.from_numpy(synthetic.draw_prior(cl, index=rank)).to(dev)
    b = torch.empty_like(x_true)
    plan.apply_A(x_true, b)  # b = A x_true (FP64), the paper's synthetic protocol
    x = torch.empty_like(b)

    # calibration (outside the timed region): fewest cycles reaching < 1 uK
    def cycles_to(mode, cap=12):
        for c in range(1, cap + 1):
            plan.solve(b, x, eps=0.0, max_cycles=c, mode=mode | binding.CR_FIXED, check=False)
            err = max_pixel_error(plan, x, x_true, npix, dev)
            if err < 1.0:
                return c, err
        return cap, err

    def best_mode(base):
        # stationary CR-Solve (Fig. code:mg) or CR-Cycle-preconditioned
        # flexible CG; fewer cycles wins, the stationary form on a tie
        c1, e1 = cycles_to(base)
        c2, e2 = cycles_to(base | binding.CR_PCG, cap=c1)
        return (base | binding.CR_PCG, c2, e2) if (c2 < c1 and e2 < 1.0) else (base, c1, e1)

    mode_mixed, cyc_mixed, err_mixed = best_mode(binding.CR_MIXED)
    mode_f64, cyc_f64, err_f64 = best_mode(binding.CR_F64)

    def solve_mixed():
        plan.solve(b, x, eps=0.0, max_cycles=cyc_mixed, mode=mode_mixed | binding.CR_FIXED, check=False)

    # the fixed-count solve captured once into a CUDA graph (stationary form):
    # one launch per realization; the direct launches are timed beside it
    graph = None
    if not (mode_mixed & binding.CR_PCG) and not args.no_graph:
        graph = binding.Batch([plan], [x], [b], cyc_mixed, mode_mixed)

    def step():
        if graph is not None:
            graph.run()
        else:
            solve_mixed()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = binding.launch_count()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    launches = (graph.kernel_nodes() * args.steps) if graph is not None else binding.launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    # the same solves launched directly, with per-stage CUDA events (the
    # kernel-level breakdown and the roofline come from this region)
    plan.set_timing(True)
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    d0.record(stream)
    for _ in range(args.steps):
        solve_mixed()
    d1.record(stream)
    torch.cuda.synchronize()
    ms_direct = d0.elapsed_time(d1) / args.steps
    stages = plan.timing()
    stages_exec = plan.timing_exec()
    plan.set_timing(False)
    ms, ms_job = whole_job(ms, world, dev)
    err_timed = max_pixel_error(plan, x, x_true, npix, dev)

    # plain FP64 solve (same protocol), one timed run
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    plan.solve(b, x, eps=0.0, max_cycles=cyc_f64, mode=mode_f64 | binding.CR_FIXED, check=False)
    f1.record(stream)
    torch.cuda.synchronize()
    f64_s = f0.elapsed_time(f1) * 1e-3

    # SHT pair throughput (apply_A) in both precisions
    def pair_rate(dtype_c, reps=3):
        xx = x_true.to(dtype_c)
        yy = torch.empty_like(xx)
        plan.apply_A(xx, yy)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            plan.apply_A(xx, yy)
        a1.record(stream)
        torch.cuda.synchronize()
        return reps / (a0.elapsed_time(a1) * 1e-3)

    pairs_f64 = pair_rate(torch.complex128)
    pairs_f32 = pair_rate(torch.complex64, reps=10)

    # end to end through the C ABI with host buffers
    bh = b.cpu().pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps // 2)):
        b.copy_(bh, non_blocking=True)  # the graph reads b and writes x at their bound addresses
        step()
        xh.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = whole_job((time.perf_counter() - t0) / max(1, args.steps // 2), world, dev)[1]

    # the same realization with the FP64 Legendre stages (outer residual) in
    # double-float arithmetic on the FP32 pipes (plan option fp64_df)
    level_nsides = [plan.level(h)["nside_h"] for h in range(1, plan.nlevels() + 1)]
    level_rows = []
    for h in range(1, plan.nlevels() + 1):
        lv = plan.level(h)
        kind, nring, npx = plan.level_grid(h)
        level_rows.append((lv["nside_h"], lv["lmax_h"], lv["n_rec"], (nring, npx // nring) if kind == "gl" else None))
    mixed_df = None
    if graph is not None:
        graph.close()
    if not args.no_df:
        del plan
        torch.cuda.synchronize()
        mixed_df = df_variant(binding, synthetic, dev, stream, args, cfg, cl, bl, ninv, x_true, npix)

    schwarz = None if not args.schwarz else schwarz_variant(binding, synthetic, dev, stream, args, cfg, cl, bl, ninv,
                                                             x_true, npix)
    cg_cmp = None if args.no_cg else cg_comparison(binding, synthetic, dev, stream)
    batch = None if args.no_batch else batch_measurement(binding, synthetic, dev, args)
    batch2048 = None if args.no_batch else batch_nside2048(binding, synthetic, dev, args)

    if rank != 0:
        return
    clocks = clk.summary()
    value = ms_job * 1e-3  # whole job: seconds per realization over all replicas
    out = {
        "metric": METRIC, "value": value, "unit": "s/realization", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "nside": nside, "lmax": lmax,
                   "step": "one realization: CR-Solve of b = A x_true, FP32 W-cycles under FP64 refinement, "
                           "fixed cycle count reaching < 1 uK max-pixel error (found before the timed region)",
                   "cycles": cyc_mixed, "levels": level_nsides,
                   "l2": "inputs larger than L2 (N^-1 403 MB, phase 393 MB, smoother factors ~20 GB)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "max_pixel_error_uK": {"mixed": err_timed, "mixed_calibration": err_mixed, "fp64": err_f64},
        "launch": "cuda_graph" if graph is not None else "direct",
        "direct_launch_s_per_realization": ms_direct * 1e-3,
        "fp64": {"s_per_realization": f64_s, "cycles": cyc_f64, "pcg": bool(mode_f64 & binding.CR_PCG)},
        "mixed_pcg": bool(mode_mixed & binding.CR_PCG),
        "sht_pairs_per_s": {"f64": pairs_f64, "f32": pairs_f32},
        "precompute_s": precompute_s,
        "precompute_split": precompute_split,
        "autotune": autotune,
        "e2e": {"value": e2e_s, "unit": "s/realization", "h2d_bytes_per_step": int(bh.numel() * 16),
                "d2h_bytes_per_step": int(xh.numel() * 16)},
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
        "stages_work_per_step": {k: v[2] / args.steps for k, v in stages.items() if v[2] > 0},
        "roofline": roofline_of(stages, stages_exec, args.steps, peaks_live),
        "fma_peaks_tflops": peaks_live,
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    if mixed_df is not None:
        out["mixed_df_residual"] = mixed_df
    if schwarz is not None:
        out["schwarz_smoother"] = schwarz
    if cg_cmp is not None:
        out["cg_comparison"] = cg_cmp
    if batch is not None:
        out["batch"] = batch
    if batch2048 is not None:
        batch2048["fp64_single_s_per_realization"] = f64_s
        batch2048["mixed_single_s_per_realization"] = value
        out["batch_nside2048"] = batch2048
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(nside, lmax, level_rows, cyc_mixed)
        if cg_cmp is not None:
            out["cpu_baseline"]["oracle_cg_nside256"] = oracle_cg_baseline(cg_cmp["cg_diag_f64"]["iterations"])
    print(json.dumps(out))


if __name__ == "__main__":
    main()
