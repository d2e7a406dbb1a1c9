"""Timed runs of single library calls on synthetic inputs, one JSON line each.

    python -m paper_1308_5299_gb300.cases tc --nside 512 --lmax 1023 --nrhs 16
    python -m paper_1308_5299_gb300.cases sht --nside 1024 --lmax 2047 --dtype f32
    python -m paper_1308_5299_gb300.cases diag --workload nside256_lmax767
    python -m paper_1308_5299_gb300.cases grad --workload nside512_lmax1023 --nrhs 8

``tc``: batched synthesis, adjoint synthesis and system-matrix application
with the Legendre contractions on the tensor cores (BF16 operands, FP32
accumulation) for ``nrhs`` right-hand sides, against the same number of
FP32 CUDA-core calls, timed with CUDA events on the plan's stream after
``--warmup`` untimed repetitions.  Inputs: random coefficients and maps of
the Planck-shaped problem of that size (prior, beam and noise of
``synthetic.problem_inputs`` where the name exists, else a damped spectrum
with a 60 arcmin beam and unit noise).

``sht``: one synthesis and one adjoint synthesis of a single right-hand side
in FP32 or FP64.

``apply``: A = S^-1 + B Y^T N^-1 Y B in FP32 or FP64 on a named workload
(``--workload``), with the per-stage CUDA-event times of the plan (Legendre
synthesis, fused ring FFTs with N^-1, Legendre adjoint) and the stages'
dense and executed Legendre flops; ``--nrhs N`` applies it to N prior draws
at once (FP64: the Legendre stages 8 right-hand sides at a time).

``smooth``: one pixel-smoother application (Y_h^T M_h Y_h r in FP32) per
pixel level of a named workload's default hierarchy, with the ICC(0)
triangular sweeps launched once per colour and as one cooperative launch:
the plan's per-stage time of the sweeps alone, per application.

``diag``: the convergence diagnostics of ``diagnostics`` on a synthetic
workload (error by scale per W-cycle, smoother-only stagnation on the first
pixel level, level filters).

``grad``: forward and backward time of the differentiable constrained
realizations (``autodiff``) for nrhs right-hand sides.
"""
import argparse
import json

import numpy as np
import torch

from . import binding, synthetic


def _problem(nside, lmax, dev):
    name = "nside%d_lmax%d" % (nside, lmax)
    if name in synthetic.CONFIGS:
        _, cl, bl, ninv = synthetic.problem_inputs(name)
        return cl, bl, torch.from_numpy(ninv).to(dev)
    cl = synthetic.cl_spectrum(lmax, True)
    bl = synthetic.gaussian_beam(lmax, 60.0)
    return cl, bl, torch.ones(12 * nside * nside, dtype=torch.float64, device=dev)


def _time(fn, stream, reps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tc_case(nside, lmax, nrhs, warmup, reps, tune=False, split=False):
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    cl, bl, ninv = _problem(nside, lmax, dev)
    plan = binding.Plan(lmax, nside=nside, cl=cl, bl=bl, ninv=ninv, stream=stream, tc_split=split)
    if tune:
        plan.autotune()
    nlm = binding.n_lm(lmax)
    a = torch.from_numpy(np.stack([synthetic.random_alm(lmax, seed=300 + j) for j in range(nrhs)]))
    a = a.to(torch.complex64).to(dev)
    m = torch.randn((nrhs, plan.npix), dtype=torch.float32, device=dev)
    maps = torch.empty_like(m)
    out = torch.empty((nrhs, nlm), dtype=torch.complex64, device=dev)
    runs = {
        "synthesis": (lambda: plan.sht_synth(a, maps, tensor_cores=True),
                      lambda: [plan.sht_synth(a[j], maps[j]) for j in range(nrhs)]),
        "adjoint": (lambda: plan.sht_adjoint(m, out, tensor_cores=True),
                    lambda: [plan.sht_adjoint(m[j], out[j]) for j in range(nrhs)]),
        "apply_A": (lambda: plan.apply_A(a, out, tensor_cores=True),
                    lambda: [plan.apply_A(a[j], out[j]) for j in range(nrhs)]),
    }
    res = {}
    for name, (tc, f32) in runs.items():
        for _ in range(warmup):
            tc()
            f32()
        torch.cuda.synchronize()
        res[name] = {"tensor_core_ms": _time(tc, stream, reps), "fp32_ms": _time(f32, stream, reps)}
    return {"case": "tc", "nside": nside, "lmax": lmax, "nrhs": nrhs, "reps": reps, "split": bool(split),
            "ms": res, "tune": [t for t in binding.tune_table() if t["lmax"] == lmax] if tune else None}


def sht_case(nside, lmax, warmup, reps, dtype, pins=()):
    """One synthesis and one adjoint synthesis (single right-hand side) in
    FP32 or FP64, default (untuned) ring blocks unless pinned: pins is a list
    of (stage, pairs per thread, m tile)."""
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    for stage, rp, mt in pins:
        binding.tune_set(4 * nside - 1, 12 * nside * nside, lmax, dtype, stage, rp, m_tile=mt)
    plan = binding.Plan(lmax, nside=nside, stream=stream)
    cdt, rdt = (torch.complex64, torch.float32) if dtype == "f32" else (torch.complex128, torch.float64)
    a = torch.from_numpy(synthetic.random_alm(lmax, seed=301)).to(cdt).to(dev)
    m = torch.empty(plan.npix, dtype=rdt, device=dev)
    out = torch.empty_like(a)
    res = {}
    for name, fn in (("synthesis", lambda: plan.sht_synth(a, m)), ("adjoint", lambda: plan.sht_adjoint(m, out))):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        res[name] = _time(fn, stream, reps)
    return {"case": "sht", "nside": nside, "lmax": lmax, "dtype": dtype, "reps": reps, "pins": list(pins),
            "ms": res}


def apply_case(name, warmup, reps, dtype, tune, pin=None, nrhs=1):
    """A x for one right-hand side on the workload's observation grid, timed
    whole and per stage (one realization's outer residual at Nside 2048 is
    one FP64 call; the FP32 cycles make many FP32 calls).  pin: (stage,
    pairs per thread) fixed for this precision before the plan is made."""
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    cfg, cl, bl, ninv = synthetic.problem_inputs(name)
    lmax = cfg["lmax"]
    if pin is not None:
        nside = cfg["nside"]
        binding.tune_set(4 * nside - 1, 12 * nside * nside, lmax, dtype, pin[0], pin[1])
    plan = binding.Plan(lmax, nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev), stream=stream)
    if tune:
        plan.autotune()
    cdt = torch.complex64 if dtype == "f32" else torch.complex128
    x = torch.from_numpy(synthetic.draw_prior(cl, index=1)).to(cdt).to(dev)
    if nrhs > 1:  # several right-hand sides (FP64: the batched Legendre stages)
        x = torch.stack([torch.from_numpy(synthetic.draw_prior(cl, index=1 + j)).to(cdt) for j in range(nrhs)]).to(dev)
    y = torch.empty_like(x)
    fn = lambda: plan.apply_A(x, y)
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms = _time(fn, stream, reps)
    plan.set_timing(True)
    for _ in range(reps):
        fn()
    st = plan.timing()
    ex = plan.timing_exec()
    plan.set_timing(False)
    stages = {k: {"ms_per_call": v[0] / reps, "work_dense": v[2] / reps, "work_exec": ex.get(k, 0.0) / reps}
              for k, v in st.items()}
    return {"case": "apply", "workload": name, "dtype": dtype, "reps": reps, "autotuned": bool(tune), "nrhs": nrhs,
            "ms_per_call": ms, "stages": stages,
            "tune": [t for t in binding.tune_table() if t["lmax"] == lmax] if tune else None}


def smooth_case(name, warmup, reps):
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    cfg, cl, bl, ninv = synthetic.problem_inputs(name)
    res = {}
    for mode in ("per_colour", "cooperative"):
        plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                            levels="default", stream=stream, smoother_sweep=mode)
        for h in range(1, plan.nlevels() + 1):
            lv = plan.level(h)
            r = torch.from_numpy(synthetic.random_alm(lv["lmax_h"], seed=7)).to(torch.complex64).to(dev)
            c = torch.empty_like(r)
            for _ in range(warmup):
                plan.smooth(h, r, c)
            torch.cuda.synchronize()
            plan.set_timing(True)
            for _ in range(reps):
                plan.smooth(h, r, c)
            st = plan.timing()
            plan.set_timing(False)
            ms = st.get("pixel_smoother", (0.0, 1, 0.0))
            res.setdefault("n%d" % lv["nside_h"], {})[mode] = {"ms": ms[0] / reps, "GB_per_s": ms[2] / ms[0] / 1e6}
        del plan
        torch.cuda.synchronize()
    return {"case": "smooth", "workload": name, "reps": reps, "levels": res}


def diag_case(name, cycles, iters):
    """Convergence diagnostics (``diagnostics``) of one synthetic problem:
    error by scale after each W-cycle, smoother-only error and residual on
    the first pixel level, and the level filters, sampled at a few l."""
    from . import diagnostics

    dev = torch.device("cuda", 0)
    cfg, cl, bl, ninv = synthetic.problem_inputs(name)
    lmax = cfg["lmax"]
    plan = binding.Plan(lmax, nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                        levels="default")
    xt = torch.from_numpy(synthetic.draw_prior(cl, index=31)).to(dev)
    b = torch.empty_like(xt)
    plan.apply_A(xt, b)
    ls = sorted({2, 8, 32, 128, lmax // 4, lmax // 2, (3 * lmax) // 4, lmax})
    cyc = diagnostics.error_by_scale(plan, b, xt, cycles)
    L1 = plan.level(1)["lmax_h"]
    x = xt.cpu().numpy()
    off = lambda mm: mm * (2 * lmax + 3 - mm) // 2
    xt1 = np.concatenate([x[off(mm):off(mm) + L1 + 1 - mm] for mm in range(L1 + 1)])
    res, rows = diagnostics.smoother_only(plan, 1, torch.from_numpy(xt1).to(dev), iters)
    l1 = [l for l in ls if l <= L1]
    filt = diagnostics.filter_curves(plan)
    return {"case": "diag", "workload": name, "l": ls,
            "error_by_scale": [[float(r[l]) for l in ls] for r in cyc],
            "smoother_only_level1": {"l": l1, "relres": [float(v) for v in res],
                                     "error_last": [float(rows[-1][l]) for l in l1],
                                     "error_first": [float(rows[0][l]) for l in l1]},
            "filters": {str(h): [float(f[l]) for l in ls] for h, f in filt.items()}}


def grad_case(name, nrhs, warmup):
    """Differentiation (configuration 5): constrained realizations of nrhs
    right-hand sides and the gradient of L = sum Re(w* x) with respect to
    C_l and N^-1 through the adjoint solve (``autodiff.realization``);
    wall-clock seconds of the forward pass (plan precompute, draws, solves)
    and of the backward pass (adjoint solves, gradient contractions)."""
    import time

    from . import autodiff

    dev = torch.device("cuda", 0)
    cfg, cl, bl, ninv = synthetic.problem_inputs(name)
    rng = np.random.default_rng(23)
    w = torch.from_numpy(rng.normal(size=(nrhs, binding.n_lm(cfg["lmax"]))) + 0j).to(dev)
    res = {}
    for it in range(warmup + 1):
        tcl = torch.tensor(cl, dtype=torch.float64, requires_grad=True)
        tn = torch.tensor(ninv, dtype=torch.float64, device=dev, requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x = autodiff.realization(tcl, tn, bl, cfg["nside"], seed=5, nrhs=nrhs)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        (torch.conj(w) * x).real.sum().backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        res = {"forward_s": t1 - t0, "backward_s": t2 - t1,
               "grad_cl_finite": bool(torch.isfinite(tcl.grad).all()),
               "grad_ninv_finite": bool(torch.isfinite(tn.grad).all())}
    return {"case": "grad", "workload": name, "nrhs": nrhs, **res,
            "note": "forward includes the plan precompute; solves to a 1e-12 relative residual (mixed PCG)"}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=["tc", "sht", "apply", "smooth", "diag", "grad"])
    ap.add_argument("--tune", action="store_true", help="apply, tc: autotune the kernel shapes first")
    ap.add_argument("--split", action="store_true", help="tc: hi + lo BF16 operands")
    ap.add_argument("--pin-adjoint", type=int, default=0,
                    help="apply, sht: ring pairs per thread of the adjoint Legendre stage (as the autotuner would pin)")
    ap.add_argument("--pin-synth", type=int, default=0,
                    help="sht: ring pairs per thread of the synthesis Legendre stage")
    ap.add_argument("--m-tile", type=int, default=1, help="sht: m tile (1 or 2) of the pinned stages")
    ap.add_argument("--workload", default="nside256_lmax767")
    ap.add_argument("--cycles", type=int, default=4)
    ap.add_argument("--iters", type=int, default=16)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--nside", type=int, default=512)
    ap.add_argument("--lmax", type=int, default=1023)
    ap.add_argument("--nrhs", type=int, default=None, help="right-hand sides (tc, grad: default 16; apply: 1)")
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args(argv)
    nrhs = args.nrhs if args.nrhs is not None else (1 if args.case == "apply" else 16)
    binding.lib()
    if args.case == "tc":
        print(json.dumps(tc_case(args.nside, args.lmax, nrhs, args.warmup, args.reps, args.tune, args.split)))
    elif args.case == "apply":
        pin = None
        if args.pin_adjoint:
            pin = ("adjoint", args.pin_adjoint)
        print(json.dumps(apply_case(args.workload, args.warmup, args.reps, args.dtype, args.tune, pin, nrhs)))
    elif args.case == "smooth":
        print(json.dumps(smooth_case(args.workload, args.warmup, args.reps)))
    elif args.case == "diag":
        print(json.dumps(diag_case(args.workload, args.cycles, args.iters)))
    elif args.case == "grad":
        print(json.dumps(grad_case(args.workload, nrhs, args.warmup)))
    else:
        pins = [(st, rp, args.m_tile) for st, rp in (("synthesis", args.pin_synth), ("adjoint", args.pin_adjoint))
                if rp]
        print(json.dumps(sht_case(args.nside, args.lmax, args.warmup, args.reps, args.dtype, pins)))


if __name__ == "__main__":
    main()
