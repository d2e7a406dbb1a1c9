"""Parity of the CUDA multi-level solver with the oracle (Sections 3.2-3.5,
Fig. code:mg): the level table and filters, the level operators A_h,
restriction and interpolation, the top-level diagonal smoother, the pixel
block-ICC smoothers (same ridge), the bottom dense solve, one CR-Cycle, and
CR-Solve in FP64 and mixed precision against the exact answer x_true of
b = A x_true."""
import numpy as np
import pytest
import torch

from gpu_util import cuda_device, rel_l2
from oracle import geometry, multilevel, operators, sht
from paper_1308_5299_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return cuda_device()


@pytest.fixture(scope="module")
def case32(dev):
    """Nside 32 / lmax 95: three pixel levels (Nside_h 32, 16, 8) and a
    dense bottom, built by the oracle; the GPU plan takes the same level
    table and ridges.  At Nside_h 32 the tiles form a 4 x 4 grid per base
    face, so the inner four of every face have only interior neighbours; at
    Nside_h 16 and 8 every tile touches a face edge."""
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside32_lmax95")
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, bl, ninv, g)
    H = multilevel.Hierarchy(prob)
    levels = [dict(nside_h=l["nside_h"], lmax_h=l["lmax_h"], n_rec=l["n_rec"], fl=l["fl"]) for l in H.levels]
    plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                        levels=levels, lmax_dense=H.ld, ridge_alpha=[p.alpha for p in H.pix])
    return dict(cfg=cfg, cl=cl, bl=bl, ninv=ninv, prob=prob, H=H, plan=plan)


def rand_alm(L, seed, cl=None):
    a = synthetic.random_alm(L, seed=seed)
    if cl is not None:
        l, m = sht.lm_arrays(L)
        a[cl[l] <= 0] = 0.0
    return a


@pytest.mark.parametrize("nside,lmax", [(32, 95), (64, 191), (128, 383)])
def test_default_level_table(dev, nside, lmax):
    cl = synthetic.cl_spectrum(lmax, True)
    bl = synthetic.gaussian_beam(lmax, 60.0)
    ninv = torch.ones(12 * nside * nside, dtype=torch.float64, device=dev)
    plan = binding.Plan(lmax, nside=nside, cl=cl, bl=bl, ninv=ninv, levels="default", ridge_bisections=8)
    t = multilevel.level_table(nside, lmax)
    assert plan.nlevels() == len(t["levels"])
    for h, ref in enumerate(t["levels"], start=1):
        lv = plan.level(h)
        assert (lv["nside_h"], lv["lmax_h"], lv["n_rec"]) == (ref["nside_h"], ref["lmax_h"], ref["n_rec"])
        np.testing.assert_allclose(lv["fl"], ref["fl"], rtol=1e-12, atol=1e-300)
    bt = plan.level(plan.nlevels() + 1)
    assert bt["lmax_h"] == t["bottom"]["lmax_h"]


def test_level_operators(case32, dev):
    H, plan, prob = case32["H"], case32["plan"], case32["prob"]
    for h in range(0, len(H.levels) + 2):
        L = H.lmax_h(h)
        x = rand_alm(L, 10 + h, prob.cl)
        y = torch.empty(sht.n_lm(L), dtype=torch.complex128, device=dev)
        plan.level_apply(h, torch.from_numpy(x).to(dev), y)
        assert rel_l2(y.cpu().numpy(), H.apply_A(h, x)) < 1e-10, h


def test_gl_downgrade_level_operators(case32, dev):
    """Section 3.4: every pixel level's A_h applied through its
    Gauss-Legendre grid (2 lmax_h + 1 rings, band-limited quadrature-weighted
    inverse-noise map) equals the oracle's A_h on the observation grid."""
    c, H = case32, case32["H"]
    levels = [dict(nside_h=l["nside_h"], lmax_h=l["lmax_h"], n_rec=l["n_rec"], fl=l["fl"]) for l in H.levels]
    plan = binding.Plan(c["cfg"]["lmax"], nside=c["cfg"]["nside"], cl=c["cl"], bl=c["bl"],
                        ninv=torch.from_numpy(c["ninv"]).to(dev), levels=levels, lmax_dense=H.ld,
                        ridge_alpha=[p.alpha for p in H.pix], gl_downgrade=1)
    for h in range(1, len(H.levels) + 1):
        L = H.lmax_h(h)
        kind, nring, npix = plan.level_grid(h)
        assert kind == "gl" and nring == 2 * L + 1, (h, kind, nring)
        x = rand_alm(L, 70 + h, c["prob"].cl)
        ref = H.apply_A(h, x)
        y = torch.empty(sht.n_lm(L), dtype=torch.complex128, device=dev)
        plan.level_apply(h, torch.from_numpy(x).to(dev), y)
        assert rel_l2(y.cpu().numpy(), ref) < 1e-10, h
        y32 = torch.empty(sht.n_lm(L), dtype=torch.complex64, device=dev)
        plan.level_apply(h, torch.from_numpy(x).to(dev).to(torch.complex64), y32)
        assert rel_l2(y32.cpu().numpy().astype(np.complex128), ref) < 2e-5, h
    assert c["plan"].level_grid(1)[0] == "healpix"


def test_gl_downgrade_nside256_matches_obs_grid(dev):
    """At Nside 256 / lmax 767 the default rule moves the coarse levels to
    Gauss-Legendre grids; their A_h agree with the observation-grid A_h of a
    plan with the downgrade off."""
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside256_lmax767")
    kw = dict(nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev), levels="default",
              ridge_lambda_target=-1.0, ridge_bisections=6)
    pa = binding.Plan(cfg["lmax"], gl_downgrade=0, **kw)
    pb = binding.Plan(cfg["lmax"], gl_downgrade=-1, **kw)
    ngl = 0
    for h in range(1, pa.nlevels() + 1):
        L = pa.level(h)["lmax_h"]
        assert pb.level_grid(h)[0] == "healpix"
        if pa.level_grid(h)[0] != "gl":
            continue
        ngl += 1
        x = torch.from_numpy(rand_alm(L, 80 + h, cl)).to(dev)
        ya = torch.empty_like(x)
        yb = torch.empty_like(x)
        pa.level_apply(h, x, ya)
        pb.level_apply(h, x, yb)
        assert rel_l2(ya.cpu().numpy(), yb.cpu().numpy()) < 1e-11, h
    assert ngl >= 3


def test_restrict_prolong(case32, dev):
    H, plan, prob = case32["H"], case32["plan"], case32["prob"]
    for h in range(0, len(H.levels) + 1):
        Lh, LH = H.lmax_h(h), H.lmax_h(h + 1)
        r = rand_alm(Lh, 20 + h)
        out = torch.empty(sht.n_lm(LH), dtype=torch.complex128, device=dev)
        plan.restrict(h, torch.from_numpy(r).to(dev), out)
        assert rel_l2(out.cpu().numpy(), H.restrict(h, r)) < 1e-14
        c = rand_alm(LH, 30 + h)
        x0 = rand_alm(Lh, 40 + h)
        x = torch.from_numpy(x0.copy()).to(dev)
        plan.prolong_add(h, torch.from_numpy(c).to(dev), x)
        assert rel_l2(x.cpu().numpy(), x0 + H.prolong(h, c)) < 1e-14


def test_top_smoother(case32, dev):
    H, plan, prob = case32["H"], case32["plan"], case32["prob"]
    r = rand_alm(prob.lmax, 50, prob.cl)
    c = torch.empty(sht.n_lm(prob.lmax), dtype=torch.complex128, device=dev)
    plan.smooth(0, torch.from_numpy(r).to(dev), c)
    assert rel_l2(c.cpu().numpy(), H.smooth(0, r)) < 1e-10


def test_bottom_solve(case32, dev):
    H, plan, prob = case32["H"], case32["plan"], case32["prob"]
    b = rand_alm(H.ld, 60, prob.cl)
    x = torch.empty(sht.n_lm(H.ld), dtype=torch.complex128, device=dev)
    plan.bottom_solve(torch.from_numpy(b).to(dev), x)
    assert rel_l2(x.cpu().numpy(), H.bottom_solve(b)) < 1e-8


def test_bottom_matrix_ring_formula_nside256(dev):
    """The bottom level's explicit matrix (Eq. Ni-dense, l <= 40) at Nside 256,
    where polar seeds P~_mm fall below 2^-300 and the scaled recurrence has to
    renormalise, against the oracle's independent ring formula."""
    nside, lmax, ld = 256, 767, 40
    cl = synthetic.cl_spectrum(lmax, True)
    bl = synthetic.gaussian_beam(lmax, 20.0)
    ninv = synthetic.mask(nside, 15.0, 20, 120.0) / synthetic.noise_rms(nside, 2.0, 30.0) ** 2
    fl = multilevel.gauss_filter(lmax, 32)
    fl[190:] = 0.0
    plan = binding.Plan(lmax, nside=nside, cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                        levels=[dict(nside_h=32, lmax_h=189, n_rec=1, fl=fl)], lmax_dense=ld, ridge_bisections=4)
    A = plan.bottom_matrix()
    g = geometry.healpix_grid(nside)
    prob = operators.Problem(ld, cl[:ld + 1], bl[:ld + 1] * fl[:ld + 1], ninv, g)
    act = operators.real_active_mask(prob, ld)
    M = operators.ring_formula_inv_noise(prob, ld)[np.ix_(act, act)]
    lv = np.concatenate([np.arange(ld + 1)] + [np.repeat(np.arange(m, ld + 1), 2) for m in range(1, ld + 1)])[act]
    bv = (bl * fl)[lv]
    ref = bv[:, None] * M * bv[None, :] + np.diag(fl[lv] ** 2 / cl[lv])
    assert np.max(np.abs(A - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("h", [1, 2, 3])
def test_pixel_smoother(case32, dev, h):
    """Y_h^T M_h Y_h r with the same ridge: FP32 assembly (interpolated
    addition theorem) and FP32 ICC(0) against the FP64 oracle."""
    H, plan, prob = case32["H"], case32["plan"], case32["prob"]
    L = H.lmax_h(h)
    r = rand_alm(L, 70 + h, prob.cl)
    c = torch.empty(sht.n_lm(L), dtype=torch.complex128, device=dev)
    plan.smooth(h, torch.from_numpy(r).to(dev), c)
    assert rel_l2(c.cpu().numpy(), H.smooth(h, r)) < 2e-4
    assert abs(plan.level(h)["ridge"] - H.pix[h - 1].alpha) <= 1e-12 * abs(H.pix[h - 1].alpha) + 1e-300


def test_sweep_forms_identical(dev):
    """The ICC(0) triangular sweeps launched once per colour and as one
    cooperative data-flow launch (per-tile readiness flags) compute the same
    products in the same order: bit-identical smoother outputs on every
    pixel level of the Nside 256 hierarchy (Nside_h 128: 3072 tiles, down to
    Nside_h 16), and the cooperative form is what the automatic choice takes
    on the coarse levels."""
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside256_lmax767")
    kw = dict(nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev), levels="default")
    per_colour = binding.Plan(cfg["lmax"], smoother_sweep="per_colour", **kw)
    ridges = [per_colour.level(h)["ridge"] for h in range(1, per_colour.nlevels() + 1)]
    coop = binding.Plan(cfg["lmax"], smoother_sweep="cooperative", ridge_alpha=ridges, **kw)
    for h in range(1, per_colour.nlevels() + 1):
        L = per_colour.level(h)["lmax_h"]
        r = torch.from_numpy(rand_alm(L, 500 + h, cl)).to(dev)
        c1 = torch.empty(sht.n_lm(L), dtype=torch.complex128, device=dev)
        c2 = torch.empty_like(c1)
        for _ in range(3):  # repeated applications: the flags are reset every launch
            per_colour.smooth(h, r, c1)
            coop.smooth(h, r, c2)
            assert torch.equal(c1, c2), h


@pytest.mark.parametrize("h", [1, 2, 3])
def test_pixel_smoother_many_maps(case32, dev, h):
    """M_h applied to several maps at once (every factor block read once for
    all of them, the form of the batched cycles) against the oracle's
    incomplete-Cholesky solve of each map (same ridge; FP32 factor), and
    against the one-map sweeps map by map."""
    H, plan = case32["H"], case32["plan"]
    lev = H.pix[h - 1]
    npix = lev.grid["npix"]
    rng = np.random.default_rng(600 + h)
    maps = rng.normal(size=(5, npix))
    out = torch.empty((5, npix), dtype=torch.float32, device=dev)
    plan.pixel_smoother(h, torch.from_numpy(maps).to(torch.float32).to(dev), out)
    got = out.cpu().numpy().astype(np.float64)
    one = torch.empty(npix, dtype=torch.float32, device=dev)
    for j in range(5):
        assert rel_l2(got[j], lev.apply_M(maps[j])) < 2e-4, j
        plan.pixel_smoother(h, torch.from_numpy(maps[j]).to(torch.float32).to(dev), one)
        assert rel_l2(got[j], one.cpu().numpy().astype(np.float64)) < 1e-5, j


def _levels_of(H):
    return [dict(nside_h=l["nside_h"], lmax_h=l["lmax_h"], n_rec=l["n_rec"], fl=l["fl"]) for l in H.levels]


@pytest.mark.parametrize("h", [1, 2, 3])
def test_gpu_icc_bracket(case32, dev, h):
    """Section 3.5's ridge bracket on the GPU factorisation: with the
    oracle's smallest working ridge alpha* (the used ridge is 1.5 alpha*), the
    GPU's FP32 block ICC(0) of level h breaks down at 0.95 alpha* and
    succeeds at 1.5 alpha* (the fixture's plan)."""
    c = case32
    H = c["H"]
    alphas = [p.alpha for p in H.pix]
    assert alphas[h - 1] > 0
    below = list(alphas)
    below[h - 1] = 0.95 * alphas[h - 1] / 1.5
    with pytest.raises(binding.CRError) as e:
        binding.Plan(c["cfg"]["lmax"], nside=c["cfg"]["nside"], cl=c["cl"], bl=c["bl"],
                     ninv=torch.from_numpy(c["ninv"]).to(dev), levels=_levels_of(H), lmax_dense=H.ld,
                     ridge_alpha=below)
    assert e.value.code == binding.CR_EICC
    assert c["plan"].level(h)["ridge"] == pytest.approx(alphas[h - 1], rel=1e-12)


def test_gpu_ridge_search(case32, dev):
    """The GPU's own ridge search (FP32 factorisations, the same bisection)
    lands within 0.1 % of the oracle's FP64 ridge on every level (measured
    within 3e-5: FP32 rounding of the assembled blocks moves the breakdown
    point only slightly)."""
    c = case32
    plan = binding.Plan(c["cfg"]["lmax"], nside=c["cfg"]["nside"], cl=c["cl"], bl=c["bl"],
                        ninv=torch.from_numpy(c["ninv"]).to(dev), levels=_levels_of(c["H"]), lmax_dense=c["H"].ld,
                        ridge_lambda_target=-1.0)
    for h in range(1, len(c["H"].levels) + 1):
        a_gpu, a_ref = plan.level(h)["ridge"], c["H"].pix[h - 1].alpha
        print("ridge level %d: gpu/oracle = %.6f" % (h, a_gpu / a_ref))
        assert abs(a_gpu / a_ref - 1.0) < 1e-3, (h, a_gpu, a_ref)


def test_one_cycle(case32, dev):
    H, plan, prob = case32["H"], case32["plan"], case32["prob"]
    b = operators.apply_A(prob, synthetic.draw_prior(case32["cl"], index=5))
    x = torch.zeros(sht.n_lm(prob.lmax), dtype=torch.complex128, device=dev)
    plan.wcycle(x, torch.from_numpy(b).to(dev))
    ref = H.cycle(0, np.zeros_like(b), b)
    assert rel_l2(x.cpu().numpy(), ref) < 2e-4


@pytest.fixture(scope="module")
def plan32_default(case32, dev):
    """The library's own level table and ridges (search plus the
    lambda_max(S_h A_h) <= 1.5 bound) on the Nside 32 problem."""
    c = case32
    plan = binding.Plan(c["cfg"]["lmax"], nside=c["cfg"]["nside"], cl=c["cl"], bl=c["bl"],
                        ninv=torch.from_numpy(c["ninv"]).to(dev), levels="default")
    for h in range(0, plan.nlevels() + 1):
        lv = plan.level(h)
        assert lv["lambda_max"] <= 1.5 or (h == 0 and lv["ridge"] < 1.0)
    return plan


@pytest.mark.parametrize("mode", [binding.CR_F64, binding.CR_MIXED])
def test_solve_to_exact_answer(case32, plan32_default, dev, mode):
    """CR-Solve converges to x_true of b = A x_true (the exact answer)."""
    prob, plan, cl = case32["prob"], plan32_default, case32["cl"]
    x_true = prob.clean(synthetic.draw_prior(cl, index=6))
    b = operators.apply_A(prob, x_true)
    x = torch.empty_like(torch.from_numpy(b)).to(dev)
    cyc, rel, hist = plan.solve(torch.from_numpy(b).to(dev), x, eps=1e-18, max_cycles=120, mode=mode, check=False)[:3]
    xh = x.cpu().numpy()
    assert rel[0] < 1e-9, (rel, hist)
    g = prob.grid
    err_map = sht.synth(xh - x_true, prob.lmax, g)
    assert np.max(np.abs(err_map)) < 1e-3  # uK, max-pixel


@pytest.mark.parametrize("mode", [binding.CR_F64 | binding.CR_PCG, binding.CR_MIXED | binding.CR_PCG])
def test_solve_nside256(dev, mode):
    """The medium configuration (Nside 256, lmax 767, modulated noise,
    galactic cut plus 200 holes, C_0 = C_1 = 0): default levels, GPU ridge
    search, CR-Cycle-preconditioned flexible CG (Fig. code:mg caption) in
    FP64 and mixed precision to a 1e-10 relative residual; max-pixel error
    against x_true below 1e-3 uK.  (The top band of this configuration is
    not noise-dominated, so the stationary form converges slowly here.)"""
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside256_lmax767")
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, bl, ninv, g)
    x_true = prob.clean(synthetic.draw_prior(cl, index=7))
    b = operators.apply_A(prob, x_true)
    plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                        levels="default")
    tb = torch.from_numpy(b).to(dev)
    x = torch.empty_like(tb)
    cyc, rel, hist = plan.solve(tb, x, eps=1e-20, max_cycles=150, mode=mode, check=False)[:3]
    assert rel[0] < 1e-10, (mode, hist[0][:cyc[0]])
    m = torch.empty(g["npix"], dtype=torch.float64, device=dev)
    plan.sht_synth(x - torch.from_numpy(x_true).to(dev), m)
    assert float(m.abs().max()) < 1e-3, mode


def test_solve_planck_shaped_nside2048(dev):
    """The Planck-143-shaped workload at full size (Nside 2048, lmax 3000,
    7.3' beam, |b| < 10 deg cut plus 3000 holes of 5', C_0 = C_1 = C_2): the
    default level table of Table cycle-cost, the mixed-precision flexible-PCG
    CR-Solve, and the property that holds at any size -- the max-pixel error
    against x_true of b = A x_true falls below 1e-3 uK within 8 cycles and
    the relative residual history decreases."""
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside2048_lmax3000")
    plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                        levels="default")
    assert [plan.level(h)["nside_h"] for h in range(1, plan.nlevels() + 1)] == [1024, 512, 256, 128, 64, 32]
    x_true = torch.from_numpy(synthetic.draw_prior(cl, index=0)).to(dev)
    b = torch.empty_like(x_true)
    plan.apply_A(x_true, b)
    x = torch.empty_like(b)
    cyc, rel, hist = plan.solve(b, x, eps=1e-24, max_cycles=8, mode=binding.CR_MIXED | binding.CR_PCG,
                                check=False)[:3]
    h = hist[0][:cyc[0]]
    assert np.all(np.diff(h) < 0), h
    m = torch.empty(12 * cfg["nside"] ** 2, dtype=torch.float64, device=dev)
    plan.sht_synth(x - x_true, m)
    assert float(m.abs().max()) < 1e-3, h


@pytest.fixture(scope="module")
def plan32_schwarz(case32, dev):
    """The oracle's level table with the additive Schwarz (block Jacobi)
    smoother and fixed ridges: 1e-3 max|A_hat| per level."""
    c = case32
    H = c["H"]
    alphas = [1e-3 * float(np.max(np.abs(pl.Ahat))) for pl in H.pix]
    levels = [dict(nside_h=l["nside_h"], lmax_h=l["lmax_h"], n_rec=l["n_rec"], fl=l["fl"]) for l in H.levels]
    plan = binding.Plan(c["cfg"]["lmax"], nside=c["cfg"]["nside"], cl=c["cl"], bl=c["bl"],
                        ninv=torch.from_numpy(c["ninv"]).to(dev), levels=levels, lmax_dense=H.ld,
                        ridge_alpha=alphas, smoother="schwarz")
    return plan, alphas


@pytest.mark.parametrize("h", [1, 2])
def test_schwarz_smoother_matches_oracle(case32, plan32_schwarz, dev, h):
    """Y_h^T M Y_h r with M = blockdiag(A_hat_pp + alpha I)^-1 (tiles as
    subdomains): FP32 assembly and tile inverses against the FP64 oracle."""
    H, prob = case32["H"], case32["prob"]
    plan, alphas = plan32_schwarz
    L = H.lmax_h(h)
    r = rand_alm(L, 170 + h, prob.cl)
    c = torch.empty(sht.n_lm(L), dtype=torch.complex128, device=dev)
    plan.smooth(h, torch.from_numpy(r).to(dev), c)
    ref = H.pix[h - 1].smooth_schwarz(r, alphas[h - 1], prob)
    assert rel_l2(c.cpu().numpy(), ref) < 2e-4


def test_schwarz_solve_converges(case32, dev):
    """The library's own ridges (search plus the lambda_max <= 1.5 bound)
    with the Schwarz smoother: mixed-precision PCG reaches the exact
    answer."""
    c = case32
    plan = binding.Plan(c["cfg"]["lmax"], nside=c["cfg"]["nside"], cl=c["cl"], bl=c["bl"],
                        ninv=torch.from_numpy(c["ninv"]).to(dev), levels="default", smoother="schwarz")
    prob = c["prob"]
    x_true = prob.clean(synthetic.draw_prior(c["cl"], index=9))
    b = torch.from_numpy(operators.apply_A(prob, x_true)).to(dev)
    x = torch.zeros_like(b)
    cyc, rel, _ = plan.solve(b, x, eps=1e-20, max_cycles=80, mode=binding.CR_MIXED | binding.CR_PCG, check=False)[:3]
    assert rel[0] < 1e-9, (cyc, rel)
    assert rel_l2(x.cpu().numpy(), x_true) < 1e-6
    for h in range(1, plan.nlevels() + 1):
        assert plan.level(h)["lambda_max"] <= 1.5 + 1e-9
