"""The split precompute of Section 5: the C_l-dependent part redone alone
(cr_plan_update_cl) and the precompute checkpoint (cr_save / cr_load).

An updated plan must equal a plan created with the new C_l from the start
(same smoothers, ridges, top and bottom levels: the solve is bit-identical),
and a plan loaded from a checkpoint must equal the plan that was saved."""
import os

import numpy as np
import pytest
import torch

from gpu_util import cuda_device, rel_l2
from oracle import geometry, operators, sht
from paper_1308_5299_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu

NAME = "nside32_lmax95"


@pytest.fixture(scope="module")
def inputs():
    dev = cuda_device()
    cfg, cl, bl, ninv = synthetic.problem_inputs(NAME)
    return dict(dev=dev, cfg=cfg, cl=cl, bl=bl, ninv=ninv, ninv_t=torch.from_numpy(ninv).to(dev))


def make(inp, cl, **kw):
    cfg = inp["cfg"]
    return binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=inp["bl"], ninv=inp["ninv_t"],
                        levels="default", **kw)


def solve(plan, inp, cl, mode=binding.CR_MIXED | binding.CR_PCG):
    cfg = inp["cfg"]
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, inp["bl"], inp["ninv"], g)
    xt = prob.clean(synthetic.draw_prior(cl, index=3))
    b = torch.from_numpy(operators.apply_A(prob, xt)).to(inp["dev"])
    x = torch.zeros_like(b)
    plan.solve(b, x, eps=1e-20, max_cycles=30, mode=mode, check=False)
    return x, xt


def level_state(plan):
    return [(lv["nside_h"], lv["lmax_h"], lv["ridge"]) for lv in (plan.level(h) for h in range(1, plan.nlevels() + 1))]


@pytest.mark.parametrize("change", ["scale", "active_set"])
def test_update_cl_equals_fresh_plan(inputs, change):
    cl = inputs["cl"]
    if change == "scale":
        # same active set: the inverse-noise terms of the smoothers are kept
        cl0 = cl * np.linspace(0.5, 2.0, cl.size)
    else:
        # C_0 = C_1 = 0 -> C_0 = C_1 = C_2: the active set changes
        cl0 = cl.copy()
        cl0[:2] = 0.0
        cl = cl.copy()
        cl[:2] = cl[2]
    upd = make(inputs, cl0)
    upd.update_cl(cl)
    fresh = make(inputs, cl)
    assert level_state(upd) == level_state(fresh)
    x1, xt = solve(upd, inputs, cl)
    x2, _ = solve(fresh, inputs, cl)
    assert torch.equal(x1, x2)
    assert rel_l2(x1.cpu().numpy(), xt) < 1e-6
    # the operator itself follows the new prior
    cfg = inputs["cfg"]
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, inputs["bl"], inputs["ninv"], g)
    v = prob.clean(synthetic.random_alm(cfg["lmax"], seed=77))
    y = torch.empty(sht.n_lm(cfg["lmax"]), dtype=torch.complex128, device=inputs["dev"])
    upd.apply_A(torch.from_numpy(v).to(inputs["dev"]), y)
    assert rel_l2(y.cpu().numpy(), operators.apply_A(prob, v)) < 1e-10


def test_update_cl_rejects_bad_prior_and_keeps_plan(inputs):
    cl = inputs["cl"]
    plan = make(inputs, cl)
    x1, _ = solve(plan, inputs, cl)
    bad = cl.copy()
    bad[5] = -1.0
    with pytest.raises(binding.CRError) as e:
        plan.update_cl(bad)
    assert e.value.code == binding.CR_EINVAL
    x2, _ = solve(plan, inputs, cl)
    assert torch.equal(x1, x2)


def test_checkpoint_round_trip(inputs, tmp_path):
    cl = inputs["cl"]
    full = make(inputs, cl)
    path = str(tmp_path / "pre.crck")
    full.save(path)
    assert os.path.getsize(path) > 0
    lazy = make(inputs, cl, defer_precompute=True)
    b = torch.zeros(sht.n_lm(inputs["cfg"]["lmax"]), dtype=torch.complex128, device=inputs["dev"])
    with pytest.raises(binding.CRError) as e:
        lazy.solve(b, torch.zeros_like(b), eps=1e-20, max_cycles=2)
    assert e.value.code == binding.CR_ESTATE
    lazy.load(path)
    assert level_state(lazy) == level_state(full)
    x1, _ = solve(full, inputs, cl)
    x2, _ = solve(lazy, inputs, cl)
    assert torch.equal(x1, x2)
    # a deferred plan can also be completed by an update
    lazy2 = make(inputs, cl, defer_precompute=True)
    lazy2.update_cl(cl)
    x3, _ = solve(lazy2, inputs, cl)
    assert torch.equal(x1, x3)


def test_checkpoint_rejects_other_inputs_and_damaged_files(inputs, tmp_path):
    cl = inputs["cl"]
    full = make(inputs, cl)
    path = str(tmp_path / "pre.crck")
    full.save(path)
    other = make(inputs, cl * 1.5, defer_precompute=True)
    with pytest.raises(binding.CRError) as e:
        other.load(path)
    assert e.value.code == binding.CR_EINVAL
    raw = open(path, "rb").read()
    cut = str(tmp_path / "cut.crck")
    open(cut, "wb").write(raw[: len(raw) // 2])
    flip = str(tmp_path / "flip.crck")
    damaged = bytearray(raw)
    damaged[len(raw) // 2] ^= 0x40
    open(flip, "wb").write(bytes(damaged))
    other_smoother = make(inputs, cl, defer_precompute=True, smoother="schwarz")
    with pytest.raises(binding.CRError) as e:
        other_smoother.load(path)
    assert e.value.code == binding.CR_EINVAL
    lazy = make(inputs, cl, defer_precompute=True)
    for bad in (cut, flip, str(tmp_path / "missing.crck")):
        with pytest.raises(binding.CRError) as e:
            lazy.load(bad)
        assert e.value.code == binding.CR_EIO
    lazy.load(path)
    x1, _ = solve(full, inputs, cl)
    x2, _ = solve(lazy, inputs, cl)
    assert torch.equal(x1, x2)
