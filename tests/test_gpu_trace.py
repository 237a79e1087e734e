"""The per-checkpoint trace (wf_params.trace, wf_get_trace): lambda, the two
residual terms and chi^2_aug at every checkpoint of every run of a solve, the
quantities Fig. 3 of the paper follows along the cooling."""

import math

import numpy as np
import pytest

from gpu_util import dev, make_plan
from paper_1704_00865_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    from paper_1704_00865_gb300 import build, wf
    build.build()
    wf.load()
    return wf


def test_trace_records_every_checkpoint(wf):
    prob = synth.make_problem(64, 128, 71, mask_frac=0.05)
    plan = make_plan(prob, residual_every=10, max_iters=60, trace=2)
    st = plan.run(wf.make_schedule("fixed", [30.0, 3.0, 1.0], [20, 20, 20]), 0.0)
    tr = plan.trace()
    assert [r["sweeps"] for r in tr] == [10, 20, 30, 40, 50, 60]
    assert [r["lam"] for r in tr] == [30.0, 30.0, 3.0, 3.0, 1.0, 1.0]
    assert all(r["run"] == 0 for r in tr)
    # the last record is the state the plan holds: its residual and chi^2_aug
    u, m = plan.residual()
    assert tr[-1]["rel_rho_u"] == pytest.approx(u, rel=1e-12) and tr[-1]["rel_rho_m"] == pytest.approx(m, rel=1e-12)
    assert tr[-1]["rel_rho_u"] == pytest.approx(st["rel_rho_u"], rel=1e-12)
    assert tr[-1]["chi2_aug"] == pytest.approx(plan.chi2_aug(), rel=1e-12)
    # Appendix A: at fixed lambda no sweep raises the augmented objective
    for a, b in zip(tr, tr[1:]):
        if a["lam"] == b["lam"]:
            assert b["chi2_aug"] <= a["chi2_aug"] * (1 + 1e-6), (a, b)
    # the residual falls along the cooling
    assert tr[-1]["rel_rho_u"] < tr[0]["rel_rho_u"]
    plan.close()


def test_trace_of_a_refined_solve_and_without_chi2(wf):
    import torch
    prob = synth.make_problem(64, 64, 72, mask_frac=0.05)
    plan = wf.Plan(64, 64, wf.parts_of(prob), wf.make_params(residual_every=10, max_iters=40, refine=2,
                                                             refine_max_iters=30, trace=1))
    out = torch.empty(64, 64, device="cuda")
    _, st = plan.solve(*[dev(a) for a in (prob.d, prob.pixel_var, prob.mask, prob.C, prob.P1f, prob.Pst,
                                          prob.stripe_amp2)], wf.make_schedule("fixed", [10.0], [20]), 0.0, out=out)
    tr = plan.trace()
    assert [r["run"] for r in tr] == [0] * 4 + [1] * 3 + [2] * 3
    assert sum(1 for r in tr if r["run"] > 0) * 10 == st["iters"] - 40
    assert all(math.isnan(r["chi2_aug"]) for r in tr)
    assert all(np.isfinite(r["rel_rho_u"]) for r in tr)
    plan.close()


def test_trace_needs_the_flag_and_chi2_the_merged_block(wf):
    prob = synth.make_problem(64, 64, 73, mask_frac=0.05)
    plan = make_plan(prob)
    with pytest.raises(wf.WFError) as e:
        plan.trace()
    assert e.value.code == wf.WF_EINVAL
    plan.close()
    with pytest.raises(wf.WFError) as e:
        wf.Plan(64, 64, wf.parts_of(prob), wf.make_params(trace=2, merge_2df=0, split_fp=0.3))
    assert e.value.code == wf.WF_EUNSUPPORTED
