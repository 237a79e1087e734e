"""The one-launch sweep (wf_params.sweep_kernel, csrc/wf_fused.cu) against the
FP64 oracle and against the two-launch sweep, at 1024 x 1024 with all three
noise parts and the 5% disc mask (the benchmark map) and with per-row stripe
amplitudes; a refined solve (corrections with their masked-pixel source) in
this form against the same solve in two launches.  The one-launch form is
opt-in: on a GB300 it measured slower than the two launches at 1024^2."""

import numpy as np
import pytest

import oracle as O
from gpu_util import dev, field, make_plan, oracle_fields, rel
from paper_1704_00865_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    from paper_1704_00865_gb300 import build, wf
    build.build()
    wf.load()
    return wf


def _time_form(plan):
    us, one = plan.time_sweeps(1.0, 4)
    return one


@pytest.mark.parametrize("rows_vary", [False, True])
def test_one_launch_sweeps_match_the_oracle_field_by_field(wf, rows_vary):
    prob = synth.make_problem(1024, 1024, 1000, mask_frac=0.05, stripe_rows_vary=rows_vary)
    kw = dict(merge_2df=1, split_f=0.5, split_fp=0.5)
    plan = make_plan(prob, sweep_kernel=1, **kw)
    ch = O.Chain(O.build_parts(prob, merge_2df=True, split_f=0.5, split_fp=0.5))
    # one launch of three sweeps at each level (the grid barriers between
    # and within sweeps), then one more launch
    for lam, n in ((40.0, 3), (4.0, 3), (1.0, 1)):
        plan.iterate(lam, n)
        for _ in range(n):
            ch.sweep(lam)
        for fid, ref in oracle_fields(ch).items():
            got = field(plan, fid)
            assert rel(got, ref) < 2e-5, (lam, fid, rel(got, ref))
    plan.close()


def test_one_launch_refined_solve_agrees_with_two_launches(wf):
    # corrections run the one-launch sweep with the masked-pixel source
    import torch
    prob = synth.cfg1_problem(1000, 1024)
    sched = wf.make_schedule("fixed", [30.0], [300])
    out = {}
    for form in (0, 1):
        plan = wf.Plan(1024, 1024, wf.parts_of(prob), wf.make_params(
            sweep_kernel=form, residual_every=50, max_iters=300, refine=2, refine_max_iters=300,
            refine_lam1_iters=100, refine_tol_scale=1.0))
        o = torch.empty(1024, 1024, device="cuda")
        _, st = plan.solve(*[dev(a) for a in (prob.d, prob.pixel_var, prob.mask, prob.C, prob.P1f, prob.Pst,
                                              prob.stripe_amp2)], sched, 0.0, out=o)
        out[form] = (o.cpu().numpy().astype(np.float64), st)
        plan.close()
    assert out[0][1]["iters"] == out[1][1]["iters"] == 900
    assert rel(out[1][0], out[0][0]) < 1e-5


def test_one_launch_and_two_launch_runs_agree(wf):
    # a scheduled run with residual checkpoints between the launches: the
    # two forms differ only in the rounding order of the column transforms
    prob = synth.make_problem(1024, 1024, 1001, mask_frac=0.05)
    sched = wf.make_schedule("fixed", [30.0, 3.0, 1.0], [100, 100, 100])
    out = {}
    for form in (0, 1):
        plan = make_plan(prob, sweep_kernel=form, residual_every=50, max_iters=300)
        st = plan.run(sched, 0.0)
        assert st["iters"] == 300 and st["lam_final"] == 1.0, st
        out[form] = (field(plan, wf.WF_FIELD_S), field(plan, wf.WF_FIELD_D_RF), st)
        plan.close()
    assert rel(out[1][0], out[0][0]) < 1e-5
    assert rel(out[1][1], out[0][1]) < 1e-5
    assert abs(out[1][2]["rel_rho_u"] - out[0][2]["rel_rho_u"]) < 1e-3 * out[0][2]["rel_rho_u"]


def test_forms_and_where_the_one_launch_form_is_refused(wf):
    prob = synth.make_problem(1024, 1024, 1002, mask_frac=0.05)
    for form, one in ((0, False), (1, True)):
        plan = make_plan(prob, sweep_kernel=form)
        assert _time_form(plan) is one
        plan.close()
    small = synth.make_problem(256, 256, 1003, mask_frac=0.05)
    with pytest.raises(wf.WFError) as e:
        wf.Plan(256, 256, wf.parts_of(small), wf.make_params(sweep_kernel=1))
    assert e.value.code == wf.WF_EUNSUPPORTED
    with pytest.raises(wf.WFError) as e:   # the plain sweep stores t_2DF: two launches only
        wf.Plan(1024, 1024, wf.parts_of(prob), wf.make_params(sweep_kernel=1, merge_2df=0, split_fp=0.3))
    assert e.value.code == wf.WF_EUNSUPPORTED


def test_one_launch_sweep_is_deterministic_and_timed(wf):
    prob = synth.make_problem(1024, 1024, 1004, mask_frac=0.05)
    res = []
    for _ in range(2):
        plan = make_plan(prob, sweep_kernel=1)
        plan.iterate(10.0, 40)
        res.append(field(plan, wf.WF_FIELD_S))
        plan.close()
    assert np.array_equal(res[0], res[1])
    t = {}
    for form in (0, 1):
        plan = make_plan(prob, sweep_kernel=form)
        t[form] = plan.time_sweeps(1.0, 200)[0]
        plan.close()
    print(f"1024^2 sweep: two launches {t[0]:.2f} us, one launch {t[1]:.2f} us")
    assert 0 < t[1] < 2 * t[0]
