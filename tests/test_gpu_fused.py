"""The one-launch sweep (wf_params.sweep_kernel, csrc/wf_fused.cu) against the
FP64 oracle and against the two-launch sweep, at 1024 x 1024 with all three
noise parts and the 5% disc mask (the benchmark map) and with per-row stripe
amplitudes.  The benchmark solve itself, corrections with their masked-pixel
source included, runs in this form by default and is checked against the
FP64 PCG solution in test_gpu_parity.py."""

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
    plan = make_plan(prob, sweep_kernel=2, **kw)
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


def test_one_launch_and_two_launch_runs_agree(wf):
    # a scheduled run with residual checkpoints between the launches: the
    # two forms differ only in the rounding order of the column transforms
    prob = synth.make_problem(1024, 1024, 1001, mask_frac=0.05)
    sched = wf.make_schedule("fixed", [30.0, 3.0, 1.0], [100, 100, 100])
    out = {}
    for form in (1, 2):
        plan = make_plan(prob, sweep_kernel=form, residual_every=50, max_iters=300)
        st = plan.run(sched, 0.0)
        assert st["iters"] == 300 and st["lam_final"] == 1.0, st
        out[form] = (field(plan, wf.WF_FIELD_S), field(plan, wf.WF_FIELD_D_RF), st)
        plan.close()
    assert rel(out[2][0], out[1][0]) < 1e-5
    assert rel(out[2][1], out[1][1]) < 1e-5
    assert abs(out[2][2]["rel_rho_u"] - out[1][2]["rel_rho_u"]) < 1e-3 * out[1][2]["rel_rho_u"]


def test_default_form_is_one_launch_where_supported(wf):
    prob = synth.make_problem(1024, 1024, 1002, mask_frac=0.05)
    plan = make_plan(prob)
    assert _time_form(plan) is True
    plan.close()
    small = synth.make_problem(256, 256, 1003, mask_frac=0.05)
    plan = make_plan(small)
    assert _time_form(plan) is False
    plan.close()
    with pytest.raises(wf.WFError) as e:
        wf.Plan(256, 256, wf.parts_of(small), wf.make_params(sweep_kernel=2))
    assert e.value.code == wf.WF_EUNSUPPORTED
    with pytest.raises(wf.WFError) as e:   # the plain sweep stores t_2DF: two launches only
        wf.Plan(1024, 1024, wf.parts_of(prob), wf.make_params(sweep_kernel=2, merge_2df=0, split_fp=0.3))
    assert e.value.code == wf.WF_EUNSUPPORTED


def test_one_launch_sweep_is_deterministic_and_times_faster(wf):
    prob = synth.make_problem(1024, 1024, 1004, mask_frac=0.05)
    res = []
    for _ in range(2):
        plan = make_plan(prob, sweep_kernel=2)
        plan.iterate(10.0, 40)
        res.append(field(plan, wf.WF_FIELD_S))
        plan.close()
    assert np.array_equal(res[0], res[1])
    t = {}
    for form in (1, 2):
        plan = make_plan(prob, sweep_kernel=form)
        t[form] = plan.time_sweeps(1.0, 200)[0]
        plan.close()
    print(f"1024^2 sweep: two launches {t[1]:.2f} us, one launch {t[2]:.2f} us")
    assert t[2] < t[1]
