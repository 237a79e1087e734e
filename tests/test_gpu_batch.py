"""Batched solves (wf_batch_create / wf_batch_solve): many maps of uneven
sizes on concurrent lanes give, map by map, exactly what wf_solve gives for
each map alone, and therefore inherit its parity with the oracle."""

import numpy as np
import pytest

import oracle as O
from gpu_util import dev, rel
from paper_1704_00865_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPES = [(64, 128), (256, 256), (128, 32), (32, 512), (128, 128), (64, 64), (512, 256), (32, 32)]


@pytest.fixture(scope="module")
def wf():
    from paper_1704_00865_gb300 import build, wf
    build.build()
    wf.load()
    return wf


def _problems():
    return [synth.make_problem(ny, nx, 500 + i, mask_frac=0.05, k_knee=4.0, k_knee_x=4.0,
                               stripe_rows_vary=(i % 2 == 1), amp_jitter=0.5)
            for i, (ny, nx) in enumerate(SHAPES)]


def _arrays(prob, on_device):
    f = dev if on_device else (lambda a: a)
    return (f(prob.d), f(prob.pixel_var), f(prob.mask), f(prob.C), f(prob.P1f), f(prob.Pst), f(prob.stripe_amp2))


@pytest.mark.parametrize("lanes", [1, 3, 8])
def test_batch_equals_single_solves_bit_for_bit(wf, lanes):
    import torch
    probs = _problems()
    params = dict(refine=1, refine_max_iters=200, refine_lam1_iters=50, residual_every=10, max_iters=400,
                  tol_u_scale=20.0)
    sched = wf.make_schedule("fixed", [30.0, 3.0], [60, 60])
    b = wf.Batch(SHAPES, params=wf.make_params(**params), lanes=lanes)
    outs = [torch.empty(ny, nx, device="cuda") for ny, nx in SHAPES]
    # device inputs for even maps, host inputs for odd ones
    rc, stats = b.solve([_arrays(p, i % 2 == 0) for i, p in enumerate(probs)], sched, 1e-5, outs)
    assert b.launch_count() > 0
    b.close()
    for i, (p, (ny, nx)) in enumerate(zip(probs, SHAPES)):
        plan = wf.Plan(ny, nx, wf.parts_of(p), wf.make_params(**params))
        ref = torch.empty(ny, nx, device="cuda")
        _, st = plan.solve(*_arrays(p, True), sched, 1e-5, out=ref)
        plan.close()
        assert stats[i]["iters"] == st["iters"], (i, stats[i], st)
        assert torch.equal(outs[i], ref), i


def test_batch_maps_reach_the_dense_solution(wf):
    import torch
    shapes = [(32, 32), (32, 64), (64, 32)]
    probs = [synth.make_problem(ny, nx, 700 + i, mask_frac=0.06, k_knee=4.0, k_knee_x=4.0)
             for i, (ny, nx) in enumerate(shapes)]
    sched = wf.make_schedule("fixed", O.cooling_levels(1e2, 5), [20] * 5)
    b = wf.Batch(shapes, params=wf.make_params(refine=1, residual_every=10, max_iters=100000, tol_u_scale=20.0),
                 lanes=3)
    outs = [np.empty((ny, nx), np.float32) for ny, nx in shapes]   # host outputs
    rc, stats = b.solve([_arrays(p, True) for p in probs], sched, 1e-5, outs)
    b.close()
    assert rc == wf.WF_OK, stats
    for p, o in zip(probs, outs):
        assert rel(o.astype(np.float64), O.dense_wf(p)) < 1e-4


def test_batch_reports_the_first_error(wf):
    import torch
    shapes = [(64, 64), (32, 32)]
    probs = [synth.make_problem(ny, nx, 900 + i, mask_frac=0.05) for i, (ny, nx) in enumerate(shapes)]
    bad = list(_arrays(probs[1], True))
    Cb = bad[3].clone()
    Cb[0, 0] = -1.0                       # a signal eigenvalue <= 0
    bad[3] = Cb
    b = wf.Batch(shapes, lanes=2)
    outs = [torch.empty(ny, nx, device="cuda") for ny, nx in shapes]
    with pytest.raises(wf.WFError) as e:
        b.solve([_arrays(probs[0], True), tuple(bad)], wf.make_schedule("fixed", [10.0], [10]), 1e-5, outs)
    assert e.value.code == wf.WF_ENOTPD
    b.close()
