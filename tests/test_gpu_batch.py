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


# ---------------------------------------------------------------- persistent mode (lanes = 0)

def _batch_solve(wf, probs, lanes, sched, tol, **params):
    import torch
    shapes = [p.shape for p in probs]
    b = wf.Batch(shapes, params=wf.make_params(**params), lanes=lanes)
    inputs = [tuple(dev(a) for a in (p.d, p.pixel_var, p.mask, p.C, p.P1f, p.Pst, p.stripe_amp2)) for p in probs]
    outs = [torch.empty(*sh, device="cuda") for sh in shapes]
    rc, stats = b.solve(inputs, sched, tol, outs)
    b.close()
    return rc, stats, [o.cpu().numpy().astype(np.float64) for o in outs]


@pytest.mark.parametrize("shape_choice", [0, 2])
def test_persistent_batch_matches_the_oracle_sweep_for_sweep(wf, shape_choice):
    # every size the persistent kernel takes, one map each (two of 256), a
    # fixed schedule run to its cap: each map's s against the FP64 oracle's
    # messenger iteration with the same schedule, for both compiled shapes
    import os
    O.set_workers(os.cpu_count() or 1)
    sizes = [256, 384, 256, 512, 768, 1024, 1536, 2048]
    probs = [synth.make_problem(n, n, 4100 + i, amp_jitter=0.5, stripe_rows_vary=(i % 2 == 1))
             for i, n in enumerate(sizes)]
    lam, its = [30.0, 3.0, 1.0], [20, 20, 20]
    sched = wf.make_schedule("fixed", lam, its)
    rc, stats, outs = _batch_solve(wf, probs, 0, sched, 0.0, residual_every=10, max_iters=60,
                                   autotune=shape_choice)
    assert rc == wf.WF_OK  # tol = 0: every map runs to max_iters, no stop test
    for p, st, s in zip(probs, stats, outs):
        assert st["iters"] == 60 and st["lam_final"] == 1.0, st
        r = O.messenger_solve(p, schedule=O.fixed_schedule(lam, its), n_iters=60, residual_every=10,
                              merge_2df=True, split_f=0.5, split_fp=0.5)
        err = rel(s, r["s"])
        assert err < 1e-4, (p.shape, err)
        # the residual each map's stop test reads
        assert abs(st["rel_rho_u"] - r["rel_u"]) < 2e-3 * r["rel_u"], (p.shape, st, r["rel_u"])


@pytest.mark.parametrize("refine,accel", [(2, 0), (4, 3)])
def test_persistent_batch_refined_solves_agree_with_single_map_solves(wf, refine, accel):
    # the whole solve (first run, corrections with their masked-pixel source,
    # plain or Anderson-combined, the refined s) for each map of a mixed
    # batch, against the same solve of each map alone (lanes = 1, the per-map
    # kernels)
    sizes = [512, 256, 1024, 384, 256]
    probs = [synth.make_problem(n, n, 4200 + i, amp_jitter=0.5) for i, n in enumerate(sizes)]
    sched = wf.make_schedule("fixed", [30.0, 3.0], [200, 200])
    kw = dict(residual_every=20, max_iters=400, refine=refine, refine_max_iters=300, refine_lam1_iters=100,
              refine_tol_scale=1.0, autotune=0, refine_accel=accel)
    rc, stats, outs = _batch_solve(wf, probs, 0, sched, 0.0, **kw)
    _, stats1, outs1 = _batch_solve(wf, probs, 1, sched, 0.0, **kw)
    for p, a, b, sa, sb in zip(probs, outs, outs1, stats, stats1):
        assert sa["iters"] == sb["iters"] == 400 + 300 * refine, (p.shape, sa, sb)
        assert rel(a, b) < 1e-5, (p.shape, rel(a, b))


def test_persistent_batch_maps_stop_on_their_own_test(wf):
    # per-map done flags: each map leaves the shared launches at the first
    # checkpoint where its own stop test passes, as it does alone
    sizes = [256, 512, 256, 384]
    probs = [synth.make_problem(n, n, 4300 + i, amp_jitter=0.5, k_knee=4.0, k_knee_x=4.0)
             for i, n in enumerate(sizes)]
    sched = wf.make_schedule("fixed", O.cooling_levels(1e2, 5), [40] * 5)
    kw = dict(residual_every=10, max_iters=20000, tol_u_scale=5.0, autotune=0)
    rc, stats, outs = _batch_solve(wf, probs, 0, sched, 2e-4, **kw)
    _, stats1, outs1 = _batch_solve(wf, probs, 1, sched, 2e-4, **kw)
    assert rc == wf.WF_OK, stats
    for p, a, b, sa, sb in zip(probs, outs, outs1, stats, stats1):
        assert sa["status"] == 0 and abs(sa["iters"] - sb["iters"]) <= 10, (p.shape, sa, sb)
        assert rel(a, b) < 1e-4, (p.shape, rel(a, b))
    assert len({s["iters"] for s in stats}) > 1, stats


def test_persistent_batch_rejects_what_its_kernel_does_not_take(wf):
    with pytest.raises(wf.WFError) as e:
        wf.Batch([(256, 256), (256, 512)], lanes=0)
    assert e.value.code == wf.WF_EUNSUPPORTED
    with pytest.raises(wf.WFError) as e:
        wf.Batch([(128, 128)], lanes=0)
    assert e.value.code == wf.WF_EUNSUPPORTED
    with pytest.raises(wf.WFError) as e:
        wf.Batch([(256, 256)], params=wf.make_params(merge_2df=0, split_fp=0.3), lanes=0)
    assert e.value.code == wf.WF_EUNSUPPORTED
