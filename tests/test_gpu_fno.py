"""The warm-start network on the GPU (wf_fno_*) against the FP64 oracle:
forward pass, gradients against the oracle's finite differences, the input
features, training, and the warm-started solve (wf_solve_warm)."""

import numpy as np
import pytest

import oracle as O
from oracle import fno_oracle as F
from gpu_util import dev, rel
from paper_1704_00865_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    from paper_1704_00865_gb300 import build, wf
    build.build()
    wf.load()
    return wf


def _net(wf, n, batch, width, mx, my, layers, seed=11):
    theta = synth.fno_init(seed, width, mx, my, layers)
    net = wf.FNO(n, batch, theta, width=width, mx=mx, my=my, layers=layers)
    p = F.unflatten(net.params(rounded=True).astype(np.float64), F.template(width, mx, my, layers))
    return net, p


@pytest.mark.parametrize("n,width,mx,my,layers", [(32, 8, 4, 4, 2), (64, 32, 16, 16, 4), (16, 6, 3, 5, 3)])
def test_forward_matches_the_oracle(wf, n, width, mx, my, layers):
    import torch
    net, p = _net(wf, n, 2, width, mx, my, layers)
    x = np.random.default_rng(n).standard_normal((2, 2, n, n)).astype(np.float32)
    y = torch.empty(2, n, n, device="cuda")
    net.forward(dev(x), y, 2)
    net.close()
    assert rel(y.cpu().numpy(), F.forward(p, x.astype(np.float64))) < 2e-5


def test_gradient_matches_oracle_finite_differences(wf):
    n, width, mx, my, layers = 16, 4, 3, 2, 2
    net, p = _net(wf, n, 2, width, mx, my, layers, seed=3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 2, n, n)).astype(np.float32)
    t = rng.standard_normal((2, n, n)).astype(np.float32)
    loss, g = net.gradient(dev(x), dev(t), 2)
    net.close()
    assert loss == pytest.approx(F.loss(p, x.astype(np.float64), t.astype(np.float64)), rel=1e-5)
    # every block of parameters: P, p, W_0, w_0, R_0, ..., Q, q
    tot = g.size
    lay = [("P", width * 2), ("p", width)]
    for l in range(layers):
        lay += [(f"W{l}", width * width), (f"w{l}", width), (f"R{l}", width * width * 2 * my * mx * 2)]
    lay += [("Q", width), ("q", 1)]
    assert sum(s for _, s in lay) == tot
    o = 0
    for name, size in lay:
        idx = list(range(o, o + size, max(1, size // 12)))
        fd = F.fd_gradient(p, x.astype(np.float64), t.astype(np.float64), idx)
        err = np.linalg.norm(g[idx] - fd) / max(np.linalg.norm(fd), 1e-30)
        assert err < 2e-3, (name, err)
        o += size


def test_features_match_the_oracle(wf):
    import torch
    prob = synth.make_problem(64, 128, 9, mask_frac=0.08)
    x = torch.empty(2, 64, 128, device="cuda")
    sg = torch.empty(1, device="cuda")
    wf.fno_features(dev(prob.d), dev(prob.pixel_var), dev(prob.mask), x, sg)
    xr, sr = F.features(prob.d, prob.pixel_var, prob.mask)
    assert sg.item() == pytest.approx(sr, rel=1e-6)
    assert rel(x.cpu().numpy(), xr) < 1e-6


def test_training_lowers_the_loss(wf):
    import torch
    n, width, mx, my, layers, B = 32, 8, 4, 4, 2, 4
    net, _ = _net(wf, n, B, width, mx, my, layers, seed=5)
    rng = np.random.default_rng(6)
    x = dev(rng.standard_normal((B, 2, n, n)).astype(np.float32))
    # a target the network can represent: a smoothed copy of the data channel
    t = torch.from_numpy(np.fft.irfft2(np.fft.rfft2(x[:, 0].cpu().numpy()) *
                                       (np.abs(np.fft.fftfreq(n))[:, None] < 0.1) *
                                       (np.fft.rfftfreq(n)[None, :] < 0.1), s=(n, n)).astype(np.float32)).cuda()
    l0 = net.gradient(x, t, B)[0]
    for _ in range(300):
        l = net.train_step(x, t, B, 3e-3)
    net.close()
    assert l < 0.2 * l0, (l0, l)


def test_warm_start_from_the_solution_needs_few_sweeps(wf):
    import torch
    prob = synth.make_problem(128, 128, 13, mask_frac=0.05, k_knee=4.0, k_knee_x=4.0)
    sched = wf.make_schedule("fixed", O.cooling_levels(1e2, 5), [40] * 5)
    params = wf.make_params(residual_every=10, max_iters=100000, tol_u_scale=20.0, refine=1,
                            refine_max_iters=2000, refine_lam1_iters=500, stall_checks=20)
    plan = wf.Plan(128, 128, wf.parts_of(prob), params)
    inp = [dev(a) for a in (prob.d, prob.pixel_var, prob.mask, prob.C, prob.P1f, prob.Pst, prob.stripe_amp2)]
    cold = torch.empty(128, 128, device="cuda")
    _, st_c = plan.solve(*inp, sched, 1e-5, out=cold)
    warm = torch.empty(128, 128, device="cuda")
    lam1 = wf.make_schedule("fixed", [1.0], [0])
    _, st_w = plan.solve_warm(*inp, cold, lam1, 1e-5, out=warm)
    plan.close()
    ref = O.dense_wf(prob) if prob.d.size <= 4096 else O.pcg_wf(prob, tol=1e-10)
    assert st_c["status"] == 0 and st_w["status"] == 0, (st_c, st_w)
    assert rel(warm.cpu().numpy(), ref) < 1e-4 and rel(cold.cpu().numpy(), ref) < 1e-4
    # the first solve of the warm start starts at the answer: it stops at its
    # first checkpoints (the correction solve runs its fixed budget either way)
    assert st_w["iters"] < st_c["iters"] - 1000, (st_c["iters"], st_w["iters"])


def test_trained_network_gains_over_the_cold_start(wf):
    # train on maps the batched solver solves, then solve held-out maps cold
    # (the benchmark's schedule) and from the network's prediction (the same
    # levels at half length): both reach the FP64 solution, the warm start in
    # fewer sweeps; a zero start with the warm schedule is the control
    import os
    import torch
    import bench
    O.set_workers(os.cpu_count() or 1)
    n, ntr, nte, B = 256, 128, 4, 8
    probs = [synth.make_problem(n, n, 8000 + i, amp_jitter=0.5) for i in range(ntr + nte)]
    inp = [tuple(dev(a) for a in (p.d, p.pixel_var, p.mask, p.C, p.P1f, p.Pst, p.stripe_amp2)) for p in probs]
    # the solve form where the prediction pays: one long first solve and one
    # correction (with the headline's short first solve and four corrections
    # a zero start needs no more sweeps for the same accuracy)
    params = bench.solver_params(wf, **bench.LONG_FIRST_SOLVE)
    sched = bench.solver_schedule(wf)
    wsched = bench.warm_schedule(wf)
    sol = [torch.empty(n, n, device="cuda") for _ in range(ntr)]
    b = wf.Batch([(n, n)] * ntr, params=bench.solver_params(wf), lanes=16)
    b.solve(inp[:ntr], sched, bench.TOL, sol)
    b.close()
    X = torch.empty(len(probs), 2, n, n, device="cuda")
    SG = torch.empty(len(probs), device="cuda")
    for i in range(len(probs)):
        wf.fno_features(inp[i][0], inp[i][1], inp[i][2], X[i], SG[i:i + 1])
    T = torch.stack(sol) / SG[:ntr, None, None]
    net = wf.FNO(n, B, synth.fno_init(2, **bench.WARM_FNO), **bench.WARM_FNO)
    rng = np.random.default_rng(1)
    for it in range(600):
        idx = torch.from_numpy(rng.choice(ntr, B, replace=False)).cuda()
        net.train_step(X[idx].contiguous(), T[idx].contiguous(), B, 2e-3 * 0.5 ** (it // 150))
    y = torch.empty(B, n, n, device="cuda")
    cold_it, warm_it, ctrl_it, errs = [], [], [], []
    for j in range(nte):
        i = ntr + j
        plan = wf.Plan(n, n, wf.parts_of(probs[i]), params)
        cold = torch.empty(n, n, device="cuda")
        _, st_c = plan.solve(*inp[i], sched, bench.TOL, out=cold)
        ctrl = torch.empty(n, n, device="cuda")
        _, st_z = plan.solve(*inp[i], wsched, bench.TOL, out=ctrl)
        net.forward(X[i:i + 1].contiguous(), y, 1)
        warm = torch.empty(n, n, device="cuda")
        _, st_w = plan.solve_warm(*inp[i], (y[0] * SG[i]).contiguous(), wsched, bench.TOL, out=warm)
        plan.close()
        ref = O.pcg_wf(probs[i], tol=1e-10)
        assert st_c["status"] == 0 and st_w["status"] == 0
        e_c, e_w, e_z = (rel(a.cpu().numpy(), ref) for a in (cold, warm, ctrl))
        errs.append((e_c, e_w, e_z))
        assert e_c < 1e-4 and e_w < 1e-4, (e_c, e_w)
        cold_it.append(st_c["iters"])
        warm_it.append(st_w["iters"])
        ctrl_it.append(st_z["iters"])
    net.close()
    print(f"256^2 sweeps per solve: cold {np.mean(cold_it):.0f}, warm-started {np.mean(warm_it):.0f}, "
          f"zero start with the warm schedule {np.mean(ctrl_it):.0f}; worst errors {np.max(errs, axis=0)}")
    assert np.mean(warm_it) < np.mean(cold_it)
