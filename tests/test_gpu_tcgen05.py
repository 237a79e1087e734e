"""The radix-16 stages of the column pass on the 5th-generation tensor cores
(tcgen05.mma kind::tf32, TMEM accumulators; wf_params.dft_precision 3 = split
TF32, 4 = one TF32 product) against the FP64 oracle, with the error stated
per result: the fields after one sweep (where only the column pass differs
between the precisions, so the error is that of its four radix-16 stages),
after several sweeps, and the benchmark's 1024 x 1024 solve against the
oracle's solution and literal residual."""

import os

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
    O.set_workers(os.cpu_count() or 1)
    return wf


@pytest.mark.parametrize("n", [512, 1024])
def test_tcgen05_stages_per_sweep_against_the_oracle(wf, n):
    prob = synth.cfg1_problem(1000, n) if n == 1024 else synth.make_problem(n, n, 1500)
    P = O.build_parts(prob, merge_2df=True, split_f=0.5, split_fp=0.5)
    lams = [10.0, 10.0, 10.0, 1.0]
    ch = O.Chain(P)
    refs = []
    for lam in lams:
        ch.sweep(lam)
        refs.append({k: v.copy() for k, v in oracle_fields(ch).items()})
    err = {}
    for prec in (0, 3, 4):
        plan = make_plan(prob, merge_2df=1, split_f=0.5, split_fp=0.5, dft_precision=prec)
        e = []
        for lam, ref in zip(lams, refs):
            plan.iterate(lam, 1)
            e.append(max(rel(field(plan, fid), r) for fid, r in ref.items()))
        err[prec] = e
        plan.close()
    # after one sweep the signal-side field d_2DF is the column pass's output:
    # four radix-16 stages (two per transform) at 1024, three at 512
    print(f"{n}^2 worst field rel L2 after sweeps 1..4: fp32 {err[0]}, tcgen05 split tf32 {err[3]}, "
          f"tcgen05 tf32 {err[4]}")
    assert max(err[0]) < 2e-5
    assert max(err[3]) < 2e-5          # the split keeps FP32 accuracy
    # one TF32 product per stage: about 2^-11 relative each, so these are the
    # tensor-core stages and not a silent FP32 fallback
    assert 1e-5 < err[4][0] and max(err[4]) < 5e-3


def test_tcgen05_benchmark_solve(wf):
    import torch
    import bench
    prob = synth.cfg1_problem(bench.SEED, bench.N)
    P = O.build_parts(prob)
    s_ref = O.pcg_wf(prob, P=P, tol=1e-10)
    plan = wf.Plan(bench.N, bench.N, wf.parts_of(prob), bench.solver_params(wf, dft_precision=3))
    out = torch.empty(bench.N, bench.N, device="cuda")
    _, st = plan.solve(dev(prob.d), dev(prob.pixel_var), dev(prob.mask), dev(prob.C), dev(prob.P1f),
                       dev(prob.Pst), dev(prob.stripe_amp2), bench.solver_schedule(wf), bench.TOL, out=out)
    plan.close()
    s = out.cpu().numpy().astype(np.float64)
    lit = O.literal_residual(prob, s, P=P, tol=1e-10)
    m = prob.mask.astype(bool)
    err, err_m = rel(s, s_ref), rel(s[m], s_ref[m])
    print(f"1024^2 benchmark solve, tcgen05 split tf32: {st['iters']} sweeps, status {st['status']}, "
          f"literal residual {lit:.2e}, rel L2 {err:.2e} (masked {err_m:.2e})")
    assert st["status"] == 0, st
    assert lit < 1e-5 and err < 1e-4 and err_m < 1e-4


def test_tcgen05_sizes(wf):
    for prec in (3, 4):
        with pytest.raises(wf.WFError) as e:
            wf.Plan(2048, 2048, 7, wf.make_params(dft_precision=prec))
        assert e.value.code == wf.WF_EUNSUPPORTED
