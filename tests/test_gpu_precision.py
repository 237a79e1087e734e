"""The radix-16 stages of the column transforms on the tensor cores
(wf_params.dft_precision: 1 = split TF32, three products per complex factor
pair; 2 = one TF32 product) against FP64, with the error stated for each
result: the 2D transform alone (forward and inverse), the fields after a few
sweeps against the oracle's sweeps, and the benchmark's 1024 x 1024 solve
against the oracle's solution and literal residual."""

import os

import numpy as np
import pytest

import oracle as O
from gpu_util import dev, field, make_plan, oracle_fields, pack_spectrum, rel, unpack_spectrum
from paper_1704_00865_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    from paper_1704_00865_gb300 import build, wf
    build.build()
    wf.load()
    O.set_workers(os.cpu_count() or 1)
    return wf


@pytest.mark.parametrize("ny,nx", [(512, 64), (1024, 128), (2048, 32), (4096, 32), (1024, 1024)])
def test_transforms_per_precision(wf, ny, nx):
    rng = np.random.default_rng(ny + 3 * nx)
    x = rng.standard_normal((ny, nx)).astype(np.float32)
    Y = np.fft.rfft2(rng.standard_normal((ny, nx)))
    ref_f = np.fft.rfft2(x.astype(np.float64))
    ref_i = np.fft.irfft2(Y, s=(ny, nx))
    err = {}
    for prec in (0, 1, 2):
        p = wf.Plan(ny, nx, wf.WF_PART_WHITE, wf.make_params(dft_precision=prec))
        ef = rel(unpack_spectrum(p.fft2(x), ny, nx), ref_f)
        ei = rel(p.fft2(pack_spectrum(Y), inverse=True).reshape(ny, nx), ref_i)
        p.close()
        err[prec] = (ef, ei)
    print(f"{ny}x{nx} rel L2 (forward, inverse): fp32 {err[0][0]:.1e} {err[0][1]:.1e}, "
          f"split tf32 {err[1][0]:.1e} {err[1][1]:.1e}, tf32 {err[2][0]:.1e} {err[2][1]:.1e}")
    assert max(err[0]) < 5e-6
    # split TF32 keeps FP32 accuracy
    assert max(err[1]) < 5e-6
    # one TF32 product per stage: about 2^-11 per stage, so the tensor-core
    # stages are demonstrably the ones that ran
    assert 1e-5 < min(err[2]) and max(err[2]) < 3e-3


def _sweeps(wf, prob, lams):
    # the oracle's sweeps once, then a plan per precision against them
    P = O.build_parts(prob, merge_2df=True, split_f=0.5, split_fp=0.5)
    ch = O.Chain(P)
    for lam in lams:
        ch.sweep(lam)
    ref = oracle_fields(ch)
    worst = {}
    for prec in (1, 2):
        plan = make_plan(prob, merge_2df=1, split_f=0.5, split_fp=0.5, dft_precision=prec)
        for lam in lams:
            plan.iterate(lam, 1)
        worst[prec] = max(rel(field(plan, fid), r) for fid, r in ref.items())
        plan.close()
    return worst


@pytest.mark.parametrize("n", [1024, 4096])
def test_sweeps_per_precision(wf, n):
    # the 1024 x 1024 benchmark map and the 4096 x 4096 map with the same noise
    prob = synth.cfg1_problem(1000, 1024) if n == 1024 else synth.make_problem(4096, 4096, 3000)
    lams = [10.0, 10.0, 10.0, 1.0] if n == 1024 else [10.0, 1.0]
    w = _sweeps(wf, prob, lams)
    print(f"{n}^2 after {len(lams)} sweeps, worst field rel L2: split tf32 {w[1]:.2e}, tf32 {w[2]:.2e}")
    assert w[1] < 2e-5
    assert w[2] < 5e-3


@pytest.fixture(scope="module")
def full_size(wf):
    import bench
    prob = synth.cfg1_problem(bench.SEED, bench.N)
    P = O.build_parts(prob)
    return prob, P, O.pcg_wf(prob, P=P, tol=1e-10)


@pytest.mark.parametrize("prec", [1, 2])
def test_benchmark_solve_per_precision(wf, full_size, prec):
    # the benchmark's solve with the tensor-core column stages: the residual,
    # the stop test and the corrections stay FP32 / FP64, so they pull the
    # solution to the oracle's even from the TF32 sweeps
    import torch
    import bench
    prob, P, s_ref = full_size
    plan = wf.Plan(bench.N, bench.N, wf.parts_of(prob), bench.solver_params(wf, dft_precision=prec))
    out = torch.empty(bench.N, bench.N, device="cuda")
    _, st = plan.solve(dev(prob.d), dev(prob.pixel_var), dev(prob.mask), dev(prob.C), dev(prob.P1f),
                       dev(prob.Pst), dev(prob.stripe_amp2), bench.solver_schedule(wf), bench.TOL, out=out)
    assert plan.shapes()[1] == 16
    plan.close()
    s = out.cpu().numpy().astype(np.float64)
    lit = O.literal_residual(prob, s, P=P, tol=1e-10)
    err = rel(s, s_ref)
    print(f"1024^2 benchmark solve, dft_precision={prec}: {st['iters']} sweeps, status {st['status']}, "
          f"literal residual {lit:.2e}, rel L2 vs oracle {err:.2e}")
    assert st["status"] == 0, st
    assert lit < 1e-5, lit
    assert err < 1e-4, err
