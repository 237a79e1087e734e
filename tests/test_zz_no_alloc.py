"""wf_fft2_noalloc -- the 2D transform for callers that may not allocate
device memory (an embedding application that owns all of it, or a pipeline
that must not allocate once running).  Its working memory is a fixed device
array inside the library, so the check is that, called twice in a row through
the C ABI, it returns what the plan-based wf_fft2 returns.  Kept last in
collection order so that a failure here never hides another test."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("ny,nx", [(1024, 1024), (64, 256), (384, 1536)])
def test_noalloc_transform_matches_plan_transform_on_two_calls(ny, nx):
    import torch
    from paper_1704_00865_gb300 import build, wf
    build.build()
    wf.load()
    rng = np.random.default_rng(ny + nx)
    plan = wf.Plan(ny, nx, wf.WF_PART_WHITE)
    stream = torch.cuda.current_stream()
    # call 1: forward transform of a map; call 2: inverse transform of a
    # different spectrum (the second call reuses the array the first filled)
    x = rng.standard_normal((ny, nx)).astype(np.float32)
    y = rng.standard_normal((ny, nx)).astype(np.float32)
    ref_fwd = plan.fft2(x)
    ref_inv = plan.fft2(y, inverse=True)
    out1 = torch.empty(ny * nx, device="cuda")
    out2 = torch.empty(ny * nx, device="cuda")
    wf.wf_fft2_noalloc(ny, nx, torch.from_numpy(x).cuda(), out1, inverse=False,
                       stream=wf.C.c_void_p(stream.cuda_stream))
    wf.wf_fft2_noalloc(ny, nx, torch.from_numpy(y).cuda(), out2, inverse=True,
                       stream=wf.C.c_void_p(stream.cuda_stream))
    stream.synchronize()
    assert _rel(out1.cpu().numpy(), ref_fwd) < 5e-6
    assert _rel(out2.cpu().numpy(), ref_inv) < 5e-6
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_array_and_host_buffers():
    import torch
    from paper_1704_00865_gb300 import build, wf
    build.build()
    lib = wf.load()
    big = torch.empty(2048 * 1024, device="cuda")
    assert lib.wf_fft2_noalloc(2048, 1024, wf.C.c_void_p(big.data_ptr()), wf.C.c_void_p(big.data_ptr()),
                               0, None) == wf.WF_EUNSUPPORTED
    host = np.zeros(64 * 64, np.float32)
    dev = torch.empty(64 * 64, device="cuda")
    assert lib.wf_fft2_noalloc(64, 64, wf.C.c_void_p(host.ctypes.data), wf.C.c_void_p(dev.data_ptr()),
                               0, None) == wf.WF_EINVAL


def test_noalloc_call_after_a_larger_one_rewrites_what_it_reads():
    # the shared array keeps the last call's contents: a 64 x 256 transform
    # after a 1024 x 1024 one (and a 1024 x 1024 one after that) must read
    # only what it wrote itself -- every twiddle and spectrum entry it uses
    import torch
    from paper_1704_00865_gb300 import build, wf
    build.build()
    wf.load()
    stream = torch.cuda.current_stream()
    sp = wf.C.c_void_p(stream.cuda_stream)
    rng = np.random.default_rng(7)
    for ny, nx in [(1024, 1024), (64, 256), (1024, 1024)]:
        plan = wf.Plan(ny, nx, wf.WF_PART_WHITE)
        for inverse in (False, True):
            x = rng.standard_normal((ny, nx)).astype(np.float32)
            ref = plan.fft2(x, inverse=inverse)
            out = torch.empty(ny * nx, device="cuda")
            wf.wf_fft2_noalloc(ny, nx, torch.from_numpy(x).cuda(), out, inverse=inverse, stream=sp)
            stream.synchronize()
            assert _rel(out.cpu().numpy(), ref) < 5e-6, (ny, nx, inverse)
        plan.close()
