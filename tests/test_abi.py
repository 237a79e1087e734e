"""CPU checks of the boundary: libwf.so builds for sm_103a, loads, and exports
every function include/wf.h declares; host-side argument checks answer
without touching a GPU; the product path never reaches the oracle."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "wf.h")).read()
    return re.findall(r"^WF_API\s+[\w\s\*]+?\b(wf_\w+)\s*\(", src, flags=re.M)


@pytest.fixture(scope="module")
def lib():
    from paper_1704_00865_gb300 import build, wf
    build.build()
    return wf.load()


def test_header_declares_the_expected_entry_points():
    names = _declared()
    from paper_1704_00865_gb300 import wf
    assert sorted(names) == sorted(wf.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n
    # and nothing else with C linkage beyond the declared ABI
    import subprocess
    from paper_1704_00865_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = sorted(l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("wf_"))
    assert exported == sorted(_declared())


def test_host_only_entry_points(lib):
    from paper_1704_00865_gb300 import wf
    assert lib.wf_version() == 3
    assert wf.strerror(0) == "ok"
    assert "converge" in wf.strerror(3)
    p = wf.wf_params_default()
    assert list(p.theta) == [0.9, 0.9, 1.0]
    assert p.split_f == 0.5 and p.split_fp == 0.5 and p.split_w == 0.0
    assert p.residual_every == 10 and p.check_every == 8
    assert p.merge_2df == 1 and p.tol_u_scale == 1.0 and p.refine == 0 and p.refine_tol_scale == 100.0
    assert p.autotune == 1 and p.stall_checks == 0 and p.refine_max_iters == 0
    assert p.dft_precision == 0 and p.refine_extra == 0 and p.sweep_kernel == 0 and p.trace == 0
    assert lib.wf_plan_shapes(None, None, None) == wf.WF_EINVAL


@pytest.mark.parametrize("ny,nx,parts,code", [
    (1024, 1000, 7, 7),      # not a power of two
    (16, 1024, 7, 7),        # below the smallest size
    (8192, 64, 7, 7),        # above the largest size
    (64, 64, 6, 1),          # white part missing
    (64, 64, 15, 1),         # unknown part bit
])
def test_plan_create_rejects_bad_arguments_before_any_cuda_call(lib, ny, nx, parts, code):
    h = C.c_void_p()
    assert lib.wf_plan_create(C.byref(h), ny, nx, parts, None, None) == code
    assert h.value is None


def test_plan_create_rejects_bad_params(lib):
    from paper_1704_00865_gb300 import wf
    for kw in (dict(theta=(0.9, 1.5, 1.0)), dict(split_f=0.5, split_fp=0.5, merge_2df=0), dict(split_f=1.01, split_fp=0.0), dict(split_f=0.6, split_fp=0.6),
               dict(residual_every=0), dict(tol_u_scale=0.0), dict(refine=-1), dict(refine=33),
               dict(refine_max_iters=-1), dict(refine_lam1_iters=-1), dict(stall_checks=-1),
               dict(autotune=3), dict(dft_precision=-1), dict(dft_precision=5), dict(sweep_kernel=2), dict(trace=3), dict(refine_accel=-1), dict(refine_accel=17),
               dict(refine_extra=-1), dict(refine_extra=33)):
        p = wf.make_params(**kw)
        h = C.c_void_p()
        assert lib.wf_plan_create(C.byref(h), 64, 64, 7, C.byref(p), None) == wf.WF_EINVAL


@pytest.mark.parametrize("ny,kw", [
    (256, dict(dft_precision=1)),                 # no 16-value column shape at 256
    (2048, dict(dft_precision=3)),                # tcgen05 stages: columns of 512 and 1024 only
    (4096, dict(dft_precision=4)),
    (1536, dict(dft_precision=2)),                # 3 * 2^k columns
    (1024, dict(dft_precision=1, merge_2df=0, split_fp=0.3)),  # plain sweep (stored t_2DF)
])
def test_tensor_core_stages_reject_unsupported_plans(lib, ny, kw):
    from paper_1704_00865_gb300 import wf
    p = wf.make_params(**kw)
    h = C.c_void_p()
    assert lib.wf_plan_create(C.byref(h), ny, 64, 7, C.byref(p), None) == wf.WF_EUNSUPPORTED
    assert h.value is None


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1704_00865_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, flags=re.M), f
                assert "wf_oracle" not in src, f


def test_schedule_struct_layout_matches_header(lib, tmp_path):
    # the binding's ctypes structs against the C compiler's layout of the
    # structs include/wf.h declares: every field's offset and the size
    import shutil
    import subprocess
    from paper_1704_00865_gb300 import wf
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = [wf.wf_schedule, wf.wf_params, wf.wf_stats, wf.wf_map]
    lines = []
    for st in structs:
        name = st.__name__
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "wf.h"\nint main(void) {\n' +
                   "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n")
               if l)
    for st in structs:
        name = st.__name__
        assert int(got[name]) == C.sizeof(st), name
        for f, _ in st._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(st, f).offset, (name, f)


@pytest.mark.parametrize("sizes,lanes,parts,code", [
    ([], 4, 7, 1),                           # no maps
    ([(64, 64)], 65, 7, 1),                  # too many lanes
    ([(64, 64), (64, 1000)], 2, 7, 7),       # one unsupported size
    ([(64, 64), (128, 32)], 2, 6, 1),        # white part missing
    ([(64, 64)], 0, 7, 7),                   # persistent mode: size its kernel does not take
    ([(256, 256), (256, 512)], 0, 7, 7),     # persistent mode: not square
    ([(256, 256)], 0, 3, 7),                 # persistent mode: no stripe part
    ([(256, 256)], -1, 7, 1),                # negative lanes
])
def test_batch_create_rejects_bad_arguments_before_any_cuda_call(lib, sizes, lanes, parts, code):
    from paper_1704_00865_gb300 import wf
    n = len(sizes)
    ny = (C.c_int * max(n, 1))(*[a for a, _ in sizes])
    nx = (C.c_int * max(n, 1))(*[b for _, b in sizes])
    h = C.c_void_p()
    p = wf.wf_params_default()
    assert lib.wf_batch_create(C.byref(h), n, ny, nx, parts, C.byref(p), lanes, None) == code
    assert h.value is None
    bad = wf.make_params(refine=33)
    if n:
        assert lib.wf_batch_create(C.byref(h), n, ny, nx, 7, C.byref(bad), 1, None) in (wf.WF_EINVAL, code)


def test_batch_solve_rejects_null_handles(lib):
    from paper_1704_00865_gb300 import wf
    s = wf.make_schedule("fixed", [10.0], [10])
    assert lib.wf_batch_solve(None, None, C.byref(s), 1e-5, None) == wf.WF_EINVAL
    assert lib.wf_batch_launch_count(None) == -1
    lib.wf_batch_destroy(None)
    assert C.sizeof(wf.wf_map) == 8 * 8


def test_pointer_rule_rejects_another_gpus_memory(tmp_path):
    # The rule every entry point applies to a caller's array (csrc/wf_ptr.h),
    # from what cudaPointerGetAttributes reports: device memory of the current
    # GPU is used in place, host memory is staged, and device memory of any
    # other GPU is rejected (WF_EINVAL) instead of being handed to a kernel
    # that would fault on it.  Compiled here with the host compiler alone.
    import shutil
    import subprocess
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "ptr_rule.cpp"
    src.write_text(r'''
#include <cstdio>
#include "wf_ptr.h"
using namespace wf;
int main() {
  int bad = 0;
  // (query ok, cudaMemoryType, pointer's device, current device) -> where
  struct { bool ok; int type, pdev, cur, want; } cases[] = {
    {true, 2, 0, 0, PTR_DEVICE},        // this GPU's memory
    {true, 2, 3, 3, PTR_DEVICE},
    {true, 2, 1, 0, PTR_OTHER_DEVICE},  // a second GPU's memory
    {true, 2, 0, 1, PTR_OTHER_DEVICE},
    {true, 3, 1, 0, PTR_DEVICE},        // managed memory, any device
    {true, 1, 0, 0, PTR_HOST},          // pinned host memory
    {true, 0, -2, 0, PTR_HOST},         // pageable host memory
    {false, 0, 0, 0, PTR_HOST},         // query failed: not device memory
  };
  for (auto& c : cases)
    if (classify_ptr(c.ok, c.type, c.pdev, c.cur) != c.want) { std::printf("case %d %d %d\n", c.type, c.pdev, c.cur); ++bad; }
  return bad;
}
''')
    exe = tmp_path / "ptr_rule"
    inc = os.path.join(ROOT, "paper_1704_00865_gb300", "csrc")
    r = subprocess.run([cxx, "-std=c++17", "-I", inc, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
