"""The library's transforms (the flat-sky stand-ins for the spherical-harmonic
transforms of Sec. 2) against brute-force FP64 DFTs and numpy's FFT."""

import numpy as np
import pytest

import oracle as O
from gpu_util import pack_spectrum, rel, unpack_rows, unpack_spectrum

pytestmark = pytest.mark.gpu

SIZES = [(32, 32), (32, 64), (64, 32), (128, 256), (256, 128), (512, 512), (1024, 1024),
         (2048, 64), (64, 4096), (4096, 32),
         # lengths 3 * 2^k (a radix-3 stage in both directions)
         (384, 384), (768, 384), (384, 768), (1536, 64), (64, 1536), (1536, 1536), (384, 32), (32, 768)]


@pytest.fixture(scope="module")
def wf():
    from paper_1704_00865_gb300 import build, wf
    build.build()
    wf.load()
    return wf


def _plan(wf, ny, nx):
    return wf.Plan(ny, nx, wf.WF_PART_WHITE)


def test_forward_2d_matches_brute_force_dft(wf):
    ny, nx = 32, 64
    x = np.random.default_rng(0).standard_normal((ny, nx)).astype(np.float32)
    p = _plan(wf, ny, nx)
    X = unpack_spectrum(p.fft2(x), ny, nx)
    ref = O.brute_dft(O.brute_dft(x.astype(np.float64), axis=0), axis=1)[:, : nx // 2 + 1]
    assert rel(X, ref) < 2e-6


@pytest.mark.parametrize("ny,nx", [(384, 32), (32, 768)])
def test_radix3_lengths_match_brute_force_dft(wf, ny, nx):
    x = np.random.default_rng(ny + nx).standard_normal((ny, nx)).astype(np.float32)
    p = _plan(wf, ny, nx)
    X = unpack_spectrum(p.fft2(x), ny, nx)
    ref = O.brute_dft(O.brute_dft(x.astype(np.float64), axis=0), axis=1)[:, : nx // 2 + 1]
    assert rel(X, ref) < 2e-6
    p.close()


@pytest.mark.parametrize("ny,nx", SIZES)
def test_forward_inverse_and_row_transforms(wf, ny, nx):
    rng = np.random.default_rng(ny * 7 + nx)
    x = rng.standard_normal((ny, nx)).astype(np.float32)
    p = _plan(wf, ny, nx)
    X = unpack_spectrum(p.fft2(x), ny, nx)
    assert rel(X, np.fft.rfft2(x.astype(np.float64))) < 5e-6
    # inverse of a given spectrum
    Y = np.fft.rfft2(rng.standard_normal((ny, nx)))
    y = p.fft2(pack_spectrum(Y), inverse=True).reshape(ny, nx)
    assert rel(y, np.fft.irfft2(Y, s=(ny, nx))) < 5e-6
    # rows only (the stripe basis)
    R = unpack_rows(p.fft2(x, rows_only=True), ny, nx)
    assert rel(R, np.fft.rfft(x.astype(np.float64), axis=1)) < 5e-6
    xb = p.fft2(p.fft2(x, rows_only=True), inverse=True, rows_only=True).reshape(ny, nx)
    assert rel(xb, x) < 5e-6
    p.close()


def test_device_and_host_buffers_agree(wf):
    import torch
    ny, nx = 256, 512
    x = np.random.default_rng(5).standard_normal((ny, nx)).astype(np.float32)
    p = _plan(wf, ny, nx)
    host = p.fft2(x)
    out = torch.empty(ny * nx, device="cuda")
    p.fft2(torch.from_numpy(x).cuda(), out=out)
    assert np.array_equal(out.cpu().numpy(), host)
