"""Helpers shared by the GPU tests: plans from synth problems, layout
conversions of the library's packed spectra, and the mapping between the
library's fields and the oracle chain's."""

import numpy as np


def dev(a):
    import torch
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_plan(prob, **params):
    from paper_1704_00865_gb300 import wf
    ny, nx = prob.shape
    plan = wf.Plan(ny, nx, wf.parts_of(prob), wf.make_params(**params))
    plan.set_problem(dev(prob.d), dev(prob.pixel_var), dev(prob.mask), dev(prob.C), dev(prob.P1f),
                     dev(prob.Pst), dev(prob.stripe_amp2))
    return plan


def field(plan, which):
    import torch
    out = torch.empty(plan.ny, plan.nx, device="cuda")
    plan.get_field(which, out)
    return out.cpu().numpy().astype(np.float64)


def unpack_spectrum(flat, ny, nx):
    """Library 2D spectrum [ny][nx/2] complex (column 0 packed) -> rfft2 layout."""
    Z = np.asarray(flat, np.float32).reshape(ny, nx).view(np.complex64).astype(np.complex128)
    h = nx // 2
    X = np.empty((ny, h + 1), np.complex128)
    X[:, 1:h] = Z[:, 1:]
    z0 = Z[:, 0]
    zm = np.conj(z0[(-np.arange(ny)) % ny])
    X[:, 0] = 0.5 * (z0 + zm)
    X[:, h] = (z0 - zm) / 2j
    return X


def pack_spectrum(X):
    """rfft2 layout [ny][nx/2+1] -> library layout (float32 flat)."""
    ny, h1 = X.shape
    h = h1 - 1
    Z = np.empty((ny, h), np.complex64)
    Z[:, 1:] = X[:, 1:h]
    Z[:, 0] = X[:, 0] + 1j * X[:, h]
    return Z.view(np.float32).ravel()


def unpack_rows(flat, ny, nx):
    Z = np.asarray(flat, np.float32).reshape(ny, nx).view(np.complex64).astype(np.complex128)
    h = nx // 2
    X = np.empty((ny, h + 1), np.complex128)
    X[:, 1:h] = Z[:, 1:]
    X[:, 0] = Z[:, 0].real
    X[:, h] = Z[:, 0].imag
    return X


def oracle_fields(chain):
    """{library field id: oracle pixel map} for the fields the chain has."""
    from paper_1704_00865_gb300 import wf
    out = {wf.WF_FIELD_S: chain.s}
    for i, part in enumerate(chain.P.parts):
        if part.name == "2DF":
            if not chain.P.merge_2df:   # t_2DF is marginalised when merged
                out[wf.WF_FIELD_T_2DF] = chain.t[i]
            out[wf.WF_FIELD_D_2DF] = chain.dd[i]
        elif part.name == "RF":
            out[wf.WF_FIELD_T_RF] = chain.t[i]
            out[wf.WF_FIELD_D_RF] = chain.dd[i]
    return out


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    dt = np.complex128 if (np.iscomplexobj(a) or np.iscomplexobj(b)) else np.float64
    a = a.astype(dt)
    b = b.astype(dt)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
