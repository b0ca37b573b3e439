"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI on
torch tensors and bring results back as numpy arrays laid out like the oracle's."""
import numpy as np

import oracle as O
import paper_1511_05578_gb300 as crv
from paper_1511_05578_gb300 import inputs


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def max_rel(a, b):
    """Element-wise error scaled by the reference's largest entry: max|a - b| / max|b|.
    One wrong entry shows here at its own size, where a norm over a whole scale would
    dilute it."""
    mb = np.abs(b).max() if np.size(b) else 0.0
    return np.abs(a - b).max() / (mb if mb > 0 else 1.0) if np.size(b) else 0.0


def map_to_device(fmap, real):
    import torch
    a = np.asarray(fmap)
    if real:
        return torch.tensor(np.ascontiguousarray(a.real)[None], device="cuda")
    return torch.tensor(np.ascontiguousarray(np.stack([a.real, a.imag], -1))[None], device="cuda")


def map_from_device(t, real):
    a = t[0].cpu().numpy()
    return a if real else a[..., 0] + 1j * a[..., 1]


def W_from_device(Wt, j, real):
    a = Wt[j][0].cpu().numpy().astype(np.float64)
    return a if real else a[..., 0] + 1j * a[..., 1]


def W_to_device(p, W_o):
    Wt = p.W_tensors(1)
    for j, v in W_o.items():
        a = np.asarray(v)
        if p.real:
            Wt[j].copy_(__import__("torch").tensor(a.real[None]))
        else:
            Wt[j].copy_(__import__("torch").tensor(np.stack([a.real, a.imag], -1)[None]))
    return Wt


def flm_to_device(f):
    import torch
    return torch.tensor(np.asarray(f, dtype=np.complex128)[None], device="cuda")


def case(L, lam, J0, s, real, seed, power=2.0):
    f = inputs.flm_gaussian(L, seed, spin=s, real=real, power=power)
    fmap = O.sht_inverse(f, L, s)
    if real:
        fmap = fmap.real
    return f, fmap
