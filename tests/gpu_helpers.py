"""Shared helpers of the GPU parity tests (marshalling only)."""
import numpy as np


def lib():
    from paper_1302_3120_gb300 import build
    build.build()
    from paper_1302_3120_gb300 import csar
    return csar


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).cuda()


def dev_mask(mask):
    import torch
    import synth
    return torch.from_numpy(synth.pack_mask(mask).view(np.int32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def crand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
