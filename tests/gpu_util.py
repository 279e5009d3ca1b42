"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import numpy as np


def rel_per_rhs(got, ref):
    got = np.asarray(got).reshape(got.shape[0], -1)
    ref = np.asarray(ref).reshape(ref.shape[0], -1)
    return np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)


def to_device(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
