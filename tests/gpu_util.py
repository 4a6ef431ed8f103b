"""Helpers of the GPU tests: numpy <-> CUDA int64 tensors holding uint64 bits."""
import numpy as np


def to_dev(x, dev="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).to(dev)


def to_host(t):
    return t.cpu().numpy().view(np.uint64)
