"""Helpers shared by the GPU tests: numpy <-> torch marshalling."""
import numpy as np

TOL = {2: 1e-24, 4: 1e-55, 8: 1e-112}


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t):
    return t.detach().cpu().numpy()
