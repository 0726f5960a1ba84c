"""Helpers shared by the GPU tests (not collected: no test_ prefix)."""
import numpy as np

from paper_0707_3548_gb300 import tqr


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def to_dev(A):
    torch = torch_cuda()
    return tqr.colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda"))


def to_host(X):
    return np.asfortranarray(X.cpu().numpy())


def t_blocks(Tflat, m, n, nb, ib):
    """Split the flat T array into {(i, k): ib x nb} following tqr_t_size's layout."""
    p, q = -(-m // nb), -(-n // nb)
    kt = min(p, q)
    out = {}
    off = 0
    for k in range(kt):
        for i in range(k, p):
            blk = Tflat[off:off + ib * nb].reshape(nb, ib).T   # column-major ib x nb
            out[(i, k)] = blk
            off += ib * nb
    return out
