"""Helpers for the GPU tests: move a CSR to the device and compare with the oracle."""
import numpy as np
import torch

import oracle


def to_dev(off, adj, device="cuda:0"):
    return (torch.from_numpy(np.ascontiguousarray(off, np.int64)).to(device),
            torch.from_numpy(np.ascontiguousarray(adj, np.int32)).to(device))


def gpu_core(k, off, adj):
    o, a = to_dev(off, adj)
    core, km = k.decompose(o, a)
    return core.cpu().numpy(), int(km.cpu()[0])


def assert_parity(k, n, off, adj, want=None):
    """GPU coreness must equal the oracle's bit for bit, and k_max its maximum."""
    if want is None:
        want = oracle.bz(n, off, adj)
    got, km = gpu_core(k, off, adj)
    np.testing.assert_array_equal(got, want)
    assert km == (int(want.max()) if n else 0)
    return got
