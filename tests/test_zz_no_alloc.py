"""The allocation-free bin sort agrees with the context-based one.

ib_bin_sort_noalloc serves callers that cannot allocate device memory (code
inside a CUDA graph capture in global mode, hosts whose runtime owns all
device memory): it takes caller-owned device buffers and keeps its radix-sort
work space in one fixed device array.  Two calls in a row, on different
inputs, must each give exactly the keys and permutation of ib_bin_sort.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import numpy as np
import pytest

from paper_math_0301321_gb300 import binding, synth
from paper_math_0301321_gb300.binding import Context, IBError

pytestmark = pytest.mark.gpu


class Grid:
    def __init__(self, n, h):
        self.n, self.h, self.rho, self.mu, self.dt = n, h, 1.0, 0.02, 1e-5


def markers(seed, n, h, m):
    L = np.array(n, float) * h
    X = synth.random_markers(seed, m) * L[:, None]
    X[:, : m // 5] = X[:, m // 5: 2 * (m // 5)]        # repeated cells
    X[0, :16] -= L[0]                                   # outside the box: wrapped
    return X


def test_noalloc_bin_sort_matches_context_sort_twice(ib):
    import torch
    for seed, n, m in ((31, (64, 32, 96), 50000), (32, (128, 128, 128), 200000)):
        h = 1.0 / 64
        g = Grid(n, h)
        X = markers(seed, n, h, m)
        ctx = Context(g, prec="fp32")
        ctx.set_structure(synth._empty_structure(X))
        k_ref, p_ref = ctx.bin_sort(X)
        ctx.close()
        Xd = torch.from_numpy(X).cuda()
        key = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        perm = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        binding.bin_sort_noalloc(n, h, Xd, key, perm)
        torch.cuda.synchronize()
        assert torch.equal(key, k_ref)
        assert torch.equal(perm, p_ref)


def test_noalloc_bin_sort_rejects_too_many_markers(ib):
    import torch
    m = (1 << 20) + 1
    X = torch.zeros((3, m), dtype=torch.float64, device="cuda")
    key = torch.empty(m, dtype=torch.int32, device="cuda")
    with pytest.raises(IBError, match="IB_NOALLOC_MAX_MARKERS"):
        binding.bin_sort_noalloc((32, 32, 32), 1 / 32, X, key, key)
