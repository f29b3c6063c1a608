"""The binding's size checks (CPU): the C ABI takes bare pointers and sizes
every array from the context, so the binding refuses any array whose element
count, type or memory does not match what the call will read or write.

The checks run before any CUDA call, so a Context object is made here
without its constructor (no device needed) and given the sizes a context of
that grid and structure would have."""
import numpy as np
import pytest
import torch

from paper_math_0301321_gb300.binding import Context


def fake(device=False, prec="fp64", n=(8, 6, 4), m=5, n_seg=3):
    c = Context.__new__(Context)
    c.device = device
    c.fp64 = prec == "fp64"
    c.dtype_np = np.float64 if c.fp64 else np.float32
    c.dtype_t = torch.float64 if c.fp64 else torch.float32
    c.n = n
    c.G = n[0] * n[1] * n[2]
    c.m, c.n_seg = m, n_seg
    return c


def test_fields_and_marker_arrays_must_have_the_calls_sizes():
    c = fake(prec="fp32")
    nx, ny, nz = c.n
    u = c._field(np.ones((3, nz, ny, nx)))
    assert u.dtype == np.float32 and u.shape == (3, nz, ny, nx)
    with pytest.raises(ValueError):
        c._field(np.ones((3, nz, ny, nx + 1)))
    assert c._field(np.ones((3, c.m)), 3 * c.m).shape == (3, c.m)        # marker forces
    with pytest.raises(ValueError):
        c._field(np.ones((3, c.m + 1)), 3 * c.m)
    assert c._pos(np.zeros((3, c.m))).dtype == np.float64
    with pytest.raises(ValueError):
        c._pos(np.zeros((3, c.m - 1)))
    assert c._pos(np.ones(c.n_seg), c.n_seg).shape == (c.n_seg,)
    with pytest.raises(ValueError):
        c._pos(np.ones(c.n_seg + 1), c.n_seg)


def test_buffers_the_library_writes_must_match_type_size_and_memory():
    h = fake(device=False, prec="fp32")
    ok = np.zeros(3 * h.m)
    assert h._out(ok, 3 * h.m, True, "lam_D_out") is ok
    assert h._out(torch.zeros(3 * h.m, dtype=torch.float64), 3 * h.m, True, "x") is not None
    for bad in (np.zeros(3 * h.m, np.float32), np.zeros(3 * h.m + 1), np.zeros((3 * h.m, 2))[:, 0]):
        with pytest.raises(ValueError):
            h._out(bad, 3 * h.m, True, "lam_D_out")
    with pytest.raises(ValueError):                       # the context's real type is float32
        h._out(np.zeros(3 * h.G), 3 * h.G, False, "lam_u_out")
    d = fake(device=True)
    for bad in (np.zeros(d.n_seg), torch.zeros(d.n_seg, dtype=torch.float64)):
        with pytest.raises(ValueError):                   # host memory for a device context
            d._out(bad, d.n_seg, True, "grad_b")
