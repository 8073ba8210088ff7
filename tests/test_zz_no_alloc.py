"""p3t_energy_noalloc: the energy sums for callers that cannot allocate device
memory (code running under stream capture, or behind an allocator that owns
all device memory).  Called through the C ABI and checked against the
allocating p3t_energy on two calls in a row, so that the shared static
scratch is exercised with leftover contents from the previous call.

Collected last on purpose (file name), so a failure here does not hide the
other tests of a run that stops at the first failure."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P3T_ERR_CAPACITY = 2


def _lib():
    from paper_1506_04553_b300 import binding
    lib = binding._lib
    lib.p3t_energy_noalloc.argtypes = [C.c_int64, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p]
    lib.p3t_energy_noalloc.restype = C.c_int
    return lib


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_energy_matches_allocating_entry_point(cuda):
    import torch
    from paper_1506_04553_b300 import Context, Params, ics
    lib = _lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ctx = Context(Params())
    for call, (n, seed) in enumerate([(300_001, 1), (70_000, 2)]):
        pos, vel, m = ics.plummer(n, seed)
        md = torch.tensor(m, device="cuda")
        vd = torch.tensor(vel, device="cuda")
        pot = torch.tensor(-np.abs(np.random.default_rng(seed).normal(size=n)),
                           device="cuda")
        ref = ctx.energy(md, vd, pot).cpu().numpy()
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.p3t_energy_noalloc(n, _ptr(md), _ptr(vd), _ptr(pot), _ptr(out),
                                    stream)
        assert rc == 0
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref)), (call, got, ref)
        # without a potential the second sum is zero
        rc = lib.p3t_energy_noalloc(n, _ptr(md), _ptr(vd), None, _ptr(out), stream)
        assert rc == 0
        got = out.cpu().numpy()
        assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0]) and got[1] == 0.0


def test_noalloc_energy_rejects_out_of_range_sizes(cuda):
    import torch
    lib = _lib()
    out = torch.zeros((2,), dtype=torch.float64, device="cuda")
    dummy = C.c_void_p(out.data_ptr())
    # rejected before any device work: n beyond the kernel's index range
    assert lib.p3t_energy_noalloc(1 << 31, dummy, dummy, None, dummy, None) == P3T_ERR_CAPACITY
    assert lib.p3t_energy_noalloc(-1, dummy, dummy, None, dummy, None) == 1
    assert lib.p3t_energy_noalloc(5, None, dummy, None, dummy, None) == 1
    # n = 0 gives zeros
    assert lib.p3t_energy_noalloc(0, None, None, None, dummy, None) == 0
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [0.0, 0.0]
