"""The misfit entry point that allocates nothing (sbfwi_misfit_noalloc).

It exists for callers that cannot let the library call cudaMalloc: for example a
framework that has already reserved nearly all device memory, or a real-time
loop that must not block in the driver's allocator.  Its per-block partial sums
live in a fixed array inside the library.  This file is collected last so that a
failure here cannot hide any other test.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_misfit_matches_the_allocating_entry_point_twice(lib):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    dt = 0.0625
    # two calls in a row with different sizes and data: the shared array must not carry anything over
    for shape in [(3, 5, 1000), (8, 32, 801)]:          # 15000 and 205056 samples (ragged last block)
        tr = torch.tensor(rng.standard_normal(shape), device="cuda")
        ob = torch.tensor(rng.standard_normal(shape), device="cuda")
        E_out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        res_out = torch.empty_like(tr)
        lib.misfit_noalloc(tr, ob, dt, E_out, res_out)
        torch.cuda.synchronize()
        E_ref, res_ref = lib.misfit(tr, ob, dt)          # the existing entry point, same device data
        assert abs(E_out.item() - E_ref) <= 1e-10 * abs(E_ref)
        assert torch.equal(res_out, res_ref)


def test_noalloc_misfit_rejects_sizes_beyond_its_limit(lib):
    torch = pytest.importorskip("torch")
    small = torch.zeros(4, dtype=torch.float64, device="cuda")
    E_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    code = lib._lib.sbfwi_misfit_noalloc(vp(small), vp(small), 4096 * 65536 + 1, 0.1, vp(E_out), None, None)
    assert code == lib.EINVAL
    assert "no-allocation limit" in lib._lib.sbfwi_last_error().decode()
