"""The allocation-free filter entry point agrees with the allocating one.

dcrf_filter_static serves callers that cannot allocate device memory when they
filter; its scratch is a fixed file-scope device array shared by all calls.
This file is collected last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

from helpers import gpu_setup, rel_err
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _static(dcrf, lat, Y, storage):
    out = torch.empty_like(Y)
    st = dcrf.lib().dcrf_filter_static(lat.handle, ctypes.c_void_p(Y.data_ptr()), Y.shape[1],
                                       ctypes.c_void_p(out.data_ptr()), dcrf.STORAGE[storage],
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def test_static_scratch_filter_matches_allocating_filter(dcrf):
    p = S.make_problem(160, 120, 10, 21, seed=77)
    g = gpu_setup(dcrf, [p], torch)
    rng = np.random.default_rng(5)
    # both entry points run the same splat, blur and slice kernels; the dense
    # splat adds float32 values with atomics, so two calls of the allocating
    # filter differ by as much as these two (measured on 160x120, L=21:
    # 4.6e-7 in float32, and 8.2e-4 in float16 storage, where a changed last
    # bit of a splat sum can flip the rounding of a stored half)
    for storage, tol in (("f32", 1e-5), ("f16", 2e-3)):
        for call in range(2):                      # two calls in a row share the array
            Y = torch.from_numpy(rng.uniform(0, 1, (p.n_pixels, 21)).astype(np.float32)).cuda()
            for lat in (g["lb"], g["ls"]):
                st, out = _static(dcrf, lat, Y, storage)
                assert st == 0
                ref = dcrf.dcrf_filter(lat, Y, storage=storage)
                torch.cuda.synchronize()
                assert rel_err(out.cpu().numpy(), ref.cpu().numpy()) <= tol, (storage, call)


def test_static_scratch_rejects_requests_beyond_capacity(dcrf):
    cap = dcrf.lib().dcrf_filter_static_capacity()
    assert cap == 16 << 20
    p = S.voc_shaped()
    g = gpu_setup(dcrf, [p], torch)
    lat = g["ls"]
    assert lat.m * 64 * 12 > cap                   # float32 values with 64 labels do not fit
    Y = torch.zeros((p.n_pixels, 64), dtype=torch.float32, device="cuda")
    st, _ = _static(dcrf, lat, Y, "f32")
    assert st == -8
