"""The paint entry point that allocates nothing, for callers that cannot
call cudaMalloc (hosts that own all device memory, loops that cannot take
cudaMalloc's implicit synchronisation).  It must give the same density as
the plan-based fpm_paint, call after call, although every call reuses the
library's fixed scratch.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

from paper_2010_11847_gb300 import inputs

pytestmark = pytest.mark.gpu


def _rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("np_,nc", [(16, 64), (32, 64), (48, 48), (64, 64)])
def test_paint_noalloc_matches_plan_paint_twice(cuda, libfpm, np_, nc):
    import torch
    from paper_2010_11847_gb300.binding import Plan, FPM_OK
    dx = torch.from_numpy(inputs.random_displacements(np_, 5.0, 41 + nc)).cuda()
    with Plan(np_, nc, 100.0, inputs.COSMO_DEFAULT) as pl:
        ref = pl.paint(dx).cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                      # the second call reuses the scratch the first left
        rho = torch.full((nc, nc, nc), -7.0, device="cuda")
        rc = libfpm.fpm_paint_noalloc(np_, nc, ctypes.c_void_p(dx.data_ptr()),
                                      ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(stream))
        assert rc == FPM_OK
        torch.cuda.synchronize()
        got = rho.cpu().numpy()
        assert _rel_l2(got, ref) < 1e-5
        assert abs(got.astype(np.float64).sum() - nc ** 3) < 1e-3 * nc ** 3


def test_paint_noalloc_rejects_sizes_beyond_its_scratch(cuda, libfpm):
    import torch
    from paper_2010_11847_gb300.binding import FPM_EINVAL
    dx = torch.zeros(3, 128 ** 3, device="cuda")
    rho = torch.zeros(128, 128, 128, device="cuda")
    rc = libfpm.fpm_paint_noalloc(128, 128, ctypes.c_void_p(dx.data_ptr()), ctypes.c_void_p(rho.data_ptr()), None)
    assert rc == FPM_EINVAL
    rc = libfpm.fpm_paint_noalloc(64, 128, ctypes.c_void_p(dx.data_ptr()), ctypes.c_void_p(rho.data_ptr()), None)
    assert rc == FPM_EINVAL
