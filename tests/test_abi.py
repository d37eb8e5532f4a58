"""The C-ABI library builds, loads and exports every symbol that
include/fpm.h declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2010_11847_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fpm_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(libfpm):
    declared = _declared()
    assert {"fpm_plan_create", "fpm_paint", "fpm_force", "fpm_kdk", "fpm_lpt", "fpm_linear_field",
            "fpm_readout"} <= declared
    for name in sorted(declared):
        assert hasattr(libfpm, name), name
    assert set(binding.EXPORTS) <= declared


def test_strerror_and_codes(libfpm):
    assert libfpm.fpm_strerror(0) == b"ok"
    assert b"invalid" in libfpm.fpm_strerror(-1)
    assert libfpm.fpm_strerror(12345) == b"unknown error"


@pytest.mark.parametrize("np_,nc", [(20, 20), (32, 48), (32, 256), (32, 0), (1024, 1024), (64, 32)])
def test_plan_rejects_bad_sizes_on_the_host(libfpm, np_, nc):
    h = ctypes.c_void_p()
    c = binding.fpm_cosmo(0.3, 0.05, 0.7, 0.96, 0.8, 2.7255)
    assert libfpm.fpm_plan_create(ctypes.byref(h), np_, nc, 100.0, ctypes.byref(c), None) == binding.FPM_EINVAL
    assert not h.value


def test_plan_rejects_bad_cosmology(libfpm):
    h = ctypes.c_void_p()
    for bad in [(0.0, 0.0, 0.7, 0.96, 0.8, 2.7), (0.3, 0.4, 0.7, 0.96, 0.8, 2.7), (0.3, 0.05, -1, 0.96, 0.8, 2.7)]:
        c = binding.fpm_cosmo(*bad)
        assert libfpm.fpm_plan_create(ctypes.byref(h), 32, 32, 100.0, ctypes.byref(c), None) == binding.FPM_EINVAL
    c = binding.fpm_cosmo(0.3, 0.05, 0.7, 0.96, 0.8, 2.7255)
    assert libfpm.fpm_plan_create(ctypes.byref(h), 32, 32, -5.0, ctypes.byref(c), None) == binding.FPM_EINVAL
    assert libfpm.fpm_plan_create(None, 32, 32, 100.0, ctypes.byref(c), None) == binding.FPM_EINVAL


def test_null_plan_entry_points(libfpm):
    assert libfpm.fpm_paint(None, None, None, None, None, None) == binding.FPM_EINVAL
    assert libfpm.fpm_force(None, None, None, None) == binding.FPM_EINVAL
    assert libfpm.fpm_kdk(None, None, None, None, 1, None, None, None) == binding.FPM_EINVAL
    assert libfpm.fpm_status(None, None) == binding.FPM_EINVAL
    assert libfpm.fpm_kdk_adj(None, None, None, None, 1, None, None, None, None) == binding.FPM_EINVAL
    assert libfpm.fpm_set_force_kernel(None, binding.GREENS["discrete"], binding.GRADIENTS["exact"]) == binding.FPM_EINVAL
    assert libfpm.fpm_set_pyramid(None, 2, 2, 16) == binding.FPM_EINVAL
    assert libfpm.fpm_adam_step(None, None, None, None, None, 8, 1.0, 1.0, 0.01, 0.9, 0.999, 1e-8, 1, None,
                                None) == binding.FPM_EINVAL
    libfpm.fpm_plan_destroy(None)


def test_no_cpu_fallback_without_device(libfpm):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    h = ctypes.c_void_p()
    c = binding.fpm_cosmo(0.3075, 0.0486, 0.6774, 0.9667, 0.8159, 2.7255)
    assert libfpm.fpm_plan_create(ctypes.byref(h), 32, 32, 100.0, ctypes.byref(c), None) == binding.FPM_ECUDA
