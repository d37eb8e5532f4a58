"""Thin Python binding of libfpm's C ABI (argument marshalling only).

Every method maps onto one ``fpm_*`` entry point of ``include/fpm.h`` with
the same name.  PyTorch provides device memory and the current CUDA stream;
all arithmetic runs in the library's CUDA kernels.  There is no CPU path:
importing this module without the built library, or calling it without a
CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

_LIB = None
_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfpm.so")

FPM_OK, FPM_EINVAL, FPM_ENOMEM, FPM_ECUDA, FPM_ETIMEOUT, FPM_EDEVICE, FPM_ENOTIMPL = 0, -1, -2, -3, -4, -5, -6

EXPORTS = [
    "fpm_plan_create", "fpm_plan_destroy", "fpm_plan_scratch_bytes", "fpm_growth", "fpm_linear_field",
    "fpm_lpt", "fpm_paint", "fpm_force", "fpm_readout", "fpm_kdk", "fpm_power", "fpm_status", "fpm_strerror",
    "fpm_profile", "fpm_profile_read", "fpm_kernel_class_name", "fpm_launch_count", "fpm_paint_noalloc",
    "fpm_chi2", "fpm_paint_adj", "fpm_readout_adj", "fpm_force_adj", "fpm_kdk_adj", "fpm_lpt_adj",
    "fpm_linear_field_adj", "fpm_batch_create", "fpm_batch_destroy", "fpm_batch_configure", "fpm_batch_kdk",
    "fpm_batch_status", "fpm_batch_info", "fpm_batch_phase_times", "fpm_batch_tune", "fpm_adam_step", "fpm_set_force_kernel", "fpm_set_pyramid", "fpm_set_pyramid_reading",
]
GREENS = {"naive": 0, "discrete": 1}     # FPM_GREEN_NAIVE, FPM_GREEN_DISCRETE (Eq. 4)
GRADIENTS = {"fd4": 0, "exact": 1}       # FPM_GRAD_FD4 (Eq. 5), FPM_GRAD_EXACT
PYR_BANDPASS = {"block": 0, "global": 1}
BATCH_KNOBS = {"readout": 0, "paint_tile": 1, "fft_slots": 2}   # FPM_BTUNE_*
BATCH_PHASES = ("keys", "kdk", "scan", "scatter", "paint", "halo", "z_r2c", "y_fwd", "x_green", "y_inv", "z_c2r",
                "gradient", "kdk_last")     # FPM_BPH_* order
PYR_KERNEL = {"matched": 0, "coarse": 1}
FPM_K_COUNT = 20


class FpmError(RuntimeError):
    def __init__(self, fn: str, code: int):
        msg = lib().fpm_strerror(code).decode()
        super().__init__(f"{fn} failed: {msg} ({code})")
        self.code = code


class fpm_cosmo(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("omega_m", "omega_b", "h", "n_s", "sigma8", "t_cmb")]


def lib() -> ctypes.CDLL:
    """Load libfpm.so (built in-tree by ``build.build()``); raise if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfpm.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    L.fpm_plan_create.argtypes = [ctypes.POINTER(vp), i, i, d, ctypes.POINTER(fpm_cosmo), vp]
    L.fpm_plan_destroy.argtypes = [vp]
    L.fpm_plan_destroy.restype = None
    L.fpm_plan_scratch_bytes.argtypes = [vp]
    L.fpm_plan_scratch_bytes.restype = i64
    L.fpm_growth.argtypes = [vp, vp, i, vp, vp]
    L.fpm_linear_field.argtypes = [vp, vp, vp, vp]
    L.fpm_lpt.argtypes = [vp, vp, d, i, vp, vp, vp]
    L.fpm_paint.argtypes = [vp, vp, vp, vp, vp, vp]
    L.fpm_force.argtypes = [vp, vp, vp, vp]
    L.fpm_readout.argtypes = [vp, vp, vp, vp, vp]
    L.fpm_kdk.argtypes = [vp, vp, vp, vp, i, vp, vp, vp]
    L.fpm_force_ckpt_floats.argtypes = [vp]
    L.fpm_force_ckpt_floats.restype = i64
    L.fpm_power.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.fpm_status.argtypes = [vp, vp]
    L.fpm_strerror.argtypes = [i]
    L.fpm_strerror.restype = ctypes.c_char_p
    L.fpm_profile.argtypes = [vp, i]
    L.fpm_profile_read.argtypes = [vp, vp, vp, i, vp]
    L.fpm_kernel_class_name.argtypes = [i]
    L.fpm_kernel_class_name.restype = ctypes.c_char_p
    L.fpm_launch_count.argtypes = []
    L.fpm_launch_count.restype = i64
    L.fpm_paint_noalloc.argtypes = [i, i, vp, vp, vp]
    L.fpm_chi2.argtypes = [vp, vp, vp, d, vp, vp, vp]
    L.fpm_adam_step.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int64, d, d, d, d, d, d, ctypes.c_int, vp, vp]
    L.fpm_set_force_kernel.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.fpm_set_pyramid.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.fpm_set_pyramid_reading.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.fpm_paint_adj.argtypes = [vp, vp, vp, vp, vp]
    L.fpm_readout_adj.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.fpm_force_adj.argtypes = [vp, vp, vp, vp]
    L.fpm_kdk_adj.argtypes = [vp, vp, vp, vp, i, vp, vp, vp, vp]
    L.fpm_lpt_adj.argtypes = [vp, vp, d, i, vp, vp, vp, vp]
    L.fpm_linear_field_adj.argtypes = [vp, vp, vp, vp]
    L.fpm_batch_create.argtypes = [ctypes.POINTER(vp), vp, i]
    L.fpm_batch_destroy.argtypes = [vp]
    L.fpm_batch_destroy.restype = None
    L.fpm_batch_configure.argtypes = [vp, i, i, i64]
    L.fpm_batch_kdk.argtypes = [vp, vp, vp, vp, i, vp]
    L.fpm_batch_status.argtypes = [vp, vp]
    L.fpm_batch_info.argtypes = [vp, vp, vp]
    L.fpm_batch_phase_times.argtypes = [vp, vp, ctypes.c_int, vp]
    L.fpm_batch_tune.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    for name in EXPORTS:
        if name not in ("fpm_plan_destroy", "fpm_plan_scratch_bytes", "fpm_strerror", "fpm_kernel_class_name",
                        "fpm_launch_count", "fpm_batch_destroy"):
            getattr(L, name).restype = i
    _LIB = L
    return L


def _check(fn: str, code: int):
    if code != FPM_OK:
        raise FpmError(fn, code)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("libfpm takes contiguous CUDA tensors")
    return t.data_ptr()


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _host_f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Plan:
    """An fpm_plan: np^3 particles on an nc^3 mesh in a periodic box (Mpc/h)."""

    def __init__(self, np_: int, nc: int, box: float, cosmo: dict, stream=None):
        import torch
        self.np, self.nc, self.box, self.cosmo = int(np_), int(nc), float(box), dict(cosmo)
        self.N, self.M = self.np ** 3, self.nc ** 3
        self.device = torch.device("cuda", torch.cuda.current_device())
        c = fpm_cosmo(**{k: float(cosmo[k]) for k in ("omega_m", "omega_b", "h", "n_s", "sigma8", "t_cmb")})
        h = ctypes.c_void_p()
        _check("fpm_plan_create", lib().fpm_plan_create(ctypes.byref(h), self.np, self.nc, self.box,
                                                         ctypes.byref(c), _stream(stream)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().fpm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # allocation helpers (torch owns the memory) ---------------------------
    def _empty(self, *shape, dtype=None):
        import torch
        return torch.empty(*shape, dtype=dtype or torch.float32, device=self.device)

    def spectrum_shape(self, n=None):
        n = n or self.np
        return (n, n // 2 + 1, n)

    # entry points ----------------------------------------------------------
    def scratch_bytes(self) -> int:
        return int(lib().fpm_plan_scratch_bytes(self._h))

    def growth(self, a, stream=None) -> np.ndarray:
        a = _host_f64(a).ravel()
        out = np.empty((a.size, 5))
        _check("fpm_growth", lib().fpm_growth(self._h, a.ctypes.data, a.size, out.ctypes.data, _stream(stream)))
        return out

    def linear_field(self, white, lin_k=None, stream=None):
        import torch
        lin_k = lin_k if lin_k is not None else self._empty(self.spectrum_shape(), dtype=torch.complex64)
        _check("fpm_linear_field", lib().fpm_linear_field(self._h, _ptr(white), _ptr(lin_k), _stream(stream)))
        return lin_k

    def lpt(self, lin_k, a0: float, order: int = 2, dx=None, p=None, stream=None):
        dx = dx if dx is not None else self._empty(3, self.N)
        p = p if p is not None else self._empty(3, self.N)
        _check("fpm_lpt", lib().fpm_lpt(self._h, _ptr(lin_k), float(a0), int(order), _ptr(dx), _ptr(p),
                                        _stream(stream)))
        return dx, p

    def paint(self, dx, rho=None, keys=False, perm=False, stream=None):
        import torch
        rho = rho if rho is not None else self._empty(self.nc, self.nc, self.nc)
        k = self._empty(self.N, dtype=torch.int32) if keys else None
        q = self._empty(self.N, dtype=torch.int32) if perm else None
        _check("fpm_paint", lib().fpm_paint(self._h, _ptr(dx), _ptr(rho), _ptr(k), _ptr(q), _stream(stream)))
        if keys or perm:
            return rho, k, q
        return rho

    def set_force_kernel(self, green="naive", gradient="fd4"):
        """Green's function ("naive" or Eq. 4's "discrete") and gradient
        ("fd4", Eq. 5, or "exact") of every later force evaluation."""
        _check("fpm_set_force_kernel", lib().fpm_set_force_kernel(self._h, GREENS[green], GRADIENTS[gradient]))

    def set_pyramid(self, levels=2, split=2, halo=16):
        """Multi-grid pyramid force (Algorithm 3) for later force evaluations;
        levels=0 switches it off."""
        _check("fpm_set_pyramid", lib().fpm_set_pyramid(self._h, int(levels), int(split), int(halo)))

    def set_pyramid_reading(self, bandpass="block", coarse_kernel="matched"):
        """Reading of Algorithm 3 for the pyramid force: the short-range
        band-pass on each padded "block" or on the assembled ("global") mesh,
        and the coarse mesh's operator "matched" to the fine mesh or Eq. 5 in
        "coarse" cell units."""
        _check("fpm_set_pyramid_reading", lib().fpm_set_pyramid_reading(
            self._h, PYR_BANDPASS[bandpass], PYR_KERNEL[coarse_kernel]))

    def force(self, rho, F=None, stream=None):
        F = F if F is not None else self._empty(3, self.nc, self.nc, self.nc)
        _check("fpm_force", lib().fpm_force(self._h, _ptr(rho), _ptr(F), _stream(stream)))
        return F

    def readout(self, F, dx, f_out=None, stream=None):
        f_out = f_out if f_out is not None else self._empty(3, self.N)
        _check("fpm_readout", lib().fpm_readout(self._h, _ptr(F), _ptr(dx), _ptr(f_out), _stream(stream)))
        return f_out

    def kdk(self, dx, p, a, ckpt=None, fckpt=None, stream=None):
        """KDK steps over the scale factors a; ckpt [len(a), 3, N] receives dx
        at every stage, fckpt [len(a), force_ckpt_floats] the force meshes and
        tile buckets."""
        a = _host_f64(a).ravel()
        _check("fpm_kdk", lib().fpm_kdk(self._h, _ptr(dx), _ptr(p), a.ctypes.data, a.size - 1, _ptr(ckpt),
                                        _ptr(fckpt), _stream(stream)))
        return dx, p

    @property
    def force_ckpt_floats(self) -> int:
        """Floats per stage of a force checkpoint (the force mesh, 4 nc^3, and
        the stage's tile buckets)."""
        return int(lib().fpm_force_ckpt_floats(self._h))

    def power(self, a, b=None, stream=None) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        nb = self.nc // 2
        pk, km, nm = np.empty(nb), np.empty(nb), np.empty(nb)
        _check("fpm_power", lib().fpm_power(self._h, _ptr(a), _ptr(b), pk.ctypes.data, km.ctypes.data,
                                            nm.ctypes.data, _stream(stream)))
        return km, pk, nm

    def status(self, stream=None) -> int:
        return int(lib().fpm_status(self._h, _stream(stream)))

    def profile(self, enable: bool = True, only: str = None):
        """Per-class device timing on or off; `only` (a class name) times
        that class's launches alone."""
        code = int(bool(enable))
        if enable and only is not None:
            names = [lib().fpm_kernel_class_name(k).decode() for k in range(FPM_K_COUNT)]
            code = 2 + names.index(only)
        _check("fpm_profile", lib().fpm_profile(self._h, code))

    def profile_read(self, stream=None) -> dict:
        """{class name: (ms, launches)} accumulated since the last read."""
        ms = np.zeros(FPM_K_COUNT)
        cnt = np.zeros(FPM_K_COUNT, dtype=np.int64)
        _check("fpm_profile_read", lib().fpm_profile_read(self._h, ms.ctypes.data, cnt.ctypes.data, FPM_K_COUNT,
                                                          _stream(stream)))
        return {lib().fpm_kernel_class_name(k).decode(): (float(ms[k]), int(cnt[k]))
                for k in range(FPM_K_COUNT) if cnt[k]}

    # adjoints -----------------------------------------------------------------
    def chi2(self, rho, target_delta, sigma=1.0, g_rho=None, want_grad=True, stream=None):
        """(loss, g_rho) of sum (rho - 1 - target)^2 / sigma^2."""
        if want_grad and g_rho is None:
            g_rho = self._empty(self.nc, self.nc, self.nc)
        loss = ctypes.c_double()
        _check("fpm_chi2", lib().fpm_chi2(self._h, _ptr(rho), _ptr(target_delta), float(sigma),
                                          _ptr(g_rho) if want_grad else None, ctypes.byref(loss), _stream(stream)))
        return loss.value, g_rho

    def adam_step(self, x, g, m, v, t, lr=0.01, betas=(0.9, 0.999), eps=1e-8, gscale=1.0, pscale=0.0,
                  want_prior=True, stream=None):
        """One Adam update of x in place with the gradient gscale g + pscale x
        (Eq. 12's prior on the white noise); returns sum(x^2)/2 before it."""
        prior = ctypes.c_double()
        _check("fpm_adam_step", lib().fpm_adam_step(self._h, _ptr(x), _ptr(g), _ptr(m), _ptr(v), int(x.numel()),
                                                    float(gscale), float(pscale), float(lr), float(betas[0]),
                                                    float(betas[1]), float(eps), int(t),
                                                    ctypes.byref(prior) if want_prior else None, _stream(stream)))
        return prior.value if want_prior else None

    def paint_adj(self, dx, g_rho, g_dx=None, stream=None):
        g_dx = g_dx if g_dx is not None else self._empty(3, self.N)
        _check("fpm_paint_adj", lib().fpm_paint_adj(self._h, _ptr(dx), _ptr(g_rho), _ptr(g_dx), _stream(stream)))
        return g_dx

    def readout_adj(self, F, dx, g_f, stream=None):
        g_F = self._empty(3, self.nc, self.nc, self.nc)
        g_dx = self._empty(3, self.N)
        _check("fpm_readout_adj", lib().fpm_readout_adj(self._h, _ptr(F), _ptr(dx), _ptr(g_f), _ptr(g_F),
                                                        _ptr(g_dx), _stream(stream)))
        return g_F, g_dx

    def force_adj(self, g_F, g_rho=None, stream=None):
        g_rho = g_rho if g_rho is not None else self._empty(self.nc, self.nc, self.nc)
        _check("fpm_force_adj", lib().fpm_force_adj(self._h, _ptr(g_F), _ptr(g_rho), _stream(stream)))
        return g_rho

    def kdk_adj(self, ckpt, a, g_dx, g_p_in=None, g_p=None, fckpt=None, stream=None):
        """Cotangents of the initial (dx, p) from those of the final ones
        (g_p_in None: the loss does not depend on the final momenta); fckpt:
        the forward's force checkpoints (None: recompute the forces)."""
        a = _host_f64(a).ravel()
        g_p = g_p if g_p is not None else self._empty(3, self.N)
        _check("fpm_kdk_adj", lib().fpm_kdk_adj(self._h, _ptr(ckpt), _ptr(fckpt), a.ctypes.data, a.size - 1,
                                                _ptr(g_dx), _ptr(g_p_in), _ptr(g_p), _stream(stream)))
        return g_dx, g_p

    def lpt_adj(self, lin_k, a0, g_dx, g_p, order=2, g_lin_k=None, stream=None):
        import torch
        g_lin_k = g_lin_k if g_lin_k is not None else self._empty(self.spectrum_shape(), dtype=torch.complex64)
        _check("fpm_lpt_adj", lib().fpm_lpt_adj(self._h, _ptr(lin_k), float(a0), int(order), _ptr(g_dx), _ptr(g_p),
                                                _ptr(g_lin_k), _stream(stream)))
        return g_lin_k

    def linear_field_adj(self, g_lin_k, g_white=None, stream=None):
        g_white = g_white if g_white is not None else self._empty(self.np, self.np, self.np)
        _check("fpm_linear_field_adj", lib().fpm_linear_field_adj(self._h, _ptr(g_lin_k), _ptr(g_white),
                                                                  _stream(stream)))
        return g_white

    # a whole forward model (Algorithm 4 + KDK) ------------------------------
    def simulate(self, white, a, order: int = 2, ckpt=None, stream=None):
        lin_k = self.linear_field(white, stream=stream)
        dx, p = self.lpt(lin_k, float(a[0]), order, stream=stream)
        self.kdk(dx, p, a, ckpt=ckpt, stream=stream)
        return dx, p, lin_k


class Batch:
    """An fpm_batch: independent simulations (one Plan each) advanced by one
    persistent launch per KDK step, graph-captured."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        _check("fpm_batch_create", lib().fpm_batch_create(ctypes.byref(h), arr, len(self.plans)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().fpm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, blocks_per_sm=-1, readout_chunks=-1, spin_limit=-1):
        _check("fpm_batch_configure", lib().fpm_batch_configure(self._h, int(blocks_per_sm), int(readout_chunks),
                                                                int(spin_limit)))

    def kdk(self, dxs, ps, a, stream=None):
        a = _host_f64(a).ravel()
        dptr = (ctypes.c_void_p * len(dxs))(*[_ptr(x) for x in dxs])
        pptr = (ctypes.c_void_p * len(ps))(*[_ptr(x) for x in ps])
        _check("fpm_batch_kdk", lib().fpm_batch_kdk(self._h, dptr, pptr, a.ctypes.data, a.size - 1,
                                                    _stream(stream)))

    def status(self, stream=None) -> int:
        return int(lib().fpm_batch_status(self._h, _stream(stream)))

    def tune(self, nc: int, knob: str, value: int):
        """Per-mesh-size layout of the batched step: knob "readout" (0 chunks,
        1 bricks 32 in z, 2 bricks 64 in z), "paint_tile" (8 or 16) or
        "fft_slots" (8 or 16), for every simulation of mesh nc."""
        _check("fpm_batch_tune", lib().fpm_batch_tune(self._h, int(nc), BATCH_KNOBS[knob], int(value)))

    def phase_times(self, stream=None) -> dict:
        """{phase: device ms} accumulated over the batched runs since the last read."""
        ms = np.zeros(len(BATCH_PHASES))
        _check("fpm_batch_phase_times", lib().fpm_batch_phase_times(self._h, ms.ctypes.data, len(BATCH_PHASES),
                                                                    _stream(stream)))
        return dict(zip(BATCH_PHASES, ms.tolist()))

    def info(self) -> dict:
        g, c = ctypes.c_int(), ctypes.c_int()
        _check("fpm_batch_info", lib().fpm_batch_info(self._h, ctypes.byref(g), ctypes.byref(c)))
        return {"grid_blocks": g.value, "graph_captured": bool(c.value)}


def paint_noalloc(np_: int, nc: int, dx, rho, stream=None):
    """fpm_paint_noalloc: the CIC paint for callers that cannot allocate
    device memory (no plan; fixed scratch inside the library, np, nc <= 64).
    The caller passes both device buffers; nothing is allocated here."""
    _check("fpm_paint_noalloc", lib().fpm_paint_noalloc(int(np_), int(nc), _ptr(dx), _ptr(rho), _stream(stream)))
    return rho


def launch_count() -> int:
    """Kernels launched by libfpm in this process so far."""
    return int(lib().fpm_launch_count())


def spectrum_to_numpy_layout(spec):
    """[kx][kz][ky] half spectrum -> numpy rfftn layout [kx][ky][kz]."""
    return spec.permute(0, 2, 1)
