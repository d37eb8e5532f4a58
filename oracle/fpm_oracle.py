"""Plain FP64 CPU oracle of the FastPM particle-mesh loop as FlowPM states it.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or
executes this module: only the tests, the package entry's smoke check and the
bench's CPU-baseline leg do.  It shares no code with the CUDA path; the two
meet only through the seeded arrays of ``paper_2010_11847_gb300.inputs``.

Every function follows one passage of the paper (Modi, Lanusse & Seljak,
"FlowPM: Distributed TensorFlow implementation of the FastPM cosmological
N-body solver") or, where the paper defers to FastPM (Feng et al. 2016) or to
Eisenstein & Hu (1998), the published equations of those papers.  It is
written for reading, not speed: library FFTs serve as steps, nothing is fused.

Units.  Positions, displacements, momenta and forces are in mesh-cell units
(x0 = L/Nc = 1) and time in 1/H0, so that the force operator of Eq. 3-5 is
box-independent; the box size enters only through the linear power spectrum.

Conventions (the paper is silent on these; each is a stated reading):
  * forward DFT unnormalised with e^{-ik.x}; inverse carries 1/N^3;
  * mesh nodes at integer coordinates, CIC weights (1-t, t) per axis;
  * particle i = (ix*Np + iy)*Np + iz sits on lattice node q = (ix,iy,iz)*Nc/Np;
  * mass per particle m = (Nc/Np)^3 so the mean density is 1 and delta = rho-1;
  * cell key: tile-major with 16^3-cell tiles (see ``cell_keys``);
  * sort order: by key, ties by Lagrangian index (stable).
"""
from __future__ import annotations

import functools
import math

import numpy as np

FFT_WORKERS = -1   # threads of the library FFT (-1: all host cores)

try:                                     # multithreaded pocketfft if present
    import scipy.fft as _fft

    def _rfftn(a):
        return _fft.rfftn(a, workers=FFT_WORKERS)

    def _irfftn(a, n):
        return _fft.irfftn(a, s=(n, n, n), workers=FFT_WORKERS)
except ImportError:                      # pragma: no cover
    def _rfftn(a):
        return np.fft.rfftn(a)

    def _irfftn(a, n):
        return np.fft.irfftn(a, s=(n, n, n))

TILE = 16          # cells per tile edge in the cell key
GROWTH_A_INIT = 1e-5
GROWTH_RK4_STEPS = 20000


# ---------------------------------------------------------------------------
# Background cosmology and growth (FastPM time stepping, Sec. 2, deferred to
# Feng et al. 2016): flat LCDM, no radiation, w = -1.
# ---------------------------------------------------------------------------
def hubble_E(a, omega_m):
    """E(a) = H(a)/H0 = sqrt(Om a^-3 + 1 - Om)."""
    a = np.asarray(a, dtype=np.float64)
    return np.sqrt(omega_m * a ** -3 + (1.0 - omega_m))


def _growth_rhs(lna, y, omega_m):
    """Growth ODEs in ln a for y = [D1, D1', D2, D2'] (' = d/dln a):
         D1'' + (2 + dlnE/dlna) D1' - 1.5 Om(a) D1 = 0
         D2'' + (2 + dlnE/dlna) D2' - 1.5 Om(a) D2 = -1.5 Om(a) D1^2
    """
    a = np.exp(lna)
    E2 = omega_m * a ** -3 + (1.0 - omega_m)
    om_a = omega_m * a ** -3 / E2
    dlnE = -1.5 * om_a
    d1, d1p, d2, d2p = y
    return np.array([
        d1p,
        -(2.0 + dlnE) * d1p + 1.5 * om_a * d1,
        d2p,
        -(2.0 + dlnE) * d2p + 1.5 * om_a * d2 - 1.5 * om_a * d1 * d1,
    ])


def _growth_raw(a_targets, omega_m):
    """Integrate the growth ODEs with RK4 (uniform steps in ln a) from
    a_i = 1e-5, where D1 = a and D2 = -3/7 a^2 (growing modes), to each
    target; returns the raw state, shape (4, len(a))."""
    a_t = np.atleast_1d(np.asarray(a_targets, dtype=np.float64))
    lna0 = math.log(GROWTH_A_INIT)
    h = (np.log(a_t) - lna0) / GROWTH_RK4_STEPS          # one step size per target
    ai = GROWTH_A_INIT
    y = np.array([np.full_like(a_t, ai), np.full_like(a_t, ai),
                  np.full_like(a_t, -3.0 / 7.0 * ai ** 2),
                  np.full_like(a_t, -6.0 / 7.0 * ai ** 2)])
    lna = np.full_like(a_t, lna0)
    for _ in range(GROWTH_RK4_STEPS):
        k1 = _growth_rhs(lna, y, omega_m)
        k2 = _growth_rhs(lna + 0.5 * h, y + 0.5 * h * k1, omega_m)
        k3 = _growth_rhs(lna + 0.5 * h, y + 0.5 * h * k2, omega_m)
        k4 = _growth_rhs(lna + h, y + h * k3, omega_m)
        y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        lna = lna + h
    return y


@functools.lru_cache(maxsize=256)
def _growth_raw_cached(a_targets, omega_m):
    """_growth_raw memoised on its (hashable) arguments; same arithmetic."""
    out = _growth_raw(np.array(a_targets), omega_m)
    out.setflags(write=False)
    return out


def growth(a, omega_m):
    """Normalised growth quantities at scale factors a.

    D1 is normalised to D1(1) = 1 and D2 to D2 / D1_raw(1)^2, so that
    D2 ~ -3/7 D1^2 in the same normalisation.  Returns a dict of arrays:
    D1, D2, f1 = dlnD1/dlna, f2 = dlnD2/dlna, dD1da = dD1/da, E.
    """
    a = np.atleast_1d(np.asarray(a, dtype=np.float64))
    raw = _growth_raw_cached(tuple(np.concatenate([a, [1.0]]).tolist()), float(omega_m))
    norm = raw[0, -1]
    d1, d1p, d2, d2p = raw[:, :-1]
    return dict(
        D1=d1 / norm,
        D2=d2 / norm ** 2,
        f1=d1p / d1,
        f2=d2p / d2,
        dD1da=d1p / norm / a,
        E=hubble_E(a, omega_m),
    )


def fastpm_factors(stages, omega_m):
    """FastPM drift and kick factors for KDK steps between the given scale
    factors (Eqs. 1-2 with the growth-factor modification of Feng et al.).

    With G_p = D1, g_p = dD1/da, G_f = a^3 E dD1/da and
    g_f = dG_f/da = 1.5 Om D1 / (a^2 E):
      drift a_i -> a_f using p at a_c:  dx += p (G_p(a_f)-G_p(a_i)) / (a_c^3 E(a_c) g_p(a_c))
      kick  a_i -> a_f using f at a_c:  p  += f (G_f(a_f)-G_f(a_i)) / (a_c^2 E(a_c) g_f(a_c))
    Step k: kick a_k -> a_h (force at a_k), drift a_k -> a_{k+1} (p at a_h),
    kick a_h -> a_{k+1} (force at a_{k+1}), with a_h = sqrt(a_k a_{k+1}).

    Returns arrays kick1[k], drift[k], kick2[k] for k = 0..n-1.
    """
    a = np.asarray(stages, dtype=np.float64)
    n = len(a) - 1
    ah = np.sqrt(a[:-1] * a[1:])
    pts = np.concatenate([a, ah])
    g = growth(pts, omega_m)
    D1, dD1da, E = g["D1"], g["dD1da"], g["E"]
    Gp = D1
    gp = dD1da
    Gf = pts ** 3 * E * dD1da
    gf = 1.5 * omega_m * D1 / (pts ** 2 * E)
    ik = np.arange(n)                 # index of a_k
    ik1 = ik + 1                      # index of a_{k+1}
    ih = n + 1 + ik                   # index of a_h
    kick1 = (Gf[ih] - Gf[ik]) / (pts[ik] ** 2 * E[ik] * gf[ik])
    drift = (Gp[ik1] - Gp[ik]) / (pts[ih] ** 3 * E[ih] * gp[ih])
    kick2 = (Gf[ik1] - Gf[ih]) / (pts[ik1] ** 2 * E[ik1] * gf[ik1])
    return kick1, drift, kick2


# ---------------------------------------------------------------------------
# Linear power spectrum: Eisenstein & Hu (1998) no-wiggle transfer function
# (their eqs. 26, 28-31), normalised to sigma8.
# ---------------------------------------------------------------------------
def eh_nowiggle_transfer(k_h, cosmo):
    """T(k) for k in h/Mpc."""
    om, ob, h = cosmo["omega_m"], cosmo["omega_b"], cosmo["h"]
    theta = cosmo["t_cmb"] / 2.7
    wm, wb = om * h * h, ob * h * h
    fb = ob / om
    s = 44.5 * np.log(9.83 / wm) / np.sqrt(1.0 + 10.0 * wb ** 0.75)         # Mpc
    alpha = 1.0 - 0.328 * np.log(431.0 * wm) * fb + 0.38 * np.log(22.3 * wm) * fb * fb
    k_mpc = np.asarray(k_h, dtype=np.float64) * h
    gamma_eff = om * h * (alpha + (1.0 - alpha) / (1.0 + (0.43 * k_mpc * s) ** 4))
    q = np.asarray(k_h, dtype=np.float64) * theta * theta / gamma_eff
    L0 = np.log(2.0 * math.e + 1.8 * q)
    C0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
    return L0 / (L0 + C0 * q * q)


def tophat_window(x):
    """W(x) = 3 (sin x - x cos x) / x^3, the Fourier transform of a sphere."""
    x = np.asarray(x, dtype=np.float64)
    return 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3


def sigma8_unnormalised(cosmo, amplitude=1.0, npts=4097):
    """sigma(R = 8 Mpc/h) of P = A k^ns T^2: sqrt(int k^3 P W^2 dlnk / 2pi^2),
    Simpson's rule on a uniform ln k grid from 1e-5 to 1e2 h/Mpc."""
    lnk = np.linspace(math.log(1e-5), math.log(1e2), npts)
    k = np.exp(lnk)
    integrand = k ** 3 * amplitude * k ** cosmo["n_s"] * eh_nowiggle_transfer(k, cosmo) ** 2 \
        * tophat_window(8.0 * k) ** 2 / (2.0 * math.pi ** 2)
    dl = lnk[1] - lnk[0]
    w = np.ones(npts)
    w[1:-1:2] = 4.0
    w[2:-1:2] = 2.0
    return math.sqrt(dl / 3.0 * float(np.dot(w, integrand)))


def pk_amplitude(cosmo):
    """Amplitude A with sigma8(A) equal to cosmo['sigma8']."""
    s = sigma8_unnormalised(cosmo, 1.0)
    return (cosmo["sigma8"] / s) ** 2


def linear_pk(k_h, cosmo, amplitude=None):
    """P(k) = A k^ns T(k)^2 in (Mpc/h)^3 for k in h/Mpc."""
    if amplitude is None:
        amplitude = pk_amplitude(cosmo)
    k_h = np.asarray(k_h, dtype=np.float64)
    return amplitude * k_h ** cosmo["n_s"] * eh_nowiggle_transfer(k_h, cosmo) ** 2


# ---------------------------------------------------------------------------
# Fourier-space helpers
# ---------------------------------------------------------------------------
def _freq_int(n):
    """Integer frequencies of an n-point DFT: 0..n/2-1, -n/2..-1."""
    return np.fft.fftfreq(n, d=1.0 / n).round().astype(np.int64)


def half_spectrum_wavenumbers(n):
    """Integer wave vectors (nx, ny, nz) of an rfftn half spectrum, shape
    broadcastable to (n, n, n//2+1)."""
    f = _freq_int(n)
    fz = np.arange(n // 2 + 1, dtype=np.int64)
    return f[:, None, None], f[None, :, None], fz[None, None, :]


def fd_gradient_kernel(n):
    """Eq. 5: the FastPM 4th-order finite-difference derivative in cell units,
    g(w) = (8 sin w - sin 2w)/6 with w = 2 pi n_d / N.  At the Nyquist
    frequency w = -pi the exact value is 0 and is set so."""
    f = _freq_int(n)
    w = 2.0 * math.pi * f / n
    g = (8.0 * np.sin(w) - np.sin(2.0 * w)) / 6.0
    g[f == -n // 2] = 0.0
    return g


def fd_gradient_kernel_half(n):
    """Eq. 5 on the last (half) axis, frequencies 0..n/2."""
    fz = np.arange(n // 2 + 1)
    w = 2.0 * math.pi * fz / n
    g = (8.0 * np.sin(w) - np.sin(2.0 * w)) / 6.0
    g[fz == n // 2] = 0.0
    return g


def exact_gradient_kernel(n):
    """The exact derivative of the band-limited interpolant, i w with
    w = 2 pi n_d / N in cell units.  At the Nyquist frequency a real field's
    derivative has no real representative, so the value there is set to 0
    (the force variant of Sec. 2 with the continuous i k)."""
    f = _freq_int(n)
    w = 2.0 * math.pi * f / n
    w[f == -n // 2] = 0.0
    return w


def exact_gradient_kernel_half(n):
    """``exact_gradient_kernel`` on the last (half) axis, frequencies 0..n/2."""
    fz = np.arange(n // 2 + 1)
    w = 2.0 * math.pi * fz / n
    w[fz == n // 2] = 0.0
    return w


GRADIENTS = ("fd4", "exact")     # Eq. 5's four-point difference; the exact i k
GREENS = ("naive", "discrete")   # -1/k^2; Eq. 4's discrete Laplacian


def _gradient_kernels(n, gradient="fd4"):
    if gradient == "fd4":
        g, gz = fd_gradient_kernel(n), fd_gradient_kernel_half(n)
    elif gradient == "exact":
        g, gz = exact_gradient_kernel(n), exact_gradient_kernel_half(n)
    else:
        raise ValueError(gradient)
    return g[:, None, None], g[None, :, None], gz[None, None, :]


def _laplacian_naive(n):
    """|w|^2 = sum_d (2 pi n_d / N)^2, the naive -1/k^2 Green's function's
    denominator in cell units."""
    nx, ny, nz = half_spectrum_wavenumbers(n)
    c = 2.0 * math.pi / n
    return (c * nx) ** 2 + (c * ny) ** 2 + (c * nz) ** 2


def _laplacian_discrete(n):
    """Eq. 4's denominator: sum_d (w_d sinc(w_d / 2))^2 = sum_d (2 sin(w_d / 2))^2
    (sinc x = sin x / x), the symbol of the seven-point discrete Laplacian in
    cell units (x0 = 1)."""
    nx, ny, nz = half_spectrum_wavenumbers(n)
    c = math.pi / n
    return sum((2.0 * np.sin(c * v)) ** 2 for v in (nx, ny, nz))


def _laplacian(n, green="naive"):
    if green == "naive":
        return _laplacian_naive(n)
    if green == "discrete":
        return _laplacian_discrete(n)
    raise ValueError(green)


# ---------------------------------------------------------------------------
# Initial conditions (Algorithm 4)
# ---------------------------------------------------------------------------
def linear_field(white, box, cosmo):
    """Algorithm 4, steps 1-2: scale white noise by the power spectrum.

    delta_L(k) = FFT(w)(k) * sqrt(P(|k|) N^3 / V), k = 2 pi n / L, with the
    k = 0 mode set to zero.  The result is the unnormalised DFT of the real
    linear density field (so <|delta_L(k)|^2> = N^6 P / V), rfftn layout.
    """
    n = white.shape[0]
    W = _rfftn(np.asarray(white, dtype=np.float64))
    nx, ny, nz = half_spectrum_wavenumbers(n)
    kmag = 2.0 * math.pi / box * np.sqrt((nx * nx + ny * ny + nz * nz).astype(np.float64))
    with np.errstate(divide="ignore", invalid="ignore"):
        pk = linear_pk(kmag, cosmo)
    scale = np.sqrt(pk * n ** 3 / box ** 3)
    scale[0, 0, 0] = 0.0
    return W * scale


def lpt_fields(lin_k):
    """Lagrangian displacement fields of 1st and 2nd order on the particle
    lattice, in lattice units (Algorithm 4 step 3 uses the force kernels; the
    2LPT extension follows the figure caption of the LPT scaling test).

      phi1 = -delta_L/|w|^2            (so that lap phi1 = delta_L)
      Psi1 = -grad phi1                 -> Psi1_d(k) = i g_d delta_L / |w|^2
      S = sum_{i<j} [phi1,ii phi1,jj - phi1,ij^2],  phi1,ij(k) = g_i g_j delta_L/|w|^2
      phi2 = -S(k)/|w|^2               (so that lap phi2 = S)
      Psi2 = +grad phi2                 -> Psi2_d(k) = i g_d phi2(k)
    Returns (Psi1[3], Psi2[3]) real arrays of shape (3, N, N, N).
    """
    n = lin_k.shape[0]
    g = _gradient_kernels(n)
    k2 = _laplacian_naive(n)
    k2[0, 0, 0] = 1.0
    inv_k2 = 1.0 / k2
    inv_k2[0, 0, 0] = 0.0

    def second_derivative(i, j):
        return _irfftn(g[i] * g[j] * lin_k * inv_k2, n)

    phi = {}
    for i in range(3):
        for j in range(i, 3):
            phi[(i, j)] = second_derivative(i, j)
    S = (phi[(0, 0)] * phi[(1, 1)] + phi[(0, 0)] * phi[(2, 2)] + phi[(1, 1)] * phi[(2, 2)]
         - phi[(0, 1)] ** 2 - phi[(0, 2)] ** 2 - phi[(1, 2)] ** 2)
    phi2_k = -_rfftn(S) * inv_k2
    psi1 = np.stack([_irfftn(1j * g[d] * lin_k * inv_k2, n) for d in range(3)])
    psi2 = np.stack([_irfftn(1j * g[d] * phi2_k, n) for d in range(3)])
    return psi1, psi2


def lpt(lin_k, nc, a0, cosmo, order=2):
    """2LPT (or 1LPT) displacements and momenta at a0 in mesh-cell units.

      dx = D1 Psi1 + D2 Psi2
      p  = a^2 E (f1 D1 Psi1 + f2 D2 Psi2)     (p = a^3 E dx/da)
    evaluated at the lattice nodes and scaled by Nc/Np to mesh cells.
    Returns dx, p of shape (3, Np^3) (Lagrangian order).
    """
    np_ = lin_k.shape[0]
    psi1, psi2 = lpt_fields(lin_k)
    if order == 1:
        psi2 = np.zeros_like(psi2)
    gr = growth([a0], cosmo["omega_m"])
    D1, D2, f1, f2, E = (float(gr[k][0]) for k in ("D1", "D2", "f1", "f2", "E"))
    r = nc / np_
    dx = (D1 * psi1 + D2 * psi2) * r
    p = a0 * a0 * E * (f1 * D1 * psi1 + f2 * D2 * psi2) * r
    return dx.reshape(3, -1), p.reshape(3, -1)


# ---------------------------------------------------------------------------
# CIC paint, keys, sort, readout (Sec. 2, the linear "cloud-in-cell" window)
# ---------------------------------------------------------------------------
def lattice(np_, nc):
    """Lattice node of each particle in mesh cells, integer array (3, Np^3)."""
    r = nc // np_
    i = np.arange(np_ ** 3, dtype=np.int64)
    ix, iy, iz = i // (np_ * np_), (i // np_) % np_, i % np_
    return np.stack([ix * r, iy * r, iz * r])


POSITIONS_FP32 = True    # positions are float32 displacements; False: keep FP64 (derivative pins)


def cic_cells(dx, np_, nc):
    """Base cell and fractional offset of each particle from its float32
    displacement dx (3, N): cell = wrap(q + floor(dx)), t = dx - floor(dx).
    floor() of the float32 value is exact, so the cell is exact."""
    if POSITIONS_FP32:
        dx64 = np.asarray(dx, dtype=np.float32).astype(np.float64)
    else:
        dx64 = np.asarray(dx, dtype=np.float64)
    fl = np.floor(dx64)
    cell = (lattice(np_, nc) + fl.astype(np.int64)) % nc
    t = dx64 - fl
    return cell, t


def cell_keys(cell, nc):
    """Tile-major cell key: the mesh is cut into 16^3-cell tiles ordered
    row-major; cells inside a tile are ordered row-major too.
      key = ((tx*NT + ty)*NT + tz) * 4096 + (lx*16 + ly)*16 + lz
    with t = cell // 16, l = cell % 16, NT = Nc/16."""
    nt = nc // TILE
    t = cell // TILE
    l = cell % TILE
    tile = (t[0] * nt + t[1]) * nt + t[2]
    local = (l[0] * TILE + l[1]) * TILE + l[2]
    return (tile * TILE ** 3 + local).astype(np.uint32)


def sort_order(keys):
    """Stable counting-sort order: by key, ties by Lagrangian index."""
    return np.argsort(keys, kind="stable").astype(np.uint32)


def _corners():
    for bx in (0, 1):
        for by in (0, 1):
            for bz in (0, 1):
                yield bx, by, bz


def _corner_weight(t, b):
    w = np.ones(t.shape[1])
    for d in range(3):
        w = w * (t[d] if b[d] else (1.0 - t[d]))
    return w


def paint_cells(cell, t, weights, nc):
    """rho_c = sum_i weight_i * W(x_i - c) with the CIC window, periodic."""
    rho = np.zeros(nc ** 3)
    for b in _corners():
        c = [(cell[d] + b[d]) % nc for d in range(3)]
        flat = (c[0] * nc + c[1]) * nc + c[2]
        rho += np.bincount(flat, weights=weights * _corner_weight(t, b), minlength=nc ** 3)
    return rho.reshape(nc, nc, nc)


def readout_cells(field, cell, t):
    """f_i = sum_c W(x_i - c) field_c, the same window as the paint."""
    nc = field.shape[-1]
    flat_field = field.reshape(field.shape[:-3] + (-1,))
    out = 0.0
    for b in _corners():
        c = [(cell[d] + b[d]) % nc for d in range(3)]
        flat = (c[0] * nc + c[1]) * nc + c[2]
        out = out + flat_field[..., flat] * _corner_weight(t, b)
    return out


def paint(dx, np_, nc):
    """CIC density of N = Np^3 particles of mass (Nc/Np)^3 (mean 1)."""
    cell, t = cic_cells(dx, np_, nc)
    m = (nc / np_) ** 3
    return paint_cells(cell, t, np.full(cell.shape[1], m), nc)


def readout(F, dx, np_, nc):
    """Force (or any vector field F[3]) read out at the particles, (3, N)."""
    cell, t = cic_cells(dx, np_, nc)
    return readout_cells(F, cell, t)


# ---------------------------------------------------------------------------
# Force (Eqs. 3-5 with the naive Green's function)
# ---------------------------------------------------------------------------
def force_from_delta(delta, omega_m, green="naive", gradient="fd4"):
    """F_d = IFFT( i g_d(w) * 1.5 Om * FFT(delta) / |w|^2 ),  F(k=0) = 0.

    Eq. 3 (f = grad grad^-2 delta) with the Poisson factor and sign of
    F = -grad phi, lap phi = 1.5 Om delta.  Default: grad^-2 is the naive
    -1/k^2 and grad the FD kernel of Eq. 5.  Variants: green="discrete" puts
    Eq. 4's discrete Laplacian in the denominator; gradient="exact" uses
    g_d = w_d (Nyquist 0).  Cell units, H0 = 1.
    """
    n = delta.shape[0]
    dk = _rfftn(delta)
    g = _gradient_kernels(n, gradient)
    k2 = _laplacian(n, green)
    k2[0, 0, 0] = 1.0
    pot = 1.5 * omega_m * dk / k2
    pot[0, 0, 0] = 0.0
    return np.stack([_irfftn(1j * g[d] * pot, n) for d in range(3)])


def force(rho, omega_m, green="naive", gradient="fd4"):
    """Force meshes from a density mesh (delta = rho - 1)."""
    return force_from_delta(np.asarray(rho, dtype=np.float64) - 1.0, omega_m, green, gradient)


def particle_force(dx, np_, nc, omega_m, green="naive", gradient="fd4", pyramid=None):
    """paint -> force -> readout for particles at displacements dx; with
    ``pyramid`` (a dict of ``pyramid_force``'s levels, split, halo) the mesh
    force is Algorithm 3's."""
    rho = paint(dx, np_, nc)
    F = pyramid_force(rho, omega_m, **pyramid) if pyramid else force(rho, omega_m, green, gradient)
    return readout(F, dx, np_, nc)


# ---------------------------------------------------------------------------
# Multi-grid pyramid force (Sec. 3.1 Eqs. 6-9, Algorithms 2-3) on one device
# ---------------------------------------------------------------------------
def bspline_kernel(order=6):
    """The order-`order` discrete B-spline: the box [1/2, 1/2] convolved
    with itself `order` times, i.e. binomial weights C(order, j) / 2^order,
    j = 0..order (7 taps for order 6), centred on tap order/2.  Its symbol
    is cos(w/2)^order."""
    k = np.array([1.0])
    for _ in range(order):
        k = np.convolve(k, [0.5, 0.5])
    return k


def _smooth_periodic(a, k):
    """Periodic convolution of a 3-D field with the separable kernel k x k x k
    (k symmetric, centred): out[x] = sum_j k[j] a[x + j - r] per axis."""
    r = len(k) // 2
    out = np.asarray(a, dtype=np.float64)
    for ax in range(3):
        out = sum(k[j] * np.roll(out, r - j, axis=ax) for j in range(len(k)))
    return out


def reduce_once(h, order=6):
    """Eq. 6, g_{l+1} = S[G * g_l]: smooth with the 3-D B-spline, keep
    every second node along each axis (a stride-2 convolution)."""
    return _smooth_periodic(h, bspline_kernel(order))[::2, ::2, ::2]


def expand_once(d, order=6):
    """Eq. 7, g'_l = G * U[g_{l+1}]: insert zeros between the nodes and
    smooth with 8 times the 3-D B-spline (Algorithm 2's EXPAND kernel), a
    stride-2 transposed convolution."""
    n = d.shape[0]
    u = np.zeros((2 * n,) * 3)
    u[::2, ::2, ::2] = d
    return _smooth_periodic(u, 2.0 * bspline_kernel(order))


def reduce(h, levels=2, order=6):
    """Algorithm 2, REDUCE: `levels` stride-2 B-spline convolutions (two in
    the paper's default, a mesh 4x coarser)."""
    for _ in range(levels):
        h = reduce_once(h, order)
    return h


def expand(d, levels=2, order=6):
    """Algorithm 2, EXPAND: `levels` stride-2 transposed convolutions."""
    for _ in range(levels):
        d = expand_once(d, order)
    return d


def coarse_force(D, omega_m, scale, kernel="matched"):
    """Force meshes, in fine-cell units, of the density contrast D on a
    coarse mesh whose cells are `scale` fine cells (Algorithm 3's ForceGrids
    on the REDUCEd mesh).  kernel="coarse": Eq. 3-5's operator in coarse-cell
    units (naive Green's function, Eq. 5's gradient with w the coarse-mesh
    frequency), times `scale`.  kernel="matched": the fine mesh's operator at
    the same physical wavenumber, i g(w/scale) / (w/scale)^2 with w the
    coarse-mesh frequency, so that the coarse force of a REDUCEd field is the
    REDUCEd fine force (up to aliasing)."""
    if kernel == "coarse":
        return scale * force_from_delta(D, omega_m)
    n = D.shape[0]
    dk = _rfftn(np.asarray(D, dtype=np.float64))
    nx, ny, nz = half_spectrum_wavenumbers(n)
    w = [2.0 * math.pi * a / n / scale for a in (nx, ny, nz)]      # fine-mesh frequency of each mode
    g = [np.where(np.abs(a) == n // 2, 0.0, (8.0 * np.sin(x) - np.sin(2.0 * x)) / 6.0) for a, x in zip((nx, ny, nz), w)]
    k2 = np.broadcast_to(w[0] ** 2 + w[1] ** 2 + w[2] ** 2, dk.shape).copy()
    k2[0, 0, 0] = 1.0
    pot = 1.5 * omega_m * dk / k2
    pot[0, 0, 0] = 0.0
    return np.stack([_irfftn(1j * np.broadcast_to(g[d], dk.shape) * pot, n) for d in range(3)])


def local_force(rho, omega_m, split, halo, bandpass=None):
    """The short-range force grids of Algorithm 3 computed with local FFTs:
    the mesh is cut into split^3 cubic blocks of m = n/split cells; each block
    is padded by `halo` cells of its periodic neighbours, its force computed
    by ``force_from_delta`` as if the padded block were periodic (its own mean
    removed), and its m^3 interior kept.  With ``bandpass`` = (levels, order)
    each padded block's force first loses its long-range band,
    F_b - EXPAND(REDUCE(F_b)) on the (periodic) padded block, before the
    interior is kept."""
    rho = np.asarray(rho, dtype=np.float64)
    n = rho.shape[0]
    m = n // split
    B = m + 2 * halo
    F = np.zeros((3, n, n, n))
    for bx in range(split):
        for by in range(split):
            for bz in range(split):
                ix = [(np.arange(B) + b * m - halo) % n for b in (bx, by, bz)]
                Fb = force_from_delta(rho[np.ix_(*ix)] - 1.0, omega_m)
                if bandpass is not None:
                    lv, od = bandpass
                    Fb = np.stack([Fb[i] - expand(reduce(Fb[i], lv, od), lv, od) for i in range(3)])
                inner = slice(halo, halo + m)
                F[:, bx * m:(bx + 1) * m, by * m:(by + 1) * m, bz * m:(bz + 1) * m] = Fb[:, inner, inner, inner]
    return F


def pyramid_force(rho, omega_m, levels=2, split=2, halo=16, order=6, bandpass="block", coarse_kernel="matched"):
    """Algorithm 3: the long-range force on the REDUCEd mesh (``coarse_force``,
    in fine-cell units), the short-range force from local FFTs, combined as
    EXPAND(F_L) + F_S - EXPAND(REDUCE(F_S)).

    Two readings of where the short-range band-pass F_S - EXPAND(REDUCE(F_S))
    acts: bandpass="block" applies it to each padded block's force before
    its interior is kept (on the local grid, as a distributed implementation
    holds it with its halo); bandpass="global" applies it to the assembled
    short-range mesh.  coarse_kernel selects ``coarse_force``'s operator."""
    rho = np.asarray(rho, dtype=np.float64)
    D = reduce(rho - 1.0, levels, order)
    FL = coarse_force(D, omega_m, 2.0 ** levels, coarse_kernel)
    if bandpass == "block":
        FS = local_force(rho, omega_m, split, halo, bandpass=(levels, order))
        return np.stack([expand(FL[i], levels, order) + FS[i] for i in range(3)])
    FS = local_force(rho, omega_m, split, halo)
    F = np.empty_like(FS)
    for i in range(3):
        FLi = expand(FL[i], levels, order)
        Fli = expand(reduce(FS[i], levels, order), levels, order)
        F[i] = FLi + FS[i] - Fli
    return F


# ---------------------------------------------------------------------------
# Time integration: KDK leapfrog (Eqs. 1-2)
# ---------------------------------------------------------------------------
def kdk(dx, p, stages, np_, nc, omega_m, round_to_float32=True, record=None, green="naive", gradient="fd4",
        pyramid=None):
    """Run len(stages)-1 KDK steps from (dx, p) at stages[0].

    The oracle performs the two half kicks of every step separately.  The
    particle-to-cell assignment uses the float32 value of dx (as the GPU
    stores it) when ``round_to_float32``; all arithmetic is FP64.
    ``record``, if a list, receives (dx, p) at the start of every step.
    ``green`` and ``gradient`` select the force variant (``force_from_delta``),
    ``pyramid`` the multi-grid force (``pyramid_force``).
    """
    kick1, drift, kick2 = fastpm_factors(stages, omega_m)
    dx = np.array(dx, dtype=np.float64)
    p = np.array(p, dtype=np.float64)

    def frc(x):
        xx = x.astype(np.float32) if round_to_float32 else x
        return particle_force(xx, np_, nc, omega_m, green, gradient, pyramid)

    f = frc(dx)
    for k in range(len(stages) - 1):
        if record is not None:
            record.append((dx.copy(), p.copy()))
        p = p + kick1[k] * f
        dx = dx + drift[k] * p
        f = frc(dx)
        p = p + kick2[k] * f
    return dx, p


# ---------------------------------------------------------------------------
# Power spectrum, transfer function, cross-correlation (Eqs. 10-11)
# ---------------------------------------------------------------------------
def _bin_weights(n):
    nx, ny, nz = half_spectrum_wavenumbers(n)
    n2 = nx * nx + ny * ny + nz * nz
    # bin j holds modes with j - 1/2 <= |n| < j + 1/2, i.e. (2j-1)^2 <= 4 n^2 < (2j+1)^2
    j = np.floor((np.sqrt(4.0 * n2) + 1.0) / 2.0).astype(np.int64)
    # guard the float sqrt against off-by-one at exact squares
    j = np.where((2 * j - 1) ** 2 > 4 * n2, j - 1, j)
    j = np.where((2 * j + 1) ** 2 <= 4 * n2, j + 1, j)
    w = np.where((nz > 0) & (nz < n // 2), 2.0, 1.0) * np.ones_like(n2, dtype=np.float64)
    return j, w, np.sqrt(n2.astype(np.float64))


def power_spectrum(field, box, other=None):
    """Binned (cross) power spectrum of mesh field(s).

    P(k_j) = V/M^2 <Re(a_k b_k^*)> over modes with j - 1/2 <= |n| < j + 1/2,
    j = 1 .. N/2, k_j = 2 pi j / L; half-spectrum modes with 0 < n_z < N/2
    count twice (their conjugate partner).  No window or shot-noise correction.
    Returns (k_mean, P, n_modes), each of length N/2.
    """
    n = field.shape[0]
    a = _rfftn(np.asarray(field, dtype=np.float64))
    b = a if other is None else _rfftn(np.asarray(other, dtype=np.float64))
    j, w, nmag = _bin_weights(n)
    nb = n // 2
    sel = (j >= 1) & (j <= nb)
    prod = (a * np.conj(b)).real
    cnt = np.bincount(j[sel], weights=w[sel], minlength=nb + 1)[1:]
    pw = np.bincount(j[sel], weights=(w * prod)[sel], minlength=nb + 1)[1:]
    kw = np.bincount(j[sel], weights=(w * nmag)[sel], minlength=nb + 1)[1:]
    V, M = box ** 3, float(n) ** 3
    with np.errstate(invalid="ignore", divide="ignore"):
        P = V / M ** 2 * pw / cnt
        kmean = 2.0 * math.pi / box * kw / cnt
    return kmean, P, cnt


def transfer_function(pa, pb):
    """Eq. 10: T_f = sqrt(P_a / P_b)."""
    return np.sqrt(np.asarray(pa) / np.asarray(pb))


def cross_correlation(pab, pa, pb):
    """Eq. 11: r_c = P_ab / sqrt(P_a P_b)."""
    return np.asarray(pab) / np.sqrt(np.asarray(pa) * np.asarray(pb))


# ---------------------------------------------------------------------------
# Whole forward model
# ---------------------------------------------------------------------------
def simulate(white, nc, box, cosmo, stages, order=2, record=None):
    """Algorithm 4 initial conditions at stages[0], then KDK to stages[-1].

    Returns dict(dx, p, rho, k, pk, lin_k, dx0, p0)."""
    np_ = white.shape[0]
    lin_k = linear_field(white, box, cosmo)
    dx0, p0 = lpt(lin_k, nc, stages[0], cosmo, order=order)
    dx, p = kdk(dx0, p0, stages, np_, nc, cosmo["omega_m"], record=record)
    rho = paint(dx.astype(np.float32), np_, nc)
    k, pk, _ = power_spectrum(rho - 1.0, box)
    return dict(dx=dx, p=p, rho=rho, k=k, pk=pk, lin_k=lin_k, dx0=dx0, p0=p0)


# ---------------------------------------------------------------------------
# Adjoint (reverse mode) of the forward model: the differentiability the
# paper names as the method's main advantage (Sec. 8), through the chi^2 of
# Eq. 12's likelihood term.  Every function returns the transpose (or the
# transposed Jacobian) of the forward function of the same name applied to a
# cotangent; cotangents of real fields are real fields of the same shape.
# ---------------------------------------------------------------------------
def chi2(rho, delta_target, sigma=1.0):
    """chi^2 = sum (delta - delta_t)^2 / sigma^2 with delta = rho - 1, and its
    gradient with respect to rho."""
    r = (np.asarray(rho, dtype=np.float64) - 1.0 - delta_target) / sigma
    return float((r * r).sum()), 2.0 * r / sigma


def _corner_grad(t, b, d):
    """d/dt_d of the CIC corner weight prod_e (b_e ? t_e : 1 - t_e)."""
    w = np.ones(t.shape[1])
    for e in range(3):
        if e == d:
            w = w * (1.0 if b[e] else -1.0)
        else:
            w = w * (t[e] if b[e] else (1.0 - t[e]))
    return w


def _gather_grad(field, cell, t):
    """sum_c dW(x_i - c)/dx_d field_c for d = 0..2 (right derivative at
    integer positions, matching the floor-based cell)."""
    nc = field.shape[-1]
    flat_field = field.reshape(-1)
    out = np.zeros((3, cell.shape[1]))
    for b in _corners():
        c = [(cell[e] + b[e]) % nc for e in range(3)]
        vals = flat_field[(c[0] * nc + c[1]) * nc + c[2]]
        for d in range(3):
            out[d] += vals * _corner_grad(t, b, d)
    return out


def paint_adj(g_rho, dx, np_, nc):
    """Transposed Jacobian of paint: g_dx_i = m sum_c grad W(x_i - c) g_rho_c."""
    cell, t = cic_cells(dx, np_, nc)
    m = (nc / np_) ** 3
    return m * _gather_grad(np.asarray(g_rho, dtype=np.float64), cell, t)


def readout_adj(F, dx, g_f, np_, nc):
    """Transposed Jacobian of readout f = R(x; F): the mesh cotangent
    g_F[d] = sum_i W(x_i - c) g_f[d][i] (a paint of g_f) and the position
    cotangent g_dx_i = sum_d g_f[d][i] sum_c grad W(x_i - c) F[d]_c."""
    cell, t = cic_cells(dx, np_, nc)
    g_F = np.stack([paint_cells(cell, t, np.asarray(g_f[d], dtype=np.float64), nc) for d in range(3)])
    g_dx = np.zeros((3, cell.shape[1]))
    for d in range(3):
        g_dx += np.asarray(g_f[d])[None, :] * _gather_grad(np.asarray(F[d], dtype=np.float64), cell, t)
    return g_F, g_dx


def force_adj(g_F, omega_m, green="naive", gradient="fd4"):
    """Transpose of delta -> F (Eqs. 3-5): each F_d is a convolution with a
    real odd kernel, so its transpose is its negative:
    g_delta = -sum_d IFFT(i g_d 1.5 Om FFT(g_F_d) / |w|^2).  Both variants
    keep the kernel real and odd (g_d odd in w_d, the Laplacian even)."""
    n = g_F.shape[-1]
    g = _gradient_kernels(n, gradient)
    k2 = _laplacian(n, green)
    k2[0, 0, 0] = 1.0
    acc = 0.0
    for d in range(3):
        acc = acc + 1j * g[d] * _rfftn(np.asarray(g_F[d], dtype=np.float64))
    acc = 1.5 * omega_m * acc / k2
    acc[0, 0, 0] = 0.0
    return -_irfftn(acc, n)


def particle_force_adj(dx, g_f, np_, nc, omega_m, green="naive", gradient="fd4"):
    """Transposed Jacobian of dx -> particle_force(dx) applied to g_f."""
    F = force(paint(dx, np_, nc), omega_m, green, gradient)
    g_F, g_dx = readout_adj(F, dx, g_f, np_, nc)
    g_rho = force_adj(g_F, omega_m, green, gradient)
    return g_dx + paint_adj(g_rho, dx, np_, nc)


def kdk_adj(xs, stages, g_dx, g_p, np_, nc, omega_m, green="naive", gradient="fd4"):
    """Reverse of ``kdk`` given the positions x_k at every stage (xs[k],
    float32-rounded as the forward used them) and the cotangents of the final
    (dx, p).  Undoes, for k = n-1..0: the closing kick at x_{k+1}, the drift,
    the opening kick at x_k.  Returns the cotangents of the initial (dx, p)."""
    kick1, drift, kick2 = fastpm_factors(stages, omega_m)
    gx = np.array(g_dx, dtype=np.float64)
    gp = np.array(g_p, dtype=np.float64)
    n = len(stages) - 1
    for k in range(n - 1, -1, -1):
        gx = gx + particle_force_adj(xs[k + 1], kick2[k] * gp, np_, nc, omega_m, green, gradient)
        gp = gp + drift[k] * gx
        gx = gx + particle_force_adj(xs[k], kick1[k] * gp, np_, nc, omega_m, green, gradient)
    return gx, gp


def lpt_adj(lin_k, nc, a0, cosmo, g_dx, g_p, order=2):
    """Reverse of ``lpt``: returns G = FFT(dL/d delta_L), the unnormalised DFT
    of the cotangent of the real linear field delta_L = IFFT(lin_k)
    (rfftn layout).  Psi1_d = B_d delta_L and Psi2_d = -B_d S with B_d the
    convolution of transfer i g_d/|w|^2 (real odd, B_d^T = -B_d), and
    phi_ij = H_ij delta_L with transfer g_i g_j/|w|^2 (real even, H^T = H)."""
    np_ = lin_k.shape[0]
    gr = growth([a0], cosmo["omega_m"])
    D1, D2, f1, f2, E = (float(gr[k][0]) for k in ("D1", "D2", "f1", "f2", "E"))
    r = nc / np_
    shape = (3, np_, np_, np_)
    gdx = np.asarray(g_dx, dtype=np.float64).reshape(shape)
    gp = np.asarray(g_p, dtype=np.float64).reshape(shape)
    pf = a0 * a0 * E
    g_psi1 = r * (D1 * gdx + pf * f1 * D1 * gp)
    g_psi2 = r * (D2 * gdx + pf * f2 * D2 * gp)
    g = _gradient_kernels(np_)
    k2 = _laplacian_naive(np_)
    k2[0, 0, 0] = 1.0
    inv_k2 = 1.0 / k2
    inv_k2[0, 0, 0] = 0.0
    # B_d^T g = -IFFT(i g_d FFT(g) / |w|^2)
    G = 0.0
    for d in range(3):
        G = G - 1j * g[d] * _rfftn(g_psi1[d]) * inv_k2
    if order == 2:
        # dL/dS = sum_d (-B_d)^T g_psi2_d = sum_d B_d g_psi2_d
        gS = _irfftn(sum(1j * g[d] * _rfftn(g_psi2[d]) for d in range(3)) * inv_k2, np_)
        phi = {}
        for i in range(3):
            for j in range(i, 3):
                phi[(i, j)] = _irfftn(g[i] * g[j] * lin_k * inv_k2, np_)
        # S = sum_{i<j} (phi_ii phi_jj - phi_ij^2)
        g_phi = {
            (0, 0): gS * (phi[(1, 1)] + phi[(2, 2)]),
            (1, 1): gS * (phi[(0, 0)] + phi[(2, 2)]),
            (2, 2): gS * (phi[(0, 0)] + phi[(1, 1)]),
            (0, 1): -2.0 * gS * phi[(0, 1)],
            (0, 2): -2.0 * gS * phi[(0, 2)],
            (1, 2): -2.0 * gS * phi[(1, 2)],
        }
        for (i, j), v in g_phi.items():
            G = G + g[i] * g[j] * inv_k2 * _rfftn(v)
    return G


def linear_field_adj(G, box, cosmo):
    """Reverse of ``linear_field`` given G = FFT(dL/d delta_L): the map
    w -> delta_L is a convolution with the real even transfer
    s(k) = sqrt(P(k) N^3 / V), so g_w = IFFT(s G)."""
    n = G.shape[0]
    nx, ny, nz = half_spectrum_wavenumbers(n)
    kmag = 2.0 * math.pi / box * np.sqrt((nx * nx + ny * ny + nz * nz).astype(np.float64))
    with np.errstate(divide="ignore", invalid="ignore"):
        pk = linear_pk(kmag, cosmo)
    s = np.sqrt(pk * n ** 3 / box ** 3)
    s[0, 0, 0] = 0.0
    return _irfftn(s * G, n)


def chi2_and_grad(white, delta_target, nc, box, cosmo, stages, sigma=1.0, order=2):
    """chi^2 of the final CIC density against delta_target and its gradient
    with respect to the white noise (the reverse of ``simulate``)."""
    np_ = white.shape[0]
    xs = []
    lin_k = linear_field(white, box, cosmo)
    dx0, p0 = lpt(lin_k, nc, stages[0], cosmo, order=order)
    dx, p = kdk(dx0, p0, stages, np_, nc, cosmo["omega_m"], record=xs, round_to_float32=POSITIONS_FP32)
    ptype = np.float32 if POSITIONS_FP32 else np.float64
    xs = [x.astype(ptype) for x, _ in xs] + [dx.astype(ptype)]
    rho = paint(xs[-1], np_, nc)
    loss, g_rho = chi2(rho, delta_target, sigma)
    g_dx = paint_adj(g_rho, xs[-1], np_, nc)
    g_dx0, g_p0 = kdk_adj(xs, stages, g_dx, np.zeros_like(g_dx), np_, nc, cosmo["omega_m"])
    G = lpt_adj(lin_k, nc, stages[0], cosmo, g_dx0, g_p0, order=order)
    return loss, linear_field_adj(G, box, cosmo)


# ---------------------------------------------------------------------------
# Reconstruction (Sec. 7.1, Eq. 12): negative log-posterior and Adam
# ---------------------------------------------------------------------------
def posterior_and_grad(white, delta_target, nc, box, cosmo, stages, sigma=1.0, order=2):
    """Eq. 12's negative log-posterior of the initial conditions and its
    gradient with respect to the white noise w:

      -log p = chi^2 / 2 + s^dagger S^-1 s / 2,   chi^2 = sum (delta - delta_t)^2 / sigma^2.

    The initial field is s = L w with L diagonal in Fourier space and S = L L^dagger
    the fiducial covariance, so s^dagger S^-1 s = w^T w (the prior of the white noise)."""
    loss, g = chi2_and_grad(white, delta_target, nc, box, cosmo, stages, sigma=sigma, order=order)
    w = np.asarray(white, dtype=np.float64)
    return 0.5 * loss + 0.5 * float((w * w).sum()), 0.5 * g + w


def adam_step(x, g, m, v, t, lr=0.01, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at step t >= 1; the
    paper's optimiser with learning rate 0.01 (Sec. 7.1).  Returns (x, m, v)."""
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return np.asarray(x, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v
