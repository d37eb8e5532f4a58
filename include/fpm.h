/*
 * fpm.h -- C ABI of the GB300-native FastPM particle-mesh library (libfpm).
 *
 * The library computes the particle-mesh force-and-integration loop of
 * FastPM as the FlowPM paper (Modi, Lanusse & Seljak, arXiv:2010.11847)
 * states it: Gaussian initial conditions displaced by 2LPT (Algorithm 4),
 * then per step a cloud-in-cell paint (Sec. 2), a real-to-complex 3D FFT,
 * the force transfer function of Eqs. 3-5 (naive -1/k^2 Green's function,
 * 4th-order finite-difference gradient), three complex-to-real inverse FFTs,
 * a CIC readout and the kick/drift updates of Eqs. 1-2 with FastPM's
 * growth-factor coefficients.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every pointer to array data is a DEVICE pointer unless stated
 *    otherwise; the caller allocates and owns it.  A plan owns only its
 *    scratch, twiddle and coefficient tables.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    stream-ordered and asynchronous; none synchronises the host except
 *    fpm_status() and the calls that return host-side results as noted.
 *  - Return value: FPM_OK (0) or a negative FPM_E* code.  Argument errors
 *    are detected on the host before anything is launched.  Device-side
 *    errors (a NaN or an out-of-range cell met by a kernel) set a flag in
 *    the plan that fpm_status() reports.
 *  - Units: displacements dx, momenta p and forces are in mesh-cell units
 *    (x0 = box/nc = 1); time is in 1/H0.  Particle i = (ix*np + iy)*np + iz
 *    sits on lattice node q = (ix, iy, iz) * (nc/np); its position is
 *    q + dx (periodic).  Particle mass (nc/np)^3, so the mean density is 1.
 *  - Particle arrays are SoA float[3][np^3] in Lagrangian order.
 *  - Meshes are C-order float[nc][nc][nc] ([x][y][z], z fastest).
 *  - Half spectra (lin_k) are complex64 (interleaved float pairs) in the
 *    layout [kx][kz][ky] with kx, ky in 0..n-1 (DFT order) and kz in
 *    0..n/2; the forward DFT is unnormalised with sign e^{-ik.x}.
 *  - Sizes: np, nc in {16, 32, 48, 64, 96, 128, 192, 256, 384, 512},
 *    nc = np, 2 np or 4 np.  The cell key uses 16^3-cell tiles.
 *  - Nothing here falls back to the CPU: without a CUDA device every call
 *    that launches work fails with FPM_ECUDA.
 */
#ifndef FPM_H
#define FPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FPM_OK 0
#define FPM_EINVAL (-1)    /* bad argument (null pointer, size, range)      */
#define FPM_ENOMEM (-2)    /* device allocation failed                       */
#define FPM_ECUDA (-3)     /* a CUDA runtime call or launch failed           */
#define FPM_ETIMEOUT (-4)  /* a bounded device wait ran out                  */
#define FPM_EDEVICE (-5)   /* device error flag: NaN / cell out of range     */
#define FPM_ENOTIMPL (-6)  /* entry point not available in this build        */

typedef struct fpm_plan fpm_plan;

/* Cosmology of a flat LCDM universe (no radiation, w = -1). */
typedef struct {
  double omega_m, omega_b, h, n_s, sigma8, t_cmb;
} fpm_cosmo;

/* Create a plan for np^3 particles on an nc^3 mesh in a periodic box of
 * side `box` Mpc/h.  Allocates the plan's device scratch and computes, on
 * the GPU in FP64, the sigma8 normalisation of the Eisenstein & Hu (1998)
 * no-wiggle power spectrum.  *plan is set only on success.  Errors:
 * FPM_EINVAL (sizes, null, non-positive box or parameters), FPM_ENOMEM,
 * FPM_ECUDA.  Blocks until the normalisation is computed. */
int fpm_plan_create(fpm_plan** plan, int np, int nc, double box,
                    const fpm_cosmo* cosmo, void* stream);

/* Free the plan and its device scratch (synchronises the device). NULL ok. */
void fpm_plan_destroy(fpm_plan* plan);

/* Bytes of device scratch the plan holds. */
int64_t fpm_plan_scratch_bytes(const fpm_plan* plan);

/* Growth quantities at `n` scale factors (HOST arrays a[n] in (1e-5, 10]):
 * out[5*i + {0..4}] = D1, D2, f1 = dlnD1/dlna, f2 = dlnD2/dlna, E = H/H0 at
 * a[i], normalised to D1(1) = 1, D2 in units of D1_raw(1)^2 (FastPM time
 * stepping, Sec. 2).  Computed on the GPU in FP64; `out` is a HOST array.
 * Synchronises `stream`.  n <= 4096. */
int fpm_growth(fpm_plan* plan, const double* a, int n, double* out, void* stream);

/* Linear field, Algorithm 4 steps 1-2:
 *   lin_k(k) = DFT(white)(k) * sqrt(P(|k|) np^3 / box^3),  lin_k(0) = 0,
 * with P the sigma8-normalised EH no-wiggle spectrum (k = 2 pi n / box).
 * white: float[np^3] (standard normal); lin_k: complex64 half spectrum of
 * the np^3 lattice in the [kx][kz][ky] layout. */
int fpm_linear_field(fpm_plan* plan, const float* white, void* lin_k, void* stream);

/* Lagrangian perturbation theory at a0 (Algorithm 4 steps 3-6, order 1 or
 * 2): dx = D1 Psi1 + D2 Psi2, p = a0^2 E (f1 D1 Psi1 + f2 D2 Psi2), with
 * Psi1(k) = i g(k) lin_k / |w|^2, Psi2(k) = -i g(k) S(k) / |w|^2 and
 * S = sum_{i<j} (phi_ii phi_jj - phi_ij^2), phi_ij(k) = g_i g_j lin_k / |w|^2
 * (g the Eq. 5 gradient, w the lattice wave vector), in mesh-cell units.
 * lin_k is read only; dx, p: float[3][np^3] written. */
int fpm_lpt(fpm_plan* plan, const void* lin_k, double a0, int order,
            float* dx, float* p, void* stream);

/* CIC paint of the particles at q + dx (Sec. 2): rho: float[nc^3] mean 1,
 * deterministic (fixed-point accumulation).  Optional outputs (NULL to
 * skip): key_out uint32[np^3], the tile-major cell key of each particle
 *   key = ((tx*NT + ty)*NT + tz)*4096 + (lx*16 + ly)*16 + lz,
 *   cell = wrap(q + floor(dx)), t = cell/16, l = cell%16, NT = nc/16;
 * perm_out uint32[np^3], the stable counting-sort order (by key, ties by
 * particle index). */
int fpm_paint(fpm_plan* plan, const float* dx, float* rho,
              uint32_t* key_out, uint32_t* perm_out, void* stream);

/* Force meshes from a density mesh (Eqs. 3-5):
 *   F_d = IDFT( i g_d(w) * 1.5 omega_m * DFT(rho - 1) / |w|^2 ),  F(0) = 0,
 * g_d(w) = (8 sin w_d - sin 2w_d)/6, w = 2 pi n / nc (the defaults of
 * fpm_set_force_kernel).  rho: float[nc^3]; F: float[3][nc^3]. */
int fpm_force(fpm_plan* plan, const float* rho, float* F, void* stream);

/* Force kernel of the plan (Sec. 2): the Green's function and the gradient
 * that fpm_force, fpm_kdk, the adjoint entry points and batches built from
 * the plan use.  green: FPM_GREEN_NAIVE (default, |w|^2 = sum w_d^2) or
 * FPM_GREEN_DISCRETE (Eq. 4, |w|^2 -> sum_d (2 sin(w_d/2))^2, the
 * seven-point discrete Laplacian).  gradient: FPM_GRAD_FD4 (default, Eq. 5)
 * or FPM_GRAD_EXACT (g_d = w_d, 0 at the Nyquist frequency).  The initial
 * conditions (fpm_lpt) always use the defaults.  Synchronises the device
 * (queued work may be reading the old tables).  Errors: FPM_EINVAL (null
 * plan, unknown kind), FPM_ECUDA (table allocation or copy).
 * fpm_batch_create returns FPM_ENOTIMPL for a plan with FPM_GRAD_EXACT. */
#define FPM_GREEN_NAIVE 0
#define FPM_GREEN_DISCRETE 1
#define FPM_GRAD_FD4 0
#define FPM_GRAD_EXACT 1
int fpm_set_force_kernel(fpm_plan* plan, int green, int gradient);

/* Multi-grid pyramid force (Sec. 3.1 Eqs. 6-9, Algorithms 2-3) for every
 * later fpm_force / fpm_kdk of the plan; levels = 0 switches it off.
 * F = EXPAND(F_L) + F_S - EXPAND(REDUCE(F_S)) with REDUCE = `levels`
 * stride-2 convolutions with the order-6 discrete B-spline (binomial
 * weights C(6, j)/64, periodic), EXPAND = the transposed convolutions with
 * 8 times that kernel, F_L the force of REDUCE(rho - 1) on the
 * (nc >> levels)^3 mesh in fine-cell units, F_S the force of local FFTs:
 * split^3 cubic blocks of nc/split cells, each padded by `halo` cells of
 * its periodic neighbours and transformed as a periodic mesh of
 * B = nc/split + 2 halo cells, its interior kept.  The reading of the
 * paper's scheme is chosen by fpm_set_pyramid_reading (default: band-pass
 * per padded block, fine-mesh operator on the coarse mesh).  Requires levels
 * in {1, 2}, nc >> levels and B among the FFT sizes (16, 32, 48, 64, 96,
 * 128, 192, 256, 384, 512), split | nc, and B divisible by 2^levels for the
 * per-block band-pass.  Synchronises the device; allocates about 9 nc^3
 * floats.  Errors: FPM_EINVAL, FPM_ENOMEM.  With a pyramid set, the adjoint
 * entry points and fpm_batch_create return FPM_ENOTIMPL. */
int fpm_set_pyramid(fpm_plan* plan, int levels, int split, int halo);

/* Reading of Algorithm 3 used by the plan's pyramid force (the paper leaves
 * both open; Sec. 3.1, Sec. 6.1).  bandpass: FPM_PYR_BANDPASS_BLOCK applies
 * F_S - EXPAND(REDUCE(F_S)) to each padded block's force (REDUCE and EXPAND
 * periodic on the block) before its interior is kept; FPM_PYR_BANDPASS_GLOBAL
 * applies it to the assembled short-range mesh.  coarse_kernel:
 * FPM_PYR_KERNEL_MATCHED gives the coarse mesh the fine mesh's operator at
 * the same wavenumber (naive Green's function, Eq. 5 gradient symbol at the
 * fine frequency; three-field spectral passes); FPM_PYR_KERNEL_COARSE uses
 * Eq. 5 in coarse-cell units.  Rebuilds a pyramid that is set (device
 * synchronised).  Errors: FPM_EINVAL (unknown value, or a set pyramid whose
 * block size the reading cannot split), FPM_ENOMEM. */
#define FPM_PYR_BANDPASS_BLOCK 0
#define FPM_PYR_BANDPASS_GLOBAL 1
#define FPM_PYR_KERNEL_MATCHED 0
#define FPM_PYR_KERNEL_COARSE 1
int fpm_set_pyramid_reading(fpm_plan* plan, int bandpass, int coarse_kernel);

/* CIC readout of three meshes at the particles: f_out[d][i] =
 * sum_c W(q_i + dx_i - c) F[d][c].  F: float[3][nc^3]; f_out float[3][np^3]. */
int fpm_readout(fpm_plan* plan, const float* F, const float* dx, float* f_out,
                void* stream);

/* KDK leapfrog (Eqs. 1-2) with FastPM factors over nsteps steps between the
 * HOST scale factors a[0..nsteps] (strictly increasing, nsteps <= 2048);
 * dx, p are updated in place (input at a[0], output at a[nsteps]).  Step k:
 * kick a_k -> a_h (force at a_k), drift a_k -> a_{k+1} (momentum at a_h),
 * kick a_h -> a_{k+1} (force at a_{k+1}), a_h = sqrt(a_k a_{k+1}); the
 * closing kick of a step and the opening kick of the next are applied as
 * one.  The coefficients are computed on the GPU in FP64.  ckpt (NULL to
 * skip): float[nsteps+1][3][np^3], receives dx at every a_k (the momenta
 * are not needed to reverse the steps: the force depends on dx only).
 * fckpt (NULL to skip): float[nsteps+1][fpm_force_ckpt_floats(plan)],
 * receives for every a_k the force mesh in the plan's internal layout
 * (float4 per cell on power-of-two meshes, else [3][nc^3]) and the tile
 * buckets of that stage's particles; fpm_kdk_adj then reuses both instead
 * of recomputing the forces and re-sorting the particles (both are written
 * straight into the checkpoint by the kernels that make them: no extra
 * traffic).  Its contents are internal: only fpm_kdk_adj reads them. */
int fpm_kdk(fpm_plan* plan, float* dx, float* p, const double* a, int nsteps,
            float* ckpt, float* fckpt, void* stream);

/* Floats per stage of fpm_kdk's force checkpoint fckpt: 4 nc^3 for the
 * force mesh plus np^3 + np^3/2 + (nc/16)^3 + 1 for the tile buckets,
 * rounded up to a multiple of 64 (0 for a NULL plan).  Not in the paper: a
 * memory-for-time choice of the reverse pass (Sec. 5 stores the states). */
int64_t fpm_force_ckpt_floats(const fpm_plan* plan);

/* Binned power spectrum (Eq. 10's ingredient) of mesh field `a`, or the
 * cross spectrum of `a` and `b` (b may be NULL):
 *   P(k_j) = box^3/nc^6 <Re(A_k B_k^*)>,  j - 1/2 <= |n| < j + 1/2,
 * j = 1..nc/2; HOST outputs pk[nc/2], kmean[nc/2] (h/Mpc), nmodes[nc/2]
 * (any may be NULL).  Synchronises `stream`. */
int fpm_power(fpm_plan* plan, const float* a, const float* b, double* pk,
              double* kmean, double* nmodes, void* stream);

/* ---------------------------------------------------------------------
 * Adjoints (reverse mode).  The paper's reconstruction (Sec. 7, Eq. 12)
 * needs the gradient of a chi^2 between the final density and data with
 * respect to the initial conditions; these entry points are the transposed
 * Jacobians of the forward steps, applied to cotangents of the same
 * layouts.  Adjoint entry points that transform meshes need power-of-two
 * np and nc (else FPM_ENOTIMPL).  The first adjoint call on a plan
 * allocates the adjoint scratch (cudaMalloc; make it before any stream
 * capture).  All return-by-argument buffers are overwritten unless stated.
 * ------------------------------------------------------------------- */

/* One Adam update (Kingma & Ba 2015, Algorithm 1; the optimiser of the
 * paper's reconstruction, Sec. 7.1, learning rate 0.01 there) on the
 * negative log-posterior of Eq. 12, with the prior of the white noise fused:
 * the gradient used is gscale * g + pscale * x (g: DEVICE float[n], e.g.
 * d chi^2 / d x; gscale = 1/2, pscale = 1 give chi^2/2 + x^T x/2).  x, m, v
 * (DEVICE float[n]) are updated in place; t >= 1 is the step count (bias
 * corrections 1/(1 - beta^t)).  prior (nullable, HOST double) receives the
 * FP64 sum of x^2 / 2 before the update; when given, `stream` is
 * synchronised.  FPM_EINVAL for n <= 0, t < 1, lr <= 0, beta outside [0, 1)
 * or eps < 0.  Asynchronous otherwise. */
int fpm_adam_step(fpm_plan* plan, float* x, const float* g, float* m, float* v, int64_t n, double gscale,
                  double pscale, double lr, double beta1, double beta2, double eps, int t, double* prior,
                  void* stream);

/* chi^2 of Eq. 12's likelihood term: loss = sum_c (rho_c - 1 - t_c)^2 /
 * sigma^2 with t = target_delta (float[nc^3]), accumulated in FP64 in a
 * fixed order; g_rho (nullable, float[nc^3]) = 2 (rho - 1 - t) / sigma^2.
 * loss (nullable) is a HOST double; when given, `stream` is synchronised. */
int fpm_chi2(fpm_plan* plan, const float* rho, const float* target_delta, double sigma,
             float* g_rho, double* loss, void* stream);

/* Transposed Jacobian of fpm_paint with respect to dx:
 * g_dx[d][i] = m sum_c dW(q_i + dx_i - c)/dx_d g_rho[c]  (m = (nc/np)^3;
 * right derivative where a particle sits exactly on a cell boundary). */
int fpm_paint_adj(fpm_plan* plan, const float* dx, const float* g_rho, float* g_dx,
                  void* stream);

/* Transposed Jacobian of fpm_readout(F, dx) applied to g_f (float[3][np^3]):
 * g_F[d][c] = sum_i W(q_i + dx_i - c) g_f[d][i] (float[3][nc^3], a
 * deterministic fixed-point scatter) and
 * g_dx[e][i] = sum_d g_f[d][i] sum_c dW/dx_e F[d][c]. */
int fpm_readout_adj(fpm_plan* plan, const float* F, const float* dx, const float* g_f,
                    float* g_F, float* g_dx, void* stream);

/* Transpose of fpm_force's linear map rho -> F: each F_d is a convolution
 * with a real odd kernel, so g_rho = -sum_d IDFT(i g_d 1.5 omega_m
 * DFT(g_F_d) / |w|^2).  g_F: float[3][nc^3]; g_rho: float[nc^3]. */
int fpm_force_adj(fpm_plan* plan, const float* g_F, float* g_rho, void* stream);

/* Reverse of fpm_kdk over the same HOST scale factors a[0..nsteps], given
 * its checkpoints ckpt (float[nsteps+1][3][np^3], dx at every a_k) and,
 * optionally, its force checkpoints fckpt (NULL: recompute).  On entry g_dx
 * holds the cotangent of the final dx and g_p_in (nullable: zero, e.g. a
 * loss on the density alone) that of the final p; on return g_dx and g_p
 * (required, may equal g_p_in) hold the cotangents of the initial dx and p.
 * Each reverse step takes the stage's force and tile buckets from fckpt (as
 * written by the fpm_kdk call over the same a; NULL: recomputes paint and
 * force), then applies the drift transpose and the transposed force
 * Jacobian (readout, force and paint transposes).  The result is bitwise
 * the same either way. */
int fpm_kdk_adj(fpm_plan* plan, const float* ckpt, const float* fckpt, const double* a, int nsteps,
                float* g_dx, const float* g_p_in, float* g_p, void* stream);

/* Reverse of fpm_lpt: from the cotangents of dx and p (float[3][np^3])
 * returns g_lin_k = DFT(dL/d delta_L), the unnormalised DFT of the
 * cotangent of the real linear field delta_L = IDFT(lin_k), in the lin_k
 * layout.  Uses Psi1_d = B_d delta_L, Psi2_d = -B_d S with B_d the real odd
 * convolution of transfer i g_d / |w|^2 (B_d^T = -B_d) and the chain rule
 * through S = sum_{i<j} (phi_ii phi_jj - phi_ij^2). */
int fpm_lpt_adj(fpm_plan* plan, const void* lin_k, double a0, int order, const float* g_dx,
                const float* g_p, void* g_lin_k, void* stream);

/* Reverse of fpm_linear_field: the map white -> delta_L is a convolution
 * with the real even transfer s(k) = sqrt(P(k) np^3 / box^3), so
 * g_white = IDFT(s g_lin_k) (float[np^3]). */
int fpm_linear_field_adj(fpm_plan* plan, const void* g_lin_k, float* g_white, void* stream);

/* ---------------------------------------------------------------------
 * Batched simulations.  Many independent simulations (each with its own
 * plan: size, box, cosmology) advance together by one persistent
 * cooperative kernel launch per KDK step; a launch runs every phase of the
 * step (readout-kick-drift and keys, tile scan, scatter, paint, halo, the
 * five FFT passes with the force transfer function) over a work list that
 * spans all simulations, with a bounded-spin grid barrier between phases
 * (FPM_ETIMEOUT instead of a hang).  A whole run is captured once into a
 * CUDA graph and replayed.  The paper's batch splitting (Sec. 4) is the
 * use case; each simulation gives the same bits as fpm_kdk on its plan.
 * Supported plans: np = nc in {32, 64, 96, 128}.
 * ------------------------------------------------------------------- */
typedef struct fpm_batch fpm_batch;

/* Group nsims plans (HOST array of plan pointers; the plans must outlive the
 * batch and are used as the simulations' scratch). */
int fpm_batch_create(fpm_batch** batch, fpm_plan* const* plans, int nsims);
void fpm_batch_destroy(fpm_batch* batch);

/* Tuning knobs (negative / zero: keep): persistent blocks per SM (0 = as
 * many as fit), 256-particle chunks per readout work item, barrier spin
 * limit (iterations of a ~64 ns sleep before FPM_ETIMEOUT). */
int fpm_batch_configure(fpm_batch* batch, int blocks_per_sm, int readout_chunks, int64_t spin_limit);

/* Run nsteps KDK steps of every simulation between the HOST scale factors
 * a[0..nsteps] (shared by all), updating dx[s], p[s] in place (HOST arrays
 * of device pointers, float[3][np_s^3] each), exactly as fpm_kdk would. */
int fpm_batch_kdk(fpm_batch* batch, float* const* dx, float* const* p, const double* a, int nsteps,
                  void* stream);

/* FPM_ETIMEOUT if a grid barrier gave up, else the plans' device flags;
 * synchronises `stream` and clears the flags. */
int fpm_batch_status(fpm_batch* batch, void* stream);

/* Persistent grid size in blocks, and whether the run was graph-captured. */
int fpm_batch_info(fpm_batch* batch, int* grid_blocks, int* graph_captured);

/* Per-mesh-size layout of the batched step, for every simulation of the
 * batch whose mesh is nc (an autotuner's knobs; none changes a result bit):
 *   FPM_BTUNE_READOUT    the fused readout's particle traversal: 0 chunks of
 *                        consecutive particles, 1 or 2 Lagrangian bricks of
 *                        4 x 32 x 32 or 4 x 16 x 64 particles (np divisible);
 *   FPM_BTUNE_PAINT_TILE the paint's tile edge, 8 or 16 cells (the particles
 *                        are bucketed and painted by tiles of that edge; 8
 *                        gives small meshes 8x more work items);
 *   FPM_BTUNE_FFT_SLOTS  points per thread of the power-of-two FFT passes,
 *                        8 or 16 (16: half the threads per line, twice the
 *                        lines per block).
 * Invalidates the batch's captured graph.  Errors: FPM_EINVAL (no such mesh
 * in the batch, or a value the mesh cannot take), FPM_ENOMEM. */
#define FPM_BTUNE_READOUT 0
#define FPM_BTUNE_PAINT_TILE 1
#define FPM_BTUNE_FFT_SLOTS 2
int fpm_batch_tune(fpm_batch* batch, int nc, int knob, int value);

/* Device milliseconds of each phase of the batched step, accumulated over
 * every fpm_batch_kdk since the last read, then reset: ms (HOST array of
 * n >= FPM_BPH_COUNT entries) in the order below.  A phase's time is the
 * first block's wall time from the end of the previous phase's grid barrier
 * to the end of its own (every block has then finished it); the last phase
 * of a launch ends when the first block finishes it.  Synchronises
 * `stream`.  Errors: FPM_EINVAL, FPM_ECUDA. */
#define FPM_BPH_KEYS 0      /* cell keys of the initial state          */
#define FPM_BPH_KDK 1       /* readout + kick + drift + keys            */
#define FPM_BPH_SCAN 2      /* tile-count scan                          */
#define FPM_BPH_SCATTER 3   /* bucketing by tile                        */
#define FPM_BPH_PAINT 4     /* tile paint                               */
#define FPM_BPH_HALO 5      /* tile-face sums                           */
#define FPM_BPH_ZF 6        /* z r2c                                    */
#define FPM_BPH_YF 7        /* y forward                                */
#define FPM_BPH_X 8         /* x pass with the Green's function         */
#define FPM_BPH_YI 9        /* y inverse                                */
#define FPM_BPH_ZI 10       /* z c2r                                    */
#define FPM_BPH_GRAD 11     /* Eq. 5 difference of the potential        */
#define FPM_BPH_KDK_LAST 12 /* closing kick                             */
#define FPM_BPH_COUNT 13
int fpm_batch_phase_times(fpm_batch* batch, double* ms, int n, void* stream);

/* CIC paint that allocates nothing.  The paper has no counterpart: this is
 * a service for callers that cannot call cudaMalloc -- hosts or plugins that
 * hand out every byte of device memory themselves, loops that cannot afford
 * cudaMalloc's implicit device synchronisation.  Same result as fpm_paint
 * without a plan: rho (float[nc^3], mean 1) of np^3 particles at q + dx
 * (dx: float[3][np^3]); both caller device buffers.  Scratch is one fixed
 * file-scope device array of about 2.9 MB that every GPU loading the library
 * keeps until exit; sizes above its maximum -- np or nc larger than 64 --
 * are rejected with FPM_EINVAL, as are unsupported sizes.  Every call looks
 * the array's device address up (cudaGetSymbolAddress, no allocation) with
 * the caller's device current; the first call on a device may load the
 * library's device code there, so make that first call before any stream
 * capture.  All calls share the array and each leaves its contents behind
 * (the call clears what must start at zero): calls whose execution overlaps
 * on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  Device-side error flags are not reported by
 * this variant: a non-finite or absurdly large displacement gives an
 * undefined density.  Asynchronous on `stream`. */
int fpm_paint_noalloc(int np, int nc, const float* dx, float* rho, void* stream);

/* Kernel classes of the per-class timing below. */
#define FPM_K_KDK 0       /* CIC readout fused with kick, drift and new keys */
#define FPM_K_KEYS 1      /* cell keys + tile histogram (first paint)        */
#define FPM_K_SCAN 2      /* scan of the tile histogram                      */
#define FPM_K_SCATTER 3   /* bucketing of particles by tile                  */
#define FPM_K_PAINT 4     /* in-tile counting sort + fixed-point CIC paint   */
#define FPM_K_HALO 5      /* tile-face sums of the paint                     */
#define FPM_K_FFT_ZF 6    /* z pass, real-to-complex (other mesh sizes)      */
#define FPM_K_FFT_YF 7    /* y pass, forward                                 */
#define FPM_K_FFT_X 8     /* x pass with the Eq. 3-5 transfer function       */
#define FPM_K_FFT_YI 9    /* y pass, inverse (3 fields)                      */
#define FPM_K_FFT_ZI 10   /* z pass, complex-to-real (3 fields)              */
#define FPM_K_READOUT 11  /* plain CIC readout                               */
#define FPM_K_IC 12       /* linear field and 2LPT                           */
#define FPM_K_COEF 13     /* FP64 growth and FastPM factors                  */
#define FPM_K_POWER 14    /* power spectrum                                  */
/* Power-of-two meshes compute the force through the potential (Eqs. 3-5):  */
#define FPM_K_POT_FWD 15  /* z r2c + y forward, one slab-ordered launch      */
#define FPM_K_POT_X 16    /* x pass with the Green's function (1 field)      */
#define FPM_K_POT_INV 17  /* y inverse + z c2r to phi, one slab-ordered launch */
#define FPM_K_POT_GRAD 18 /* Eq. 5 difference of phi to the force meshes     */
#define FPM_K_PYRAMID 19  /* multi-grid pyramid force (Algorithm 3), all passes */
#define FPM_K_COUNT 20

/* Turn per-kernel-class timing on or off for this plan (off by default).
 * When on, every launch of the plan is bracketed by CUDA events recorded on
 * the launching stream; this adds no synchronisation.  enable: 0 off, 1
 * every class; FPM_PROFILE_ONLY(cls) times the launches of class cls only
 * (two events per such launch, the rest of the plan's work untouched). */
#define FPM_PROFILE_ONLY(cls) (2 + (cls))
int fpm_profile(fpm_plan* plan, int enable);

/* Synchronise `stream`, then return the accumulated device milliseconds and
 * launch counts per class since the last read (ms, launches: HOST arrays
 * of n >= FPM_K_COUNT entries), and reset them. */
int fpm_profile_read(fpm_plan* plan, double* ms, int64_t* launches, int n, void* stream);

/* Name of a kernel class (static string). */
const char* fpm_kernel_class_name(int cls);

/* Number of CUDA kernels this library has launched in this process. */
int64_t fpm_launch_count(void);

/* Device error flag of the plan (FPM_OK or FPM_EDEVICE / FPM_ETIMEOUT);
 * synchronises `stream`, then clears the flag. */
int fpm_status(fpm_plan* plan, void* stream);

/* Static description of an FPM_* code. */
const char* fpm_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* FPM_H */
