// internal.h -- host-side declarations shared by the translation units.
#pragma once
#include "common.cuh"

namespace fpm {

struct CosmoParams {
  double omega_m, omega_b, h, n_s, sigma8, t_cmb;
};

// Scalars of the EH no-wiggle transfer function, precomputed on the host
// for the per-mode FP32 evaluation.
struct EhParams {
  float h, s, alpha, omh, theta2, n_s;
};

// Per-size FFT tables on the device.
struct FftTables {
  int n = 0;
  float2* tw = nullptr;    // exp(-2 pi i m / n), m = 0..n-1 (host FP64, rounded)
  float* g = nullptr;      // gradient symbol of bin m, 0 at Nyquist: Eq. 5's (8 sin w - sin 2w)/6, or w
  float* w2 = nullptr;     // Laplacian symbol of bin m: w^2 (naive), or (2 sin(w/2))^2 (Eq. 4)
};                         // w = 2 pi f / n, f the signed frequency of bin m

// Buffers of the sort + paint pipeline.
struct PaintCtx {
  Geom g;
  size_t N = 0, M = 0;
  int ntiles = 0;
  uint32_t* keys = nullptr;        // [N]
  uint32_t* items = nullptr;       // [N] particle indices bucketed by tile
  uint16_t* cells = nullptr;       // [N] in-tile cell (key & 4095) of each item, written with the
                                   // cube bucketing; null: the paint recomputes it from dx
  uint32_t* tile_count = nullptr;  // [ntiles]
  uint32_t* tile_start = nullptr;  // [ntiles + 1]
  uint32_t* tile_cursor = nullptr; // [ntiles]
  unsigned long long* halo = nullptr;  // [ntiles * SHELL] fixed-point shell partials
  uint32_t* tile_done = nullptr;   // [ntiles] shells counted toward each tile's faces (zero between paints);
                                   // null: the faces are summed by a separate halo launch
  int* err = nullptr;
  int* big_flag = nullptr;
};

// cosmo.cu
int launch_sigma8(const CosmoParams& c, double* d_amp, cudaStream_t s);
int launch_growth(const double* d_a, int n, double om, double* d_raw, double* d_out, cudaStream_t s);
int launch_factors(const double* d_pts, int nsteps, double om, double* d_raw, double* d_gr, double* d_fac,
                   cudaStream_t s);

// fft.cu
// green: 0 naive w^2, 1 Eq. 4 discrete; grad: 0 Eq. 5 difference, 1 exact w.
// grad_scale s != 1 (with grad 0): the gradient symbol of a mesh s times
// finer at the same wavenumber, in this mesh's units: s g(w / s).
int fft_tables_create(FftTables* t, int n, int green = 0, int grad = 0, double grad_scale = 1.0);
void fft_tables_destroy(FftTables* t);
int fft_zfwd(const FftTables& t, const float* in, float2* spec, int nf, size_t in_fs, size_t out_fs,
             cudaStream_t s);
int fft_y(const FftTables& t, float2* spec, int nf, size_t fs, bool inverse, cudaStream_t s);
int fft_zinv(const FftTables& t, const float2* spec, float* out, int nf, size_t in_fs, size_t out_fs,
             cudaStream_t s);
int fft_xforce(const FftTables& t, const float2* in, float2* out, size_t out_fs, float coef, cudaStream_t s);
// c2r z pass of 3 fields written interleaved (float4 per cell); pow2 sizes only.
bool fft_has_interleaved(int n);
int fft_zinv3(const FftTables& t, const float2* spec, float4* out, size_t in_fs, cudaStream_t s);

// fft_slab.cu: the force through the potential, power-of-two meshes.
// ctr: 1 + n words of device scratch (zeroed by the calls); err: device flag.
bool fft_has_potential(int n);
int fft_slab_planes(int n);
int fft_pot_forward(const FftTables& t, const float* rho, float2* spec, unsigned* ctr, int* err, cudaStream_t s);
int fft_pot_xgreen(const FftTables& t, float2* spec, float coef, unsigned* ctr, int* err, cudaStream_t s);
int fft_pot_inverse(const FftTables& t, float2* spec, float* phi, unsigned* ctr, int* err, cudaStream_t s);
// F: interleaved float4 per cell (f4) or [3][M].
int fft_pot_gradient(const FftTables& t, const float* phi, float* F, bool f4, size_t M, cudaStream_t s);
// out = -sum_d D_d g_d, g = [3][n^3]: the transpose of the gradient
int fft_pot_divergence_neg(const FftTables& t, const float* g, float* out, cudaStream_t s);

// ic.cu
int fft_xlinear(const FftTables& t, const float2* in, float2* out, const EhParams& e, const double* d_amp,
                float kf, float n3v, cudaStream_t s);
int fft_xlpt_hessian(const FftTables& t, const float2* lin_k, float2* out, size_t out_fs, float coef,
                     cudaStream_t s);
int fft_xlpt_disp(const FftTables& t, const float2* specS, const float2* lin_k, float2* out, size_t out_fs,
                  const double* gr, float a0, float coef, bool second, cudaStream_t s);
int fft_xpower(const FftTables& t, const float2* sa, const float2* sb, double* bins, cudaStream_t s);
int launch_lpt_source(const float* phi, size_t n, float* S, cudaStream_t s);
// 2LPT through potentials (power-of-two lattices): psi = IFFT[coef lin/|w|^2]
// (x pass), the real-space source S of psi, and the two potentials of the
// displacement and the momentum (x pass with both outputs).
bool ic_has_potential(int n);
int fft_xpot(const FftTables& t, const float2* lin, float2* out, float coef, cudaStream_t s);
int fft_xdisp2(const FftTables& t, const float2* specS, const float2* lin, float2* out0, float2* out1,
               const double* gr, float a0, float coef, bool second, cudaStream_t s);
int launch_lpt_source_fd(int n, const float* psi, float* S, cudaStream_t s);
// the six phi_ij = IFFT[g_i g_j lin / |w|^2] / N^3 from psi, [6][n^3] (00, 11, 22, 01, 02, 12)
int launch_lpt_hessian_fd(int n, const float* psi, float* phi6, cudaStream_t s);

// paint.cu
int paint_setup();
Geom make_geom(int np, int nc);
size_t paint_halo_elems(int ntiles);
int launch_keys(const PaintCtx& c, const float* dx, cudaStream_t s);
int launch_scan(const PaintCtx& c, cudaStream_t s);
int launch_scatter(const PaintCtx& c, cudaStream_t s);
int launch_paint_tiles(const PaintCtx& c, const float* dx, float* rho, uint32_t* perm, cudaStream_t s);
int launch_perm_big(const PaintCtx& c, uint32_t* perm, cudaStream_t s);
int launch_halo(const PaintCtx& c, float* rho, cudaStream_t s);
int launch_readout(const PaintCtx& c, const float* F, const float* dx, float* f_out, cudaStream_t s);
// dx_out: where the drifted displacements go (null: dx itself; a separate
// buffer needs the brick traversal)
int launch_kdk(const PaintCtx& c, float* dx, float* p, const float* F, bool f4, const double* fac, int ik1,
               int ik2, int idr, bool emit_keys, cudaStream_t s, float* dx_out = nullptr);
// readout.cu: whether launch_kdk takes the brick traversal (and so accepts a
// separate dx_out)
bool kdk_brick_fits(const PaintCtx& c, bool f4);
// readout.cu: the brick traversal of the fused readout (interleaved float4
// force, lattice divisible by the brick); keys == nullptr emits no keys.
int launch_kdk_brick(const PaintCtx& c, const float* dx, float* dx_out, float* p, const float4* F, const double* fac,
                     int ik1, int ik2, int idr, uint32_t* keys, cudaStream_t s);

// paint.cu: adjoints at fixed positions
// v_i = K v[i] with K from vk (scaled v needs the brick gather: FPM_EINVAL elsewhere)
int launch_gather_adj(const PaintCtx& c, const float* dx, const float* g_rho, const float* F, bool f4,
                      const float* v, float* g_dx, bool accumulate, cudaStream_t s, KScale vk = KScale{});
// The three channels v_i = K v[ch][i] (K from vk); vmax_ready: *vmax
// already holds max |K v| (bit pattern), e.g. from launch_gather_adj_dk.
// With halo3 (3 shell buffers of paint_halo_elems) and done3 (3 x ntiles
// face counters, zero between paints) meshes of at most VEC3_MAX_TILES
// tiles (nc <= 128) have their channels painted by one launch, side by side
// (one channel's 512 tiles alone leave most of the GPU idle: 128^3 forward
// + adjoint 3.90 -> 3.63 ms); larger meshes, or without the buffers, take
// one launch per channel on the plan's buffers (at 512^3 the side-by-side
// launch measured slower, 4.53 vs 4.34 ms per reverse step).
constexpr int VEC3_MAX_TILES = 512;
int launch_paint_vec(const PaintCtx& c, const float* dx, const float* v, KScale vk, unsigned* vmax, float* out,
                     cudaStream_t s, bool vmax_ready = false, unsigned long long* halo3 = nullptr,
                     uint32_t* done3 = nullptr);
// launch_gather_adj (accumulating, float4 force, brick lattices) with the
// cotangent velocities v = K gp taken from the momentum cotangents gp (K
// from vk), followed per particle by the next reverse step's drift and kick
// transposes (gp += D g_dx in place, K' from fac[ik1] (+ fac[ik2])) and
// max |K' gp| into *vmax; FPM_ENOTIMPL where the lattice or layout has no
// brick gather (the caller then runs them apart).
int launch_gather_adj_dk(const PaintCtx& c, const float* dx, const float* g_rho, const float* F, bool f4, float* gp,
                         KScale vk, float* g_dx, const double* fac, int idr, int ik1, int ik2, unsigned* vmax,
                         cudaStream_t s);

// adjoint.cu: spectral adjoints (power-of-two sizes) and elementwise steps
enum SrcKernel : int {
  SK_FORCE_NEG = 0,   // -i g_d 1.5 Om / |w|^2   (transpose of the force operator, axis d)
  SK_B = 1,           // i g_d / |w|^2            (B_d: displacement from density, axis d)
  SK_BCONJ = 2,       // -i g_d / |w|^2           (B_d^T)
  SK_H = 3,           // g_i g_j / |w|^2          (H_ij, second derivatives)
  SK_LINEAR = 4,      // sqrt(P(|k|) N^3 / V)     (linear-field transfer)
};
struct XSource {
  const float2* spec;   // half spectrum [kx][kz][ky]
  int kind;             // SrcKernel
  int a, b;             // axes (d, or i and j)
  int in_k;             // 1: already in k space, 0: x axis still to transform
};
constexpr int XCOMBINE_MAX = 9;
// out = sum_s K_s(k) X_s(k) * coef, then an inverse x transform when
// inverse != 0 (out stays in k space otherwise).  out may alias a source.
int fft_xcombine(const FftTables& t, const XSource* src, int nsrc, float coef, double omega_m, const EhParams* eh,
                 const double* d_amp, float kf, float n3v, float2* out, int inverse, cudaStream_t s);
int launch_adam(float* x, const float* g, float* m, float* v, size_t n, float gscale, float pscale, float lr,
                float b1, float b2, float o1, float o2, float eps, float c1, float c2, double* partial, int npartial,
                double* prior, cudaStream_t s);
int launch_chi2(const float* rho, const float* target, size_t M, float sigma, float* g_rho, double* partial,
                int npartial, double* loss, cudaStream_t s);
int launch_adj_drift_kick(float* gx, float* gp, float* v, size_t n, const double* fac, int idr, int ik1, int ik2,
                          cudaStream_t s);
int launch_scale_copy(const float* src, float* dst, size_t n, const double* fac, int ik, cudaStream_t s);
int launch_lpt_gpsi(const float* gdx, const float* gp, size_t n, const double* gr, float a0, float r, float* out6,
                    cudaStream_t s);
int launch_lpt_gphi(const float* gS, float* phi6, size_t n, cudaStream_t s);

// batch.cu: many simulations, one persistent launch per step
struct BatchPlanView {
  PaintCtx pc;
  int nc = 0, np = 0, f4 = 0;
  float* F = nullptr;
  float* rho = nullptr;
  float2* spec = nullptr;
  size_t specmax = 0;
  const double* fac = nullptr;
  FftTables tab;
  float force_coef = 0.f;
};
struct Batch;
bool batch_size_ok(int nc, int np);

// Multi-grid pyramid force (pyramid.cu): coarse mesh nc >> levels, split^3
// local blocks of nc/split cells padded by `halo` (B = nc/split + 2 halo).
struct Pyramid {
  int nc = 0, levels = 0, split = 0, halo = 0, nco = 0, m = 0, B = 0;
  int block_bandpass = 1;           // band-pass each padded block before cropping (else the assembled F_S)
  int matched = 1;                  // coarse force with the fine mesh's operator (else coarse-cell Eq. 5)
  float* bco = nullptr;             // REDUCEd block force [3][(B >> levels)^3] (block band-pass)
  size_t spec_co = 0, spec_b = 0;   // complex elements of one coarse / block half spectrum
  FftTables tco, tb;                // coarse and block FFT tables (default force kernel)
  float* dco = nullptr;             // coarse density contrast, nco^3
  float2* sco = nullptr;            // 3 coarse half spectra
  float* FL = nullptr;              // coarse force [3][nco^3], then F_L - REDUCE(F_S)
  float* blk = nullptr;             // padded block density, B^3
  float2* sb = nullptr;             // 3 block half spectra
  float* Fb = nullptr;              // block force [3][B^3]
  float* FS = nullptr;              // short-range force [3][nc^3]
  float* ping = nullptr;            // resampling scratch, 3 max(nc^3, B^3) / 2 each
  float* pong = nullptr;
  int64_t bytes = 0;
};
int pyramid_create(Pyramid* y, int nc, int levels, int split, int halo, int block_bandpass, int matched);
void pyramid_destroy(Pyramid* y);
// Force meshes of rho (mean 1) by Algorithm 3: planar F[3][nc^3] or float4
// per cell (f4); `launches` is incremented by the kernels enqueued.
int pyramid_force(const Pyramid& y, const float* rho, float* F, bool f4, double omega_m, unsigned* ctr, int* err,
                  cudaStream_t s, int* launches);
int batch_create(Batch** out, const BatchPlanView* views, int nsims);
void batch_destroy(Batch* b);
int batch_configure(Batch* b, int blocks_per_sm, int ro_iters, long long spin_limit);
int batch_kdk(Batch* b, float* const* dx, float* const* p, int nsteps, cudaStream_t s);
int batch_status(Batch* b, cudaStream_t s);
int batch_info(const Batch* b, int* grid, int* graph_captured);
int batch_phase_times(Batch* b, double* ms, int n, cudaStream_t s);
// Per-mesh-size configuration of the batched step (every simulation of mesh nc):
enum BatchTuneKnob : int { BT_READOUT = 0, BT_PAINT_TILE = 1, BT_FFT_SLOTS = 2 };
int batch_tune(Batch* b, int nc, int knob, int value);

inline size_t spec_elems(int n) { return (size_t)n * (n / 2 + 1) * n; }

}  // namespace fpm
