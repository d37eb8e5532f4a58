// api.cu -- the extern "C" entry points of libfpm and the plan that owns the
// scratch.  Every entry point validates its arguments on the host, then
// enqueues kernels on the caller's stream; nothing runs on the CPU.
#include "internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <utility>
#include <vector>

using namespace fpm;

namespace {
std::atomic<long long> g_launches{0};

// Optional per-kernel-class timing: an event pair around each launch.
struct Profiler {
  bool on = false;
  int only = -1;               // >= 0: time only the launches of this class
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<int, size_t>> recs;   // (class, index of the start event)
  cudaEvent_t next() {
    if (used == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[used++];
  }
};
}  // namespace

struct fpm_plan {
  int np = 0, nc = 0;
  double box = 0;
  CosmoParams cosmo{};
  EhParams eh{};
  size_t N = 0, M = 0;
  FftTables tc, tp;            // mesh (nc) and lattice (np) tables
  bool share_tables = false;
  FftTables tf;                // force tables of a non-default force kernel (else tc is used)
  bool own_tf = false;
  int green = FPM_GREEN_NAIVE, grad = FPM_GRAD_FD4;
  Pyramid* pyr = nullptr;      // multi-grid force (Algorithm 3) when set
  int pyr_block = 1;           // its reading: band-pass per padded block (else on the assembled F_S)
  int pyr_matched = 1;         // and the fine mesh's operator on the coarse mesh (else coarse-cell Eq. 5)
  bool f4 = false;             // internal force meshes interleaved (float4 per cell)
  size_t specmax = 0;          // complex elements of one half spectrum
  float2* spec = nullptr;      // 6 half spectra
  float* real6 = nullptr;      // 6 real lattice fields (2LPT Hessian)
  float* rho = nullptr;        // density mesh
  float* F = nullptr;          // 3 force meshes
  unsigned* slab_ctr = nullptr;  // work counters of the slab-ordered FFT launches
  PaintCtx pc;
  double* d_amp = nullptr;     // P(k) amplitude (sigma8 normalisation)
  double* d_pts = nullptr;     // scale factors of a coefficient request
  double* d_raw = nullptr;
  double* d_gr = nullptr;
  double* d_fac = nullptr;
  std::vector<double> fac_pts;   // the points (stages, half stages) d_fac was computed for
  double* d_bins = nullptr;
  int* d_err = nullptr;
  int64_t scratch_bytes = 0;
  Profiler prof;
  // adjoint scratch, allocated by the first adjoint call
  float2* aspec = nullptr;     // 9 half spectra of the lattice
  float* adj6 = nullptr;       // 6 lattice fields (cotangents of Psi1, Psi2)
  float* gS = nullptr;         // lattice field (cotangent of the 2LPT source)
  float* gF = nullptr;         // 3 meshes (cotangent of the force meshes)
  float* vbuf = nullptr;       // [3][N] kick-weighted momentum cotangent
  unsigned* vmax = nullptr;    // max |v| bits for the signed fixed point
  unsigned long long* halo3 = nullptr;   // 3 shell buffers of the three-channel vector paint
  uint32_t* done3 = nullptr;   // its 3 x ntiles face counters (zero between paints)
  double* partial = nullptr;   // chi^2 block partials
  double* d_loss = nullptr;
};

namespace {

constexpr int MAX_STEPS = 2048;

bool size_ok(int n) { return fft_size_ok(n); }

template <typename T>
int dalloc(fpm_plan* p, T** ptr, size_t count) {
  if (count == 0) {
    *ptr = nullptr;
    return FPM_OK;
  }
  if (cudaMalloc(reinterpret_cast<void**>(ptr), count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return FPM_ENOMEM;
  }
  p->scratch_bytes += (int64_t)(count * sizeof(T));
  return FPM_OK;
}

void free_plan(fpm_plan* p) {
  if (!p) return;
  cudaFree(p->spec);
  cudaFree(p->real6);
  cudaFree(p->rho);
  cudaFree(p->F);
  cudaFree(p->slab_ctr);
  cudaFree(p->pc.keys);
  cudaFree(p->pc.items);
  cudaFree(p->pc.cells);
  cudaFree(p->pc.tile_count);
  cudaFree(p->pc.tile_start);
  cudaFree(p->pc.tile_cursor);
  cudaFree(p->pc.tile_done);
  cudaFree(p->pc.halo);
  cudaFree(p->pc.big_flag);
  cudaFree(p->d_amp);
  cudaFree(p->d_pts);
  cudaFree(p->d_raw);
  cudaFree(p->d_gr);
  cudaFree(p->d_fac);
  cudaFree(p->d_bins);
  cudaFree(p->d_err);
  cudaFree(p->aspec);
  cudaFree(p->adj6);
  cudaFree(p->halo3);
  cudaFree(p->done3);
  cudaFree(p->gS);
  cudaFree(p->gF);
  cudaFree(p->vbuf);
  cudaFree(p->vmax);
  cudaFree(p->partial);
  cudaFree(p->d_loss);
  for (cudaEvent_t e : p->prof.pool) cudaEventDestroy(e);
  if (p->tc.tw) fft_tables_destroy(&p->tc);
  if (!p->share_tables && p->tp.tw) fft_tables_destroy(&p->tp);
  if (p->own_tf) fft_tables_destroy(&p->tf);
  if (p->pyr) {
    pyramid_destroy(p->pyr);
    delete p->pyr;
  }
  delete p;
}

EhParams make_eh(const CosmoParams& c) {
  // EH98 eqs. 26 and 31: sound horizon (Mpc) and the baryon suppression.
  const double wm = c.omega_m * c.h * c.h, wb = c.omega_b * c.h * c.h, fb = c.omega_b / c.omega_m;
  EhParams e;
  e.h = (float)c.h;
  e.s = (float)(44.5 * log(9.83 / wm) / sqrt(1.0 + 10.0 * pow(wb, 0.75)));
  e.alpha = (float)(1.0 - 0.328 * log(431.0 * wm) * fb + 0.38 * log(22.3 * wm) * fb * fb);
  e.omh = (float)(c.omega_m * c.h);
  e.theta2 = (float)((c.t_cmb / 2.7) * (c.t_cmb / 2.7));
  e.n_s = (float)c.n_s;
  return e;
}

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Copy n doubles from the host and append 1.0 (the growth normalisation point).
int stage_points(fpm_plan* p, const double* host, int n, cudaStream_t s) {
  std::vector<double> v(host, host + n);
  v.push_back(1.0);
  FPM_CUDA_TRY(cudaMemcpyAsync(p->d_pts, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  // pageable source: the copy is staged before the call returns, but keep
  // the vector alive until the stream has consumed it
  FPM_CUDA_TRY(cudaStreamSynchronize(s));
  return FPM_OK;
}

// Run one launcher (which enqueues `nk` kernels) and, when profiling,
// bracket it with events on the same stream.
template <typename Fn>
int timed(fpm_plan* p, int cls, int nk, cudaStream_t s, Fn fn) {
  size_t i0 = 0;
  const bool rec = p->prof.on && (p->prof.only < 0 || p->prof.only == cls);
  if (rec) {
    i0 = p->prof.used;
    cudaEvent_t a = p->prof.next();
    if (!a || cudaEventRecord(a, s) != cudaSuccess) return FPM_ECUDA;
  }
  const int rc = fn();
  g_launches += nk;
  if (rec) {
    cudaEvent_t b = p->prof.next();
    if (!b || cudaEventRecord(b, s) != cudaSuccess) return FPM_ECUDA;
    p->prof.recs.push_back({cls, i0});
  }
  return rc;
}

// Tables of the plan's force kernel (Green's function and gradient symbols).
const FftTables& force_tables(const fpm_plan* p) { return p->own_tf ? p->tf : p->tc; }

// The potential form F_d = D_d phi needs the gradient to be Eq. 5's
// real-space difference; the exact gradient takes the three-field path.
bool force_via_potential(const fpm_plan* p) { return fft_has_potential(p->nc) && p->grad == FPM_GRAD_FD4; }

int force_impl(fpm_plan* p, const float* rho, float* F, cudaStream_t s, bool interleaved = false) {
  if (p->pyr)
    return timed(p, FPM_K_PYRAMID, 0, s, [&] {
      int nl = 0;
      const int rc = pyramid_force(*p->pyr, rho, F, interleaved, p->cosmo.omega_m, p->slab_ctr, p->d_err, s, &nl);
      g_launches += nl;
      return rc;
    });
  const FftTables& t = force_tables(p);
  const float coef = (float)(1.5 * p->cosmo.omega_m / (double)p->M);
  if (force_via_potential(p)) {
    // phi = IFFT[coef delta / |w|^2] in the second half spectrum's memory,
    // then F_d = D_d phi (the Eq. 5 difference) in real space
    float* phi = reinterpret_cast<float*>(p->spec + p->specmax);
    const int fused = t.n >= 128 ? 1 : 2;
    FPM_TRY(timed(p, FPM_K_POT_FWD, fused, s,
                  [&] { return fft_pot_forward(t, rho, p->spec, p->slab_ctr, p->d_err, s); }));
    FPM_TRY(timed(p, FPM_K_POT_X, 1, s, [&] { return fft_pot_xgreen(t, p->spec, coef, p->slab_ctr, p->d_err, s); }));
    FPM_TRY(timed(p, FPM_K_POT_INV, fused, s,
                  [&] { return fft_pot_inverse(t, p->spec, phi, p->slab_ctr, p->d_err, s); }));
    return timed(p, FPM_K_POT_GRAD, 1, s, [&] { return fft_pot_gradient(t, phi, F, interleaved, p->M, s); });
  }
  FPM_TRY(timed(p, FPM_K_FFT_ZF, 1, s, [&] { return fft_zfwd(t, rho, p->spec, 1, 0, 0, s); }));
  FPM_TRY(timed(p, FPM_K_FFT_YF, 1, s, [&] { return fft_y(t, p->spec, 1, 0, false, s); }));
  FPM_TRY(timed(p, FPM_K_FFT_X, 1, s, [&] { return fft_xforce(t, p->spec, p->spec, p->specmax, coef, s); }));
  FPM_TRY(timed(p, FPM_K_FFT_YI, 1, s, [&] { return fft_y(t, p->spec, 3, p->specmax, true, s); }));
  FPM_TRY(timed(p, FPM_K_FFT_ZI, 1, s, [&] {
    return interleaved ? fft_zinv3(t, p->spec, reinterpret_cast<float4*>(F), p->specmax, s)
                       : fft_zinv(t, p->spec, F, 3, p->specmax, p->M, s);
  }));
  return FPM_OK;
}

// Sort the particles (keys already in c.keys, tile histogram filled) and paint.
int sort_paint_impl(fpm_plan* p, const PaintCtx& c, const float* dx, float* rho, uint32_t* perm, cudaStream_t s) {
  FPM_TRY(timed(p, FPM_K_SCAN, 1, s, [&] { return launch_scan(c, s); }));
  FPM_TRY(timed(p, FPM_K_SCATTER, 1, s, [&] { return launch_scatter(c, s); }));
  FPM_TRY(timed(p, FPM_K_PAINT, 1, s, [&] { return launch_paint_tiles(c, dx, rho, perm, s); }));
  if (perm) FPM_TRY(timed(p, FPM_K_PAINT, 1, s, [&] { return launch_perm_big(c, perm, s); }));
  if (perm || !c.tile_done) FPM_TRY(timed(p, FPM_K_HALO, 1, s, [&] { return launch_halo(c, rho, s); }));
  return FPM_OK;
}

int paint_impl(fpm_plan* p, const float* dx, float* rho, uint32_t* keys, uint32_t* perm, cudaStream_t s) {
  PaintCtx c = p->pc;
  if (keys) c.keys = keys;
  FPM_TRY(timed(p, FPM_K_KEYS, 1, s, [&] { return launch_keys(c, dx, s); }));
  return sort_paint_impl(p, c, dx, rho, perm, s);
}

// One stage of a force checkpoint: the force mesh (4 nc^3 floats), then the
// tile buckets of the stage's positions -- items (np^3 u32), in-tile cells
// (np^3 u16), tile starts (ntiles + 1 u32) -- padded to 64 floats.
size_t ckpt_stage_floats(const fpm_plan* p) {
  const size_t f = 4 * p->M + p->N + (p->N + 1) / 2 + (size_t)p->pc.ntiles + 1;
  return (f + 63) & ~(size_t)63;
}

// The plan's paint context with its buckets in stage k of fckpt.
PaintCtx stage_ctx(const fpm_plan* p, const float* fckpt, int k) {
  PaintCtx c = p->pc;
  float* b = const_cast<float*>(fckpt) + (size_t)k * ckpt_stage_floats(p) + 4 * p->M;
  c.items = reinterpret_cast<uint32_t*>(b);
  c.cells = reinterpret_cast<uint16_t*>(b + p->N);
  c.tile_start = reinterpret_cast<uint32_t*>(b + p->N + (p->N + 1) / 2);
  return c;
}

}  // namespace

extern "C" {

const char* fpm_strerror(int code) {
  switch (code) {
    case FPM_OK: return "ok";
    case FPM_EINVAL: return "invalid argument";
    case FPM_ENOMEM: return "device allocation failed";
    case FPM_ECUDA: return "CUDA runtime error";
    case FPM_ETIMEOUT: return "bounded device wait ran out";
    case FPM_EDEVICE: return "device error flag set (non-finite or out-of-range particle)";
    case FPM_ENOTIMPL: return "not implemented";
    default: return "unknown error";
  }
}

int fpm_plan_create(fpm_plan** out, int np, int nc, double box, const fpm_cosmo* cosmo, void* stream) {
  if (!out || !cosmo) return FPM_EINVAL;
  if (!size_ok(np) || !size_ok(nc) || nc % np != 0 || nc / np > 4 || nc % TILE != 0) return FPM_EINVAL;
  if (!(box > 0) || !(cosmo->omega_m > 0 && cosmo->omega_m <= 1) || !(cosmo->h > 0) || !(cosmo->sigma8 > 0) ||
      !(cosmo->omega_b >= 0 && cosmo->omega_b < cosmo->omega_m) || !(cosmo->t_cmb > 0) || !isfinite(cosmo->n_s))
    return FPM_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return FPM_ECUDA;
  }
  cudaStream_t s = S(stream);
  fpm_plan* p = new fpm_plan();
  p->np = np;
  p->nc = nc;
  p->box = box;
  p->cosmo = CosmoParams{cosmo->omega_m, cosmo->omega_b, cosmo->h, cosmo->n_s, cosmo->sigma8, cosmo->t_cmb};
  p->eh = make_eh(p->cosmo);
  p->N = (size_t)np * np * np;
  p->M = (size_t)nc * nc * nc;
  int rc = FPM_OK;
#define TRY(x)              \
  do {                      \
    rc = (x);               \
    if (rc != FPM_OK) {     \
      free_plan(p);         \
      return rc;            \
    }                       \
  } while (0)
  TRY(paint_setup());
  TRY(fft_tables_create(&p->tc, nc));
  if (np == nc) {
    p->tp = p->tc;
    p->share_tables = true;
  } else {
    TRY(fft_tables_create(&p->tp, np));
  }
  p->specmax = spec_elems(nc);
  TRY(dalloc(p, &p->spec, 6 * p->specmax));
  TRY(dalloc(p, &p->real6, 6 * p->N));
  TRY(dalloc(p, &p->rho, p->M));
  TRY(dalloc(p, &p->F, 4 * p->M));
  TRY(dalloc(p, &p->slab_ctr, (size_t)(1 + MAX_N)));
  p->f4 = fft_has_interleaved(nc);
  PaintCtx& c = p->pc;
  c.g = make_geom(np, nc);
  c.N = p->N;
  c.M = p->M;
  c.ntiles = c.g.nt * c.g.nt * c.g.nt;
  TRY(dalloc(p, &c.keys, p->N));
  TRY(dalloc(p, &c.items, p->N));
  TRY(dalloc(p, &c.cells, p->N));
  TRY(dalloc(p, &c.tile_count, (size_t)c.ntiles));
  TRY(dalloc(p, &c.tile_start, (size_t)c.ntiles + 1));
  TRY(dalloc(p, &c.tile_cursor, (size_t)c.ntiles));
  TRY(dalloc(p, &c.halo, paint_halo_elems(c.ntiles)));
  TRY(dalloc(p, &c.tile_done, (size_t)c.ntiles));
  if (cudaMemsetAsync(c.tile_done, 0, sizeof(uint32_t) * c.ntiles, s) != cudaSuccess) TRY(FPM_ECUDA);
  TRY(dalloc(p, &c.big_flag, 1));
  TRY(dalloc(p, &p->d_amp, 1));
  TRY(dalloc(p, &p->d_pts, 2 * MAX_STEPS + 2));
  TRY(dalloc(p, &p->d_raw, 4 * (2 * MAX_STEPS + 2)));
  TRY(dalloc(p, &p->d_gr, 6 * (2 * MAX_STEPS + 2)));
  TRY(dalloc(p, &p->d_fac, 3 * MAX_STEPS));
  TRY(dalloc(p, &p->d_bins, 3 * (size_t)(nc / 2)));
  TRY(dalloc(p, &p->d_err, 1));
  c.err = p->d_err;
  if (cudaMemsetAsync(p->d_err, 0, sizeof(int), s) != cudaSuccess) TRY(FPM_ECUDA);
  TRY(launch_sigma8(p->cosmo, p->d_amp, s));
  g_launches += 1;
  if (cudaStreamSynchronize(s) != cudaSuccess) TRY(FPM_ECUDA);
#undef TRY
  *out = p;
  return FPM_OK;
}

void fpm_plan_destroy(fpm_plan* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  free_plan(p);
}

int64_t fpm_plan_scratch_bytes(const fpm_plan* p) { return p ? p->scratch_bytes : 0; }

int fpm_growth(fpm_plan* p, const double* a, int n, double* out, void* stream) {
  if (!p || !a || !out || n <= 0 || n > 2 * MAX_STEPS + 1) return FPM_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!(a[i] > 1e-5 && a[i] <= 10.0)) return FPM_EINVAL;
  cudaStream_t s = S(stream);
  FPM_TRY(stage_points(p, a, n, s));
  FPM_TRY(timed(p, FPM_K_COEF, 2, s, [&] { return launch_growth(p->d_pts, n, p->cosmo.omega_m, p->d_raw, p->d_gr, s); }));
  std::vector<double> rows(6 * (size_t)n);
  FPM_CUDA_TRY(cudaMemcpyAsync(rows.data(), p->d_gr, rows.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  FPM_CUDA_TRY(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 5; ++k) out[5 * i + k] = rows[6 * i + k];
  return FPM_OK;
}

int fpm_linear_field(fpm_plan* p, const float* white, void* lin_k, void* stream) {
  if (!p || !white || !lin_k) return FPM_EINVAL;
  cudaStream_t s = S(stream);
  const FftTables& t = p->tp;
  float2* out = reinterpret_cast<float2*>(lin_k);
  const double n3v = (double)p->N / (p->box * p->box * p->box);
  const bool pot = fft_has_potential(p->np);
  return timed(p, FPM_K_IC, pot && p->np >= 128 ? 2 : 3, s, [&] {
    if (pot) {
      FPM_TRY(fft_pot_forward(t, white, p->spec, p->slab_ctr, p->d_err, s));
    } else {
      FPM_TRY(fft_zfwd(t, white, p->spec, 1, 0, 0, s));
      FPM_TRY(fft_y(t, p->spec, 1, 0, false, s));
    }
    return fft_xlinear(t, p->spec, out, p->eh, p->d_amp, (float)(6.283185307179586 / p->box), (float)n3v, s);
  });
}

int fpm_lpt(fpm_plan* p, const void* lin_k, double a0, int order, float* dx, float* mom, void* stream) {
  if (!p || !lin_k || !dx || !mom || (order != 1 && order != 2) || !(a0 > 1e-5 && a0 <= 10.0))
    return FPM_EINVAL;
  cudaStream_t s = S(stream);
  const FftTables& t = p->tp;
  const float2* lk = reinterpret_cast<const float2*>(lin_k);
  FPM_TRY(stage_points(p, &a0, 1, s));
  FPM_TRY(timed(p, FPM_K_COEF, 2, s, [&] { return launch_growth(p->d_pts, 1, p->cosmo.omega_m, p->d_raw, p->d_gr, s); }));
  const float inv_n3 = (float)(1.0 / (double)p->N);
  const bool second = order == 2;
  const float r = (float)(p->nc / p->np);
  if (ic_has_potential(p->np)) {
    // psi = IFFT[lin / |w|^2] / N^3, S from its real-space second differences,
    // then the displacement and momentum potentials and their Eq. 5 gradients
    float* psi = p->real6;
    float* phx = p->real6 + p->N;
    float* php = p->real6 + 2 * p->N;
    float2* s0 = p->spec;
    float2* s1 = p->spec + p->specmax;
    float2* s2 = p->spec + 2 * p->specmax;
    const int fused = p->np >= 128 ? 1 : 2;
    return timed(p, FPM_K_IC, second ? 5 + 4 * fused : 3 + 2 * fused, s, [&] {
      if (second) {
        FPM_TRY(fft_xpot(t, lk, s0, inv_n3, s));
        FPM_TRY(fft_pot_inverse(t, s0, psi, p->slab_ctr, p->d_err, s));
        FPM_TRY(launch_lpt_source_fd(p->np, psi, p->rho, s));
        FPM_TRY(fft_pot_forward(t, p->rho, s0, p->slab_ctr, p->d_err, s));
      }
      FPM_TRY(fft_xdisp2(t, s0, lk, s1, s2, p->d_gr, (float)a0, inv_n3 * r, second, s));
      FPM_TRY(fft_pot_inverse(t, s1, phx, p->slab_ctr, p->d_err, s));
      FPM_TRY(fft_pot_inverse(t, s2, php, p->slab_ctr, p->d_err, s));
      FPM_TRY(fft_pot_gradient(t, phx, dx, false, p->N, s));
      return fft_pot_gradient(t, php, mom, false, p->N, s);
    });
  }
  return timed(p, FPM_K_IC, second ? 11 : 4, s, [&] {
    if (second) {
      FPM_TRY(fft_xlpt_hessian(t, lk, p->spec, p->specmax, inv_n3, s));
      FPM_TRY(fft_y(t, p->spec, 6, p->specmax, true, s));
      FPM_TRY(fft_zinv(t, p->spec, p->real6, 6, p->specmax, p->N, s));
      FPM_TRY(launch_lpt_source(p->real6, p->N, p->rho, s));
      FPM_TRY(fft_zfwd(t, p->rho, p->spec, 1, 0, 0, s));
      FPM_TRY(fft_y(t, p->spec, 1, 0, false, s));
    }
    FPM_TRY(fft_xlpt_disp(t, p->spec, lk, p->spec, p->specmax, p->d_gr, (float)a0, inv_n3 * r, second, s));
    FPM_TRY(fft_y(t, p->spec, 6, p->specmax, true, s));
    FPM_TRY(fft_zinv(t, p->spec, dx, 3, p->specmax, p->N, s));
    return fft_zinv(t, p->spec + 3 * p->specmax, mom, 3, p->specmax, p->N, s);
  });
}

int fpm_paint(fpm_plan* p, const float* dx, float* rho, uint32_t* key_out, uint32_t* perm_out, void* stream) {
  if (!p || !dx || !rho) return FPM_EINVAL;
  return paint_impl(p, dx, rho, key_out, perm_out, S(stream));
}

int fpm_force(fpm_plan* p, const float* rho, float* F, void* stream) {
  if (!p || !rho || !F) return FPM_EINVAL;
  return force_impl(p, rho, F, S(stream));
}

int fpm_readout(fpm_plan* p, const float* F, const float* dx, float* f_out, void* stream) {
  if (!p || !F || !dx || !f_out) return FPM_EINVAL;
  cudaStream_t s = S(stream);
  return timed(p, FPM_K_READOUT, 1, s, [&] { return launch_readout(p->pc, F, dx, f_out, s); });
}

int fpm_kdk(fpm_plan* p, float* dx, float* mom, const double* a, int nsteps, float* ckpt, float* fckpt,
            void* stream) {
  if (!p || !dx || !mom || !a || nsteps < 0 || nsteps > MAX_STEPS) return FPM_EINVAL;
  if (nsteps == 0) return FPM_OK;
  for (int k = 0; k <= nsteps; ++k)
    if (!(a[k] > 1e-5 && a[k] <= 10.0) || (k > 0 && !(a[k] > a[k - 1]))) return FPM_EINVAL;
  cudaStream_t s = S(stream);
  std::vector<double> pts(a, a + nsteps + 1);
  for (int k = 0; k < nsteps; ++k) pts.push_back(sqrt(a[k] * a[k + 1]));
  FPM_TRY(stage_points(p, pts.data(), (int)pts.size(), s));
  FPM_TRY(timed(p, FPM_K_COEF, 3, s, [&] {
    return launch_factors(p->d_pts, nsteps, p->cosmo.omega_m, p->d_raw, p->d_gr, p->d_fac, s);
  }));
  p->fac_pts = pts;
  const size_t N = p->N;
  // the force of stage k is computed straight into its checkpoint slot, and
  // the stage's tile buckets are written there by its sort
  auto Fk = [&](int k) { return fckpt ? fckpt + (size_t)k * ckpt_stage_floats(p) : p->F; };
  auto Ck = [&](int k) { return fckpt ? stage_ctx(p, fckpt, k) : p->pc; };
  // with checkpoints and the brick readout, the drift of step k writes
  // straight into stage k+1 of ckpt and the steps run on the checkpoints
  // (the closing kick writes dx): no copies
  const bool in_ckpt = ckpt && kdk_brick_fits(p->pc, p->f4);
  auto X = [&](int k) { return in_ckpt ? ckpt + (size_t)k * 3 * N : dx; };
  if (ckpt) FPM_CUDA_TRY(cudaMemcpyAsync(ckpt, dx, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  {
    const PaintCtx c0 = Ck(0);
    FPM_TRY(timed(p, FPM_K_KEYS, 1, s, [&] { return launch_keys(c0, dx, s); }));
    FPM_TRY(sort_paint_impl(p, c0, dx, p->rho, nullptr, s));
  }
  FPM_TRY(force_impl(p, p->rho, Fk(0), s, p->f4));
  for (int k = 0; k < nsteps; ++k) {
    // closing kick of step k-1 and opening kick of step k share the force at a_k
    const int ik2 = k > 0 ? 3 * (k - 1) + 2 : -1;
    FPM_TRY(timed(p, FPM_K_KDK, 1, s, [&] {
      return launch_kdk(p->pc, X(k), mom, Fk(k), p->f4, p->d_fac, 3 * k + 0, ik2, 3 * k + 1, true, s, X(k + 1));
    }));
    if (ckpt && !in_ckpt)
      FPM_CUDA_TRY(cudaMemcpyAsync(ckpt + (size_t)(k + 1) * 3 * N, dx, 3 * N * sizeof(float),
                                   cudaMemcpyDeviceToDevice, s));
    FPM_TRY(sort_paint_impl(p, Ck(k + 1), X(k + 1), p->rho, nullptr, s));
    FPM_TRY(force_impl(p, p->rho, Fk(k + 1), s, p->f4));
  }
  return timed(p, FPM_K_KDK, 1, s, [&] {
    return launch_kdk(p->pc, X(nsteps), mom, Fk(nsteps), p->f4, p->d_fac, 3 * (nsteps - 1) + 2, -1, -1, false, s,
                      dx);
  });
}

static int set_pyramid_impl(fpm_plan* p, int levels, int split, int halo) {
  if (levels > 0) {
    const int nco = levels <= 2 ? p->nc >> levels : 0;
    const int B = p->nc / (split > 0 ? split : 1) + 2 * halo;
    if (levels > 2 || split < 1 || halo < 0 || p->nc % split != 0 || (nco << levels) != p->nc ||
        !size_ok(nco) || !size_ok(B) || (p->pyr_block && B % (1 << levels) != 0))
      return FPM_EINVAL;
  }
  FPM_CUDA_TRY(cudaDeviceSynchronize());
  if (p->pyr) {
    pyramid_destroy(p->pyr);
    delete p->pyr;
    p->pyr = nullptr;
  }
  if (levels == 0) return FPM_OK;
  Pyramid* y = new Pyramid();
  const int rc = pyramid_create(y, p->nc, levels, split, halo, p->pyr_block, p->pyr_matched);
  if (rc != FPM_OK) {
    pyramid_destroy(y);
    delete y;
    return rc == FPM_ECUDA ? FPM_ENOMEM : rc;
  }
  p->pyr = y;
  return FPM_OK;
}

int fpm_set_pyramid(fpm_plan* p, int levels, int split, int halo) {
  if (!p || levels < 0) return FPM_EINVAL;
  return set_pyramid_impl(p, levels, split, halo);
}

int fpm_set_pyramid_reading(fpm_plan* p, int bandpass, int coarse_kernel) {
  if (!p || (bandpass != FPM_PYR_BANDPASS_BLOCK && bandpass != FPM_PYR_BANDPASS_GLOBAL) ||
      (coarse_kernel != FPM_PYR_KERNEL_MATCHED && coarse_kernel != FPM_PYR_KERNEL_COARSE))
    return FPM_EINVAL;
  const int block = bandpass == FPM_PYR_BANDPASS_BLOCK, matched = coarse_kernel == FPM_PYR_KERNEL_MATCHED;
  if (block == p->pyr_block && matched == p->pyr_matched) return FPM_OK;
  const int old_block = p->pyr_block, old_matched = p->pyr_matched;
  p->pyr_block = block;
  p->pyr_matched = matched;
  if (!p->pyr) return FPM_OK;
  const int rc = set_pyramid_impl(p, p->pyr->levels, p->pyr->split, p->pyr->halo);   // rebuilt with the reading
  if (rc == FPM_EINVAL) {
    p->pyr_block = old_block;
    p->pyr_matched = old_matched;
  }
  return rc;
}

int fpm_set_force_kernel(fpm_plan* p, int green, int gradient) {
  if (!p || (green != FPM_GREEN_NAIVE && green != FPM_GREEN_DISCRETE) ||
      (gradient != FPM_GRAD_FD4 && gradient != FPM_GRAD_EXACT))
    return FPM_EINVAL;
  if (green == p->green && gradient == p->grad) return FPM_OK;
  FPM_CUDA_TRY(cudaDeviceSynchronize());
  if (p->own_tf) fft_tables_destroy(&p->tf);
  p->own_tf = false;
  p->green = FPM_GREEN_NAIVE;
  p->grad = FPM_GRAD_FD4;
  if (green != FPM_GREEN_NAIVE || gradient != FPM_GRAD_FD4) {
    const int rc = fft_tables_create(&p->tf, p->nc, green, gradient);
    if (rc != FPM_OK) {
      fft_tables_destroy(&p->tf);
      return rc;
    }
    p->own_tf = true;
  }
  p->green = green;
  p->grad = gradient;
  return FPM_OK;
}

int fpm_power(fpm_plan* p, const float* a, const float* b, double* pk, double* kmean, double* nmodes,
              void* stream) {
  if (!p || !a) return FPM_EINVAL;
  cudaStream_t s = S(stream);
  const FftTables& t = p->tc;
  const int nb = p->nc / 2;
  FPM_CUDA_TRY(cudaMemsetAsync(p->d_bins, 0, 3 * nb * sizeof(double), s));
  float2* sb = b ? p->spec + p->specmax : nullptr;
  const bool pot = fft_has_potential(p->nc);
  const int zy = pot && p->nc >= 128 ? 1 : 2;
  FPM_TRY(timed(p, FPM_K_POWER, b ? 1 + 2 * zy : 1 + zy, s, [&] {
    if (pot) {
      FPM_TRY(fft_pot_forward(t, a, p->spec, p->slab_ctr, p->d_err, s));
      if (b) FPM_TRY(fft_pot_forward(t, b, sb, p->slab_ctr, p->d_err, s));
    } else {
      FPM_TRY(fft_zfwd(t, a, p->spec, 1, 0, 0, s));
      FPM_TRY(fft_y(t, p->spec, 1, 0, false, s));
      if (b) {
        FPM_TRY(fft_zfwd(t, b, sb, 1, 0, 0, s));
        FPM_TRY(fft_y(t, sb, 1, 0, false, s));
      }
    }
    return fft_xpower(t, p->spec, sb, p->d_bins, s);
  }));
  std::vector<double> h(3 * nb);
  FPM_CUDA_TRY(cudaMemcpyAsync(h.data(), p->d_bins, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  FPM_CUDA_TRY(cudaStreamSynchronize(s));
  const double V = p->box * p->box * p->box, M = (double)p->M;
  for (int j = 0; j < nb; ++j) {
    const double cnt = h[nb + j];
    if (pk) pk[j] = cnt > 0 ? V / (M * M) * h[j] / cnt : 0.0;
    if (kmean) kmean[j] = cnt > 0 ? 6.283185307179586 / p->box * h[2 * nb + j] / cnt : 0.0;
    if (nmodes) nmodes[j] = cnt;
  }
  return FPM_OK;
}

int fpm_profile(fpm_plan* p, int enable) {
  if (!p || enable < 0 || enable >= 2 + FPM_K_COUNT) return FPM_EINVAL;
  p->prof.on = enable != 0;
  p->prof.only = enable >= 2 ? enable - 2 : -1;
  p->prof.used = 0;
  p->prof.recs.clear();
  return FPM_OK;
}

int fpm_profile_read(fpm_plan* p, double* ms, int64_t* launches, int n, void* stream) {
  if (!p || !ms || !launches || n < FPM_K_COUNT) return FPM_EINVAL;
  for (int k = 0; k < n; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  FPM_CUDA_TRY(cudaStreamSynchronize(S(stream)));
  for (const auto& r : p->prof.recs) {
    float t = 0.f;
    FPM_CUDA_TRY(cudaEventElapsedTime(&t, p->prof.pool[r.second], p->prof.pool[r.second + 1]));
    ms[r.first] += t;
    launches[r.first] += 1;
  }
  p->prof.used = 0;
  p->prof.recs.clear();
  return FPM_OK;
}

const char* fpm_kernel_class_name(int cls) {
  static const char* names[FPM_K_COUNT] = {"kdk_readout_kick_drift", "cell_keys", "tile_scan", "tile_scatter",
                                           "paint_tiles", "paint_halo", "fft_z_r2c", "fft_y_fwd",
                                           "fft_x_green", "fft_y_inv", "fft_z_c2r", "readout",
                                           "initial_conditions", "coefficients_fp64", "power_spectrum",
                                           "pot_fft_fwd_zy", "pot_fft_x_green", "pot_fft_inv_yz",
                                           "pot_gradient", "pyramid_force"};
  return (cls >= 0 && cls < FPM_K_COUNT) ? names[cls] : "unknown";
}

int64_t fpm_launch_count(void) { return (int64_t)g_launches.load(); }

int64_t fpm_force_ckpt_floats(const fpm_plan* p) { return p ? (int64_t)ckpt_stage_floats(p) : 0; }

// ---------------------------------------------------------------- adjoints
static constexpr int CHI_PARTIALS = 1024;

static int ensure_adjoint(fpm_plan* p) {
  if (p->gF) return FPM_OK;
  if (!fft_has_interleaved(p->np) || !fft_has_interleaved(p->nc)) return FPM_ENOTIMPL;
  const size_t sp = spec_elems(p->np);
  int rc;
  if ((rc = dalloc(p, &p->aspec, 9 * sp)) || (rc = dalloc(p, &p->adj6, 6 * p->N)) || (rc = dalloc(p, &p->gS, p->N)) ||
      (rc = dalloc(p, &p->vbuf, 3 * p->N)) || (rc = dalloc(p, &p->vmax, 1)) ||
      (rc = dalloc(p, &p->partial, CHI_PARTIALS)) || (rc = dalloc(p, &p->d_loss, 1)) ||
      (rc = dalloc(p, &p->gF, 3 * p->M)))
    return rc;
  if (p->pc.tile_done && p->pc.ntiles <= VEC3_MAX_TILES) {   // the three-channel vector paint
    if ((rc = dalloc(p, &p->halo3, 3 * paint_halo_elems(p->pc.ntiles))) ||
        (rc = dalloc(p, &p->done3, 3 * (size_t)p->pc.ntiles)))
      return rc;
    if (cudaMemset(p->done3, 0, 3 * sizeof(uint32_t) * p->pc.ntiles) != cudaSuccess) return FPM_ECUDA;
  }
  return FPM_OK;
}

// g_rho = -sum_d A_d g_F_d (A_d^T = -A_d for the real odd force kernels).
static int force_adj_impl(fpm_plan* p, const float* gF, float* g_rho, cudaStream_t s) {
  if (p->pyr) return FPM_ENOTIMPL;   // the pyramid force has no adjoint here
  const FftTables& t = force_tables(p);
  if (force_via_potential(p)) {
    // F_d = D_d G rho with G symmetric and D^T = -D: g_rho = G (-sum_d D_d g_F_d)
    const float coef = (float)(1.5 * p->cosmo.omega_m / (double)p->M);
    const int fused = t.n >= 128 ? 1 : 2;
    FPM_TRY(timed(p, FPM_K_POT_GRAD, 1, s, [&] { return fft_pot_divergence_neg(t, gF, g_rho, s); }));
    FPM_TRY(timed(p, FPM_K_POT_FWD, fused, s,
                  [&] { return fft_pot_forward(t, g_rho, p->spec, p->slab_ctr, p->d_err, s); }));
    FPM_TRY(timed(p, FPM_K_POT_X, 1, s, [&] { return fft_pot_xgreen(t, p->spec, coef, p->slab_ctr, p->d_err, s); }));
    return timed(p, FPM_K_POT_INV, fused, s,
                 [&] { return fft_pot_inverse(t, p->spec, g_rho, p->slab_ctr, p->d_err, s); });
  }
  FPM_TRY(timed(p, FPM_K_FFT_ZF, 1, s, [&] { return fft_zfwd(t, gF, p->spec, 3, p->M, p->specmax, s); }));
  FPM_TRY(timed(p, FPM_K_FFT_YF, 1, s, [&] { return fft_y(t, p->spec, 3, p->specmax, false, s); }));
  XSource src[3];
  for (int d = 0; d < 3; ++d) src[d] = XSource{p->spec + d * p->specmax, SK_FORCE_NEG, d, 0, 0};
  FPM_TRY(timed(p, FPM_K_FFT_X, 1, s, [&] {
    return fft_xcombine(t, src, 3, (float)(1.0 / (double)p->M), p->cosmo.omega_m, nullptr, nullptr, 0.f, 0.f,
                        p->spec, 1, s);
  }));
  FPM_TRY(timed(p, FPM_K_FFT_YI, 1, s, [&] { return fft_y(t, p->spec, 1, 0, true, s); }));
  FPM_TRY(timed(p, FPM_K_FFT_ZI, 1, s, [&] { return fft_zinv(t, p->spec, g_rho, 1, 0, 0, s); }));
  return FPM_OK;
}

// The next reverse step's drift and kick transposes, when the transposed
// gather can apply them on the fly (idr >= 0).
struct NextDriftKick {
  int idr = -1, ik1 = -1, ik2 = -1;
};

// gx += J^T v at positions x (paint, force and readout transposes), v_i =
// K v[i] with K from vk.  With vmax_ready the vector paint takes max |v|
// from p->vmax.  With `next` (and v = the momentum cotangents gp) the gather
// then applies next's drift and kick transposes to (gx, gp) and leaves
// max |K' gp| for the next step; *fused tells whether it did.
static int force_jt_impl(fpm_plan* p, const PaintCtx& c, const float* x, float* v, KScale vk, float* gx,
                         const float* F, cudaStream_t s, bool vmax_ready = false, NextDriftKick next = {},
                         bool* fused = nullptr) {
  if (fused) *fused = false;
  const int nvec = (vmax_ready ? 0 : 1) + (c.tile_done && p->halo3 ? 1 : (c.tile_done ? 3 : 6));
  FPM_TRY(timed(p, FPM_K_PAINT, nvec, s,
                [&] { return launch_paint_vec(c, x, v, vk, p->vmax, p->gF, s, vmax_ready, p->halo3, p->done3); }));
  FPM_TRY(force_adj_impl(p, p->gF, p->rho, s));
  if (next.idr >= 0 && fused) {
    FPM_TRY(timed(p, FPM_K_READOUT, 1, s, [&] {
      return launch_gather_adj_dk(c, x, p->rho, F, p->f4, v, vk, gx, p->d_fac, next.idr, next.ik1, next.ik2,
                                  p->vmax, s);
    }));
    *fused = true;
    return FPM_OK;
  }
  return timed(p, FPM_K_READOUT, 1, s,
               [&] { return launch_gather_adj(c, x, p->rho, F, p->f4, v, gx, true, s, vk); });
}

extern "C" {

int fpm_chi2(fpm_plan* p, const float* rho, const float* target, double sigma, float* g_rho, double* loss,
             void* stream) {
  if (!p || !rho || !target || !(sigma > 0)) return FPM_EINVAL;
  FPM_TRY(ensure_adjoint(p));
  cudaStream_t s = S(stream);
  FPM_TRY(launch_chi2(rho, target, p->M, (float)sigma, g_rho, p->partial, CHI_PARTIALS, p->d_loss, s));
  g_launches += 2;
  if (loss) {
    FPM_CUDA_TRY(cudaMemcpyAsync(loss, p->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    FPM_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return FPM_OK;
}

int fpm_adam_step(fpm_plan* p, float* x, const float* g, float* m, float* v, int64_t n, double gscale,
                  double pscale, double lr, double beta1, double beta2, double eps, int t, double* prior,
                  void* stream) {
  if (!p || !x || !g || !m || !v || n <= 0 || t < 1 || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) ||
      !(beta2 >= 0 && beta2 < 1) || !(eps >= 0))
    return FPM_EINVAL;
  FPM_TRY(ensure_adjoint(p));
  cudaStream_t s = S(stream);
  const double c1 = 1.0 / (1.0 - pow(beta1, t)), c2 = 1.0 / (1.0 - pow(beta2, t));
  FPM_TRY(launch_adam(x, g, m, v, (size_t)n, (float)gscale, (float)pscale, (float)lr, (float)beta1, (float)beta2,
                      (float)(1.0 - beta1), (float)(1.0 - beta2), (float)eps, (float)c1, (float)c2, p->partial,
                      CHI_PARTIALS, p->d_loss, s));
  g_launches += 2;
  if (prior) {
    FPM_CUDA_TRY(cudaMemcpyAsync(prior, p->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    FPM_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return FPM_OK;
}

int fpm_paint_adj(fpm_plan* p, const float* dx, const float* g_rho, float* g_dx, void* stream) {
  if (!p || !dx || !g_rho || !g_dx) return FPM_EINVAL;
  cudaStream_t s = S(stream);
  return timed(p, FPM_K_READOUT, 1, s,
               [&] { return launch_gather_adj(p->pc, dx, g_rho, nullptr, false, nullptr, g_dx, false, s); });
}

int fpm_readout_adj(fpm_plan* p, const float* F, const float* dx, const float* g_f, float* g_F, float* g_dx,
                    void* stream) {
  if (!p || !F || !dx || !g_f || !g_F || !g_dx) return FPM_EINVAL;
  FPM_TRY(ensure_adjoint(p));
  cudaStream_t s = S(stream);
  PaintCtx c = p->pc;
  FPM_TRY(timed(p, FPM_K_KEYS, 1, s, [&] { return launch_keys(c, dx, s); }));
  FPM_TRY(timed(p, FPM_K_SCAN, 1, s, [&] { return launch_scan(c, s); }));
  FPM_TRY(timed(p, FPM_K_SCATTER, 1, s, [&] { return launch_scatter(c, s); }));
  FPM_TRY(timed(p, FPM_K_PAINT, c.tile_done && p->halo3 ? 2 : (c.tile_done ? 4 : 7), s,
                [&] { return launch_paint_vec(c, dx, g_f, KScale{}, p->vmax, g_F, s, false, p->halo3, p->done3); }));
  return timed(p, FPM_K_READOUT, 1, s,
               [&] { return launch_gather_adj(c, dx, nullptr, F, false, g_f, g_dx, false, s); });
}

int fpm_force_adj(fpm_plan* p, const float* g_F, float* g_rho, void* stream) {
  if (!p || !g_F || !g_rho) return FPM_EINVAL;
  if (!fft_has_interleaved(p->nc)) return FPM_ENOTIMPL;
  return force_adj_impl(p, g_F, g_rho, S(stream));
}

int fpm_kdk_adj(fpm_plan* p, const float* ckpt, const float* fckpt, const double* a, int nsteps, float* g_dx,
                const float* g_p_in, float* g_p, void* stream) {
  if (!p || !ckpt || !a || !g_dx || !g_p || nsteps < 1 || nsteps > MAX_STEPS) return FPM_EINVAL;
  for (int k = 0; k <= nsteps; ++k)
    if (!(a[k] > 1e-5 && a[k] <= 10.0) || (k > 0 && !(a[k] > a[k - 1]))) return FPM_EINVAL;
  FPM_TRY(ensure_adjoint(p));
  cudaStream_t s = S(stream);
  std::vector<double> pts(a, a + nsteps + 1);
  for (int k = 0; k < nsteps; ++k) pts.push_back(sqrt(a[k] * a[k + 1]));
  FPM_TRY(stage_points(p, pts.data(), (int)pts.size(), s));
  FPM_TRY(timed(p, FPM_K_COEF, 3, s, [&] {
    return launch_factors(p->d_pts, nsteps, p->cosmo.omega_m, p->d_raw, p->d_gr, p->d_fac, s);
  }));
  p->fac_pts = pts;
  const size_t N3 = 3 * p->N;
  float* gp = g_p;
  if (g_p_in) {
    if (g_p_in != g_p)
      FPM_CUDA_TRY(cudaMemcpyAsync(gp, g_p_in, N3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  } else {     // the loss does not depend on the final momenta: start from zero
    FPM_CUDA_TRY(cudaMemsetAsync(gp, 0, N3 * sizeof(float), s));
  }
  // the force at stage k and the tile buckets of x_k: both from the
  // forward's force checkpoint, or recomputed (paint + force)
  const float* Fk = p->F;
  PaintCtx Ck = p->pc;
  auto prepare = [&](int k, const float* x) -> int {
    if (fckpt) {
      Fk = fckpt + (size_t)k * ckpt_stage_floats(p);
      Ck = stage_ctx(p, fckpt, k);
      return FPM_OK;
    }
    Fk = p->F;
    Ck = p->pc;
    FPM_TRY(paint_impl(p, x, p->rho, nullptr, nullptr, s));
    return force_impl(p, p->rho, p->F, s, p->f4);
  };
  // drift transpose of step k, then the merged kick at x_k (opening kick of
  // step k and closing kick of step k-1 share the force at a_k)
  auto drift_kick = [](int k) {
    NextDriftKick d;
    d.idr = 3 * k + 1;
    d.ik1 = 3 * k + 0;
    d.ik2 = k > 0 ? 3 * (k - 1) + 2 : -1;
    return d;
  };
  auto kick_of = [&](const NextDriftKick& d) {
    KScale k;
    k.fac = p->d_fac;
    k.ik1 = d.ik1;
    k.ik2 = d.ik2;
    return k;
  };
  // On brick lattices the velocity cotangents v = K gp are never stored:
  // the vector paint and the gather scale gp as they read it, and each
  // gather applies the next step's drift and kick transposes (chain).
  // Elsewhere v is materialised in vbuf by the drift-kick kernel.
  const bool chain = kdk_brick_fits(p->pc, p->f4);
  bool ready = false;   // the last gather applied this step's drift-kick transposes and max |v|
  if (g_p_in) {   // closing half kick at a_n: gx += J^T(x_n) (K gp)
    const float* xn = ckpt + (size_t)nsteps * N3;
    KScale kn;
    kn.fac = p->d_fac;
    kn.ik1 = 3 * (nsteps - 1) + 2;
    FPM_TRY(prepare(nsteps, xn));
    if (chain) {
      FPM_TRY(force_jt_impl(p, Ck, xn, gp, kn, g_dx, Fk, s, false, drift_kick(nsteps - 1), &ready));
    } else {
      FPM_TRY(launch_scale_copy(gp, p->vbuf, N3, p->d_fac, kn.ik1, s));
      FPM_TRY(force_jt_impl(p, Ck, xn, p->vbuf, KScale{}, g_dx, Fk, s));
    }
  }
  for (int k = nsteps - 1; k >= 0; --k) {
    const float* xk = ckpt + (size_t)k * N3;
    const NextDriftKick d = drift_kick(k);
    if (!ready)
      FPM_TRY(launch_adj_drift_kick(g_dx, gp, chain ? nullptr : p->vbuf, N3, p->d_fac, d.idr, d.ik1, d.ik2, s));
    FPM_TRY(prepare(k, xk));
    if (chain) {
      const bool vmax_ready = ready;
      FPM_TRY(force_jt_impl(p, Ck, xk, gp, kick_of(d), g_dx, Fk, s, vmax_ready,
                            k > 0 ? drift_kick(k - 1) : NextDriftKick{}, &ready));
    } else {
      FPM_TRY(force_jt_impl(p, Ck, xk, p->vbuf, KScale{}, g_dx, Fk, s));
    }
  }
  g_launches += 1 + 2 * nsteps;
  return FPM_OK;
}

int fpm_lpt_adj(fpm_plan* p, const void* lin_k, double a0, int order, const float* g_dx, const float* g_p,
                void* g_lin_k, void* stream) {
  if (!p || !lin_k || !g_dx || !g_p || !g_lin_k || (order != 1 && order != 2) || !(a0 > 1e-5 && a0 <= 10.0))
    return FPM_EINVAL;
  FPM_TRY(ensure_adjoint(p));
  cudaStream_t s = S(stream);
  const FftTables& t = p->tp;
  const size_t sp = spec_elems(p->np), N = p->N;
  const float2* lk = reinterpret_cast<const float2*>(lin_k);
  float2* out = reinterpret_cast<float2*>(g_lin_k);
  const float inv_n3 = (float)(1.0 / (double)N);
  FPM_TRY(stage_points(p, &a0, 1, s));
  FPM_TRY(timed(p, FPM_K_COEF, 2, s, [&] { return launch_growth(p->d_pts, 1, p->cosmo.omega_m, p->d_raw, p->d_gr, s); }));
  return timed(p, FPM_K_IC, order == 2 ? 17 : 4, s, [&] {
    FPM_TRY(launch_lpt_gpsi(g_dx, g_p, N, p->d_gr, (float)a0, (float)(p->nc / p->np), p->adj6, s));
    XSource src[9];
    int ns = 0;
    if (order == 2) {
      // phi_ij of the forward model, then g_S = sum_d B_d g_Psi2_d
      if (ic_has_potential(p->np)) {
        // psi = IFFT[lin / |w|^2] / N^3 in the gS slot, phi_ij from its second differences
        FPM_TRY(fft_xpot(t, lk, p->spec, inv_n3, s));
        FPM_TRY(fft_pot_inverse(t, p->spec, p->gS, p->slab_ctr, p->d_err, s));
        FPM_TRY(launch_lpt_hessian_fd(p->np, p->gS, p->real6, s));
      } else {
        FPM_TRY(fft_xlpt_hessian(t, lk, p->spec, p->specmax, inv_n3, s));
        FPM_TRY(fft_y(t, p->spec, 6, p->specmax, true, s));
        FPM_TRY(fft_zinv(t, p->spec, p->real6, 6, p->specmax, N, s));
      }
      FPM_TRY(fft_zfwd(t, p->adj6 + 3 * N, p->aspec, 3, N, sp, s));
      FPM_TRY(fft_y(t, p->aspec, 3, sp, false, s));
      for (int d = 0; d < 3; ++d) src[d] = XSource{p->aspec + d * sp, SK_B, d, 0, 0};
      FPM_TRY(fft_xcombine(t, src, 3, inv_n3, 0.0, nullptr, nullptr, 0.f, 0.f, p->aspec, 1, s));
      FPM_TRY(fft_y(t, p->aspec, 1, 0, true, s));
      FPM_TRY(fft_zinv(t, p->aspec, p->gS, 1, 0, 0, s));
      FPM_TRY(launch_lpt_gphi(p->gS, p->real6, N, s));
      FPM_TRY(fft_zfwd(t, p->real6, p->aspec + 3 * sp, 6, N, sp, s));
      FPM_TRY(fft_y(t, p->aspec + 3 * sp, 6, sp, false, s));
      const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
      for (int q = 0; q < 6; ++q) src[ns++] = XSource{p->aspec + (3 + q) * sp, SK_H, pi[q], pj[q], 0};
    }
    FPM_TRY(fft_zfwd(t, p->adj6, p->aspec, 3, N, sp, s));
    FPM_TRY(fft_y(t, p->aspec, 3, sp, false, s));
    for (int d = 0; d < 3; ++d) src[ns++] = XSource{p->aspec + d * sp, SK_BCONJ, d, 0, 0};
    return fft_xcombine(t, src, ns, 1.f, 0.0, nullptr, nullptr, 0.f, 0.f, out, 0, s);
  });
}

int fpm_linear_field_adj(fpm_plan* p, const void* g_lin_k, float* g_white, void* stream) {
  if (!p || !g_lin_k || !g_white) return FPM_EINVAL;
  FPM_TRY(ensure_adjoint(p));
  cudaStream_t s = S(stream);
  const FftTables& t = p->tp;
  const double n3v = (double)p->N / (p->box * p->box * p->box);
  XSource src{reinterpret_cast<const float2*>(g_lin_k), SK_LINEAR, 0, 0, 1};
  return timed(p, FPM_K_IC, 3, s, [&] {
    FPM_TRY(fft_xcombine(t, &src, 1, (float)(1.0 / (double)p->N), 0.0, &p->eh, p->d_amp,
                         (float)(6.283185307179586 / p->box), (float)n3v, p->aspec, 1, s));
    FPM_TRY(fft_y(t, p->aspec, 1, 0, true, s));
    return fft_zinv(t, p->aspec, g_white, 1, 0, 0, s);
  });
}

// ---------------------------------------------------------------- batched
struct fpm_batch {
  Batch* impl = nullptr;
  std::vector<fpm_plan*> plans;
};

int fpm_batch_create(fpm_batch** out, fpm_plan* const* plans, int nsims) {
  if (!out || !plans || nsims < 1 || nsims > 4096) return FPM_EINVAL;
  std::vector<BatchPlanView> views(nsims);
  for (int s = 0; s < nsims; ++s) {
    fpm_plan* p = plans[s];
    if (!p || !batch_size_ok(p->nc, p->np)) return FPM_EINVAL;
    BatchPlanView& v = views[s];
    v.pc = p->pc;
    v.nc = p->nc;
    v.np = p->np;
    v.f4 = p->f4 ? 1 : 0;
    v.F = p->F;
    v.rho = p->rho;
    v.spec = p->spec;
    v.specmax = p->specmax;
    v.fac = p->d_fac;
    if (p->grad != FPM_GRAD_FD4 || p->pyr) return FPM_ENOTIMPL;   // batched phases use the potential form
    v.tab = force_tables(p);
    v.force_coef = (float)(1.5 * p->cosmo.omega_m / (double)p->M);
  }
  fpm_batch* b = new fpm_batch();
  b->plans.assign(plans, plans + nsims);
  const int rc = batch_create(&b->impl, views.data(), nsims);
  if (rc != FPM_OK) {
    delete b;
    return rc;
  }
  *out = b;
  return FPM_OK;
}

void fpm_batch_destroy(fpm_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  batch_destroy(b->impl);
  delete b;
}

int fpm_batch_configure(fpm_batch* b, int blocks_per_sm, int readout_chunks, int64_t spin_limit) {
  if (!b) return FPM_EINVAL;
  return batch_configure(b->impl, blocks_per_sm, readout_chunks, (long long)spin_limit);
}

int fpm_batch_kdk(fpm_batch* b, float* const* dx, float* const* mom, const double* a, int nsteps, void* stream) {
  if (!b || !dx || !mom || !a || nsteps < 1 || nsteps > MAX_STEPS) return FPM_EINVAL;
  for (int k = 0; k <= nsteps; ++k)
    if (!(a[k] > 1e-5 && a[k] <= 10.0) || (k > 0 && !(a[k] > a[k - 1]))) return FPM_EINVAL;
  const int ns = (int)b->plans.size();
  for (int s = 0; s < ns; ++s)
    if (!dx[s] || !mom[s]) return FPM_EINVAL;
  cudaStream_t s = S(stream);
  std::vector<double> pts(a, a + nsteps + 1);
  for (int k = 0; k < nsteps; ++k) pts.push_back(sqrt(a[k] * a[k + 1]));
  // FP64 factors of every simulation's own cosmology, unless its plan
  // already holds them for these stages; the stages are staged from the
  // host once and copied on the device to the other plans
  const fpm_plan* staged = nullptr;
  for (fpm_plan* p : b->plans) {
    if (p->fac_pts == pts) continue;
    if (!staged) {
      FPM_TRY(stage_points(p, pts.data(), (int)pts.size(), s));
      staged = p;
    } else {
      FPM_CUDA_TRY(cudaMemcpyAsync(p->d_pts, staged->d_pts, (pts.size() + 1) * sizeof(double),
                                   cudaMemcpyDeviceToDevice, s));
    }
    FPM_TRY(launch_factors(p->d_pts, nsteps, p->cosmo.omega_m, p->d_raw, p->d_gr, p->d_fac, s));
    p->fac_pts = pts;
    g_launches += 3;
  }
  FPM_TRY(batch_kdk(b->impl, dx, mom, nsteps, s));
  g_launches += nsteps + 2;
  return FPM_OK;
}

int fpm_batch_status(fpm_batch* b, void* stream) {
  if (!b) return FPM_EINVAL;
  const int rc = batch_status(b->impl, S(stream));
  if (rc != FPM_OK) return rc;
  for (fpm_plan* p : b->plans) FPM_TRY(fpm_status(p, stream));
  return FPM_OK;
}

int fpm_batch_info(fpm_batch* b, int* grid_blocks, int* graph_captured) {
  if (!b) return FPM_EINVAL;
  return batch_info(b->impl, grid_blocks, graph_captured);
}

int fpm_batch_tune(fpm_batch* b, int nc, int knob, int value) {
  if (!b) return FPM_EINVAL;
  static_assert(FPM_BTUNE_READOUT == BT_READOUT && FPM_BTUNE_PAINT_TILE == BT_PAINT_TILE &&
                    FPM_BTUNE_FFT_SLOTS == BT_FFT_SLOTS, "knob codes");
  return batch_tune(b->impl, nc, knob, value);
}

int fpm_batch_phase_times(fpm_batch* b, double* ms, int n, void* stream) {
  if (!b || !ms) return FPM_EINVAL;
  return batch_phase_times(b->impl, ms, n, S(stream));
}

}  // extern "C"

extern "C" int fpm_status(fpm_plan* p, void* stream) {
  if (!p) return FPM_EINVAL;
  cudaStream_t s = S(stream);
  int h = 0;
  FPM_CUDA_TRY(cudaMemcpyAsync(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  FPM_CUDA_TRY(cudaStreamSynchronize(s));
  FPM_CUDA_TRY(cudaMemsetAsync(p->d_err, 0, sizeof(int), s));
  if (h & ERR_TIMEOUT) return FPM_ETIMEOUT;
  if (h) return FPM_EDEVICE;
  return FPM_OK;
}

}  // extern "C"
