// ic.cu -- linear field (Algorithm 4 steps 1-2), 2LPT displacements and
// momenta (Algorithm 4 steps 3-6, second order per the LPT scaling test),
// and the binned power spectrum used by Eqs. 10-11.  All of them are x-axis
// passes of the 3D FFT with a spectral operator in the middle.  Power-of-two
// lattices use the register FFT and build 2LPT through potentials
// (ic_reg.cuh); the shared-memory kernels below serve 48/96/192/384.
#include "internal.h"
#include "fft_passes.cuh"
#include "ic_reg.cuh"

namespace fpm {

// ------------------------------------------------------------ linear field
// Forward x transform of DFT_zy(white), then scale each mode by
// sqrt(P(|k|) N^3 / V); the k = 0 mode is set to zero.  In place allowed.
template <int N>
__global__ void __launch_bounds__(FFT_THREADS) k_xlinear(const float2* in, float2* out, EhParams e,
                                                         const double* __restrict__ d_amp, float kf,
                                                         float n3_over_v, const float2* __restrict__ g_tw) {
  extern __shared__ float2 smem[];
  constexpr int LS = sp_size(N);
  constexpr int NB = N / XB;
  float2* s0 = smem;
  float2* s1 = s0 + XB * LS;
  float2* tw = s1 + XB * LS;
  load_twiddles<N>(tw, g_tw);
  const int kz = blockIdx.x / NB, ky0 = (blockIdx.x % NB) * XB;
  xload<N>(s0, in, kz, ky0);
  __syncthreads();
  float2* d = FftPlan<N>::template run<false>(s0, s1, XB, LS, tw);
  const float amp = (float)d_amp[0];
  for (int idx = threadIdx.x; idx < N * XB; idx += blockDim.x) {
    const int j = idx / N, x = idx - j * N;
    const int fx = freq_of(x, N), fy = freq_of(ky0 + j, N), fz = kz;
    const int n2 = fx * fx + fy * fy + fz * fz;
    float sc = 0.f;
    if (n2 > 0) {
      const float k = kf * sqrtf((float)n2);
      const float T = eh_nowiggle_T32(k, e);
      const float pk = amp * powf(k, e.n_s) * T * T;
      sc = sqrtf(pk * n3_over_v);
    }
    d[j * LS + sp(x)] = cscale(d[j * LS + sp(x)], sc);
  }
  __syncthreads();
  xstore<N>(out, d, kz, ky0);
}

// ------------------------------------------------------------ 2LPT, first pass
// phi_ij(k) = g_i g_j lin_k / |w|^2 (inverse-normalised by coef = 1/N^3)
// for (ij) = 00, 11, 22, 01, 02, 12; inverse x transform of each.
template <int N>
__global__ void __launch_bounds__(FFT_THREADS) k_xlpt_hessian(const float2* __restrict__ lin_k, float2* out,
                                                              size_t out_fs, float coef,
                                                              const float2* __restrict__ g_tw,
                                                              const float* __restrict__ g_g,
                                                              const float* __restrict__ g_w2) {
  extern __shared__ float2 smem[];
  constexpr int LS = sp_size(N);
  constexpr int NB = N / XB;
  float2* src = smem;
  float2* f1 = src + XB * LS;
  float2* f2 = f1 + XB * LS;
  float2* tw = f2 + XB * LS;
  load_twiddles<N>(tw, g_tw);
  const int kz = blockIdx.x / NB, ky0 = (blockIdx.x % NB) * XB;
  xload<N>(src, lin_k, kz, ky0);
  __syncthreads();
  const int pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
  for (int o = 0; o < 6; ++o) {
    for (int idx = threadIdx.x; idx < N * XB; idx += blockDim.x) {
      const int j = idx / N, x = idx - j * N;
      const int ky = ky0 + j;
      const int kk[3] = {x, ky, kz};
      const float k2 = __ldg(g_w2 + x) + __ldg(g_w2 + ky) + __ldg(g_w2 + kz);
      const float s = k2 > 0.f ? __ldg(g_g + kk[pi[o]]) * __ldg(g_g + kk[pj[o]]) * coef / k2 : 0.f;
      f1[j * LS + sp(x)] = cscale(src[j * LS + sp(x)], s);
    }
    __syncthreads();
    const float2* r = FftPlan<N>::template run<true>(f1, f2, XB, LS, tw);
    xstore<N>(out + o * out_fs, r, kz, ky0);
    __syncthreads();
  }
}

// S = phi00 phi11 + phi00 phi22 + phi11 phi22 - phi01^2 - phi02^2 - phi12^2
__global__ void k_lpt_source(const float* __restrict__ phi, size_t n, float* __restrict__ S) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float a = phi[i], b = phi[n + i], c = phi[2 * n + i];
  const float xy = phi[3 * n + i], xz = phi[4 * n + i], yz = phi[5 * n + i];
  S[i] = a * b + a * c + b * c - xy * xy - xz * xz - yz * yz;
}

// ------------------------------------------------------------ 2LPT, second pass
// Forward x transform of DFT_zy(S) (when second order), then for d = x,y,z:
//   dx_d(k) = i g_d (D1 lin_k - D2 S(k)) / |w|^2 * r / N^3
//   p_d(k)  = i g_d a^2 E (f1 D1 lin_k - f2 D2 S(k)) / |w|^2 * r / N^3
// (Psi1 = i g lin_k/|w|^2, Psi2 = i g phi2, phi2 = -S/|w|^2), inverse x
// transform of each of the six.  gr = growth row at a0 (D1, D2, f1, f2, E).
template <int N, bool SECOND>
__global__ void __launch_bounds__(FFT_THREADS) k_xlpt_disp(const float2* specS,
                                                           const float2* __restrict__ lin_k, float2* out,
                                                           size_t out_fs, const double* __restrict__ gr,
                                                           float a0, float coef,
                                                           const float2* __restrict__ g_tw,
                                                           const float* __restrict__ g_g,
                                                           const float* __restrict__ g_w2) {
  extern __shared__ float2 smem[];
  constexpr int LS = sp_size(N);
  constexpr int NB = N / XB;
  float2* sl = smem;              // lin_k block
  float2* s0 = sl + XB * LS;      // S block / work
  float2* s1 = s0 + XB * LS;
  float2* s2 = s1 + XB * LS;
  float2* tw = s2 + XB * LS;
  load_twiddles<N>(tw, g_tw);
  const int kz = blockIdx.x / NB, ky0 = (blockIdx.x % NB) * XB;
  xload<N>(sl, lin_k, kz, ky0);
  float2* sk = nullptr;
  if (SECOND) xload<N>(s0, specS, kz, ky0);
  __syncthreads();
  float2 *f1, *f2;
  if (SECOND) {
    sk = FftPlan<N>::template run<false>(s0, s1, XB, LS, tw);
    f1 = (sk == s0) ? s1 : s0;
    f2 = s2;
  } else {
    f1 = s0;
    f2 = s1;
  }
  const float D1 = (float)gr[0], D2 = (float)gr[1], F1 = (float)gr[2], F2 = (float)gr[3], E = (float)gr[4];
  const float pfac = a0 * a0 * E;
  for (int o = 0; o < 6; ++o) {
    const int d = o % 3;
    const bool mom = o >= 3;
    const float c1 = mom ? pfac * F1 * D1 : D1;
    const float c2 = mom ? pfac * F2 * D2 : D2;
    for (int idx = threadIdx.x; idx < N * XB; idx += blockDim.x) {
      const int j = idx / N, x = idx - j * N;
      const int ky = ky0 + j;
      const int kk[3] = {x, ky, kz};
      const float k2 = __ldg(g_w2 + x) + __ldg(g_w2 + ky) + __ldg(g_w2 + kz);
      const float s = k2 > 0.f ? __ldg(g_g + kk[d]) * coef / k2 : 0.f;
      float2 v = cscale(sl[j * LS + sp(x)], c1);
      if (SECOND) {
        const float2 sv = sk[j * LS + sp(x)];
        v.x -= c2 * sv.x;
        v.y -= c2 * sv.y;
      }
      f1[j * LS + sp(x)] = mul_i(cscale(v, s));
    }
    __syncthreads();
    const float2* r = FftPlan<N>::template run<true>(f1, f2, XB, LS, tw);
    xstore<N>(out + o * out_fs, r, kz, ky0);
    __syncthreads();
  }
}

// ------------------------------------------------------------ power spectrum
// Forward x transform of DFT_zy(a) (and of b), then per mode accumulate
// w Re(A B*), w and w |n| into bin j (j - 1/2 <= |n| < j + 1/2, 1 <= j <= N/2)
// with w = 2 for 0 < kz < N/2 (the conjugate partner), else 1.
template <int N>
__global__ void __launch_bounds__(FFT_THREADS) k_xpower(const float2* __restrict__ sa,
                                                        const float2* __restrict__ sb,
                                                        double* __restrict__ bins,
                                                        const float2* __restrict__ g_tw) {
  extern __shared__ float2 smem[];
  constexpr int LS = sp_size(N);
  constexpr int NB = N / XB;
  constexpr int NBIN = N / 2;
  float2* s0 = smem;
  float2* s1 = s0 + XB * LS;
  float2* s2 = s1 + XB * LS;
  float2* s3 = s2 + XB * LS;
  float2* tw = s3 + XB * LS;
  double* acc = reinterpret_cast<double*>(tw + N);   // 3 * NBIN doubles
  load_twiddles<N>(tw, g_tw);
  for (int k = threadIdx.x; k < 3 * NBIN; k += blockDim.x) acc[k] = 0.0;
  const int kz = blockIdx.x / NB, ky0 = (blockIdx.x % NB) * XB;
  xload<N>(s0, sa, kz, ky0);
  if (sb) xload<N>(s2, sb, kz, ky0);
  __syncthreads();
  const float2* A = FftPlan<N>::template run<false>(s0, s1, XB, LS, tw);
  const float2* B = A;
  if (sb) B = FftPlan<N>::template run<false>(s2, s3, XB, LS, tw);
  const double w = (kz > 0 && kz < N / 2) ? 2.0 : 1.0;
  for (int idx = threadIdx.x; idx < N * XB; idx += blockDim.x) {
    const int j = idx / N, x = idx - j * N;
    const int fx = freq_of(x, N), fy = freq_of(ky0 + j, N);
    const int n2 = fx * fx + fy * fy + kz * kz;
    int b = (int)floorf(sqrtf((float)n2) + 0.5f);
    if ((2 * b - 1) * (2 * b - 1) > 4 * n2) --b;
    if ((2 * b + 1) * (2 * b + 1) <= 4 * n2) ++b;
    if (b < 1 || b > NBIN) continue;
    const float2 va = A[j * LS + sp(x)], vb = B[j * LS + sp(x)];
    const double pr = (double)va.x * vb.x + (double)va.y * vb.y;
    atomicAdd(acc + (b - 1), w * pr);
    atomicAdd(acc + NBIN + (b - 1), w);
    atomicAdd(acc + 2 * NBIN + (b - 1), w * sqrt((double)n2));
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 3 * NBIN; k += blockDim.x)
    if (acc[k] != 0.0) atomicAdd(bins + k, acc[k]);
}

// ------------------------------------------------------------ host side
template <typename K>
static int set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    FPM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return FPM_OK;
}

#define FPM_DISPATCH_N(n, CALL)                  \
  switch (n) {                                   \
    case 16: { constexpr int N = 16; CALL; }     \
    case 32: { constexpr int N = 32; CALL; }     \
    case 48: { constexpr int N = 48; CALL; }     \
    case 64: { constexpr int N = 64; CALL; }     \
    case 96: { constexpr int N = 96; CALL; }     \
    case 128: { constexpr int N = 128; CALL; }   \
    case 192: { constexpr int N = 192; CALL; }   \
    case 256: { constexpr int N = 256; CALL; }   \
    case 384: { constexpr int N = 384; CALL; }   \
    case 512: { constexpr int N = 512; CALL; }   \
    default: return FPM_EINVAL;                  \
  }

template <int N>
static int xlinear_impl(const FftTables& t, const float2* in, float2* out, const EhParams& e,
                        const double* d_amp, float kf, float n3v, cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using C = RegCfg<N>;
    FPM_TRY(set_smem(k_xlin_r<N>, C::SMEM));
    k_xlin_r<N><<<((N / 2 + 1) * N + C::L - 1) / C::L, C::THREADS, C::SMEM, s>>>(in, out, e, d_amp, kf, n3v, t.tw);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  } else {
    const size_t sm = xpass_smem<N>(2);
    FPM_TRY(set_smem(k_xlinear<N>, sm));
    k_xlinear<N><<<(N / 2 + 1) * (N / XB), FFT_THREADS, sm, s>>>(in, out, e, d_amp, kf, n3v, t.tw);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
}

template <int N>
static int xhess_impl(const FftTables& t, const float2* lin_k, float2* out, size_t out_fs, float coef,
                      cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    return FPM_ENOTIMPL;                 // power-of-two lattices take the potential path
  } else {
    const size_t sm = xpass_smem<N>(3);
    FPM_TRY(set_smem(k_xlpt_hessian<N>, sm));
    k_xlpt_hessian<N><<<(N / 2 + 1) * (N / XB), FFT_THREADS, sm, s>>>(lin_k, out, out_fs, coef, t.tw, t.g, t.w2);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
}

template <int N>
static int xdisp_impl(const FftTables& t, const float2* specS, const float2* lin_k, float2* out, size_t out_fs,
                      const double* gr, float a0, float coef, bool second, cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    return FPM_ENOTIMPL;                 // power-of-two lattices take the potential path
  } else {
    const size_t sm = xpass_smem<N>(4);
    const int grid = (N / 2 + 1) * (N / XB);
    if (second) {
      FPM_TRY(set_smem(k_xlpt_disp<N, true>, sm));
      k_xlpt_disp<N, true><<<grid, FFT_THREADS, sm, s>>>(specS, lin_k, out, out_fs, gr, a0, coef, t.tw, t.g, t.w2);
    } else {
      FPM_TRY(set_smem(k_xlpt_disp<N, false>, sm));
      k_xlpt_disp<N, false><<<grid, FFT_THREADS, sm, s>>>(specS, lin_k, out, out_fs, gr, a0, coef, t.tw, t.g, t.w2);
    }
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
}

template <int N>
static int xpower_impl(const FftTables& t, const float2* sa, const float2* sb, double* bins, cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using C = RegCfg<N>;
    const size_t sm = C::SMEM + 3 * (N / 2) * sizeof(float);
    FPM_TRY(set_smem(k_xpow_r<N>, sm));
    int dev = 0, nsm = 0, per = 0;
    FPM_CUDA_TRY(cudaGetDevice(&dev));
    FPM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_xpow_r<N>, C::THREADS, sm));
    const int items = ((N / 2 + 1) * N + C::L - 1) / C::L;
    const int grid = per > 0 && nsm * per < items ? nsm * per : items;
    k_xpow_r<N><<<grid, C::THREADS, sm, s>>>(sa, sb, bins, t.tw, items);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  } else {
    const size_t sm = xpass_smem<N>(4) + 3 * (N / 2) * sizeof(double);
    FPM_TRY(set_smem(k_xpower<N>, sm));
    k_xpower<N><<<(N / 2 + 1) * (N / XB), FFT_THREADS, sm, s>>>(sa, sb, bins, t.tw);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
}

int fft_xlinear(const FftTables& t, const float2* in, float2* out, const EhParams& e, const double* d_amp,
                float kf, float n3v, cudaStream_t s) {
  FPM_DISPATCH_N(t.n, return xlinear_impl<N>(t, in, out, e, d_amp, kf, n3v, s));
}

int fft_xlpt_hessian(const FftTables& t, const float2* lin_k, float2* out, size_t out_fs, float coef,
                     cudaStream_t s) {
  FPM_DISPATCH_N(t.n, return xhess_impl<N>(t, lin_k, out, out_fs, coef, s));
}

int fft_xlpt_disp(const FftTables& t, const float2* specS, const float2* lin_k, float2* out, size_t out_fs,
                  const double* gr, float a0, float coef, bool second, cudaStream_t s) {
  FPM_DISPATCH_N(t.n, return xdisp_impl<N>(t, specS, lin_k, out, out_fs, gr, a0, coef, second, s));
}

int fft_xpower(const FftTables& t, const float2* sa, const float2* sb, double* bins, cudaStream_t s) {
  FPM_DISPATCH_N(t.n, return xpower_impl<N>(t, sa, sb, bins, s));
}

// ------------------------------------------------------------ 2LPT through potentials (power-of-two lattices)
bool ic_has_potential(int n) { return is_pow2_size(n); }

template <int N>
static int xpot_impl(const FftTables& t, const float2* lin, float2* out, float coef, cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using C = RegCfg<N>;
    FPM_TRY(set_smem(k_xpot_r<N>, C::SMEM));
    k_xpot_r<N><<<((N / 2 + 1) * N + C::L - 1) / C::L, C::THREADS, C::SMEM, s>>>(lin, out, coef, t.tw, t.w2);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  return FPM_ENOTIMPL;
}

template <int N>
static int xdisp2_impl(const FftTables& t, const float2* specS, const float2* lin, float2* out0, float2* out1,
                       const double* gr, float a0, float coef, bool second, cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using C = RegCfg<N>;
    const size_t sm = C::SMEM + (size_t)N * C::L * sizeof(float2);
    const int grid = ((N / 2 + 1) * N + C::L - 1) / C::L;
    if (second) {
      FPM_TRY(set_smem(k_xdisp_r<N, true>, sm));
      k_xdisp_r<N, true><<<grid, C::THREADS, sm, s>>>(specS, lin, out0, out1, gr, a0, coef, t.tw, t.w2);
    } else {
      FPM_TRY(set_smem(k_xdisp_r<N, false>, sm));
      k_xdisp_r<N, false><<<grid, C::THREADS, sm, s>>>(specS, lin, out0, out1, gr, a0, coef, t.tw, t.w2);
    }
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  return FPM_ENOTIMPL;
}

template <int N>
static int source_fd_impl(const float* psi, float* S, bool hess, cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using H = HsCfg<N>;
    const dim3 grid(N / H::TZ, N / H::TY, N / H::XC);
    if (hess) k_lpt_source_fd<N, true><<<grid, 256, 0, s>>>(psi, S);
    else k_lpt_source_fd<N, false><<<grid, 256, 0, s>>>(psi, S);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  return FPM_ENOTIMPL;
}

int fft_xpot(const FftTables& t, const float2* lin, float2* out, float coef, cudaStream_t s) {
  FPM_DISPATCH_N(t.n, return xpot_impl<N>(t, lin, out, coef, s));
}

int fft_xdisp2(const FftTables& t, const float2* specS, const float2* lin, float2* out0, float2* out1,
               const double* gr, float a0, float coef, bool second, cudaStream_t s) {
  FPM_DISPATCH_N(t.n, return xdisp2_impl<N>(t, specS, lin, out0, out1, gr, a0, coef, second, s));
}

int launch_lpt_source_fd(int n, const float* psi, float* S, cudaStream_t s) {
  FPM_DISPATCH_N(n, return source_fd_impl<N>(psi, S, false, s));
}

int launch_lpt_hessian_fd(int n, const float* psi, float* phi6, cudaStream_t s) {
  FPM_DISPATCH_N(n, return source_fd_impl<N>(psi, phi6, true, s));
}

int launch_lpt_source(const float* phi, size_t n, float* S, cudaStream_t s) {
  k_lpt_source<<<(int)((n + 255) / 256), 256, 0, s>>>(phi, n, S);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

}  // namespace fpm
