// fft.cu -- host launchers of the 3D FFT passes and their tables.
#include "internal.h"
#include "fft_passes.cuh"
#include "fft_reg.cuh"

#include <math.h>
#include <vector>

namespace fpm {

int fft_tables_create(FftTables* t, int n, int green, int grad, double grad_scale) {
  t->n = n;
  std::vector<float2> tw(n);
  std::vector<float> g(n), w2(n);
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < n; ++m) {
    const double ang = -two_pi * m / n;
    tw[m] = make_float2((float)cos(ang), (float)sin(ang));
    const int f = m < n / 2 ? m : m - n;            // signed frequency
    const double w = two_pi * f / n;
    if (m == n / 2) g[m] = 0.f;                                   // 0 at Nyquist either way
    else if (grad) g[m] = (float)w;                               // exact
    else if (grad_scale == 1.0) g[m] = (float)((8.0 * sin(w) - sin(2.0 * w)) / 6.0);   // Eq. 5
    else {                                                        // Eq. 5 of a mesh grad_scale x finer
      const double wf = w / grad_scale;
      g[m] = (float)(grad_scale * (8.0 * sin(wf) - sin(2.0 * wf)) / 6.0);
    }
    const double s = 2.0 * sin(0.5 * w);                          // Eq. 4: w sinc(w/2)
    w2[m] = (float)(green ? s * s : w * w);
  }
  FPM_CUDA_TRY(cudaMalloc(&t->tw, n * sizeof(float2)));
  FPM_CUDA_TRY(cudaMalloc(&t->g, n * sizeof(float)));
  FPM_CUDA_TRY(cudaMalloc(&t->w2, n * sizeof(float)));
  FPM_CUDA_TRY(cudaMemcpy(t->tw, tw.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
  FPM_CUDA_TRY(cudaMemcpy(t->g, g.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  FPM_CUDA_TRY(cudaMemcpy(t->w2, w2.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  return FPM_OK;
}

void fft_tables_destroy(FftTables* t) {
  cudaFree(t->tw);
  cudaFree(t->g);
  cudaFree(t->w2);
  t->tw = nullptr;
  t->g = t->w2 = nullptr;
}

#define FPM_DISPATCH_N(n, CALL)            \
  switch (n) {                             \
    case 16: { constexpr int N = 16; CALL; } \
    case 32: { constexpr int N = 32; CALL; } \
    case 48: { constexpr int N = 48; CALL; } \
    case 64: { constexpr int N = 64; CALL; } \
    case 96: { constexpr int N = 96; CALL; } \
    case 128: { constexpr int N = 128; CALL; } \
    case 192: { constexpr int N = 192; CALL; } \
    case 256: { constexpr int N = 256; CALL; } \
    case 384: { constexpr int N = 384; CALL; } \
    case 512: { constexpr int N = 512; CALL; } \
    default: return FPM_EINVAL;            \
  }

template <typename K>
static int set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    FPM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return FPM_OK;
}

template <int N>
static int zfwd_impl(const FftTables& t, const float* in, float2* spec, int nf, size_t in_fs, size_t out_fs,
                     cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using C = RegCfg<N>;
    FPM_TRY(set_smem(k_zfwd_r<N>, C::SMEM));
    k_zfwd_r<N><<<dim3(N * N / (2 * C::L), nf), C::THREADS, C::SMEM, s>>>(in, spec, in_fs, out_fs, t.tw);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  const size_t sm = zpass_smem<N>();
  FPM_TRY(set_smem(k_zfwd<N>, sm));
  dim3 grid(N * (N / (2 * ZG)), nf);
  k_zfwd<N><<<grid, FFT_THREADS, sm, s>>>(in, spec, in_fs, out_fs, t.tw);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

template <int N>
static int y_impl(const FftTables& t, float2* spec, int nf, size_t fs, bool inverse, cudaStream_t s) {
  const int nlines = N * (N / 2 + 1);
  if constexpr (is_pow2_size(N)) {
    using C = RegCfg<N>;
    dim3 grid((nlines + C::L - 1) / C::L, nf);
    if (inverse) {
      FPM_TRY(set_smem(k_yfft_r<N, true>, C::SMEM));
      k_yfft_r<N, true><<<grid, C::THREADS, C::SMEM, s>>>(spec, nlines, fs, t.tw);
    } else {
      FPM_TRY(set_smem(k_yfft_r<N, false>, C::SMEM));
      k_yfft_r<N, false><<<grid, C::THREADS, C::SMEM, s>>>(spec, nlines, fs, t.tw);
    }
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  const size_t sm = ypass_smem<N>();
  dim3 grid((nlines + YL - 1) / YL, nf);
  if (inverse) {
    FPM_TRY(set_smem(k_yfft<N, true>, sm));
    k_yfft<N, true><<<grid, FFT_THREADS, sm, s>>>(spec, nlines, fs, t.tw);
  } else {
    FPM_TRY(set_smem(k_yfft<N, false>, sm));
    k_yfft<N, false><<<grid, FFT_THREADS, sm, s>>>(spec, nlines, fs, t.tw);
  }
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

template <int N>
static int zinv_impl(const FftTables& t, const float2* spec, float* out, int nf, size_t in_fs, size_t out_fs,
                     cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using C = RegCfg<N>;
    FPM_TRY(set_smem(k_zinv_r<N>, C::SMEM));
    k_zinv_r<N><<<dim3(N * N / (2 * C::L), nf), C::THREADS, C::SMEM, s>>>(spec, out, in_fs, out_fs, t.tw);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  const size_t sm = zpass_smem<N>();
  FPM_TRY(set_smem(k_zinv<N>, sm));
  dim3 grid(N * (N / (2 * ZG)), nf);
  k_zinv<N><<<grid, FFT_THREADS, sm, s>>>(spec, out, in_fs, out_fs, t.tw);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

template <int N>
static int xforce_impl(const FftTables& t, const float2* in, float2* out, size_t out_fs, float coef,
                       cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using C = RegCfg<N>;
    FPM_TRY(set_smem(k_xforce_r<N>, C::SMEM));
    const int lines = (N / 2 + 1) * N;
    k_xforce_r<N><<<(lines + C::L - 1) / C::L, C::THREADS, C::SMEM, s>>>(in, out, out_fs, coef, t.tw, t.g, t.w2);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  const size_t sm = xpass_smem<N>(3);
  FPM_TRY(set_smem(k_xforce<N>, sm));
  dim3 grid((N / 2 + 1) * (N / XB));
  k_xforce<N><<<grid, FFT_THREADS, sm, s>>>(in, out, out_fs, coef, t.tw, t.g, t.w2);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int fft_zfwd(const FftTables& t, const float* in, float2* spec, int nf, size_t in_fs, size_t out_fs,
             cudaStream_t s) {
  FPM_DISPATCH_N(t.n, return zfwd_impl<N>(t, in, spec, nf, in_fs, out_fs, s));
}

int fft_y(const FftTables& t, float2* spec, int nf, size_t fs, bool inverse, cudaStream_t s) {
  FPM_DISPATCH_N(t.n, return y_impl<N>(t, spec, nf, fs, inverse, s));
}

int fft_zinv(const FftTables& t, const float2* spec, float* out, int nf, size_t in_fs, size_t out_fs,
             cudaStream_t s) {
  FPM_DISPATCH_N(t.n, return zinv_impl<N>(t, spec, out, nf, in_fs, out_fs, s));
}

int fft_xforce(const FftTables& t, const float2* in, float2* out, size_t out_fs, float coef, cudaStream_t s) {
  FPM_DISPATCH_N(t.n, return xforce_impl<N>(t, in, out, out_fs, coef, s));
}

template <int N>
static int zinv3_impl(const FftTables& t, const float2* spec, float4* out, size_t in_fs, cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using C = RegCfg<N>;
    FPM_TRY(set_smem(k_zinv3_r<N>, C::SMEM));
    k_zinv3_r<N><<<N * N / (2 * C::L), C::THREADS, C::SMEM, s>>>(spec, out, in_fs, t.tw);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  return FPM_ENOTIMPL;
}

bool fft_has_interleaved(int n) { return is_pow2_size(n); }

int fft_zinv3(const FftTables& t, const float2* spec, float4* out, size_t in_fs, cudaStream_t s) {
  FPM_DISPATCH_N(t.n, return zinv3_impl<N>(t, spec, out, in_fs, s));
}

}  // namespace fpm
