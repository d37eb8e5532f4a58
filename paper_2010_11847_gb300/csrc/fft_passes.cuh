// fft_passes.cuh -- the three axis passes of the 3D real FFT (internal).
//
// Spectral layout [kx][kz][ky] (ky fastest): the z pass transposes while it
// transforms, so that every pass moves whole >=128-byte segments.
//   z pass  (r2c): real rows along z -> half spectrum lines along ky
//   y pass       : contiguous lines along ky, in place
//   x pass       : lines along kx (stride (n/2+1)*n), XB adjacent ky per CTA;
//                  the spectral operator of the step is applied here
//   z pass  (c2r): lines along kz for 2*ZG adjacent y -> real rows along z
// Two real rows share one complex transform (row a in the real part, row b
// in the imaginary part) and are separated / recombined by the symmetry
// Z(N-k) = conj(A(k)) + i conj(B(k)).
#pragma once
#include "fft.cuh"
#include "internal.h"

namespace fpm {

constexpr int ZG = 8;          // complex lines (= row pairs) per CTA in z passes
constexpr int YL = 8;          // lines per CTA in the y pass
constexpr int XB = 8;          // adjacent ky lines per CTA in x passes
constexpr int FFT_THREADS = 256;

template <int N>
constexpr size_t zpass_smem() { return (size_t)(2 * ZG * sp_size(N) + N) * sizeof(float2); }
template <int N>
constexpr size_t ypass_smem() { return (size_t)(2 * YL * sp_size(N) + N) * sizeof(float2); }
template <int N>
constexpr size_t xpass_smem(int nbuf) { return (size_t)(nbuf * XB * sp_size(N) + N) * sizeof(float2); }

// ---------------------------------------------------------------- z r2c
template <int N>
__device__ __forceinline__ void body_zfwd(const float* __restrict__ in, float2* __restrict__ out,
                                                      size_t in_fs, size_t out_fs, const float2* __restrict__ g_tw, float2* smem, int bx, int by) {
  constexpr int LS = sp_size(N);
  constexpr int NH = N / 2 + 1;
  constexpr int GROUPS = N / (2 * ZG);
  float2* a = smem;
  float2* b = a + ZG * LS;
  float2* tw = b + ZG * LS;
  load_twiddles<N>(tw, g_tw);
  const int x = bx / GROUPS;
  const int y0 = (bx % GROUPS) * 2 * ZG;
  const float* src = in + by * in_fs + ((size_t)x * N + y0) * N;
  for (int idx = threadIdx.x; idx < ZG * N; idx += blockDim.x) {
    const int g = idx / N, z = idx - g * N;
    a[g * LS + sp(z)] = make_float2(__ldcg(src + (2 * g) * N + z), __ldcg(src + (2 * g + 1) * N + z));
  }
  __syncthreads();
  const float2* r = FftPlan<N>::template run<false>(a, b, ZG, LS, tw);
  float4* dst = reinterpret_cast<float4*>(out + by * out_fs + (size_t)x * NH * N + y0);
  for (int idx = threadIdx.x; idx < NH * ZG; idx += blockDim.x) {
    const int kz = idx / ZG, g = idx - kz * ZG;
    const float2 zk = r[g * LS + sp(kz)];
    const float2 zn = conjf2(r[g * LS + sp((N - kz) % N)]);
    const float2 A = cscale(cadd(zk, zn), 0.5f);
    const float2 B = cscale(mul_mi(csub(zk, zn)), 0.5f);
    dst[((size_t)kz * N) / 2 + g] = make_float4(A.x, A.y, B.x, B.y);
  }
}

template <int N>
__global__ void __launch_bounds__(FFT_THREADS) k_zfwd(const float* __restrict__ in, float2* __restrict__ out,
                                                      size_t in_fs, size_t out_fs, const float2* __restrict__ g_tw) {
  extern __shared__ float2 smem[];
  body_zfwd<N>(in, out, in_fs, out_fs, g_tw, smem, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- y (in place)
template <int N, bool INV>
__device__ __forceinline__ void body_yfft(float2* __restrict__ data, int nlines, size_t fs,
                                                      const float2* __restrict__ g_tw, float2* smem, int bx, int by) {
  constexpr int LS = sp_size(N);
  float2* a = smem;
  float2* b = a + YL * LS;
  float2* tw = b + YL * LS;
  load_twiddles<N>(tw, g_tw);
  const int line0 = bx * YL;
  const int nl = min(YL, nlines - line0);
  float2* base = data + by * fs + (size_t)line0 * N;
  for (int idx = threadIdx.x; idx < YL * N; idx += blockDim.x) {
    const int l = idx / N, e = idx - l * N;
    a[l * LS + sp(e)] = (l < nl) ? base[(size_t)l * N + e] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2* r = FftPlan<N>::template run<INV>(a, b, YL, LS, tw);
  for (int idx = threadIdx.x; idx < nl * N; idx += blockDim.x) {
    const int l = idx / N, e = idx - l * N;
    base[(size_t)l * N + e] = r[l * LS + sp(e)];
  }
}

template <int N, bool INV>
__global__ void __launch_bounds__(FFT_THREADS) k_yfft(float2* __restrict__ data, int nlines, size_t fs,
                                                      const float2* __restrict__ g_tw) {
  extern __shared__ float2 smem[];
  body_yfft<N, INV>(data, nlines, fs, g_tw, smem, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- z c2r
template <int N>
__device__ __forceinline__ void body_zinv(const float2* __restrict__ in, float* __restrict__ out,
                                                      size_t in_fs, size_t out_fs, const float2* __restrict__ g_tw, float2* smem, int bx, int by) {
  constexpr int LS = sp_size(N);
  constexpr int NH = N / 2 + 1;
  constexpr int GROUPS = N / (2 * ZG);
  float2* a = smem;
  float2* b = a + ZG * LS;
  float2* tw = b + ZG * LS;
  load_twiddles<N>(tw, g_tw);
  const int x = bx / GROUPS;
  const int y0 = (bx % GROUPS) * 2 * ZG;
  const float4* src = reinterpret_cast<const float4*>(in + by * in_fs + (size_t)x * NH * N + y0);
  for (int idx = threadIdx.x; idx < NH * ZG; idx += blockDim.x) {
    const int kz = idx / ZG, g = idx - kz * ZG;
    const float4 v = __ldcg(src + ((size_t)kz * N) / 2 + g);   // A = (x, y), B = (z, w)
    if (kz == 0 || kz == N / 2) {
      a[g * LS + sp(kz)] = make_float2(v.x, v.z);
    } else {
      a[g * LS + sp(kz)] = make_float2(v.x - v.w, v.y + v.z);
      a[g * LS + sp(N - kz)] = make_float2(v.x + v.w, v.z - v.y);
    }
  }
  __syncthreads();
  const float2* r = FftPlan<N>::template run<true>(a, b, ZG, LS, tw);
  float* dst = out + by * out_fs + ((size_t)x * N + y0) * N;
  for (int idx = threadIdx.x; idx < ZG * N; idx += blockDim.x) {
    const int g = idx / N, z = idx - g * N;
    const float2 v = r[g * LS + sp(z)];
    dst[(2 * g) * N + z] = v.x;
    dst[(2 * g + 1) * N + z] = v.y;
  }
}

template <int N>
__global__ void __launch_bounds__(FFT_THREADS) k_zinv(const float2* __restrict__ in, float* __restrict__ out,
                                                      size_t in_fs, size_t out_fs, const float2* __restrict__ g_tw) {
  extern __shared__ float2 smem[];
  body_zinv<N>(in, out, in_fs, out_fs, g_tw, smem, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- x pass helpers
// Load XB adjacent ky lines of a half spectrum (all kx) into smem lines.
template <int N>
__device__ __forceinline__ void xload(float2* dst, const float2* __restrict__ spec, int kz, int ky0) {
  constexpr int LS = sp_size(N);
  constexpr size_t S = (size_t)(N / 2 + 1) * N;
  for (int idx = threadIdx.x; idx < N * XB; idx += blockDim.x) {
    const int x = idx / XB, j = idx - x * XB;
    dst[j * LS + sp(x)] = __ldcg(spec + x * S + (size_t)kz * N + ky0 + j);
  }
}

template <int N>
__device__ __forceinline__ void xstore(float2* __restrict__ spec, const float2* src, int kz, int ky0) {
  constexpr int LS = sp_size(N);
  constexpr size_t S = (size_t)(N / 2 + 1) * N;
  for (int idx = threadIdx.x; idx < N * XB; idx += blockDim.x) {
    const int x = idx / XB, j = idx - x * XB;
    spec[x * S + (size_t)kz * N + ky0 + j] = src[j * LS + sp(x)];
  }
}

// Force transfer function (Eqs. 3-5): forward x transform of delta(k), then
// for each axis d: F_d(k) = i g_d 1.5 Om delta(k) / |w|^2 (coef = 1.5 Om / M
// folds in the inverse normalisation), inverse x transform.  out may alias in.
template <int N>
__device__ __forceinline__ void body_xforce(const float2* in, float2* out, size_t out_fs,
                                                        float coef, const float2* __restrict__ g_tw,
                                                        const float* __restrict__ g_g,
                                                        const float* __restrict__ g_w2, float2* smem, int bx, int by) {
  constexpr int LS = sp_size(N);
  constexpr int NB = N / XB;
  float2* s0 = smem;
  float2* s1 = s0 + XB * LS;
  float2* s2 = s1 + XB * LS;
  float2* tw = s2 + XB * LS;
  load_twiddles<N>(tw, g_tw);
  const int kz = bx / NB;
  const int ky0 = (bx % NB) * XB;
  xload<N>(s0, in, kz, ky0);
  __syncthreads();
  float2* d = FftPlan<N>::template run<false>(s0, s1, XB, LS, tw);
  float2* f1 = (d == s0) ? s1 : s0;
  float2* f2 = s2;
  const float w2z = __ldg(g_w2 + kz);
  for (int axis = 0; axis < 3; ++axis) {
    for (int idx = threadIdx.x; idx < N * XB; idx += blockDim.x) {
      const int j = idx / N, x = idx - j * N;
      const int ky = ky0 + j;
      const float k2 = __ldg(g_w2 + x) + __ldg(g_w2 + ky) + w2z;
      const int kd = axis == 0 ? x : (axis == 1 ? ky : kz);
      const float gd = __ldg(g_g + kd);
      const float s = (k2 > 0.f) ? gd * coef / k2 : 0.f;
      f1[j * LS + sp(x)] = mul_i(cscale(d[j * LS + sp(x)], s));
    }
    __syncthreads();
    const float2* r = FftPlan<N>::template run<true>(f1, f2, XB, LS, tw);
    xstore<N>(out + axis * out_fs, r, kz, ky0);
    __syncthreads();
  }
}

template <int N>
__global__ void __launch_bounds__(FFT_THREADS) k_xforce(const float2* in, float2* out, size_t out_fs,
                                                        float coef, const float2* __restrict__ g_tw,
                                                        const float* __restrict__ g_g,
                                                        const float* __restrict__ g_w2) {
  extern __shared__ float2 smem[];
  body_xforce<N>(in, out, out_fs, coef, g_tw, g_g, g_w2, smem, blockIdx.x, blockIdx.y);
}

}  // namespace fpm
