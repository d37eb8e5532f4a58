// adjoint.cu -- spectral and elementwise steps of the reverse (adjoint)
// model: the transpose of the force operator (Eqs. 3-5), of the 2LPT
// displacement field (Algorithm 4 with second order) and of the linear-field
// scaling, plus the chi^2 likelihood term of Eq. 12 and the reverse
// kick/drift.  The spectral steps are x-axis passes of the 3D FFT that take
// several sources, apply a transfer function to each and sum them.
#include "internal.h"
#include "fft_reg.cuh"

namespace fpm {

struct XSources {
  XSource s[XCOMBINE_MAX];
  int n;
};

__device__ __forceinline__ float eh_T32(float k_h, const EhParams& e) {
  const float ks = 0.43f * k_h * e.h * e.s;
  const float ks2 = ks * ks;
  const float gamma = e.omh * (e.alpha + (1.f - e.alpha) / (1.f + ks2 * ks2));
  const float q = k_h * e.theta2 / gamma;
  const float L0 = logf(5.43656365691809f + 1.8f * q);   // 2e + 1.8 q
  const float C0 = 14.2f + 731.f / (1.f + 62.5f * q);
  return L0 / (L0 + C0 * q * q);
}

// sum_s K_s(k) X_s(k) over the sources of one x line, times coef, then an
// optional inverse x transform.  Line mapping as in the force x pass.
template <int N>
__global__ void __launch_bounds__(RegCfg<N>::THREADS, 1024 / RegCfg<N>::THREADS)
    k_xcombine(XSources src, float coef, float one5om, EhParams eh, const double* __restrict__ d_amp, float kf,
               float n3v, float2* out, int inverse, const float2* __restrict__ g_tw,
               const float* __restrict__ g_g, const float* __restrict__ g_w2) {
  using C = RegCfg<N>;
  constexpr int T = C::T, L = C::L, NH = N / 2 + 1;
  constexpr size_t S = (size_t)NH * N;
  extern __shared__ float2 smem[];
  float2* tw = smem;
  float2* xb = tw + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g_tw[i];
  const int line = threadIdx.x % L, t = threadIdx.x / L;
  const int gl = blockIdx.x * L + line;
  const bool valid = gl < NH * N;
  const int kz = valid ? gl / N : 0, ky = valid ? gl - kz * N : 0;
  float2* buf = xb + line * rline<N>();
  const float amp = d_amp ? (float)d_amp[0] : 0.f;
  float2 acc[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) acc[s] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int q = 0; q < src.n; ++q) {
    const XSource x = src.s[q];
    float2 v[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) v[s] = valid ? x.spec[(size_t)(t + T * s) * S + gl] : make_float2(0.f, 0.f);
    if (!x.in_k) RegFft<N>::template run<false>(v, buf, t, tw);
    const int fyz[2] = {freq_of(ky, N), kz};
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int kx = t + T * s;
      const float k2 = __ldg(g_w2 + kx) + __ldg(g_w2 + ky) + __ldg(g_w2 + kz);
      if (!(k2 > 0.f)) continue;
      const int kk[3] = {kx, ky, kz};
      float2 r;
      if (x.kind == SK_H) {
        r = cscale(v[s], __ldg(g_g + kk[x.a]) * __ldg(g_g + kk[x.b]) / k2);
      } else if (x.kind == SK_LINEAR) {
        const int fx = freq_of(kx, N);
        const float k = kf * sqrtf((float)(fx * fx + fyz[0] * fyz[0] + fyz[1] * fyz[1]));
        const float T_ = eh_T32(k, eh);
        r = cscale(v[s], sqrtf(amp * powf(k, eh.n_s) * T_ * T_ * n3v));
      } else {
        float c = __ldg(g_g + kk[x.a]) / k2;
        if (x.kind == SK_FORCE_NEG) c = -c * one5om;
        if (x.kind == SK_BCONJ) c = -c;
        r = mul_i(cscale(v[s], c));
      }
      acc[s] = cadd(acc[s], r);
    }
  }
#pragma unroll
  for (int s = 0; s < 8; ++s) acc[s] = cscale(acc[s], coef);
  if (inverse) RegFft<N>::template run<true>(acc, buf, t, tw);
  if (valid) {
#pragma unroll
    for (int s = 0; s < 8; ++s) out[(size_t)(t + T * s) * S + gl] = acc[s];
  }
}

template <int N>
static int xcombine_impl(const FftTables& t, const XSources& xs, float coef, float one5om, const EhParams& eh,
                         const double* d_amp, float kf, float n3v, float2* out, int inverse, cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using C = RegCfg<N>;
    if (C::SMEM > 48 * 1024)
      FPM_CUDA_TRY(cudaFuncSetAttribute(k_xcombine<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    const int lines = (N / 2 + 1) * N;
    k_xcombine<N><<<(lines + C::L - 1) / C::L, C::THREADS, C::SMEM, s>>>(xs, coef, one5om, eh, d_amp, kf, n3v, out,
                                                                        inverse, t.tw, t.g, t.w2);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  return FPM_ENOTIMPL;
}

int fft_xcombine(const FftTables& t, const XSource* src, int nsrc, float coef, double omega_m, const EhParams* eh,
                 const double* d_amp, float kf, float n3v, float2* out, int inverse, cudaStream_t s) {
  if (nsrc < 1 || nsrc > XCOMBINE_MAX) return FPM_EINVAL;
  XSources xs{};
  for (int i = 0; i < nsrc; ++i) xs.s[i] = src[i];
  xs.n = nsrc;
  const EhParams e = eh ? *eh : EhParams{};
  const float one5om = (float)(1.5 * omega_m);
  switch (t.n) {
    case 16: return xcombine_impl<16>(t, xs, coef, one5om, e, d_amp, kf, n3v, out, inverse, s);
    case 32: return xcombine_impl<32>(t, xs, coef, one5om, e, d_amp, kf, n3v, out, inverse, s);
    case 64: return xcombine_impl<64>(t, xs, coef, one5om, e, d_amp, kf, n3v, out, inverse, s);
    case 128: return xcombine_impl<128>(t, xs, coef, one5om, e, d_amp, kf, n3v, out, inverse, s);
    case 256: return xcombine_impl<256>(t, xs, coef, one5om, e, d_amp, kf, n3v, out, inverse, s);
    case 512: return xcombine_impl<512>(t, xs, coef, one5om, e, d_amp, kf, n3v, out, inverse, s);
    default: return FPM_ENOTIMPL;
  }
}

// ------------------------------------------------------------ chi^2 (Eq. 12)
// r = (rho - 1 - target) / sigma; loss = sum r^2 in FP64 with a fixed-order
// reduction (per-block tree, then one block over the block partials);
// g_rho = 2 r / sigma.
constexpr int CHI_THREADS = 256;
__global__ void __launch_bounds__(CHI_THREADS) k_chi2(const float* __restrict__ rho, const float* __restrict__ tgt,
                                                      size_t M, float inv_sigma, float* __restrict__ g_rho,
                                                      double* __restrict__ partial) {
  __shared__ double sm[CHI_THREADS];
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
    const float r = (rho[i] - 1.f - tgt[i]) * inv_sigma;
    if (g_rho) g_rho[i] = 2.f * r * inv_sigma;
    acc += (double)r * (double)r;
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = CHI_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void __launch_bounds__(CHI_THREADS) k_sum_partials(const double* __restrict__ partial, int n,
                                                              double* __restrict__ out) {
  __shared__ double sm[CHI_THREADS];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = CHI_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sm[0];
}

int launch_chi2(const float* rho, const float* target, size_t M, float sigma, float* g_rho, double* partial,
                int npartial, double* loss, cudaStream_t s) {
  k_chi2<<<npartial, CHI_THREADS, 0, s>>>(rho, target, M, 1.f / sigma, g_rho, partial);
  FPM_CUDA_TRY(cudaGetLastError());
  k_sum_partials<<<1, CHI_THREADS, 0, s>>>(partial, npartial, loss);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

// ------------------------------------------------------------ Adam on the posterior (Sec. 7.1, Eq. 12)
// g' = gscale g + pscale x (the prior term of the white noise), then one Adam
// update (Kingma & Ba 2015, Algorithm 1) of x, m, v in place; c1, c2 are the
// bias corrections 1/(1 - beta^t) and o1, o2 = 1 - beta, all formed in FP64
// on the host (1 - 0.999f in float32 would be off by 1e-5).  The FP64 sum of x^2 / 2 before the update
// (the prior's value) goes to per-block partials in a fixed order.
__global__ void __launch_bounds__(CHI_THREADS) k_adam(float* __restrict__ x, const float* __restrict__ g,
                                                      float* __restrict__ m, float* __restrict__ v, size_t n,
                                                      float gscale, float pscale, float lr, float b1, float b2,
                                                      float o1, float o2, float eps, float c1, float c2,
                                                      double* __restrict__ partial) {
  __shared__ double sm[CHI_THREADS];
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float xi = x[i];
    acc += 0.5 * (double)xi * (double)xi;
    const float gi = fmaf(gscale, g[i], pscale * xi);
    const float mi = fmaf(b1, m[i], o1 * gi);
    const float vi = fmaf(b2, v[i], o2 * gi * gi);
    m[i] = mi;
    v[i] = vi;
    x[i] = xi - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = CHI_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

int launch_adam(float* x, const float* g, float* m, float* v, size_t n, float gscale, float pscale, float lr,
                float b1, float b2, float o1, float o2, float eps, float c1, float c2, double* partial, int npartial,
                double* prior, cudaStream_t s) {
  k_adam<<<npartial, CHI_THREADS, 0, s>>>(x, g, m, v, n, gscale, pscale, lr, b1, b2, o1, o2, eps, c1, c2, partial);
  FPM_CUDA_TRY(cudaGetLastError());
  k_sum_partials<<<1, CHI_THREADS, 0, s>>>(partial, npartial, prior);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

// ------------------------------------------------------------ reverse kick / drift
// gp += D gx (drift transpose), then v = K gp with K = fac[ik1] (+ fac[ik2])
// (v null: gp only).
__global__ void k_adj_drift_kick(float* __restrict__ gx, float* __restrict__ gp, float* __restrict__ v, size_t n,
                                 const double* __restrict__ fac, int idr, int ik1, int ik2) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float D = (float)fac[idr];
  const float K = (float)(fac[ik1] + (ik2 >= 0 ? fac[ik2] : 0.0));
  const float g = fmaf(D, gx[i], gp[i]);
  gp[i] = g;
  if (v) v[i] = K * g;
}

__global__ void k_scale_copy(const float* __restrict__ src, float* __restrict__ dst, size_t n,
                             const double* __restrict__ fac, int ik) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)fac[ik] * src[i];
}

int launch_adj_drift_kick(float* gx, float* gp, float* v, size_t n, const double* fac, int idr, int ik1, int ik2,
                          cudaStream_t s) {
  k_adj_drift_kick<<<(int)((n + 255) / 256), 256, 0, s>>>(gx, gp, v, n, fac, idr, ik1, ik2);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_scale_copy(const float* src, float* dst, size_t n, const double* fac, int ik, cudaStream_t s) {
  k_scale_copy<<<(int)((n + 255) / 256), 256, 0, s>>>(src, dst, n, fac, ik);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

// ------------------------------------------------------------ 2LPT reverse, elementwise parts
// dx = r (D1 Psi1 + D2 Psi2), p = r a^2 E (f1 D1 Psi1 + f2 D2 Psi2):
//   g_Psi1 = r (D1 g_dx + a^2 E f1 D1 g_p),  g_Psi2 = r (D2 g_dx + a^2 E f2 D2 g_p).
__global__ void k_lpt_gpsi(const float* __restrict__ gdx, const float* __restrict__ gp, size_t n,
                           const double* __restrict__ gr, float a0, float r, float* __restrict__ out6) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  const float D1 = (float)gr[0], D2 = (float)gr[1], F1 = (float)gr[2], F2 = (float)gr[3], E = (float)gr[4];
  const float pf = a0 * a0 * E;
  const float gx = gdx[i], gv = gp[i];
  out6[i] = r * (D1 * gx + pf * F1 * D1 * gv);
  out6[3 * n + i] = r * (D2 * gx + pf * F2 * D2 * gv);
}

// S = phi00 phi11 + phi00 phi22 + phi11 phi22 - phi01^2 - phi02^2 - phi12^2:
// replace the phi fields (order 00, 11, 22, 01, 02, 12) by g_S dS/dphi.
__global__ void k_lpt_gphi(const float* __restrict__ gS, float* __restrict__ phi, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = gS[i];
  const float a = phi[i], b = phi[n + i], c = phi[2 * n + i];
  phi[i] = g * (b + c);
  phi[n + i] = g * (a + c);
  phi[2 * n + i] = g * (a + b);
  phi[3 * n + i] *= -2.f * g;
  phi[4 * n + i] *= -2.f * g;
  phi[5 * n + i] *= -2.f * g;
}

int launch_lpt_gpsi(const float* gdx, const float* gp, size_t n, const double* gr, float a0, float r, float* out6,
                    cudaStream_t s) {
  k_lpt_gpsi<<<(int)((3 * n + 255) / 256), 256, 0, s>>>(gdx, gp, n, gr, a0, r, out6);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_lpt_gphi(const float* gS, float* phi6, size_t n, cudaStream_t s) {
  k_lpt_gphi<<<(int)((n + 255) / 256), 256, 0, s>>>(gS, phi6, n);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

}  // namespace fpm
