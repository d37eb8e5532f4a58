// ic_reg.cuh -- x passes of the initial conditions and of P(k) on the
// register FFT, and the real-space 2LPT source (internal).
//
// Power-of-two lattices build 2LPT through potentials, as the force does:
//   psi   = IFFT[ lin / |w|^2 ] / N^3,
//   S     = sum_{i<j} (psi_ii psi_jj - psi_ij^2),  psi_ij = D_i D_j psi,
//   Phi_x = IFFT[ (D1 lin - D2 S(k)) / |w|^2 ] r / N^3,   dx_d = D_d Phi_x,
//   Phi_p = IFFT[ a^2 E (f1 D1 lin - f2 D2 S(k)) / |w|^2 ] r / N^3,  p_d = D_d Phi_p,
// with D the Eq. 5 difference (symbol i g), so that D_i D_j has the symbol
// -g_i g_j: the same operators as the spectral form, one or two fields
// through the inverse transforms instead of six.
#pragma once
#include "fft_reg.cuh"

namespace fpm {

// Eisenstein & Hu (1998) no-wiggle transfer function in FP32 (their eqs.
// 26, 28-31), k in h/Mpc.
__device__ __forceinline__ float eh_nowiggle_T32(float k_h, const EhParams& e) {
  const float ks = 0.43f * k_h * e.h * e.s;
  const float ks2 = ks * ks;
  const float gamma = e.omh * (e.alpha + (1.f - e.alpha) / (1.f + ks2 * ks2));
  const float q = k_h * e.theta2 / gamma;
  const float L0 = logf(5.43656365691809f + 1.8f * q);   // 2e + 1.8 q
  const float C0 = 14.2f + 731.f / (1.f + 62.5f * q);
  return L0 / (L0 + C0 * q * q);
}

// sqrt(P(|n| kf) N^3 / V) for the integer wavevector n (0 at n = 0).
__device__ __forceinline__ float linear_scale(int fx, int fy, int fz, const EhParams& e, float amp, float kf,
                                              float n3v) {
  const int n2 = fx * fx + fy * fy + fz * fz;
  if (n2 == 0) return 0.f;
  const float k = kf * sqrtf((float)n2);
  const float T = eh_nowiggle_T32(k, e);
  const float pk = amp * powf(k, e.n_s) * T * T;
  return sqrtf(pk * n3v);
}

// ---------------------------------------------------------------- x passes
// Lines l = kz*N + ky, L per CTA, line fastest across threads (64-byte
// rows of the [kx][kz][ky] half spectrum).
template <int N>
struct XLine {
  static constexpr int T = RegCfg<N>::T, L = RegCfg<N>::L;
  static constexpr size_t S = (size_t)(N / 2 + 1) * N;
  int line, t, gl, kz, ky;
  bool valid;
  __device__ XLine(int bx) {
    line = threadIdx.x % L;
    t = threadIdx.x / L;
    gl = bx * L + line;
    valid = gl < (N / 2 + 1) * N;
    kz = gl / N;
    ky = gl - kz * N;
  }
  __device__ size_t at(int s) const { return (size_t)(t + T * s) * S + gl; }
};

// Linear field: forward x transform of DFT_zy(w), times linear_scale.
template <int N>
__device__ __forceinline__ void body_xlin_r(const float2* in, float2* out, EhParams e, float amp, float kf,
                                            float n3v, const float2* __restrict__ g_tw, float2* smem, int bx) {
  using X = XLine<N>;
  float2* tw = smem;
  float2* xb = tw + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g_tw[i];
  const X x(bx);
  float2 d[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) d[s] = x.valid ? __ldcg(in + x.at(s)) : make_float2(0.f, 0.f);
  __syncthreads();
  RegFft<N>::template run<false>(d, xb + x.line * rline<N>(), x.t, tw);
  const int fy = freq_of(x.ky, N), fz = x.kz;
  if (x.valid) {
#pragma unroll
    for (int s = 0; s < 8; ++s)
      out[x.at(s)] = cscale(d[s], linear_scale(freq_of(x.t + X::T * s, N), fy, fz, e, amp, kf, n3v));
  }
}

// Potential of a full spectrum: coef * lin / |w|^2 (0 at k = 0), inverse x.
template <int N>
__device__ __forceinline__ void body_xpot_r(const float2* __restrict__ lin, float2* out, float coef,
                                            const float2* __restrict__ g_tw, const float* __restrict__ g_w2,
                                            float2* smem, int bx) {
  using X = XLine<N>;
  float2* tw = smem;
  float2* xb = tw + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g_tw[i];
  const X x(bx);
  const float w2yz = x.valid ? __ldg(g_w2 + x.ky) + __ldg(g_w2 + x.kz) : 1.f;
  float2 d[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const float k2 = __ldg(g_w2 + x.t + X::T * s) + w2yz;
    d[s] = x.valid ? cscale(__ldg(lin + x.at(s)), k2 > 0.f ? coef / k2 : 0.f) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  RegFft<N>::template run<true>(d, xb + x.line * rline<N>(), x.t, tw);
  if (x.valid) {
#pragma unroll
    for (int s = 0; s < 8; ++s) out[x.at(s)] = d[s];
  }
}

// 2LPT potentials: forward x transform of DFT_zy(S) (SECOND), then
//   out0 = coef (c1d lin - c2d S) / |w|^2,  out1 = coef (c1p lin - c2p S) / |w|^2,
// each inverse x transformed.  S(k) waits in shared memory between the two.
template <int N, bool SECOND>
__device__ __forceinline__ void body_xdisp_r(const float2* specS, const float2* __restrict__ lin, float2* out0,
                                             float2* out1, float c1d, float c2d, float c1p, float c2p,
                                             float coef, const float2* __restrict__ g_tw,
                                             const float* __restrict__ g_w2, float2* smem, int bx) {
  using X = XLine<N>;
  float2* tw = smem;
  float2* xb = tw + N;
  float2* sk = xb + X::L * rline<N>();        // [kx][L] transformed S of this CTA's lines
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g_tw[i];
  const X x(bx);
  float2* buf = xb + x.line * rline<N>();
  if (SECOND) {
    float2 d[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) d[s] = x.valid ? __ldcg(specS + x.at(s)) : make_float2(0.f, 0.f);
    __syncthreads();
    RegFft<N>::template run<false>(d, buf, x.t, tw);
#pragma unroll
    for (int s = 0; s < 8; ++s) sk[(x.t + X::T * s) * X::L + x.line] = d[s];
  } else {
    __syncthreads();
  }
  const float w2yz = x.valid ? __ldg(g_w2 + x.ky) + __ldg(g_w2 + x.kz) : 1.f;
#pragma unroll 1
  for (int o = 0; o < 2; ++o) {
    const float c1 = o == 0 ? c1d : c1p, c2 = o == 0 ? c2d : c2p;
    float2 v[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const float k2 = __ldg(g_w2 + x.t + X::T * s) + w2yz;
      float2 a = x.valid ? cscale(__ldg(lin + x.at(s)), c1) : make_float2(0.f, 0.f);
      if (SECOND) {
        const float2 b = sk[(x.t + X::T * s) * X::L + x.line];
        a.x -= c2 * b.x;
        a.y -= c2 * b.y;
      }
      v[s] = cscale(a, k2 > 0.f ? coef / k2 : 0.f);
    }
    RegFft<N>::template run<true>(v, buf, x.t, tw);
    if (x.valid) {
      float2* o_ = o == 0 ? out0 : out1;
#pragma unroll
      for (int s = 0; s < 8; ++s) o_[x.at(s)] = v[s];
    }
  }
}

// Binned power: forward x transform of DFT_zy(a) (and b); every mode adds
// w Re(A B*), w and w |n| to bin j (j - 1/2 <= |n| < j + 1/2, 1 <= j <= N/2),
// w = 2 for 0 < kz < N/2 (the conjugate partner), else 1.  acc: 3 N/2
// floats of shared memory (native shared atomics; a block's partial sums of
// at most a few thousand positive terms per bin), flushed in FP64 by the
// caller.
template <int N>
__device__ __forceinline__ void body_xpow_r(const float2* __restrict__ sa, const float2* __restrict__ sb,
                                            float* acc, const float2* __restrict__ g_tw, float2* smem, int bx) {
  using X = XLine<N>;
  constexpr int NBIN = N / 2;
  float2* tw = smem;
  float2* xb = tw + N;
  const X x(bx);
  float2 A[8], B[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) A[s] = x.valid ? __ldg(sa + x.at(s)) : make_float2(0.f, 0.f);
  __syncthreads();
  RegFft<N>::template run<false>(A, xb + x.line * rline<N>(), x.t, tw);
  if (sb) {
#pragma unroll
    for (int s = 0; s < 8; ++s) B[s] = x.valid ? __ldg(sb + x.at(s)) : make_float2(0.f, 0.f);
    RegFft<N>::template run<false>(B, xb + x.line * rline<N>(), x.t, tw);
  } else {
#pragma unroll
    for (int s = 0; s < 8; ++s) B[s] = A[s];
  }
  const float w = (x.kz > 0 && x.kz < N / 2) ? 2.f : 1.f;
  const int fy = freq_of(x.ky, N);
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int fx = freq_of(x.t + X::T * s, N);
    const int n2 = fx * fx + fy * fy + x.kz * x.kz;
    int b = (int)floorf(sqrtf((float)n2) + 0.5f);
    if ((2 * b - 1) * (2 * b - 1) > 4 * n2) --b;
    if ((2 * b + 1) * (2 * b + 1) <= 4 * n2) ++b;
    const bool in = x.valid && b >= 1 && b <= NBIN;
    float v0 = in ? w * (A[s].x * B[s].x + A[s].y * B[s].y) : 0.f;
    float v1 = in ? w : 0.f;
    float v2 = in ? w * sqrtf((float)n2) : 0.f;
    // neighbouring lanes usually share the bin: then one atomic per warp
    const int b0 = __shfl_sync(full, b, 0);
    if (__all_sync(full, in && b == b0)) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        v0 += __shfl_xor_sync(full, v0, off);
        v1 += __shfl_xor_sync(full, v1, off);
        v2 += __shfl_xor_sync(full, v2, off);
      }
      if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc + (b - 1), v0);
        atomicAdd(acc + NBIN + (b - 1), v1);
        atomicAdd(acc + 2 * NBIN + (b - 1), v2);
      }
    } else if (in) {
      atomicAdd(acc + (b - 1), v0);
      atomicAdd(acc + NBIN + (b - 1), v1);
      atomicAdd(acc + 2 * NBIN + (b - 1), v2);
    }
  }
}

// ---------------------------------------------------------------- 2LPT source in real space
// psi_ii = sum_m e_m psi(x + m e_i) with e = c * c (the Eq. 5 difference c
// applied twice: offsets -4..4), psi_ij = sum_{a,b} c_a c_b psi(x + a e_i + b e_j).
// A block owns a TZ x TY patch and marches through XC planes of x with a
// ring of nine halo-padded planes (halo 4).
__host__ __device__ constexpr float fd_c(int o) {
  return o == 1 ? 8.f / 12.f : o == -1 ? -8.f / 12.f : o == 2 ? -1.f / 12.f : o == -2 ? 1.f / 12.f : 0.f;
}
__host__ __device__ constexpr float fd_e(int m) {   // (c * c)[m]
  float s = 0.f;
  for (int a = -2; a <= 2; ++a) s += fd_c(a) * fd_c(m - a);
  return s;
}

template <int N>
struct HsCfg {
  static constexpr int TZ = N < 32 ? N : 32;
  static constexpr int TY = 256 / TZ;
  static constexpr int PZ = TZ + 8, PY = TY + 8, PLANE = PZ * PY;
  static constexpr int XC = N < 32 ? N : 32;
  static constexpr int LOADS = (PLANE + 255) / 256;
};

// HESS = false: S; HESS = true: the six fields phi_ij = -psi_ij (the
// spectral g_i g_j lin / |w|^2 convention), [6][N^3] in the order 00, 11,
// 22, 01, 02, 12, for the adjoint.
template <int N, bool HESS>
__global__ void __launch_bounds__(256) k_lpt_source_fd(const float* __restrict__ psi, float* __restrict__ S) {
  using C = HsCfg<N>;
  constexpr int TZ = C::TZ, TY = C::TY, PZ = C::PZ, PLANE = C::PLANE, XC = C::XC;
  __shared__ float ring[9 * PLANE];
  const int z0 = blockIdx.x * TZ, y0 = blockIdx.y * TY, x0 = blockIdx.z * XC;
  const int tz = threadIdx.x % TZ, ty = threadIdx.x / TZ;
  float pre[C::LOADS];
  auto fetch = [&](int x) {
    const float* pl = psi + (size_t)(x & (N - 1)) * N * N;
#pragma unroll
    for (int k = 0; k < C::LOADS; ++k) {
      const int e = threadIdx.x + 256 * k;
      if (e < PLANE) {
        const int r = e / PZ, c = e - r * PZ;
        pre[k] = __ldg(pl + (size_t)((y0 - 4 + r) & (N - 1)) * N + ((z0 - 4 + c) & (N - 1)));
      }
    }
  };
  auto stash = [&](int slot) {
#pragma unroll
    for (int k = 0; k < C::LOADS; ++k) {
      const int e = threadIdx.x + 256 * k;
      if (e < PLANE) ring[slot * PLANE + e] = pre[k];
    }
  };
  for (int j = 0; j < 8; ++j) {            // planes x0-4 .. x0+3
    fetch(x0 - 4 + j);
    stash(j);
  }
  fetch(x0 + 4);
  const int cidx = (ty + 4) * PZ + tz + 4;
  for (int j = 0; j < XC; ++j) {
    stash((j + 8) % 9);                    // plane x0+j+4
    __syncthreads();
    if (j + 1 < XC) fetch(x0 + j + 5);
    auto P = [&](int dx_, int dy_, int dz_) { return ring[((j + 4 + dx_) % 9) * PLANE + cidx + dy_ * PZ + dz_]; };
    float hxx = 0.f, hyy = 0.f, hzz = 0.f, hxy = 0.f, hxz = 0.f, hyz = 0.f;
#pragma unroll
    for (int m = -4; m <= 4; ++m) {
      const float e = fd_e(m);
      hxx = fmaf(e, P(m, 0, 0), hxx);
      hyy = fmaf(e, P(0, m, 0), hyy);
      hzz = fmaf(e, P(0, 0, m), hzz);
    }
#pragma unroll
    for (int a = -2; a <= 2; ++a) {
      if (a == 0) continue;
#pragma unroll
      for (int b = -2; b <= 2; ++b) {
        if (b == 0) continue;
        const float cc = fd_c(a) * fd_c(b);
        hxy = fmaf(cc, P(a, b, 0), hxy);
        hxz = fmaf(cc, P(a, 0, b), hxz);
        hyz = fmaf(cc, P(0, a, b), hyz);
      }
    }
    const size_t o = ((size_t)(x0 + j) * N + (y0 + ty)) * N + z0 + tz;
    if (HESS) {
      constexpr size_t M = (size_t)N * N * N;
      S[o] = -hxx;
      S[M + o] = -hyy;
      S[2 * M + o] = -hzz;
      S[3 * M + o] = -hxy;
      S[4 * M + o] = -hxz;
      S[5 * M + o] = -hyz;
    } else {
      S[o] = hxx * hyy + hxx * hzz + hyy * hzz - hxy * hxy - hxz * hxz - hyz * hyz;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- kernels
template <int N>
__global__ void __launch_bounds__(RegCfg<N>::THREADS, 1024 / RegCfg<N>::THREADS)
    k_xlin_r(const float2* in, float2* out, EhParams e, const double* __restrict__ d_amp, float kf, float n3v,
             const float2* __restrict__ g_tw) {
  extern __shared__ float2 smem[];
  body_xlin_r<N>(in, out, e, (float)d_amp[0], kf, n3v, g_tw, smem, blockIdx.x);
}

template <int N>
__global__ void __launch_bounds__(RegCfg<N>::THREADS, 1024 / RegCfg<N>::THREADS)
    k_xpot_r(const float2* __restrict__ lin, float2* out, float coef, const float2* __restrict__ g_tw,
             const float* __restrict__ g_w2) {
  extern __shared__ float2 smem[];
  body_xpot_r<N>(lin, out, coef, g_tw, g_w2, smem, blockIdx.x);
}

template <int N, bool SECOND>
__global__ void __launch_bounds__(RegCfg<N>::THREADS, 1024 / RegCfg<N>::THREADS)
    k_xdisp_r(const float2* specS, const float2* __restrict__ lin, float2* out0, float2* out1,
              const double* __restrict__ gr, float a0, float coef, const float2* __restrict__ g_tw,
              const float* __restrict__ g_w2) {
  extern __shared__ float2 smem[];
  const float D1 = (float)gr[0], D2 = (float)gr[1], F1 = (float)gr[2], F2 = (float)gr[3], E = (float)gr[4];
  const float pfac = a0 * a0 * E;
  body_xdisp_r<N, SECOND>(specS, lin, out0, out1, D1, D2, pfac * F1 * D1, pfac * F2 * D2, coef, g_tw, g_w2, smem,
                          blockIdx.x);
}

// Persistent over x items: shared bins, one flush per block.
template <int N>
__global__ void __launch_bounds__(RegCfg<N>::THREADS, 1024 / RegCfg<N>::THREADS)
    k_xpow_r(const float2* __restrict__ sa, const float2* __restrict__ sb, double* __restrict__ bins,
             const float2* __restrict__ g_tw, int items) {
  extern __shared__ float2 smem[];
  constexpr int NBIN = N / 2;
  float* acc = reinterpret_cast<float*>(smem + N + RegCfg<N>::L * rline<N>());
  float2* tw = smem;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g_tw[i];
  for (int k = threadIdx.x; k < 3 * NBIN; k += blockDim.x) acc[k] = 0.f;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    __syncthreads();
    body_xpow_r<N>(sa, sb, acc, g_tw, smem, it);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 3 * NBIN; k += blockDim.x)
    if (acc[k] != 0.f) atomicAdd(bins + k, (double)acc[k]);
}

}  // namespace fpm
