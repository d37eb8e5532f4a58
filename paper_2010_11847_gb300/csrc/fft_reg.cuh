// fft_reg.cuh -- register-resident Stockham FFT for power-of-two lengths
// (internal), and the hot axis passes of the force step built on it.
//
// A line of N points is held by T = N/V threads, thread t owning the
// elements t + T*s, s = 0..V-1 (its V "slots"; V = 8, or 16 for one warp per
// line at N = 512).  A stage of radix R applies V/R butterflies per thread;
// butterfly j = t + T*q reads slots q + (V/R)*r,
// so the inputs of every stage are in the thread's registers.  Between two
// stages the outputs go through shared memory once (write at the Stockham
// position (j/Ns)*Ns*R + j%Ns + r*Ns, barrier, read back t + T*s).  The
// last stage's outputs land exactly on the thread's own slots, so a
// transform ends in registers in natural order: a forward transform, a
// pointwise operator and an inverse transform chain without touching memory.
// N = 512 = 8*8*8 needs two exchanges; twiddles come from the host FP64
// table staged in shared memory.
//
// Field data is loaded with ld.global.cg (L2, never the read-only path):
// the same bodies run inside persistent launches where another block wrote
// the data earlier in the launch.
#pragma once
#include "fft.cuh"
#include "internal.h"

namespace fpm {

__host__ __device__ __forceinline__ constexpr int rp(int i) { return i + (i >> 3); }   // padded exchange index
// Exchange index of a line: padded (LAY 0, line stride rline), or XOR-swizzled
// within 16-element rows (LAY 1, line stride N + 2).  The swizzle makes both
// the Stockham writes and the contiguous read-back free of bank conflicts
// when a line's threads are consecutive lanes; the padding suits lines that
// are interleaved across lanes (the x pass).
// sw16 is linear over XOR (each bit of the mask it XORs in is one input
// bit), so for indices made of disjoint bit fields, e.g. t + T*s with t < T
// a power of two, sw16(a + b) = sw16(a) ^ sw16(b): the run-time part is
// swizzled once and each compile-time part costs one XOR.
__host__ __device__ __forceinline__ constexpr int sw16(int i) { return i ^ (((i >> 4) & 7) | ((i >> 3) & 8)); }
template <int LAY>
__device__ __forceinline__ int xidx(int i) { return LAY == 0 ? rp(i) : sw16(i); }
template <int N>
__host__ __device__ constexpr int rline() { return N + N / 8 + 1; }   // odd: lines start on distinct banks

// Barrier between exchange steps: the whole block (sid < 0), or only the
// threads of one line -- named barrier sid for lines of >= 64 threads, the
// warp for shorter lines.
template <int T>
__device__ __forceinline__ void xsync(int sid) {
  if (sid < 0) {
    __syncthreads();
  } else if (T >= 64) {
    asm volatile("bar.sync %0, %1;" ::"r"(sid), "n"(T) : "memory");
  } else {
    __syncwarp();
  }
}

template <int N, int V, int R, int NS, bool INV, bool LAST, int LAY>
__device__ __forceinline__ void reg_stage(float2 (&v)[V], float2* buf, int t, const float2* tw, int sid) {
  constexpr int T = N / V, Q = V / R, TWS = N / (NS * R);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = t + T * q;
    const int k = (NS == 1) ? 0 : (j % NS);
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = v[q + Q * r];
    if (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[k * r * TWS];
        if (INV) w.y = -w.y;
        x[r] = cmul(x[r], w);
      }
    }
    Dft<R, INV>::run(x);
    if (LAST) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[q + Q * r] = x[r];
    } else {
      const int base = (j / NS) * NS * R + k;     // zero in the bits of r * NS
      if (LAY == 1) {
        const int sb = sw16(base);
#pragma unroll
        for (int r = 0; r < R; ++r) buf[sb ^ sw16(r * NS)] = x[r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) buf[xidx<LAY>(base + r * NS)] = x[r];
      }
    }
  }
  if (!LAST) {
    xsync<T>(sid);
    if (LAY == 1) {
      const int st = sw16(t);                    // t < T
#pragma unroll
      for (int s = 0; s < V; ++s) v[s] = buf[st ^ sw16(T * s)];
    } else {
#pragma unroll
      for (int s = 0; s < V; ++s) v[s] = buf[xidx<LAY>(t + T * s)];
    }
    xsync<T>(sid);
  }
}

template <int N, int V, bool INV, int LAY, int NS, int... Rs>
struct RegStages;
template <int N, int V, bool INV, int LAY, int NS>
struct RegStages<N, V, INV, LAY, NS> {
  static __device__ __forceinline__ void run(float2 (&)[V], float2*, int, const float2*, int) {}
};
template <int N, int V, bool INV, int LAY, int NS, int R, int... Rs>
struct RegStages<N, V, INV, LAY, NS, R, Rs...> {
  static __device__ __forceinline__ void run(float2 (&v)[V], float2* buf, int t, const float2* tw, int sid) {
    reg_stage<N, V, R, NS, INV, sizeof...(Rs) == 0, LAY>(v, buf, t, tw, sid);
    RegStages<N, V, INV, LAY, NS * R, Rs...>::run(v, buf, t, tw, sid);
  }
};

// Radix plan of each length (the same for V = 8 and 16).
template <int N, int V, bool INV, int LAY>
struct RegPlan;
#define FPM_REG_PLAN(NN, ...)                                                                  \
  template <int V, bool INV, int LAY>                                                          \
  struct RegPlan<NN, V, INV, LAY> : RegStages<NN, V, INV, LAY, 1, __VA_ARGS__> {};
FPM_REG_PLAN(16, 8, 2)
FPM_REG_PLAN(32, 8, 4)
FPM_REG_PLAN(64, 8, 8)
FPM_REG_PLAN(128, 8, 8, 2)
FPM_REG_PLAN(256, 8, 8, 4)
FPM_REG_PLAN(512, 8, 8, 8)
#undef FPM_REG_PLAN

template <int N, int V = 8>
struct RegFft {
  template <bool INV, int LAY = 0>
  static __device__ __forceinline__ void run(float2 (&v)[V], float2* buf, int t, const float2* tw, int sid = -1) {
    RegPlan<N, V, INV, LAY>::run(v, buf, t, tw, sid);
  }
};

__host__ __device__ constexpr bool is_pow2_size(int n) { return n >= 16 && n <= 512 && (n & (n - 1)) == 0; }

// Lines per CTA: 256 threads, at least 8 lines; V slots (points) per thread.
template <int N, int V = 8>
struct RegCfg {
  static constexpr int T = N / V;
  static constexpr int L = (256 / T) > 8 ? 256 / T : 8;
  static constexpr int THREADS = T * L;
  static constexpr size_t SMEM = (size_t)(L * rline<N>() + N) * sizeof(float2);
};

// ---------------------------------------------------------------- z r2c
// L complex lines = 2L consecutive real rows (row = x*N + y) per CTA.
template <int N, int V = 8>
__device__ __forceinline__ void body_zfwd_r(const float* __restrict__ in,
                                                               float2* __restrict__ out, size_t in_fs,
                                                               size_t out_fs, const float2* __restrict__ g_tw, float2* smem, int bx, int by) {
  using C = RegCfg<N, V>;
  constexpr int T = C::T, L = C::L, NH = N / 2 + 1;
  float2* tw = smem;
  float2* xb = tw + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g_tw[i];
  const int g = threadIdx.x / T, t = threadIdx.x - g * T;
  const size_t r0 = (size_t)bx * 2 * L;
  const float* src = in + by * in_fs + (r0 + 2 * g) * N;
  float2 v[V];
#pragma unroll
  for (int s = 0; s < V; ++s) v[s] = make_float2(__ldcg(src + t + T * s), __ldcg(src + N + t + T * s));
  __syncthreads();
  float2* buf = xb + g * rline<N>();
  RegFft<N, V>::template run<false>(v, buf, t, tw);
#pragma unroll
  for (int s = 0; s < V; ++s) buf[rp(t + T * s)] = v[s];
  __syncthreads();
  float2* dst = out + by * out_fs;
  for (int idx = threadIdx.x; idx < NH * L; idx += blockDim.x) {
    const int kz = idx / L, gg = idx - kz * L;
    const float2* b = xb + gg * rline<N>();
    const float2 zk = b[rp(kz)];
    const float2 zn = conjf2(b[rp((N - kz) & (N - 1))]);
    const float2 A = cscale(cadd(zk, zn), 0.5f);
    const float2 B = cscale(mul_mi(csub(zk, zn)), 0.5f);
    const size_t row = r0 + 2 * gg;
    const size_t x = row / N, y = row - x * N;
    *reinterpret_cast<float4*>(dst + (x * NH + kz) * N + y) = make_float4(A.x, A.y, B.x, B.y);
  }
}

template <int N>
__global__ void __launch_bounds__(RegCfg<N>::THREADS, 1024 / RegCfg<N>::THREADS) k_zfwd_r(const float* __restrict__ in,
                                                               float2* __restrict__ out, size_t in_fs,
                                                               size_t out_fs, const float2* __restrict__ g_tw) {
  extern __shared__ float2 smem[];
  body_zfwd_r<N>(in, out, in_fs, out_fs, g_tw, smem, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- y (in place, contiguous lines)
template <int N, bool INV, int V = 8>
__device__ __forceinline__ void body_yfft_r(float2* __restrict__ data, int nlines, size_t fs,
                                                               const float2* __restrict__ g_tw, float2* smem, int bx, int by) {
  using C = RegCfg<N, V>;
  constexpr int T = C::T, L = C::L;
  float2* tw = smem;
  float2* xb = tw + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g_tw[i];
  const int line = threadIdx.x / T, t = threadIdx.x - line * T;
  const int gl = bx * L + line;
  const bool valid = gl < nlines;
  float2* base = data + by * fs + (size_t)gl * N;
  float2 v[V];
#pragma unroll
  for (int s = 0; s < V; ++s) v[s] = valid ? __ldcg(base + t + T * s) : make_float2(0.f, 0.f);
  __syncthreads();
  RegFft<N, V>::template run<INV>(v, xb + line * rline<N>(), t, tw);
  if (valid) {
#pragma unroll
    for (int s = 0; s < V; ++s) base[t + T * s] = v[s];
  }
}

template <int N, bool INV>
__global__ void __launch_bounds__(RegCfg<N>::THREADS, 1024 / RegCfg<N>::THREADS) k_yfft_r(float2* __restrict__ data, int nlines, size_t fs,
                                                               const float2* __restrict__ g_tw) {
  extern __shared__ float2 smem[];
  body_yfft_r<N, INV>(data, nlines, fs, g_tw, smem, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- z c2r
template <int N, int V = 8>
__device__ __forceinline__ void body_zinv_r(const float2* __restrict__ in,
                                                               float* __restrict__ out, size_t in_fs,
                                                               size_t out_fs, const float2* __restrict__ g_tw, float2* smem, int bx, int by) {
  using C = RegCfg<N, V>;
  constexpr int T = C::T, L = C::L, NH = N / 2 + 1;
  float2* tw = smem;
  float2* xb = tw + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g_tw[i];
  const size_t r0 = (size_t)bx * 2 * L;
  const float2* src = in + by * in_fs;
  for (int idx = threadIdx.x; idx < NH * L; idx += blockDim.x) {
    const int kz = idx / L, gg = idx - kz * L;
    const size_t row = r0 + 2 * gg;
    const size_t x = row / N, y = row - x * N;
    const float4 v = __ldcg(reinterpret_cast<const float4*>(src + (x * NH + kz) * N + y));
    float2* b = xb + gg * rline<N>();
    if (kz == 0 || kz == N / 2) {
      b[rp(kz)] = make_float2(v.x, v.z);
    } else {
      b[rp(kz)] = make_float2(v.x - v.w, v.y + v.z);
      b[rp(N - kz)] = make_float2(v.x + v.w, v.z - v.y);
    }
  }
  __syncthreads();
  const int g = threadIdx.x / T, t = threadIdx.x - g * T;
  float2* buf = xb + g * rline<N>();
  float2 v[V];
#pragma unroll
  for (int s = 0; s < V; ++s) v[s] = buf[rp(t + T * s)];
  __syncthreads();
  RegFft<N, V>::template run<true>(v, buf, t, tw);
  float* dst = out + by * out_fs + (r0 + 2 * g) * N;
#pragma unroll
  for (int s = 0; s < V; ++s) {
    dst[t + T * s] = v[s].x;
    dst[N + t + T * s] = v[s].y;
  }
}

template <int N>
__global__ void __launch_bounds__(RegCfg<N>::THREADS, 1024 / RegCfg<N>::THREADS) k_zinv_r(const float2* __restrict__ in,
                                                               float* __restrict__ out, size_t in_fs,
                                                               size_t out_fs, const float2* __restrict__ g_tw) {
  extern __shared__ float2 smem[];
  body_zinv_r<N>(in, out, in_fs, out_fs, g_tw, smem, blockIdx.x, blockIdx.y);
}

// Three fields in one CTA, written interleaved as float4 (F0, F1, F2, 0)
// per cell: the readout then fetches a CIC corner with one 16-byte load.
template <int N>
__device__ __forceinline__ void body_zinv3_r(const float2* __restrict__ in, float4* __restrict__ out, size_t in_fs,
              const float2* __restrict__ g_tw, float2* smem, int bx, int by) {
  using C = RegCfg<N>;
  constexpr int T = C::T, L = C::L, NH = N / 2 + 1;
  float2* tw = smem;
  float2* xb = tw + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g_tw[i];
  const size_t r0 = (size_t)bx * 2 * L;
  const int g = threadIdx.x / T, t = threadIdx.x - g * T;
  float2* buf = xb + g * rline<N>();
  float2 res[3][8];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const float2* src = in + f * in_fs;
    for (int idx = threadIdx.x; idx < NH * L; idx += blockDim.x) {
      const int kz = idx / L, gg = idx - kz * L;
      const size_t row = r0 + 2 * gg;
      const size_t x = row / N, y = row - x * N;
      const float4 v = __ldcg(reinterpret_cast<const float4*>(src + (x * NH + kz) * N + y));
      float2* b = xb + gg * rline<N>();
      if (kz == 0 || kz == N / 2) {
        b[rp(kz)] = make_float2(v.x, v.z);
      } else {
        b[rp(kz)] = make_float2(v.x - v.w, v.y + v.z);
        b[rp(N - kz)] = make_float2(v.x + v.w, v.z - v.y);
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 8; ++s) res[f][s] = buf[rp(t + T * s)];
    __syncthreads();
    RegFft<N>::template run<true>(res[f], buf, t, tw);
  }
  float4* dst = out + (r0 + 2 * g) * N;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    dst[t + T * s] = make_float4(res[0][s].x, res[1][s].x, res[2][s].x, 0.f);
    dst[N + t + T * s] = make_float4(res[0][s].y, res[1][s].y, res[2][s].y, 0.f);
  }
}

template <int N>
__global__ void __launch_bounds__(RegCfg<N>::THREADS, 1024 / RegCfg<N>::THREADS) k_zinv3_r(const float2* __restrict__ in, float4* __restrict__ out, size_t in_fs,
              const float2* __restrict__ g_tw) {
  extern __shared__ float2 smem[];
  body_zinv3_r<N>(in, out, in_fs, g_tw, smem, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- x pass: force transfer function
// L consecutive lines l = kz*N + ky per CTA (line fastest across threads);
// forward x transform of delta(k), then per axis d the Eq. 3-5 operator
// F_d = i g_d coef delta / |w|^2 and the inverse x transform, from registers.
template <int N>
__device__ __forceinline__ void body_xforce_r(const float2* in, float2* out, size_t out_fs,
                                                                 float coef, const float2* __restrict__ g_tw,
                                                                 const float* __restrict__ g_g,
                                                                 const float* __restrict__ g_w2, float2* smem, int bx, int by) {
  using C = RegCfg<N>;
  constexpr int T = C::T, L = C::L, NH = N / 2 + 1;
  constexpr size_t S = (size_t)NH * N;
  float2* tw = smem;
  float2* xb = tw + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g_tw[i];
  const int line = threadIdx.x % L, t = threadIdx.x / L;
  const int gl = bx * L + line;
  const bool valid = gl < NH * N;
  const int kz = gl / N, ky = gl - kz * N;
  float2 d[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) d[s] = valid ? __ldcg(in + (size_t)(t + T * s) * S + gl) : make_float2(0.f, 0.f);
  __syncthreads();
  float2* buf = xb + line * rline<N>();
  RegFft<N>::template run<false>(d, buf, t, tw);
  const float w2yz = valid ? __ldg(g_w2 + ky) + __ldg(g_w2 + kz) : 1.f;
  float sc[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const float k2 = __ldg(g_w2 + t + T * s) + w2yz;
    sc[s] = k2 > 0.f ? coef / k2 : 0.f;
  }
  const float gy = valid ? __ldg(g_g + ky) : 0.f, gz = valid ? __ldg(g_g + kz) : 0.f;
#pragma unroll 1
  for (int axis = 0; axis < 3; ++axis) {
    float2 v[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const float gd = axis == 0 ? __ldg(g_g + t + T * s) : (axis == 1 ? gy : gz);
      v[s] = mul_i(cscale(d[s], gd * sc[s]));
    }
    RegFft<N>::template run<true>(v, buf, t, tw);
    if (valid) {
      float2* o = out + axis * out_fs;
#pragma unroll
      for (int s = 0; s < 8; ++s) o[(size_t)(t + T * s) * S + gl] = v[s];
    }
  }
}

// ---------------------------------------------------------------- x pass: potential
// One field in place: forward x transform of delta(k), the Green's function
// phi = coef delta / |w|^2 (0 at k = 0, Eq. 3), inverse x transform.  The
// Eq. 5 finite-difference gradient is then applied in real space to phi.
template <int N, int V = 8>
__device__ __forceinline__ void body_xgreen_r(float2* data, float coef, const float2* __restrict__ g_tw,
                                              const float* __restrict__ g_w2, float2* smem, int bx) {
  using C = RegCfg<N, V>;
  constexpr int T = C::T, L = C::L, NH = N / 2 + 1;
  constexpr size_t S = (size_t)NH * N;
  float2* tw = smem;
  float2* xb = tw + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g_tw[i];
  const int line = threadIdx.x % L, t = threadIdx.x / L;
  const int gl = bx * L + line;
  const bool valid = gl < NH * N;
  const int kz = gl / N, ky = gl - kz * N;
  float2 d[V];
#pragma unroll
  for (int s = 0; s < V; ++s) d[s] = valid ? __ldcg(data + (size_t)(t + T * s) * S + gl) : make_float2(0.f, 0.f);
  __syncthreads();
  float2* buf = xb + line * rline<N>();
  RegFft<N, V>::template run<false>(d, buf, t, tw);
  const float w2yz = valid ? __ldg(g_w2 + ky) + __ldg(g_w2 + kz) : 1.f;
#pragma unroll
  for (int s = 0; s < V; ++s) {
    const float k2 = __ldg(g_w2 + t + T * s) + w2yz;
    d[s] = cscale(d[s], k2 > 0.f ? coef / k2 : 0.f);
  }
  RegFft<N, V>::template run<true>(d, buf, t, tw);
  if (valid) {
#pragma unroll
    for (int s = 0; s < V; ++s) data[(size_t)(t + T * s) * S + gl] = d[s];
  }
}

template <int N>
__global__ void __launch_bounds__(RegCfg<N>::THREADS, 1024 / RegCfg<N>::THREADS) k_xgreen_r(float2* data, float coef,
                                                                 const float2* __restrict__ g_tw,
                                                                 const float* __restrict__ g_w2) {
  extern __shared__ float2 smem[];
  body_xgreen_r<N>(data, coef, g_tw, g_w2, smem, blockIdx.x);
}

// ---------------------------------------------------------------- real-space gradient
// F_d(c) = [8 (phi(c + e_d) - phi(c - e_d)) - (phi(c + 2 e_d) - phi(c - 2 e_d))] / 12,
// whose Fourier symbol is i (8 sin w - sin 2w) / 6 = i g(w) of Eq. 5 (zero
// at the Nyquist frequency by itself).  A block owns a TZ x TY patch of a
// y-z plane and marches through XC planes of x, keeping a ring of RING
// halo-padded planes in shared memory; each plane is fetched by per-thread
// asynchronous copies PF planes ahead of its first use (one commit group
// per plane), so that several planes' loads are in flight per block.
constexpr int ST_XC = 32;                  // x planes per block
constexpr int ST_PF = 3;                   // planes fetched ahead
template <int N>
struct StCfg {
  static constexpr int TZ = N < 32 ? N : 32;
  static constexpr int TY = 256 / TZ;
  static constexpr int PZ = TZ + 4, PY = TY + 4, PLANE = PZ * PY;
  static constexpr int XC = N < ST_XC ? N : ST_XC;
  static constexpr int LOADS = (PLANE + 255) / 256;
  static constexpr int RING = 6 + ST_PF;   // 5 planes in use, PF in flight, 1 being refilled
  static constexpr size_t SMEM = (size_t)RING * PLANE * sizeof(float);
};

__device__ __forceinline__ float fd4(float m2, float m1, float p1, float p2) {
  return fmaf(0.6666666666666666f, p1 - m1, -0.08333333333333333f * (p2 - m2));
}

__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gsrc) : "memory");
}

// ring: RING * PLANE floats of shared memory (4-byte aligned).
template <int N, bool F4>
__device__ __forceinline__ void body_stencil(const float* __restrict__ phi, float* __restrict__ F, size_t M,
                                             float* ring, int bz, int by, int bx) {
  using C = StCfg<N>;
  constexpr int TZ = C::TZ, TY = C::TY, PZ = C::PZ, PLANE = C::PLANE, XC = C::XC, RING = C::RING;
  const int z0 = bz * TZ, y0 = by * TY, x0 = bx * XC;
  const int tz = threadIdx.x % TZ, ty = threadIdx.x / TZ;
  // plane q (x = x0 - 2 + q, q = 0 .. XC + 3) goes to slot q % RING; one
  // commit group per call, empty past the last plane, so that the count of
  // groups in flight after plane q is always ST_PF
  auto fetch = [&](int q) {
    if (q < XC + 4) {
      const float* pl = phi + (size_t)((x0 - 2 + q) & (N - 1)) * N * N;
      float* dst = ring + (q % RING) * PLANE;
#pragma unroll
      for (int k = 0; k < C::LOADS; ++k) {
        const int e = threadIdx.x + 256 * k;
        if (e < PLANE) {
          const int r = e / PZ, c = e - r * PZ;
          cp_async4(dst + e, pl + (size_t)((y0 - 2 + r) & (N - 1)) * N + ((z0 - 2 + c) & (N - 1)));
        }
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  for (int q = 0; q < 5 + ST_PF; ++q) fetch(q);
  const int cidx = (ty + 2) * PZ + tz + 2;
  for (int j = 0; j < XC; ++j) {
    // planes j .. j+4 complete (ST_PF later groups may still be in flight),
    // visible to the block, and slot (j + 5 + ST_PF) % RING (plane j - 1,
    // last read in iteration j - 1) free for refilling
    asm volatile("cp.async.wait_group %0;" ::"n"(ST_PF) : "memory");
    __syncthreads();
    fetch(j + 5 + ST_PF);
    const float* c = ring + ((j + 2) % RING) * PLANE;
    const float fx = fd4(ring[(j % RING) * PLANE + cidx], ring[((j + 1) % RING) * PLANE + cidx],
                         ring[((j + 3) % RING) * PLANE + cidx], ring[((j + 4) % RING) * PLANE + cidx]);
    const float fy = fd4(c[cidx - 2 * PZ], c[cidx - PZ], c[cidx + PZ], c[cidx + 2 * PZ]);
    const float fz = fd4(c[cidx - 2], c[cidx - 1], c[cidx + 1], c[cidx + 2]);
    const size_t o = ((size_t)(x0 + j) * N + (y0 + ty)) * N + z0 + tz;
    if (F4) {
      reinterpret_cast<float4*>(F)[o] = make_float4(fx, fy, fz, 0.f);
    } else {
      F[o] = fx;
      F[M + o] = fy;
      F[2 * M + o] = fz;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();                         // the ring may be reused after return
}

// Transpose of the gradient: out = -sum_d D_d g_d for g = [3][N^3] (D is
// antisymmetric: D^T = -D).  A block owns a TZ x TY patch of y-z columns
// (the stencil's StCfg) and each thread marches XC planes of x: the x
// difference comes from a five-plane window of g_x in registers (one new
// load per cell, fetched a plane ahead), the y and z differences from
// neighbour loads in the current plane, shared through L1.
template <int N>
__global__ void __launch_bounds__(256) k_div_neg(const float* __restrict__ g, float* __restrict__ out) {
  using C = StCfg<N>;
  constexpr size_t M = (size_t)N * N * N;
  const int z = blockIdx.x * C::TZ + threadIdx.x % C::TZ, y = blockIdx.y * C::TY + threadIdx.x / C::TZ;
  const int x0 = blockIdx.z * C::XC;
  auto at = [](int xx, int yy, int zz) {
    return ((size_t)(xx & (N - 1)) * N + (yy & (N - 1))) * N + (zz & (N - 1));
  };
  const float* gx = g;
  const float* gy = g + M;
  const float* gz = g + 2 * M;
  float w[5];
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = __ldg(gx + at(x0 - 2 + k, y, z));
  float nxt = __ldg(gx + at(x0 + 2, y, z));
  for (int j = 0; j < C::XC; ++j) {
    const int x = x0 + j;
    w[4] = nxt;
    if (j + 1 < C::XC) nxt = __ldg(gx + at(x + 3, y, z));
    const float dx_ = fd4(w[0], w[1], w[3], w[4]);
    const float dy_ = fd4(__ldg(gy + at(x, y - 2, z)), __ldg(gy + at(x, y - 1, z)), __ldg(gy + at(x, y + 1, z)),
                          __ldg(gy + at(x, y + 2, z)));
    const float dz_ = fd4(__ldg(gz + at(x, y, z - 2)), __ldg(gz + at(x, y, z - 1)), __ldg(gz + at(x, y, z + 1)),
                          __ldg(gz + at(x, y, z + 2)));
    out[at(x, y, z)] = -(dx_ + dy_ + dz_);
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = w[k + 1];
  }
}

template <int N, bool F4>
__global__ void __launch_bounds__(256) k_stencil(const float* __restrict__ phi, float* __restrict__ F, size_t M) {
  __shared__ float ring[StCfg<N>::RING * StCfg<N>::PLANE];
  body_stencil<N, F4>(phi, F, M, ring, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int N>
__global__ void __launch_bounds__(RegCfg<N>::THREADS, 1024 / RegCfg<N>::THREADS) k_xforce_r(const float2* in, float2* out, size_t out_fs,
                                                                 float coef, const float2* __restrict__ g_tw,
                                                                 const float* __restrict__ g_g,
                                                                 const float* __restrict__ g_w2) {
  extern __shared__ float2 smem[];
  body_xforce_r<N>(in, out, out_fs, coef, g_tw, g_g, g_w2, smem, blockIdx.x, blockIdx.y);
}

}  // namespace fpm
