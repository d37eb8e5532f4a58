// fft.cuh -- shared-memory Stockham FFT engine (internal).
//
// A CTA transforms L lines of N complex points held in shared memory.  Each
// stage of radix R reads R points spaced N/R apart, twiddles them by
// w^(k r) with k = j mod Ns (the position inside the current sub-transform
// of span Ns), applies an R-point DFT and writes the results Ns apart at
// (j / Ns) * Ns * R + k: the self-sorting (Stockham) form, out of place
// between two buffers.  Mixed radices 8, 4, 2 and 3 cover every supported
// N = 2^a 3^b.  Twiddles come from a table tw[m] = exp(-2 pi i m / N)
// computed on the host in FP64 and staged in shared memory.
#pragma once
#include "common.cuh"

namespace fpm {

// Padded shared-memory index: one complex of padding per 32 keeps the
// strided Stockham writes of radix-8/4 stages off a single pair of banks.
__device__ __forceinline__ int sp(int i) { return i + (i >> 5); }
__host__ __device__ constexpr int sp_size(int n) { return n + (n >> 5) + 1; }

template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

// multiply by -i for the forward transform, +i for the inverse
template <bool INV>
__device__ __forceinline__ float2 rot_q(float2 a) { return INV ? mul_i(a) : mul_mi(a); }

template <bool INV>
struct Dft<4, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = rot_q<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <bool INV>
struct Dft<8, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    const float c = 0.70710678118654752440f;   // cos(pi/4)
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, INV>::run(e);
    Dft<4, INV>::run(o);
    // w8^k = exp(-+ 2 pi i k / 8); the products are rounded on their own
    // (never fused into the adds below), the same in every instantiation
    float2 o1 = INV ? make_float2(__fmul_rn(c, o[1].x - o[1].y), __fmul_rn(c, o[1].x + o[1].y))
                    : make_float2(__fmul_rn(c, o[1].x + o[1].y), __fmul_rn(c, o[1].y - o[1].x));
    float2 o2 = rot_q<INV>(o[2]);
    float2 o3 = INV ? make_float2(__fmul_rn(-c, o[3].x + o[3].y), __fmul_rn(c, o[3].x - o[3].y))
                    : make_float2(__fmul_rn(c, o[3].y - o[3].x), __fmul_rn(-c, o[3].x + o[3].y));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

template <bool INV>
struct Dft<3, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    const float s3 = 0.86602540378443864676f;   // sin(pi/3)
    float2 s = cadd(v[1], v[2]);
    float2 d = csub(v[1], v[2]);
    float2 m = make_float2(v[0].x - __fmul_rn(0.5f, s.x), v[0].y - __fmul_rn(0.5f, s.y));
    // forward: y1 = m - i s3 d, y2 = m + i s3 d ; inverse swaps the signs
    float2 t = make_float2(__fmul_rn(-s3, d.y), __fmul_rn(s3, d.x));   // i * s3 * d
    v[0] = cadd(v[0], s);
    if (INV) {
      v[1] = cadd(m, t);
      v[2] = csub(m, t);
    } else {
      v[1] = csub(m, t);
      v[2] = cadd(m, t);
    }
  }
};

// One Stockham stage over L lines (line stride LS complex in smem, padded index).
template <int N, int R, int NS, bool INV>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ in, float2* __restrict__ out,
                                          int L, int LS, const float2* __restrict__ tw) {
  constexpr int B = N / R;
  constexpr int TWS = N / (NS * R);
  const int total = L * B;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int line = idx / B;
    const int j = idx - line * B;
    const float2* src = in + line * LS;
    float2* dst = out + line * LS;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[sp(j + r * B)];
    const int k = (NS == 1) ? 0 : (j % NS);
    if (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[k * r * TWS];
        if (INV) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    Dft<R, INV>::run(v);
    const int base = (j / NS) * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[sp(base + r * NS)] = v[r];
  }
}

template <int N, bool INV, int NS, int... Rs>
struct Stages;

template <int N, bool INV, int NS>
struct Stages<N, INV, NS> {
  static __device__ __forceinline__ float2* run(float2* a, float2*, int, int, const float2*) { return a; }
};

template <int N, bool INV, int NS, int R, int... Rs>
struct Stages<N, INV, NS, R, Rs...> {
  static __device__ __forceinline__ float2* run(float2* a, float2* b, int L, int LS, const float2* tw) {
    fft_stage<N, R, NS, INV>(a, b, L, LS, tw);
    __syncthreads();
    return Stages<N, INV, NS * R, Rs...>::run(b, a, L, LS, tw);
  }
};

// Radix plan per size.  run() transforms L lines starting in buffer a using
// b as the ping-pong buffer and returns the buffer holding the result.
template <int N>
struct FftPlan;
#define FPM_FFT_PLAN(NN, ...)                                                             \
  template <>                                                                             \
  struct FftPlan<NN> {                                                                    \
    template <bool INV>                                                                   \
    static __device__ __forceinline__ float2* run(float2* a, float2* b, int L, int LS,   \
                                                  const float2* tw) {                     \
      return Stages<NN, INV, 1, __VA_ARGS__>::run(a, b, L, LS, tw);                       \
    }                                                                                     \
  };
FPM_FFT_PLAN(16, 4, 4)
FPM_FFT_PLAN(32, 8, 4)
FPM_FFT_PLAN(48, 4, 4, 3)
FPM_FFT_PLAN(64, 8, 8)
FPM_FFT_PLAN(96, 8, 4, 3)
FPM_FFT_PLAN(128, 8, 4, 4)
FPM_FFT_PLAN(192, 8, 8, 3)
FPM_FFT_PLAN(256, 8, 8, 4)
FPM_FFT_PLAN(384, 8, 8, 2, 3)
FPM_FFT_PLAN(512, 8, 8, 8)
#undef FPM_FFT_PLAN

// Stage the twiddle table of an N-point transform into shared memory.
template <int N>
__device__ __forceinline__ void load_twiddles(float2* s_tw, const float2* __restrict__ g_tw) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) s_tw[i] = g_tw[i];
}

}  // namespace fpm
