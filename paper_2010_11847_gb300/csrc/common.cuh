// common.cuh -- shared device/host helpers of libfpm (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/fpm.h"

namespace fpm {

constexpr int TILE = 16;                 // cells per tile edge (cell key)
constexpr int TILE3 = TILE * TILE * TILE;
constexpr int TILE1 = TILE + 1;          // paint accumulator edge (tile + upper halo)
constexpr int SHELL = 2 * TILE1 * TILE1 + 2 * (TILE - 1) * TILE1 + 2 * (TILE - 1) * (TILE - 1);
constexpr float FIX_ONE = 2147483648.0f;       // 2^31: fixed-point unit of a CIC weight
constexpr float FIX_INV = 4.656612873077393e-10f;  // 2^-31
constexpr int MAX_N = 512;

// device error flag bits
constexpr int ERR_NAN = 1;
constexpr int ERR_RANGE = 2;
constexpr int ERR_TIMEOUT = 4;

__host__ __device__ inline bool fft_size_ok(int n) {
  return n == 16 || n == 32 || n == 48 || n == 64 || n == 96 || n == 128 || n == 192 ||
         n == 256 || n == 384 || n == 512;
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// Complex product with its rounding fixed by explicit fused multiply-adds,
// so that every instantiation of a transform (any number of points per
// thread) rounds it the same way: re = fma(ax, bx, -(ay by)), im = fma(ax, by, ay bx).
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -(a.y * b.y)), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
// Real scaling, rounded on its own (never fused into a later add), so that
// its rounding does not depend on how a kernel is instantiated.
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(__fmul_rn(a.x, s), __fmul_rn(a.y, s)); }
// multiply by +i or -i
__device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

// Frequency index of DFT bin j of an n-point transform: j or j - n.
__device__ __forceinline__ int freq_of(int j, int n) { return j < n / 2 ? j : j - n; }

// Unsigned division by a runtime constant d for n < 2^31 with a multiply:
// m = ceil(2^(31+l) / d), l = ceil(log2 d), q = umulhi(n, m) >> (l - 1)
// (Granlund & Montgomery 1994, round-up variant).  d >= 2.
struct FastDiv {
  uint32_t d, m;
  int sh;
};

inline FastDiv make_fastdiv(uint32_t d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.d = d;
  f.m = (uint32_t)(((1ull << (31 + l)) + d - 1) / d);
  f.sh = l - 1;
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) { return __umulhi(n, f.m) >> f.sh; }

// A kick factor read from the FP64 factor table on the device: fac[ik1]
// (+ fac[ik2] when ik2 >= 0), rounded once to float; 1 when fac is null.
struct KScale {
  const double* fac = nullptr;
  int ik1 = -1, ik2 = -1;
};
__device__ __forceinline__ float kscale(const KScale& k) {
  return k.fac ? (float)(k.fac[k.ik1] + (k.ik2 >= 0 ? k.fac[k.ik2] : 0.0)) : 1.f;
}

// Geometry constants handed to kernels.
struct Geom {
  int np;          // particles per side
  int nc;          // mesh cells per side
  int ratio;       // nc / np
  int nt;          // tiles per side (nc / 16)
  float mass;      // (nc/np)^3
  FastDiv div_np, div_np2;
};

}  // namespace fpm

// Host-side error helpers
#define FPM_CUDA_TRY(expr)                           \
  do {                                               \
    cudaError_t e__ = (expr);                        \
    if (e__ != cudaSuccess) return FPM_ECUDA;        \
  } while (0)

#define FPM_TRY(expr)                                \
  do {                                               \
    int r__ = (expr);                                \
    if (r__ != FPM_OK) return r__;                   \
  } while (0)
