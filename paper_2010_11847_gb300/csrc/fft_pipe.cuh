// fft_pipe.cuh -- pipelined persistent FFT passes for power-of-two meshes
// (internal).
//
// A persistent block claims work items in order from a global counter and
// keeps two shared-memory stage buffers: while it transforms item i out of
// one, the cp.async copies of item i+1 fill the other, so the load latency
// of HBM/L2 is hidden behind the butterflies.  Twiddles are staged once per
// block.  Inside a transform the exchange steps synchronise only the threads
// of one line (named barrier or warp), not the block.
//
// Item kinds (all stage 32 KB at N = 512):
//   ZF  z r2c: 2L consecutive real rows of rho        -> staged [2L][N] floats
//   Y   y pass: L consecutive lines of a half spectrum  -> staged line-major
//   ZI  z c2r: the 2L-row strip of every kz plane        -> staged [kz][2L]
//   X   x pass with the Green's function: L lines, all kx -> staged [kx][L]
// The same buffer then holds the line-major exchange area (stride RL).
#pragma once
#include <cuda.h>
#include "bulk.cuh"
#include "fft_reg.cuh"

namespace fpm {

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Slots per thread and lines per block: the x pass keeps RegCfg's (8 slots,
// 64-byte rows at N = 512).  At N = 512 the z and y passes give each thread
// 16 slots (SLAB16: a line is one warp, its exchanges synchronise the warp
// only) and take SLAB_L lines per block.
// (16 slots in the x pass, whose exchanges synchronise the block anyway,
// measured slower: half the resident warps.)
constexpr bool SLAB16 = true;
constexpr int SLAB_L = 4;
template <int N, bool XP = false>
struct PipeCfg {
  static constexpr int V = (!XP && N == 512 && SLAB16) ? 16 : 8;
  static constexpr int T = N / V;
  static constexpr int L = (!XP && N == 512) ? SLAB_L : RegCfg<N>::L;
  static constexpr int THREADS = T * L;
  // resident blocks the launch bounds ask for: 16-slot passes get up to 102
  // registers (5 blocks of 128), or 128 where the inverse pass would spill
  static constexpr int MINB = V == 8 ? 1024 / THREADS : (640 / THREADS > 0 ? 640 / THREADS : 1);
  static constexpr int MINB_INV = V == 8 ? MINB : (512 / THREADS > 0 ? 512 / THREADS : 1);
  static constexpr int NH = N / 2 + 1;
  static constexpr int RL = N + 2;                  // line-major exchange (swizzled), 16-byte aligned
  static constexpr int RLX = N + N / 8 + (N == 128 ? 1 : 2);   // x pass exchange (padded)
  static constexpr int BUF = (L * RLX + 15) & ~15;  // float2 per stage buffer (a multiple of 128 bytes)
  static constexpr size_t SMEM = (size_t)(N + 2 * BUF) * sizeof(float2);
  static constexpr int ZI_PER = (NH * L + THREADS - 1) / THREADS;
  static constexpr int ZI = N / (2 * L);            // z items per x plane
  static_assert(L * N <= BUF && (NH + 1) * 2 * L <= BUF && L * RL <= BUF, "stage buffer too small");
  static_assert((N * sizeof(float2)) % 128 == 0 && (BUF * sizeof(float2)) % 128 == 0, "buffers 128-byte aligned");
  static_assert(L % 2 == 0 && N % L == 0, "x items must be whole 16-byte chunks of one kz row");
};

// ---------------------------------------------------------------- staging
template <int N>
__device__ __forceinline__ void issue_y(const float2* base, int l0, int nlines, float2* buf) {
  using P = PipeCfg<N>;
  constexpr int CPL = N / 2;
  for (int c = threadIdx.x; c < P::L * CPL; c += P::THREADS) {
    const int g = c / CPL, o = 2 * (c - g * CPL);
    if (l0 + g < nlines) cp_async16(buf + g * P::RL + o, base + (size_t)(l0 + g) * N + o);
  }
}

template <int N>
__device__ __forceinline__ void issue_zf(const float* rho, size_t r0, float2* buf) {
  using P = PipeCfg<N>;
  constexpr int CH = 2 * P::L * N / 4;
  const float* src = rho + r0 * N;
  float* dst = reinterpret_cast<float*>(buf);
  for (int c = threadIdx.x; c < CH; c += P::THREADS) cp_async16(dst + 4 * c, src + 4 * c);
}

template <int N>
__device__ __forceinline__ void issue_zi(const float2* spec, size_t r0, float2* buf) {
  using P = PipeCfg<N>;
  constexpr int L = P::L, NH = P::NH;
  const size_t x = r0 / N, y0 = r0 - x * N;
  for (int c = threadIdx.x; c < NH * L; c += P::THREADS) {
    const int kz = c / L, j = c - kz * L;
    cp_async16(buf + kz * 2 * L + 2 * j, spec + (x * NH + kz) * N + y0 + 2 * j);
  }
}

template <int N>
__device__ __forceinline__ void issue_x(const float2* spec, int gl0, float2* buf) {
  using P = PipeCfg<N, true>;
  constexpr int L = P::L, CPK = L / 2;
  constexpr size_t S = (size_t)P::NH * N;
  for (int c = threadIdx.x; c < N * CPK; c += P::THREADS) {
    const int kx = c / CPK, j = c - kx * CPK;
    cp_async16(buf + kx * L + 2 * j, spec + kx * S + gl0 + 2 * j);
  }
}

// ---------------------------------------------------------------- staging by the tensor memory accelerator
// The same stage-buffer layouts filled by one thread's bulk copies (TMA),
// completing on the buffer's mbarrier: the z r2c rows and the y lines are
// contiguous (1-D bulk copies); the z c2r strips ([kz][2L]) and the x lines
// ([kx][L]) are boxes of 2-D tensor maps of the half spectrum.  Returns the
// bytes the barrier must expect.
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* tm, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(tm), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

template <int N>
__device__ __forceinline__ uint32_t tma_issue_zf(const float* rho, size_t r0, float2* buf, unsigned long long* bar,
                                                 unsigned long long pol) {
  using P = PipeCfg<N>;
  constexpr uint32_t bytes = 2 * P::L * N * sizeof(float);
  mbar_expect_tx(bar, bytes);
  bulk_g2s(buf, rho + r0 * N, bytes, bar, pol);
  return bytes;
}

template <int N>
__device__ __forceinline__ uint32_t tma_issue_y(const float2* base, int l0, int nlines, float2* buf,
                                                unsigned long long* bar, unsigned long long pol) {
  using P = PipeCfg<N>;
  const int nl = nlines - l0 < P::L ? nlines - l0 : P::L;
  const uint32_t bytes = (uint32_t)nl * N * sizeof(float2);
  mbar_expect_tx(bar, bytes);
  for (int g = 0; g < nl; ++g) bulk_g2s(buf + g * P::RL, base + (size_t)(l0 + g) * N, N * sizeof(float2), bar, pol);
  return bytes;
}

// z c2r strip of plane x, rows y0 .. y0 + 2L - 1, every kz: boxes of
// ZiBox<N>::ROWS kz rows (a box of at most 256 rows, each box's destination
// 128-byte aligned; rows past kz = N/2 land in the buffer's spare room and
// are not used)
template <int N>
struct ZiBox {
  static constexpr int NH = N / 2 + 1;
  static constexpr int ROWS = NH <= 256 ? NH : 86;
  static constexpr int BOXES = (NH + ROWS - 1) / ROWS;
};
template <int N>
__device__ __forceinline__ void tma_issue_zi(const CUtensorMap* tm, size_t r0, float2* buf, unsigned long long* bar) {
  using P = PipeCfg<N>;
  using Z = ZiBox<N>;
  static_assert((Z::ROWS * 2 * P::L * sizeof(float2)) % 128 == 0 || Z::BOXES == 1, "box destinations 128-byte aligned");
  static_assert(Z::BOXES * Z::ROWS * 2 * P::L <= P::BUF, "boxes fit the stage buffer");
  const int x = (int)(r0 / N), y0 = (int)(r0 - (size_t)x * N);
  mbar_expect_tx(bar, Z::BOXES * Z::ROWS * 4 * P::L * sizeof(float));
#pragma unroll
  for (int b = 0; b < Z::BOXES; ++b) tma_2d(buf + b * Z::ROWS * 2 * P::L, tm, 2 * y0, x * P::NH + b * Z::ROWS, bar);
}

// x pass: lines gl0 .. gl0 + L - 1 of every kx, two boxes of N/2 kx rows
template <int N>
__device__ __forceinline__ void tma_issue_x(const CUtensorMap* tm, int gl0, float2* buf, unsigned long long* bar) {
  using P = PipeCfg<N, true>;
  mbar_expect_tx(bar, N * 2 * P::L * sizeof(float));
  tma_2d(buf, tm, 2 * gl0, 0, bar);
  tma_2d(buf + (N / 2) * P::L, tm, 2 * gl0, N / 2, bar);
}

// ---------------------------------------------------------------- transforms from the stage buffer
template <int N, bool INV>
__device__ __forceinline__ void comp_y(float2* base, int l0, int nlines, float2* buf, const float2* tw) {
  using P = PipeCfg<N>;
  constexpr int T = P::T;
  const int g = threadIdx.x / T, t = threadIdx.x - g * T;
  float2* lb = buf + g * P::RL;
  float2 v[P::V];
#pragma unroll
  for (int s = 0; s < P::V; ++s) v[s] = lb[t + T * s];
  xsync<T>(1 + g);
  RegFft<N, P::V>::template run<INV, 1>(v, lb, t, tw, 1 + g);
  if (l0 + g < nlines) {
    float2* o = base + (size_t)(l0 + g) * N;
#pragma unroll
    for (int s = 0; s < P::V; ++s) o[t + T * s] = v[s];
  }
}

template <int N>
__device__ __forceinline__ void comp_zf(float2* spec, size_t r0, float2* buf, const float2* tw) {
  using P = PipeCfg<N>;
  constexpr int T = P::T, L = P::L, NH = P::NH, RL = P::RL;
  const int g = threadIdx.x / T, t = threadIdx.x - g * T;
  const float* rows = reinterpret_cast<const float*>(buf);
  float2 v[P::V];
#pragma unroll
  for (int s = 0; s < P::V; ++s) v[s] = make_float2(rows[(2 * g) * N + t + T * s], rows[(2 * g + 1) * N + t + T * s]);
  __syncthreads();                       // the exchange area overlaps other lines' rows
  float2* lb = buf + g * RL;
  RegFft<N, P::V>::template run<false, 1>(v, lb, t, tw, 1 + g);
  const int st = sw16(t);                        // t < T: sw16(t + T s) = sw16(t) ^ sw16(T s)
#pragma unroll
  for (int s = 0; s < P::V; ++s) lb[st ^ sw16(T * s)] = v[s];
  __syncthreads();
  const size_t x = r0 / N, y0 = r0 - x * N;
  for (int idx = threadIdx.x; idx < NH * L; idx += P::THREADS) {
    const int kz = idx / L, gg = idx - kz * L;
    const float2* b = buf + gg * RL;
    const float2 zk = b[sw16(kz)];
    const float2 zn = conjf2(b[sw16((N - kz) & (N - 1))]);
    const float2 A = cscale(cadd(zk, zn), 0.5f);
    const float2 B = cscale(mul_mi(csub(zk, zn)), 0.5f);
    *reinterpret_cast<float4*>(spec + (x * NH + kz) * N + y0 + 2 * gg) = make_float4(A.x, A.y, B.x, B.y);
  }
}

template <int N>
__device__ __forceinline__ void comp_zi(float* phi, size_t r0, float2* buf, const float2* tw) {
  using P = PipeCfg<N>;
  constexpr int T = P::T, L = P::L, NH = P::NH, RL = P::RL;
  float4 q[P::ZI_PER];
#pragma unroll
  for (int m = 0; m < P::ZI_PER; ++m) {
    const int idx = threadIdx.x + P::THREADS * m;
    if (idx < NH * L) {
      const int kz = idx / L, gg = idx - kz * L;
      q[m] = *reinterpret_cast<const float4*>(buf + kz * 2 * L + 2 * gg);
    }
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < P::ZI_PER; ++m) {
    const int idx = threadIdx.x + P::THREADS * m;
    if (idx < NH * L) {
      const int kz = idx / L, gg = idx - kz * L;
      float2* b = buf + gg * RL;
      const float4 u = q[m];
      if (kz == 0 || kz == N / 2) {
        b[sw16(kz)] = make_float2(u.x, u.z);
      } else {
        b[sw16(kz)] = make_float2(u.x - u.w, u.y + u.z);
        b[sw16(N - kz)] = make_float2(u.x + u.w, u.z - u.y);
      }
    }
  }
  __syncthreads();
  const int g = threadIdx.x / T, t = threadIdx.x - g * T;
  float2* lb = buf + g * RL;
  float2 v[P::V];
  const int st = sw16(t);
#pragma unroll
  for (int s = 0; s < P::V; ++s) v[s] = lb[st ^ sw16(T * s)];
  xsync<T>(1 + g);
  RegFft<N, P::V>::template run<true, 1>(v, lb, t, tw, 1 + g);
  float* dst = phi + (r0 + 2 * g) * N;
#pragma unroll
  for (int s = 0; s < P::V; ++s) {
    dst[t + T * s] = v[s].x;
    dst[N + t + T * s] = v[s].y;
  }
}

// x pass: forward x transform, phi = coef delta / |w|^2 (0 at k = 0), inverse.
// Lines are fastest across threads (64-byte output segments), so a line's
// threads span every warp and the exchanges synchronise the block.
template <int N>
__device__ __forceinline__ void comp_x(float2* spec, int gl0, float coef, float2* buf, const float2* tw,
                                       const float* __restrict__ g_w2) {
  using P = PipeCfg<N, true>;
  constexpr int T = P::T, L = P::L;
  constexpr size_t S = (size_t)P::NH * N;
  const int line = threadIdx.x % L, t = threadIdx.x / L;
  const int gl = gl0 + line;
  const int kz = gl / N, ky = gl - kz * N;
  constexpr int V = P::V;
  float2 d[V];
#pragma unroll
  for (int s = 0; s < V; ++s) d[s] = buf[(t + T * s) * L + line];
  __syncthreads();
  float2* lb = buf + line * P::RLX;
  RegFft<N, V>::template run<false>(d, lb, t, tw);
  const float w2yz = __ldg(g_w2 + ky) + __ldg(g_w2 + kz);
#pragma unroll
  for (int s = 0; s < V; ++s) {
    const float k2 = __ldg(g_w2 + t + T * s) + w2yz;
    d[s] = cscale(d[s], k2 > 0.f ? coef / k2 : 0.f);
  }
  RegFft<N, V>::template run<true>(d, lb, t, tw);
#pragma unroll
  for (int s = 0; s < V; ++s) spec[(size_t)(t + T * s) * S + gl] = d[s];
}

}  // namespace fpm
