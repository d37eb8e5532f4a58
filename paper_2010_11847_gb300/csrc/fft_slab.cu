// fft_slab.cu -- the force mesh through the potential (internal).
//
// For power-of-two meshes the PM force of Eqs. 3-5 is computed as
//   phi = IFFT[ coef delta(k) / |w|^2 ],   F_d = D_d phi,
// with D_d the four-point difference whose symbol is the i g(w) of Eq. 5:
// one field goes through the three inverse passes instead of three, and the
// gradient is a streaming stencil in real space (fft_reg.cuh).
//
// The z (r2c) and y passes of the forward transform, and the y and z (c2r)
// passes of the inverse, each run as ONE persistent launch whose work items
// are ordered by slabs of x planes: the first-phase items of slab s+1 are
// queued before the second-phase items of slab s, and a second-phase item
// waits (bounded) until all first-phase items of its slab are done.  A
// slab's intermediate spectrum is then still in L2 when the second phase
// reads it, so each pair of passes moves the data through HBM once.  After
// the inverse z pass has read a slab's y-transformed spectrum, the consumed
// 128-byte lines are dropped from L2 without write-back (discard.global.L2):
// they are dead.
//
// Blocks claim items from a global counter in order, so an item only ever
// waits on items claimed before it by running blocks: the launch needs no
// co-residency guarantee and cannot deadlock.  A wait that runs past the
// spin limit records ERR_TIMEOUT and proceeds (results are then invalid and
// fpm_status reports FPM_ETIMEOUT); once the flag is up no block waits again.
#include "internal.h"
#include "fft_reg.cuh"

namespace fpm {

struct SlabArgs {
  const float* rho;     // forward: real mesh
  float2* spec;         // half spectrum [x][kz][y]
  float* phi;           // inverse: real potential
  const float2* tw;
  unsigned* ctr;        // [0] item counter, [1 + s] finished first-phase items of slab s
  int* err;
  int S;                // x planes per slab
  long long spin_limit;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void wait_count(const unsigned* c, unsigned target, long long limit, int* err) {
  long long spins = 0;
  while (ld_acquire_u32(c) < target) {
    if ((*(volatile int*)err & ERR_TIMEOUT) || ++spins > limit) {
      atomicOr(err, ERR_TIMEOUT);
      return;
    }
    __nanosleep(32);
  }
}

// Item order: A(0), then for k = 1 .. ns-1: A(k), B(k-1); then B(ns-1).
__device__ __forceinline__ void slab_item(int item, int ns, int nA, int nB, int* ph, int* s, int* j) {
  if (item < nA) {
    *ph = 0; *s = 0; *j = item;
    return;
  }
  const int r0 = item - nA, per = nA + nB;
  const int k = 1 + r0 / per, r = r0 - (k - 1) * per;
  if (k < ns && r < nA) {
    *ph = 0; *s = k; *j = r;
  } else if (k < ns) {
    *ph = 1; *s = k - 1; *j = r - nA;
  } else {
    *ph = 1; *s = ns - 1; *j = r;
  }
}

template <int N>
struct SlabShape {
  using C = RegCfg<N>;
  static constexpr int NH = N / 2 + 1;
  static constexpr int ZI = N / (2 * C::L);                 // z items per plane
  static __host__ __device__ int y_items(int S) { return (S * NH + C::L - 1) / C::L; }
};

// Drop the 128-byte lines of the half spectrum that z item bx has read.
template <int N>
__device__ __forceinline__ void discard_z_item(const float2* spec, int bx) {
  using C = RegCfg<N>;
  constexpr int NH = N / 2 + 1, LPR = (2 * C::L * 8) / 128;
  static_assert((2 * C::L * 8) % 128 == 0, "z item rows must cover whole lines");
  const size_t r0 = (size_t)bx * 2 * C::L;
  const size_t x = r0 / N, y0 = r0 - x * N;
  for (int e = threadIdx.x; e < NH * LPR; e += blockDim.x) {
    const int kz = e / LPR, l = e - kz * LPR;
    const float2* q = spec + (x * NH + kz) * N + y0 + 16 * l;
    if (((uintptr_t)q & 127) == 0) asm volatile("discard.global.L2 [%0], 128;" ::"l"(q) : "memory");
  }
}

template <int N, bool INV>
__global__ void __launch_bounds__(RegCfg<N>::THREADS, 1024 / RegCfg<N>::THREADS) k_slab(SlabArgs a) {
  extern __shared__ float2 smem[];
  __shared__ int s_item;
  using SH = SlabShape<N>;
  constexpr int NH = SH::NH, ZI = SH::ZI;
  const int S = a.S, ns = N / S;
  const int nA = INV ? SH::y_items(S) : S * ZI;
  const int nB = INV ? S * ZI : SH::y_items(S);
  const int total = ns * (nA + nB);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(a.ctr, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    int ph, s, j;
    slab_item(item, ns, nA, nB, &ph, &s, &j);
    float2* slab = a.spec + (size_t)s * S * NH * N;
    if (ph == 0) {
      if (INV) body_yfft_r<N, true>(slab, S * NH, 0, a.tw, smem, j, 0);
      else body_zfwd_r<N>(a.rho, a.spec, 0, 0, a.tw, smem, s * S * ZI + j, 0);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(a.ctr + 1 + s, 1u);
      }
    } else {
      if (threadIdx.x == 0) wait_count(a.ctr + 1 + s, (unsigned)nA, a.spin_limit, a.err);
      __syncthreads();
      if (INV) {
        const int bx = s * S * ZI + j;
        body_zinv_r<N>(a.spec, a.phi, 0, 0, a.tw, smem, bx, 0);
        __syncthreads();
        discard_z_item<N>(a.spec, bx);
      } else {
        body_yfft_r<N, false>(slab, S * NH, 0, a.tw, smem, j, 0);
      }
    }
  }
}

// ---------------------------------------------------------------- host side
template <typename K>
static int smem_attr(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    FPM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return FPM_OK;
}

// Planes per slab: about 12 MB of half spectrum, a power of two <= n.
int fft_slab_planes(int n) {
  const size_t plane = (size_t)(n / 2 + 1) * n * sizeof(float2);
  int S = 1;
  while (S * 2 <= n && (size_t)(S * 2) * plane <= ((size_t)12 << 20)) S *= 2;
  return S;
}

bool fft_has_potential(int n) { return is_pow2_size(n); }

template <int N, bool INV>
static int slab_launch(const FftTables& t, const float* rho, float2* spec, float* phi, unsigned* ctr, int* err,
                       cudaStream_t s) {
  using C = RegCfg<N>;
  static int grid = 0;                      // per instantiation: device-independent here (one GPU type)
  FPM_TRY(smem_attr(k_slab<N, INV>, C::SMEM));
  if (grid == 0) {
    int dev = 0, nsm = 0, per = 0;
    FPM_CUDA_TRY(cudaGetDevice(&dev));
    FPM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_slab<N, INV>, C::THREADS, C::SMEM));
    if (per < 1) return FPM_ECUDA;
    grid = nsm * per;
  }
  SlabArgs a;
  a.rho = rho;
  a.spec = spec;
  a.phi = phi;
  a.tw = t.tw;
  a.ctr = ctr;
  a.err = err;
  a.S = fft_slab_planes(N);
  a.spin_limit = 1ll << 20;
  FPM_CUDA_TRY(cudaMemsetAsync(ctr, 0, (size_t)(1 + N / a.S) * sizeof(unsigned), s));
  k_slab<N, INV><<<grid, C::THREADS, C::SMEM, s>>>(a);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

template <int N>
static int pot_fwd_impl(const FftTables& t, const float* rho, float2* spec, unsigned* ctr, int* err,
                        cudaStream_t s) {
  if constexpr (is_pow2_size(N) && N >= 128) {
    return slab_launch<N, false>(t, rho, spec, nullptr, ctr, err, s);
  } else {
    FPM_TRY(fft_zfwd(t, rho, spec, 1, 0, 0, s));
    return fft_y(t, spec, 1, 0, false, s);
  }
}

template <int N>
static int pot_inv_impl(const FftTables& t, float2* spec, float* phi, unsigned* ctr, int* err, cudaStream_t s) {
  if constexpr (is_pow2_size(N) && N >= 128) {
    return slab_launch<N, true>(t, nullptr, spec, phi, ctr, err, s);
  } else {
    FPM_TRY(fft_y(t, spec, 1, 0, true, s));
    return fft_zinv(t, spec, phi, 1, 0, 0, s);
  }
}

template <int N>
static int xgreen_impl(const FftTables& t, float2* spec, float coef, cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using C = RegCfg<N>;
    FPM_TRY(smem_attr(k_xgreen_r<N>, C::SMEM));
    const int lines = (N / 2 + 1) * N;
    k_xgreen_r<N><<<(lines + C::L - 1) / C::L, C::THREADS, C::SMEM, s>>>(spec, coef, t.tw, t.w2);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  return FPM_ENOTIMPL;
}

template <int N>
static int stencil_impl(const float* phi, float* F, bool f4, size_t M, cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using C = StCfg<N>;
    const dim3 grid(N / C::TZ, N / C::TY, N / C::XC);
    if (f4) k_stencil<N, true><<<grid, 256, 0, s>>>(phi, F, M);
    else k_stencil<N, false><<<grid, 256, 0, s>>>(phi, F, M);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  return FPM_ENOTIMPL;
}

#define FPM_DISPATCH_POW2(n, CALL)                \
  switch (n) {                                    \
    case 16: { constexpr int N = 16; CALL; }      \
    case 32: { constexpr int N = 32; CALL; }      \
    case 64: { constexpr int N = 64; CALL; }      \
    case 128: { constexpr int N = 128; CALL; }    \
    case 256: { constexpr int N = 256; CALL; }    \
    case 512: { constexpr int N = 512; CALL; }    \
    default: return FPM_ENOTIMPL;                 \
  }

int fft_pot_forward(const FftTables& t, const float* rho, float2* spec, unsigned* ctr, int* err, cudaStream_t s) {
  FPM_DISPATCH_POW2(t.n, return pot_fwd_impl<N>(t, rho, spec, ctr, err, s));
}

int fft_pot_xgreen(const FftTables& t, float2* spec, float coef, cudaStream_t s) {
  FPM_DISPATCH_POW2(t.n, return xgreen_impl<N>(t, spec, coef, s));
}

int fft_pot_inverse(const FftTables& t, float2* spec, float* phi, unsigned* ctr, int* err, cudaStream_t s) {
  FPM_DISPATCH_POW2(t.n, return pot_inv_impl<N>(t, spec, phi, ctr, err, s));
}

int fft_pot_gradient(const FftTables& t, const float* phi, float* F, bool f4, size_t M, cudaStream_t s) {
  FPM_DISPATCH_POW2(t.n, return stencil_impl<N>(phi, F, f4, M, s));
}

}  // namespace fpm
