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
// reads it, so each pair of passes moves the data through HBM once.
//
// Blocks claim items from a global counter in order, so an item only ever
// waits on items claimed before it by running blocks.  A block claims and
// prefetches its next item while it transforms the current one (the
// pipelined engine of fft_pipe.cuh); a second-phase item whose slab is not
// finished yet is fetched only after the current item is done, so no block
// waits while it holds an unfinished item: the launch needs no co-residency
// guarantee and cannot deadlock.  The x pass runs on the same engine
// without dependencies.  A wait that runs past the
// spin limit records ERR_TIMEOUT and proceeds (results are then invalid and
// fpm_status reports FPM_ETIMEOUT); once the flag is up no block waits again.
#include "internal.h"
#include "fft_pipe.cuh"

#include <cudaTypedefs.h>

#include <mutex>
#include <vector>

namespace fpm {

struct PipeArgs {
  CUtensorMap tm_zi;    // the half spectrum as [x * NH + kz][2N floats] rows (z c2r strips)
  CUtensorMap tm_x;     // the half spectrum as [kx][2 NH N floats] rows (x lines)
  const float* rho;     // forward: real mesh
  float2* spec;         // half spectrum [x][kz][y]
  float* phi;           // inverse: real potential
  const float2* tw;
  const float* w2;
  float coef;
  unsigned* ctr;        // [0] item counter, [1 + s] finished first-phase items of slab s
  int* err;
  int S;                // x planes per slab
  int D;                // lag of second-phase items, in slabs (1 <= D <= N / S)
  long long wait_ns;     // limit of one dependency wait
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded by time (%globaltimer): a profiler that slows the producers down
// does not turn a normal wait into a reported timeout.
__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void wait_count(const unsigned* c, unsigned target, long long limit_ns, int* err) {
  const unsigned long long t0 = gtimer_ns();
  while (ld_acquire_u32(c) < target) {
    if ((*(volatile int*)err & ERR_TIMEOUT) || (long long)(gtimer_ns() - t0) > limit_ns) {
      atomicOr(err, ERR_TIMEOUT);
      return;
    }
    __nanosleep(64);
  }
}

// Item order with a lag of D slabs: A(0) .. A(D-1), then for k = D .. ns-1:
// A(k), B(k-D); then B(ns-D) .. B(ns-1).  D is chosen so that a slab's
// first-phase items are normally finished when its second-phase items are
// claimed (every block holds up to two items in flight).
__device__ __forceinline__ void slab_item(int item, int ns, int D, int nA, int nB, int* ph, int* s, int* j) {
  const int head = D * nA, per = nA + nB;
  if (item < head) {
    *ph = 0; *s = item / nA; *j = item - (item / nA) * nA;
    return;
  }
  const int r0 = item - head;
  const int k = D + r0 / per;
  if (k < ns) {
    const int r = r0 - (k - D) * per;
    if (r < nA) {
      *ph = 0; *s = k; *j = r;
    } else {
      *ph = 1; *s = k - D; *j = r - nA;
    }
    return;
  }
  const int r1 = r0 - (ns - D) * per;
  *ph = 1; *s = ns - D + r1 / nB; *j = r1 - (r1 / nB) * nB;
}

enum PipeKind : int { PK_FWD = 0, PK_INV = 1, PK_X = 2 };

// KIND PK_FWD: A = z r2c (ZF), B = y forward; PK_INV: A = y inverse, B = z
// c2r to phi (ZI); PK_X: x items only, no dependencies.
template <int N, int KIND>
struct PipeSched {
  using P = PipeCfg<N, KIND == PK_X>;
  int S, ns, D, nA, nB, total;
  __device__ PipeSched(int S_, int D_) : S(S_), ns(N / S_), D(D_) {
    const int ny = (S * P::NH + P::L - 1) / P::L, nz = S * P::ZI;
    if (KIND == PK_X) {
      nA = P::NH * N / P::L;
      nB = 0;
      ns = 1;
      D = 1;
    } else {
      nA = KIND == PK_FWD ? nz : ny;
      nB = KIND == PK_FWD ? ny : nz;
    }
    total = ns * (nA + nB);
  }
  __device__ void decode(int item, int* ph, int* s, int* j) const {
    if (KIND == PK_X) {
      *ph = 0; *s = 0; *j = item;
    } else {
      slab_item(item, ns, D, nA, nB, ph, s, j);
    }
  }
};

template <int N, int KIND>
__device__ __forceinline__ void pipe_issue(const PipeArgs& a, const PipeSched<N, KIND>& sc, int item, float2* buf) {
  using P = PipeCfg<N, KIND == PK_X>;
  int ph, s, j;
  sc.decode(item, &ph, &s, &j);
  float2* slab = a.spec + (size_t)s * sc.S * P::NH * N;
  const bool zitem = (KIND == PK_FWD && ph == 0) || (KIND == PK_INV && ph == 1);
  if (KIND == PK_X) issue_x<N>(a.spec, j * P::L, buf);
  else if (zitem && KIND == PK_FWD) issue_zf<N>(a.rho, (size_t)(s * sc.S * P::ZI + j) * 2 * P::L, buf);
  else if (zitem) issue_zi<N>(a.spec, (size_t)(s * sc.S * P::ZI + j) * 2 * P::L, buf);
  else issue_y<N>(slab, j * P::L, sc.S * P::NH, buf);
}

template <int N, int KIND>
__device__ __forceinline__ void pipe_issue_tma(const PipeArgs& a, const PipeSched<N, KIND>& sc, int item, float2* buf,
                                               unsigned long long* bar, unsigned long long pol) {
  using P = PipeCfg<N, KIND == PK_X>;
  int ph, s, j;
  sc.decode(item, &ph, &s, &j);
  float2* slab = a.spec + (size_t)s * sc.S * P::NH * N;
  const bool zitem = (KIND == PK_FWD && ph == 0) || (KIND == PK_INV && ph == 1);
  if (KIND == PK_X) tma_issue_x<N>(&a.tm_x, j * P::L, buf, bar);
  else if (zitem && KIND == PK_FWD) tma_issue_zf<N>(a.rho, (size_t)(s * sc.S * P::ZI + j) * 2 * P::L, buf, bar, pol);
  else if (zitem) tma_issue_zi<N>(&a.tm_zi, (size_t)(s * sc.S * P::ZI + j) * 2 * P::L, buf, bar);
  else tma_issue_y<N>(slab, j * P::L, sc.S * P::NH, buf, bar, pol);
}

template <int N, int KIND>
__device__ __forceinline__ void pipe_compute(const PipeArgs& a, const PipeSched<N, KIND>& sc, int item,
                                             float2* buf, const float2* tw) {
  using P = PipeCfg<N, KIND == PK_X>;
  int ph, s, j;
  sc.decode(item, &ph, &s, &j);
  float2* slab = a.spec + (size_t)s * sc.S * P::NH * N;
  const int bx = s * sc.S * P::ZI + j;
  if (KIND == PK_X) {
    comp_x<N>(a.spec, j * P::L, a.coef, buf, tw, a.w2);
  } else if (KIND == PK_FWD) {
    if (ph == 0) comp_zf<N>(a.spec, (size_t)bx * 2 * P::L, buf, tw);
    else comp_y<N, false>(slab, j * P::L, sc.S * P::NH, buf, tw);
  } else {
    if (ph == 0) comp_y<N, true>(slab, j * P::L, sc.S * P::NH, buf, tw);
    else comp_zi<N>(a.phi, (size_t)bx * 2 * P::L, buf, tw);
  }
  if (KIND != PK_X && ph == 0) {            // publish a finished first-phase item
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.ctr + 1 + s, 1u);
    }
  }
}

// TMA: the stage buffers are filled by one thread's bulk / tensor copies
// completing on a per-buffer mbarrier (item i: buffer i & 1, its (i >> 1)-th
// fill, phase parity (i >> 1) & 1); else by every thread's cp.async.  Every
// thread fences its generic accesses of a buffer before the block barrier
// that hands it back to the copy engine.
template <int N, int KIND, bool TMA>
__global__ void __launch_bounds__(PipeCfg<N, KIND == PK_X>::THREADS,
                                  KIND == PK_INV ? PipeCfg<N>::MINB_INV : PipeCfg<N, KIND == PK_X>::MINB)
    k_pipe(const __grid_constant__ PipeArgs a) {
  using P = PipeCfg<N, KIND == PK_X>;
  extern __shared__ __align__(128) float2 smem_raw[];
  __shared__ int s_item, s_ready;
  __shared__ __align__(8) unsigned long long bars[2];
  // tensor copies need 128-byte aligned destinations: align the base (the
  // launch adds 128 bytes), the buffers then start at multiples of 128 bytes
  float2* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u) / sizeof(float2);
  float2* tw = smem;
  float2* bufs = smem + N;
  for (int i = threadIdx.x; i < N; i += P::THREADS) tw[i] = a.tw[i];
  const PipeSched<N, KIND> sc(a.S, a.D);
  // second-phase items wait until every first-phase item of their slab is done
  auto slab_of = [&](int item) {
    int ph, s, j;
    sc.decode(item, &ph, &s, &j);
    return ph == 1 ? s : -1;
  };
  unsigned long long pol = 0;
  if (TMA && threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init_fence();
    pol = l2_evict_first();
  }
  auto issue = [&](int item, int i) {      // stage `item` as the block's i-th item
    float2* dst = bufs + (i & 1) * P::BUF;
    if (TMA) {
      if (threadIdx.x == 0) pipe_issue_tma<N, KIND>(a, sc, item, dst, &bars[i & 1], pol);
    } else {
      pipe_issue<N, KIND>(a, sc, item, dst);
    }
  };
  bool live = true;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int it = (int)atomicAdd(a.ctr, 1u);
    s_item = it;
    if (it < sc.total && slab_of(it) >= 0) wait_count(a.ctr + 1 + slab_of(it), sc.nA, a.wait_ns, a.err);
  }
  __syncthreads();
  int cur = s_item;
  if (cur < sc.total) issue(cur, 0);
  if (!TMA) cp_async_commit();
  for (int i = 0; cur < sc.total; ++i) {
    float2* b = bufs + (i & 1) * P::BUF;
    __syncthreads();                       // bn (item i-1's buffer) and s_item are free
    if (threadIdx.x == 0) {
      const int it = (int)atomicAdd(a.ctr, 1u);
      s_item = it;
      const int sl = it < sc.total ? slab_of(it) : -1;
      s_ready = sl < 0 || ld_acquire_u32(a.ctr + 1 + sl) >= (unsigned)sc.nA;
    }
    __syncthreads();
    const int nxt = s_item;
    const bool ready = s_ready != 0;
    if (nxt < sc.total && ready) issue(nxt, i + 1);
    if (TMA) {   // after a wait that ran out, later ones keep waiting, but briefly
      live = mbar_wait(&bars[i & 1], (uint32_t)((i >> 1) & 1), live ? a.wait_ns : 1000000ll, a.err) && live;
    } else {
      cp_async_commit();
      cp_async_wait1();
      __syncthreads();
    }
    pipe_compute<N, KIND>(a, sc, cur, b, tw);
    if (TMA) fence_proxy_async();          // this buffer goes back to the copy engine
    if (nxt < sc.total && !ready) {        // wait only while holding no unfinished item
      if (threadIdx.x == 0) wait_count(a.ctr + 1 + slab_of(nxt), sc.nA, a.wait_ns, a.err);
      __syncthreads();
      issue(nxt, i + 1);
      if (!TMA) cp_async_commit();
    }
    cur = nxt;
  }
  if (!TMA) cp_async_wait0();
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

// Tensor maps of a half spectrum at `spec` (N^3 mesh) for the z c2r strips
// and the x lines, encoded once per buffer through the driver's
// cuTensorMapEncodeTiled (reached through the runtime, no driver library
// link) and cached.
namespace {
struct MapEntry {
  const void* spec;
  int n;
  CUtensorMap zi, x;
};
std::mutex g_map_mu;
std::vector<MapEntry> g_maps;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
bool g_encode_tried = false;

bool encode_2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint64_t row_bytes,
               uint32_t box_inner, uint32_t box_rows) {
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N>
bool spectrum_maps(const float2* spec, CUtensorMap* zi, CUtensorMap* x) {
  std::lock_guard<std::mutex> lock(g_map_mu);
  if (!g_encode_tried) {
    g_encode_tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    cudaGetLastError();
  }
  if (!g_encode) return false;
  for (const MapEntry& e : g_maps)
    if (e.spec == spec && e.n == N) {
      *zi = e.zi;
      *x = e.x;
      return true;
    }
  using PS = PipeCfg<N>;
  using PX = PipeCfg<N, true>;
  constexpr int NH = N / 2 + 1;
  MapEntry e;
  e.spec = spec;
  e.n = N;
  // z c2r: rows x * NH + kz of N complex (2N floats); box 2L complex x ZiBox rows
  // x pass: rows kx of NH N complex; box L complex x N/2 rows
  if (!encode_2d(&e.zi, spec, 2ull * N, (uint64_t)N * NH, 2ull * N * sizeof(float), 4 * PS::L, ZiBox<N>::ROWS) ||
      !encode_2d(&e.x, spec, 2ull * NH * N, (uint64_t)N, 2ull * NH * N * sizeof(float), 2 * PX::L, N / 2))
    return false;
  if (g_maps.size() > 64) g_maps.clear();
  g_maps.push_back(e);
  *zi = e.zi;
  *x = e.x;
  return true;
}
}  // namespace

// Stage the pencils with the tensor memory accelerator where the buffers
// allow it (16-byte aligned mesh and spectrum, tensor maps available), else
// with cp.async.
constexpr bool PIPE_TMA = true;

template <int N, int KIND>
static int pipe_launch(const FftTables& t, const float* rho, float2* spec, float* phi, float coef, unsigned* ctr,
                       int* err, cudaStream_t s) {
  using P = PipeCfg<N, KIND == PK_X>;
  PipeArgs a;
  bool tma = PIPE_TMA && (uintptr_t)spec % 16 == 0 && (KIND != PK_FWD || (uintptr_t)rho % 16 == 0) &&
             spectrum_maps<N>(spec, &a.tm_zi, &a.tm_x);
  auto kern = tma ? k_pipe<N, KIND, true> : k_pipe<N, KIND, false>;
  static int grid[2] = {0, 0};              // blocks that fit the device at once (persistent)
  constexpr size_t smem = P::SMEM + 128;    // + the alignment pad of the stage buffers
  FPM_TRY(smem_attr(kern, smem));
  if (grid[tma] == 0) {
    int dev = 0, nsm = 0, per = 0;
    FPM_CUDA_TRY(cudaGetDevice(&dev));
    FPM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, P::THREADS, smem));
    if (per < 1) return FPM_ECUDA;
    grid[tma] = nsm * per;
  }
  a.rho = rho;
  a.spec = spec;
  a.phi = phi;
  a.tw = t.tw;
  a.w2 = t.w2;
  a.coef = coef;
  a.ctr = ctr;
  a.err = err;
  a.S = KIND == PK_X ? N : fft_slab_planes(N);
  {
    // lag: about three grids' worth of items between a slab's two phases
    const int ns = N / a.S, ny = (a.S * P::NH + P::L - 1) / P::L, nz = a.S * P::ZI;
    int D = 1;
    while (D < ns && D * (ny + nz) < 3 * grid[tma]) ++D;
    a.D = D;
  }
  a.wait_ns = 4000000000ll;
  FPM_CUDA_TRY(cudaMemsetAsync(ctr, 0, (size_t)(1 + N / a.S) * sizeof(unsigned), s));
  kern<<<grid[tma], P::THREADS, smem, s>>>(a);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

template <int N>
static int pot_fwd_impl(const FftTables& t, const float* rho, float2* spec, unsigned* ctr, int* err,
                        cudaStream_t s) {
  if constexpr (is_pow2_size(N) && N >= 128) {
    return pipe_launch<N, PK_FWD>(t, rho, spec, nullptr, 0.f, ctr, err, s);
  } else {
    FPM_TRY(fft_zfwd(t, rho, spec, 1, 0, 0, s));
    return fft_y(t, spec, 1, 0, false, s);
  }
}

template <int N>
static int pot_inv_impl(const FftTables& t, float2* spec, float* phi, unsigned* ctr, int* err, cudaStream_t s) {
  if constexpr (is_pow2_size(N) && N >= 128) {
    return pipe_launch<N, PK_INV>(t, nullptr, spec, phi, 0.f, ctr, err, s);
  } else {
    FPM_TRY(fft_y(t, spec, 1, 0, true, s));
    return fft_zinv(t, spec, phi, 1, 0, 0, s);
  }
}

template <int N>
static int xgreen_impl(const FftTables& t, float2* spec, float coef, unsigned* ctr, int* err, cudaStream_t s) {
  if constexpr (is_pow2_size(N) && N >= 128) {
    return pipe_launch<N, PK_X>(t, nullptr, spec, nullptr, coef, ctr, err, s);
  } else if constexpr (is_pow2_size(N)) {
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

int fft_pot_xgreen(const FftTables& t, float2* spec, float coef, unsigned* ctr, int* err, cudaStream_t s) {
  FPM_DISPATCH_POW2(t.n, return xgreen_impl<N>(t, spec, coef, ctr, err, s));
}

int fft_pot_inverse(const FftTables& t, float2* spec, float* phi, unsigned* ctr, int* err, cudaStream_t s) {
  FPM_DISPATCH_POW2(t.n, return pot_inv_impl<N>(t, spec, phi, ctr, err, s));
}

template <int N>
static int div_impl(const float* g, float* out, cudaStream_t s) {
  if constexpr (is_pow2_size(N)) {
    using C = StCfg<N>;
    k_div_neg<N><<<dim3(N / C::TZ, N / C::TY, N / C::XC), 256, 0, s>>>(g, out);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  return FPM_ENOTIMPL;
}

int fft_pot_divergence_neg(const FftTables& t, const float* g, float* out, cudaStream_t s) {
  FPM_DISPATCH_POW2(t.n, return div_impl<N>(g, out, s));
}

int fft_pot_gradient(const FftTables& t, const float* phi, float* F, bool f4, size_t M, cudaStream_t s) {
  FPM_DISPATCH_POW2(t.n, return stencil_impl<N>(phi, F, f4, M, s));
}

}  // namespace fpm
