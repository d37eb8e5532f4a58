// batch.cu -- many independent simulations advanced by one persistent
// cooperative launch per KDK step.
//
// Each simulation keeps its own plan (sizes, cosmology, FP64 kick/drift
// factors, scratch).  A launch runs the phases of one step -- readout +
// kick + drift + keys, tile scan, scatter, paint, halo, z/y/x/y/z FFT passes
// to the potential and its finite-difference gradient (power-of-two meshes;
// 96 keeps the three-field spectral gradient) -- over a work list that spans every
// simulation: work item j of a phase is mapped to (simulation, local block)
// through per-phase prefix offsets, and the body of the matching kernel runs
// with that local block index, dispatching on the simulation's mesh size.
// Data written earlier in the same launch is read L2-coherently (ld.cg),
// never through the read-only path.
// Phases are separated by a grid barrier whose wait is bounded: past the
// spin limit the block records FPM_ETIMEOUT and stops, so a broken barrier
// can end the run early but never hang the GPU.  A whole run (initial force,
// every step, closing kick) is captured once into a CUDA graph and replayed.
#include "internal.h"
#include "fft_passes.cuh"
#include "fft_reg.cuh"
#include "paint_dev.cuh"
#include "readout_dev.cuh"

#include <algorithm>
#include <vector>

namespace fpm {

constexpr int BT = 256;        // threads of the persistent kernel
constexpr size_t BATCH_SMEM = 40 * 1024;

enum Phase : int {
  PH_KEYS = 0, PH_KDK, PH_SCAN, PH_SCATTER, PH_PAINT, PH_HALO, PH_ZF, PH_YF, PH_X, PH_YI, PH_ZI, PH_GRAD, PH_KDK_LAST,
  NPH
};

struct SimDesc {
  Geom g;
  size_t N, M;
  int nc, ntiles, f4;
  float *dx, *p, *F, *rho;
  float2* spec;
  size_t specmax;
  uint32_t *keys, *items, *tile_count, *tile_start, *tile_cursor;
  uint16_t* cells;               // in-tile cell of each item (written by the scatter phase)
  unsigned long long* halo;
  int* err;
  const double* fac;
  const float2* tw;
  const float *gk, *w2;
  float force_coef;
  int rshape;                    // readout form: 0 chunked (body_readout), 1/2 bricks of 32/64 in z
  int te;                        // paint tile edge (16: the plan's tiles; 8: batch-owned tile tables)
  int fv;                        // FFT slots per thread of the power-of-two passes (8 or 16)
  int items_of[NPH];
};

using Brick32 = BrickShape<32, 4, 4>;
using Brick64 = BrickShape<64, 4, 4>;

struct BatchArgs {
  const SimDesc* sims;
  const int* off;        // [NPH][nsims + 1] prefix offsets of work items
  int nsims;
  unsigned* bar;         // [0] arrival count, [1] generation
  long long spin_limit;
  int* status;           // FPM_ETIMEOUT bit set by a barrier that gave up
  int kind;              // 0: initial force, 1: KDK step k, 2: closing kick
  int k;                 // step index for kind 1 (closing kick of step n-1 for kind 2)
  int ro_iters;          // particle chunks of 256 per readout work item
  unsigned long long* ptime;   // [NPH] device ns per phase (block 0's view, barrier to barrier), accumulated
};

__device__ __forceinline__ unsigned long long batch_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded grid barrier (all blocks are co-resident under a cooperative
// launch).  Returns false when this block gave up or another block already
// reported a timeout; the caller then stops.
__device__ bool grid_barrier(const BatchArgs& a) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = a.bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(a.bar, 1u);
    if (arrived == gridDim.x - 1) {
      a.bar[0] = 0u;
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g0) {
        if (++spins > a.spin_limit || *(volatile int*)a.status) {
          atomicOr(a.status, ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ int find_sim(const int* off, int nsims, int item) {
  int lo = 0, hi = nsims - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Power-of-two meshes: the force through the potential, as in the
// single-simulation path (same bodies, hence the same bits): phi in the
// memory of the second half spectrum, then the Eq. 5 difference.
template <int N, int V>
__device__ void fft_phase_pow2(int ph, const SimDesc& d, int local, float2* sm) {
  const int nlines = (N / 2 + 1) * N;
  float* phi = reinterpret_cast<float*>(d.spec + d.specmax);
  switch (ph) {
    case PH_ZF: body_zfwd_r<N, V>(d.rho, d.spec, 0, 0, d.tw, sm, local, 0); break;
    case PH_YF: body_yfft_r<N, false, V>(d.spec, nlines, 0, d.tw, sm, local, 0); break;
    case PH_X: body_xgreen_r<N, V>(d.spec, d.force_coef, d.tw, d.w2, sm, local); break;
    case PH_YI: body_yfft_r<N, true, V>(d.spec, nlines, 0, d.tw, sm, local, 0); break;
    case PH_ZI: body_zinv_r<N, V>(d.spec, phi, 0, 0, d.tw, sm, local, 0); break;
    case PH_GRAD: {
      using SC = StCfg<N>;
      constexpr int nbz = N / SC::TZ, nby = N / SC::TY;
      const int bz = local % nbz, by = (local / nbz) % nby, bx = local / (nbz * nby);
      if (d.f4) body_stencil<N, true>(phi, d.F, d.M, reinterpret_cast<float*>(sm), bz, by, bx);
      else body_stencil<N, false>(phi, d.F, d.M, reinterpret_cast<float*>(sm), bz, by, bx);
      break;
    }
    default: break;
  }
}

template <int N>
__device__ void fft_phase_smem(int ph, const SimDesc& d, int local, float2* sm) {
  const int nlines = (N / 2 + 1) * N;
  const int ylines = (nlines + YL - 1) / YL;
  const int zitems = N * (N / (2 * ZG));
  switch (ph) {
    case PH_ZF: body_zfwd<N>(d.rho, d.spec, 0, 0, d.tw, sm, local, 0); break;
    case PH_YF: body_yfft<N, false>(d.spec, nlines, 0, d.tw, sm, local, 0); break;
    case PH_X: body_xforce<N>(d.spec, d.spec, d.specmax, d.force_coef, d.tw, d.gk, d.w2, sm, local, 0); break;
    case PH_YI: body_yfft<N, true>(d.spec, nlines, d.specmax, d.tw, sm, local % ylines, local / ylines); break;
    case PH_ZI: body_zinv<N>(d.spec, d.F, d.specmax, d.M, d.tw, sm, local % zitems, local / zitems); break;
    default: break;
  }
}

// 3 blocks per SM: the union of all phase bodies fits 80 registers.
__global__ void __launch_bounds__(BT, 3) k_batch_step(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  uint32_t* su = reinterpret_cast<uint32_t*>(smraw);
  int phases[12];
  int nph = 0;
  if (a.kind == 2) {
    phases[nph++] = PH_KDK_LAST;
  } else {
    phases[nph++] = a.kind == 0 ? PH_KEYS : PH_KDK;
    for (int ph = PH_SCAN; ph <= PH_GRAD; ++ph) phases[nph++] = ph;
  }
  const bool clock = blockIdx.x == 0 && threadIdx.x == 0;
  unsigned long long t_prev = clock ? batch_clock_ns() : 0ull;
  for (int q = 0; q < nph; ++q) {
    const int ph = phases[q];
    const int* off = a.off + ph * (a.nsims + 1);
    const int total = off[a.nsims];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
      const int s = find_sim(off, a.nsims, item);
      const SimDesc& d = a.sims[s];
      const int local = item - off[s];
      switch (ph) {
        case PH_KEYS:
          if (d.te == 8) body_keys<8>(d.dx, d.g, d.N, d.keys, d.tile_count, d.err, local);
          else body_keys<16>(d.dx, d.g, d.N, d.keys, d.tile_count, d.err, local);
          break;
        case PH_KDK:
        case PH_KDK_LAST: {
          const bool last = ph == PH_KDK_LAST;
          const int k = a.k;
          const int ik1 = last ? 3 * k + 2 : 3 * k, ik2 = last ? -1 : (k > 0 ? 3 * (k - 1) + 2 : -1);
          const int idr = last ? -1 : 3 * k + 1;
          uint32_t* keys = last ? nullptr : d.keys;
          // the force mesh was written by the previous launch: read-only path
          const float4* F4p = reinterpret_cast<const float4*>(d.F);
          if (d.te == 8) {
            if (d.f4 && d.rshape == 1)
              body_kdk_brick<Brick32, 8>(d.dx, d.dx, d.p, F4p, d.g, d.N, d.fac, ik1, ik2, idr, keys, d.tile_count, d.err, local);
            else if (d.f4 && d.rshape == 2)
              body_kdk_brick<Brick64, 8>(d.dx, d.dx, d.p, F4p, d.g, d.N, d.fac, ik1, ik2, idr, keys, d.tile_count, d.err, local);
            else if (d.f4)
              body_readout<true, true, true, 8>(d.dx, d.p, d.F, d.g, d.N, d.M, d.fac, ik1, ik2, idr, nullptr, keys,
                                                d.tile_count, d.err, a.ro_iters, local);
            else
              body_readout<true, false, true, 8>(d.dx, d.p, d.F, d.g, d.N, d.M, d.fac, ik1, ik2, idr, nullptr, keys,
                                                 d.tile_count, d.err, a.ro_iters, local);
          } else {
            if (d.f4 && d.rshape == 1)
              body_kdk_brick<Brick32>(d.dx, d.dx, d.p, F4p, d.g, d.N, d.fac, ik1, ik2, idr, keys, d.tile_count, d.err, local);
            else if (d.f4 && d.rshape == 2)
              body_kdk_brick<Brick64>(d.dx, d.dx, d.p, F4p, d.g, d.N, d.fac, ik1, ik2, idr, keys, d.tile_count, d.err, local);
            else if (d.f4)
              body_readout<true, true, true>(d.dx, d.p, d.F, d.g, d.N, d.M, d.fac, ik1, ik2, idr, nullptr, keys,
                                             d.tile_count, d.err, a.ro_iters, local);
            else
              body_readout<true, false, true>(d.dx, d.p, d.F, d.g, d.N, d.M, d.fac, ik1, ik2, idr, nullptr, keys,
                                              d.tile_count, d.err, a.ro_iters, local);
          }
          break;
        }
        case PH_SCAN: body_scan_tiles(d.tile_count, d.ntiles, d.tile_start, d.tile_cursor, su, 1); break;
        case PH_SCATTER:
          if (d.te == 8) body_scatter_cube<BT, 8>(d.keys, d.g.np, d.tile_cursor, d.items, d.cells, local, su, d.err);
          else body_scatter_cube<BT, 16>(d.keys, d.g.np, d.tile_cursor, d.items, d.cells, local, su, d.err);
          break;
        case PH_PAINT:
          if (d.te == 8)
            body_paint_bucket_acc<true, Acc32, 8>(d.dx, d.N, d.items, d.tile_start, d.g, d.rho, d.halo, d.err,
                                                  Acc32{su, su + TileC<8>::ACC}, local, d.cells);
          else
            body_paint_bucket_acc<true, Acc32, 16>(d.dx, d.N, d.items, d.tile_start, d.g, d.rho, d.halo, d.err,
                                                   Acc32{su, su + TileC<16>::ACC}, local, d.cells);
          break;
        case PH_HALO:
          if (d.te == 8) body_paint_halo<8>(d.halo, d.g, d.rho, su, local);
          else body_paint_halo<16>(d.halo, d.g, d.rho, su, local);
          break;
        default:
          switch (d.nc * 2 + (d.fv == 16)) {
            case 64: fft_phase_pow2<32, 8>(ph, d, local, sm); break;
            case 65: fft_phase_pow2<32, 16>(ph, d, local, sm); break;
            case 128: fft_phase_pow2<64, 8>(ph, d, local, sm); break;
            case 129: fft_phase_pow2<64, 16>(ph, d, local, sm); break;
            case 256: fft_phase_pow2<128, 8>(ph, d, local, sm); break;
            case 257: fft_phase_pow2<128, 16>(ph, d, local, sm); break;
            case 192: case 193: fft_phase_smem<96>(ph, d, local, sm); break;
            default: break;
          }
      }
      __syncthreads();   // shared memory is reused by the next item
    }
    if (q + 1 < nph && !grid_barrier(a)) return;
    if (clock) {   // every block has finished phase ph (past the barrier), or block 0 alone for the last
      const unsigned long long t = batch_clock_ns();
      atomicAdd(a.ptime + ph, t - t_prev);
      t_prev = t;
    }
  }
}

// Work items of each phase for one simulation (must match the bodies).
static void items_for(SimDesc& d, int ro_iters) {
  const int nc = d.nc, nh = nc / 2 + 1, nlines = nh * nc;
  const int pchunk = BT * ro_iters;
  d.items_of[PH_KEYS] = (int)((d.N + BT - 1) / BT);
  d.items_of[PH_KDK] = d.rshape == 1 ? Brick32::blocks(d.g.np)
                     : d.rshape == 2 ? Brick64::blocks(d.g.np) : (int)((d.N + pchunk - 1) / pchunk);
  d.items_of[PH_KDK_LAST] = d.items_of[PH_KDK];
  d.items_of[PH_SCAN] = 1;
  d.items_of[PH_SCATTER] = scatter_cube_items(d.g.np, BT);
  d.items_of[PH_PAINT] = d.ntiles;
  d.items_of[PH_HALO] = d.ntiles;
  int L = 0;
  switch (nc * 2 + (d.fv == 16)) {
    case 64: L = RegCfg<32>::L; break;
    case 65: L = RegCfg<32, 16>::L; break;
    case 128: L = RegCfg<64>::L; break;
    case 129: L = RegCfg<64, 16>::L; break;
    case 256: L = RegCfg<128>::L; break;
    case 257: L = RegCfg<128, 16>::L; break;
    default: break;
  }
  if (L) {
    const int tz = nc < 32 ? nc : 32, ty = 256 / tz, xc = nc < ST_XC ? nc : ST_XC;
    d.items_of[PH_ZF] = nc * nc / (2 * L);
    d.items_of[PH_YF] = (nlines + L - 1) / L;
    d.items_of[PH_X] = (nlines + L - 1) / L;
    d.items_of[PH_YI] = (nlines + L - 1) / L;
    d.items_of[PH_ZI] = nc * nc / (2 * L);
    d.items_of[PH_GRAD] = (nc / tz) * (nc / ty) * (nc / xc);
  } else {   // 96 = 3 * 32: shared-memory Stockham passes
    d.items_of[PH_ZF] = nc * (nc / (2 * ZG));
    d.items_of[PH_YF] = (nlines + YL - 1) / YL;
    d.items_of[PH_X] = nh * (nc / XB);
    d.items_of[PH_YI] = 3 * ((nlines + YL - 1) / YL);
    d.items_of[PH_ZI] = 3 * nc * (nc / (2 * ZG));
    d.items_of[PH_GRAD] = 0;
  }
}

bool batch_size_ok(int nc, int np) { return nc == np && (nc == 32 || nc == 64 || nc == 96 || nc == 128); }

struct Batch {
  int nsims = 0;
  std::vector<BatchPlanView> plans;
  std::vector<SimDesc> host_sims;
  SimDesc* d_sims = nullptr;
  int* d_off = nullptr;
  unsigned* d_bar = nullptr;
  int* d_status = nullptr;
  unsigned long long* d_ptime = nullptr;   // [NPH] accumulated phase ns
  long long spin_limit = 1ll << 22;
  int blocks_per_sm = 0;      // 0: as many as fit
  int ro_iters = 1;
  int grid = 0;
  cudaGraphExec_t exec = nullptr;
  bool graph_ok = false;
  int graph_steps = -1;
  std::vector<float*> graph_dx, graph_p;
  // tile tables of simulations painted by 8^3 tiles (the plan's are sized for 16^3)
  struct Tiles8 {
    uint32_t *count = nullptr, *start = nullptr, *cursor = nullptr;
    unsigned long long* halo = nullptr;
  };
  std::vector<Tiles8> tiles8;
};

// Point simulation s at the tile tables of edge te (allocating the 8^3 ones once).
static int set_tiles(Batch* b, int s, int te) {
  SimDesc& d = b->host_sims[s];
  const BatchPlanView& v = b->plans[s];
  if (te == 16) {
    d.te = 16;
    d.ntiles = v.pc.ntiles;
    d.tile_count = v.pc.tile_count;
    d.tile_start = v.pc.tile_start;
    d.tile_cursor = v.pc.tile_cursor;
    d.halo = v.pc.halo;
    return FPM_OK;
  }
  if (te != 8 || v.nc % 8 != 0) return FPM_EINVAL;
  const int nt = v.nc / 8, ntiles = nt * nt * nt;
  Batch::Tiles8& t = b->tiles8[s];
  if (!t.count) {
    if (cudaMalloc(&t.count, ntiles * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&t.start, (ntiles + 1) * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&t.cursor, ntiles * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&t.halo, (size_t)ntiles * TileC<8>::SHELL * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      return FPM_ENOMEM;
    }
  }
  d.te = 8;
  d.ntiles = ntiles;
  d.tile_count = t.count;
  d.tile_start = t.start;
  d.tile_cursor = t.cursor;
  d.halo = t.halo;
  return FPM_OK;
}

static int batch_grid(Batch* b) {
  int dev = 0, nsm = 0, per = 0;
  FPM_CUDA_TRY(cudaGetDevice(&dev));
  FPM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  FPM_CUDA_TRY(cudaFuncSetAttribute(k_batch_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BATCH_SMEM));
  FPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_step, BT, BATCH_SMEM));
  if (per < 1) return FPM_ECUDA;
  const int use = b->blocks_per_sm > 0 ? std::min(b->blocks_per_sm, per) : per;
  b->grid = nsm * use;
  return FPM_OK;
}

static int upload_tables(Batch* b) {
  const int ns = b->nsims;
  std::vector<int> off((size_t)NPH * (ns + 1));
  for (int ph = 0; ph < NPH; ++ph) {
    int run = 0;
    for (int s = 0; s < ns; ++s) {
      off[(size_t)ph * (ns + 1) + s] = run;
      run += b->host_sims[s].items_of[ph];
    }
    off[(size_t)ph * (ns + 1) + ns] = run;
  }
  FPM_CUDA_TRY(cudaMemcpy(b->d_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
  FPM_CUDA_TRY(cudaMemcpy(b->d_sims, b->host_sims.data(), ns * sizeof(SimDesc), cudaMemcpyHostToDevice));
  return FPM_OK;
}

static int launch_step(Batch* b, int kind, int k, cudaStream_t s) {
  BatchArgs a;
  a.sims = b->d_sims;
  a.off = b->d_off;
  a.nsims = b->nsims;
  a.bar = b->d_bar;
  a.spin_limit = b->spin_limit;
  a.status = b->d_status;
  a.kind = kind;
  a.k = k;
  a.ro_iters = b->ro_iters;
  a.ptime = b->d_ptime;
  FPM_CUDA_TRY(cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), s));
  void* args[] = {&a};
  FPM_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_batch_step, dim3(b->grid), dim3(BT), args, BATCH_SMEM, s));
  return FPM_OK;
}

int batch_create(Batch** out, const BatchPlanView* views, int nsims) {
  Batch* b = new Batch();
  b->nsims = nsims;
  b->plans.assign(views, views + nsims);
  b->host_sims.resize(nsims);
  int rc = FPM_OK;
  auto fail = [&](int r) {
    batch_destroy(b);
    return r;
  };
  for (int s = 0; s < nsims; ++s) {
    const BatchPlanView& v = views[s];
    SimDesc& d = b->host_sims[s];
    d = SimDesc{};
    d.g = v.pc.g;
    d.N = v.pc.N;
    d.M = v.pc.M;
    d.nc = v.nc;
    d.ntiles = v.pc.ntiles;
    d.f4 = v.f4;
    d.F = v.F;
    d.rho = v.rho;
    d.spec = v.spec;
    d.specmax = v.specmax;
    d.keys = v.pc.keys;
    d.items = v.pc.items;
    d.cells = v.pc.cells;
    d.tile_count = v.pc.tile_count;
    d.tile_start = v.pc.tile_start;
    d.tile_cursor = v.pc.tile_cursor;
    d.halo = v.pc.halo;
    d.err = v.pc.err;
    d.fac = v.fac;
    d.tw = v.tab.tw;
    d.gk = v.tab.g;
    d.w2 = v.tab.w2;
    d.force_coef = v.force_coef;
    d.te = 16;
    d.fv = 8;
    d.rshape = !d.f4 ? 0 : Brick64::fits(d.g.np) ? 2 : Brick32::fits(d.g.np) ? 1 : 0;
    items_for(d, b->ro_iters);
  }
  b->tiles8.resize(nsims);
  if (cudaMalloc(&b->d_sims, nsims * sizeof(SimDesc)) != cudaSuccess ||
      cudaMalloc(&b->d_off, (size_t)NPH * (nsims + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_bar, 2 * sizeof(unsigned)) != cudaSuccess || cudaMalloc(&b->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_ptime, NPH * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return fail(FPM_ENOMEM);
  }
  if (cudaMemset(b->d_status, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(b->d_ptime, 0, NPH * sizeof(unsigned long long)) != cudaSuccess)
    return fail(FPM_ECUDA);
  if ((rc = batch_grid(b)) != FPM_OK) return fail(rc);
  if ((rc = upload_tables(b)) != FPM_OK) return fail(rc);
  *out = b;
  return FPM_OK;
}

void batch_destroy(Batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  cudaFree(b->d_sims);
  cudaFree(b->d_off);
  cudaFree(b->d_bar);
  cudaFree(b->d_status);
  cudaFree(b->d_ptime);
  for (auto& t : b->tiles8) {
    cudaFree(t.count);
    cudaFree(t.start);
    cudaFree(t.cursor);
    cudaFree(t.halo);
  }
  delete b;
}

int batch_configure(Batch* b, int blocks_per_sm, int ro_iters, long long spin_limit) {
  if (blocks_per_sm >= 0) b->blocks_per_sm = blocks_per_sm;
  if (ro_iters >= 1) b->ro_iters = ro_iters;
  if (spin_limit >= 1) b->spin_limit = spin_limit;
  for (auto& d : b->host_sims) items_for(d, b->ro_iters);
  FPM_TRY(batch_grid(b));
  FPM_TRY(upload_tables(b));
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_steps = -1;
  }
  return FPM_OK;
}

// Advance every simulation over the same nsteps KDK steps (factors already
// computed per plan).  The step launches are captured once into a CUDA
// graph per (nsteps, particle buffers) and replayed.
int batch_kdk(Batch* b, float* const* dx, float* const* p, int nsteps, cudaStream_t s) {
  bool same = b->exec && b->graph_steps == nsteps;
  for (int i = 0; same && i < b->nsims; ++i) same = b->graph_dx[i] == dx[i] && b->graph_p[i] == p[i];
  if (!same) {
    for (int i = 0; i < b->nsims; ++i) {
      b->host_sims[i].dx = dx[i];
      b->host_sims[i].p = p[i];
    }
    FPM_TRY(upload_tables(b));
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    cudaStream_t cs;
    FPM_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    int rc = FPM_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = FPM_ECUDA;
    for (int i = 0; rc == FPM_OK && i < b->nsims; ++i)
      if (cudaMemsetAsync(b->host_sims[i].tile_count, 0, sizeof(uint32_t) * b->host_sims[i].ntiles, cs) != cudaSuccess)
        rc = FPM_ECUDA;
    if (rc == FPM_OK) rc = launch_step(b, 0, 0, cs);
    for (int k = 0; rc == FPM_OK && k < nsteps; ++k) rc = launch_step(b, 1, k, cs);
    if (rc == FPM_OK) rc = launch_step(b, 2, nsteps - 1, cs);
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess && rc == FPM_OK) rc = FPM_ECUDA;
    if (rc == FPM_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) rc = FPM_ECUDA;
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    if (rc != FPM_OK) {   // capture unavailable: launch the steps directly
      if (b->exec) cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
      b->graph_steps = -1;
      b->graph_ok = false;
      for (int i = 0; i < b->nsims; ++i)
        FPM_CUDA_TRY(cudaMemsetAsync(b->host_sims[i].tile_count, 0, sizeof(uint32_t) * b->host_sims[i].ntiles, s));
      FPM_TRY(launch_step(b, 0, 0, s));
      for (int k = 0; k < nsteps; ++k) FPM_TRY(launch_step(b, 1, k, s));
      return launch_step(b, 2, nsteps - 1, s);
    }
    b->graph_ok = true;
    b->graph_steps = nsteps;
    b->graph_dx.assign(dx, dx + b->nsims);
    b->graph_p.assign(p, p + b->nsims);
  }
  FPM_CUDA_TRY(cudaGraphLaunch(b->exec, s));
  return FPM_OK;
}

int batch_status(Batch* b, cudaStream_t s) {
  int h = 0;
  FPM_CUDA_TRY(cudaMemcpyAsync(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  FPM_CUDA_TRY(cudaStreamSynchronize(s));
  FPM_CUDA_TRY(cudaMemsetAsync(b->d_status, 0, sizeof(int), s));
  return (h & ERR_TIMEOUT) ? FPM_ETIMEOUT : FPM_OK;
}

int batch_tune(Batch* b, int nc, int knob, int value) {
  bool any = false;
  for (int s = 0; s < b->nsims; ++s) {     // validate first: all or nothing
    const SimDesc& d = b->host_sims[s];
    if (d.nc != nc) continue;
    any = true;
    if (knob == BT_READOUT) {
      const bool ok = value == 0 || (d.f4 && ((value == 1 && Brick32::fits(d.g.np)) || (value == 2 && Brick64::fits(d.g.np))));
      if (!ok) return FPM_EINVAL;
    } else if (knob == BT_PAINT_TILE) {
      if (value != 8 && value != 16) return FPM_EINVAL;
    } else if (knob == BT_FFT_SLOTS) {
      if ((value != 8 && value != 16) || !is_pow2_size(nc)) return FPM_EINVAL;
    } else {
      return FPM_EINVAL;
    }
  }
  if (!any) return FPM_EINVAL;
  for (int s = 0; s < b->nsims; ++s) {
    SimDesc& d = b->host_sims[s];
    if (d.nc != nc) continue;
    if (knob == BT_READOUT) d.rshape = value;
    else if (knob == BT_FFT_SLOTS) d.fv = value;
    else FPM_TRY(set_tiles(b, s, value));
    items_for(d, b->ro_iters);
  }
  FPM_TRY(upload_tables(b));
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_steps = -1;
  }
  return FPM_OK;
}

int batch_phase_times(Batch* b, double* ms, int n, cudaStream_t s) {
  if (n < NPH) return FPM_EINVAL;
  unsigned long long h[NPH];
  FPM_CUDA_TRY(cudaMemcpyAsync(h, b->d_ptime, sizeof(h), cudaMemcpyDeviceToHost, s));
  FPM_CUDA_TRY(cudaStreamSynchronize(s));
  FPM_CUDA_TRY(cudaMemsetAsync(b->d_ptime, 0, sizeof(h), s));
  for (int k = 0; k < NPH; ++k) ms[k] = 1e-6 * (double)h[k];
  return FPM_OK;
}

int batch_info(const Batch* b, int* grid, int* graph_captured) {
  if (grid) *grid = b->grid;
  if (graph_captured) *graph_captured = b->graph_ok ? 1 : 0;
  return FPM_OK;
}

}  // namespace fpm
