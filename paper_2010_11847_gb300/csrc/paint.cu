// paint.cu -- cell keys, counting sort, deterministic CIC paint, CIC readout
// fused with the KDK kick and drift (Sec. 2 and Eqs. 1-2).
//
// Sort.  The mesh is cut into 16^3-cell tiles.  Each particle's tile-major
// cell key is computed from its float32 displacement (cell = wrap(q +
// floor(dx)), exact in float), tile counts are histogrammed with
// warp-aggregated atomics into an L2-resident table, scanned, and the
// particles are bucketed by tile (a counting sort on the tile part of the
// key), one Lagrangian block of particles per thread block, which records
// each item's in-tile cell beside it.  When the caller asks for the
// permutation, a shared-memory counting sort by local cell plus an index
// tie-fix completes the stable order.
//
// Paint.  One CTA per tile accumulates the CIC weights of its bucket into a
// 17^3 shared-memory block (the tile plus its upper halo).  Each weight is
// a fixed-point fraction in units of 2^-24, added with 32-bit shared
// atomics; a thread whose add wraps the 32-bit word (it sees it in the
// returned old value) adds the carry to a second word, so every cell holds
// the exact 64-bit sum.  Before adding, a warp that holds long runs of the
// same cell merges them (one redux.sync per corner over each run's lanes).
// Integer addition is associative, so the density does not depend on the
// order of anything: it is deterministic.  The particle mass multiplies the
// sums at write-out.  Cells that only this tile touches are written
// directly; the shell of the 17^3 block goes to a per-tile halo buffer, and
// the last of the (up to 8) blocks whose shells cover a tile's lower faces
// sums them (a separate face-sum kernel where no face counters are kept).
#include "paint_dev.cuh"
#include "readout_dev.cuh"

namespace fpm {

// ---------------------------------------------------------------- kernels
constexpr int SCAN_THREADS = 1024;

__global__ void k_keys(const float* __restrict__ dx, Geom g, size_t N, uint32_t* __restrict__ keys,
                       uint32_t* __restrict__ tile_count, int* __restrict__ err) {
  body_keys(dx, g, N, keys, tile_count, err, blockIdx.x);
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(uint32_t* __restrict__ count, int ntiles,
                                                             uint32_t* __restrict__ start,
                                                             uint32_t* __restrict__ cursor) {
  __shared__ uint32_t part[SCAN_THREADS];
  body_scan_tiles(count, ntiles, start, cursor, part, 0);
}


constexpr int SC_THREADS = 512;
// The cube bucketing also records each item's in-tile cell for the paints.
constexpr bool PAINT_CELLS = true;

// In-tile cells recorded by the cube bucketing.
inline uint16_t* cells_of(const PaintCtx& c) { return PAINT_CELLS ? c.cells : nullptr; }

__global__ void __launch_bounds__(SC_THREADS, 4) k_scatter_cube(const uint32_t* __restrict__ keys, int np,
                                                             uint32_t* __restrict__ cursor,
                                                             uint32_t* __restrict__ items,
                                                             uint16_t* __restrict__ cells,
                                                             int* __restrict__ err) {
  __shared__ uint32_t tbl[3 * SC_TBL];
  body_scatter_cube<SC_THREADS>(keys, np, cursor, items, cells, blockIdx.x, tbl, err);
}

__global__ void __launch_bounds__(PB_THREADS) k_paint_bucket(const float* __restrict__ dx, size_t N,
                                                             const uint32_t* __restrict__ items,
                                                             const uint32_t* __restrict__ tile_start, Geom g,
                                                             float* __restrict__ rho,
                                                             unsigned long long* __restrict__ halo,
                                                             int* __restrict__ err) {
  __shared__ uint32_t lo[ACC], hi[ACC];
  body_paint_bucket(dx, N, items, tile_start, g, rho, halo, err, lo, hi, blockIdx.x);
}

// Paint with the face sums done by the last contributing block.
__global__ void __launch_bounds__(PB_THREADS) k_paint_bucket_faces(const float* __restrict__ dx, size_t N,
                                                                   const uint32_t* __restrict__ items,
                                                                   const uint32_t* __restrict__ tile_start, Geom g,
                                                                   float* __restrict__ rho,
                                                                   unsigned long long* __restrict__ halo,
                                                                   uint32_t* __restrict__ done, int* __restrict__ err,
                                                                   const uint16_t* __restrict__ cells) {
  __shared__ uint32_t lo[ACC], hi[ACC];
  __shared__ uint32_t sm[24];
  body_paint_bucket_acc<false>(dx, N, items, tile_start, g, rho, halo, err, Acc32{lo, hi}, blockIdx.x, cells);
  paint_faces_last(done, halo, g, rho, blockIdx.x, sm);
}

__global__ void __launch_bounds__(768) k_paint_halo(const unsigned long long* __restrict__ halo, Geom g,
                                                    float* __restrict__ rho) {
  __shared__ uint32_t nb[8];
  body_paint_halo(halo, g, rho, nb, blockIdx.x);
}

template <bool KDK, bool F4>
__global__ void __launch_bounds__(256) k_readout(float* __restrict__ dx, float* __restrict__ p,
                                                 const float* __restrict__ F, Geom g, size_t N, size_t M,
                                                 const double* __restrict__ fac, int ik1, int ik2, int idr,
                                                 float* __restrict__ f_out, uint32_t* __restrict__ keys,
                                                 uint32_t* __restrict__ tile_count, int* __restrict__ err,
                                                 int iters) {
  body_readout<KDK, F4>(dx, p, F, g, N, M, fac, ik1, ik2, idr, f_out, keys, tile_count, err, iters, blockIdx.x);
}

// Paint with the permutation output: counting sort of the tile's bucket by
// local cell in shared memory, index tie-fix, then the same deposit in
// sorted order.  Tiles larger than PCAP are deposited in bucket order and
// sorted by k_perm_big.
__global__ void __launch_bounds__(PS_THREADS) k_paint_sorted(const float* __restrict__ dx, size_t N,
                                                             const uint32_t* __restrict__ items,
                                                             const uint32_t* __restrict__ keys,
                                                             const uint32_t* __restrict__ tile_start, Geom g,
                                                             float* __restrict__ rho,
                                                             unsigned long long* __restrict__ halo,
                                                             uint32_t* __restrict__ perm, int* __restrict__ err) {
  extern __shared__ uint32_t smraw[];
  uint32_t* lo = smraw;
  uint32_t* hi = lo + ACC;
  uint32_t* hist = hi + ACC;
  uint32_t* sorted = hist + TILE3;
  __shared__ uint32_t part[PS_THREADS];
  const int nt = g.nt;
  const int tile = blockIdx.x;
  const int o[3] = {(tile / (nt * nt)) * TILE, ((tile / nt) % nt) * TILE, (tile % nt) * TILE};
  const uint32_t s0 = tile_start[tile], s1 = tile_start[tile + 1];
  const int n = (int)(s1 - s0);
  for (int k = threadIdx.x; k < ACC; k += blockDim.x) lo[k] = hi[k] = 0u;
  for (int k = threadIdx.x; k < TILE3; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  bool bad = false;
  const int nw = (n + 31) & ~31;
  if (n <= PCAP) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) atomicAdd(hist + (keys[items[s0 + k]] & 4095u), 1u);
    __syncthreads();
    {   // exclusive scan of the 4096 local-cell counts: 16 per thread
      constexpr int PER = TILE3 / PS_THREADS;
      uint32_t loc[PER];
      uint32_t s = 0;
      for (int k = 0; k < PER; ++k) {
        loc[k] = hist[threadIdx.x * PER + k];
        s += loc[k];
      }
      part[threadIdx.x] = s;
      __syncthreads();
      for (int off = 1; off < PS_THREADS; off <<= 1) {
        const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
      }
      uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
      for (int k = 0; k < PER; ++k) {
        hist[threadIdx.x * PER + k] = run;
        run += loc[k];
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const uint32_t i = items[s0 + k];
      sorted[atomicAdd(hist + (keys[i] & 4095u), 1u)] = i;
    }
    __syncthreads();
    // order equal cells by particle index (hist[c] is now the end of cell c)
    for (int c = threadIdx.x; c < TILE3; c += blockDim.x) {
      const int lo = c ? (int)hist[c - 1] : 0, hi = (int)hist[c];
      for (int a = lo + 1; a < hi; ++a) {
        const uint32_t v = sorted[a];
        int b = a - 1;
        while (b >= lo && sorted[b] > v) {
          sorted[b + 1] = sorted[b];
          --b;
        }
        sorted[b + 1] = v;
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) perm[s0 + k] = sorted[k];
    for (int k = threadIdx.x; k < nw; k += blockDim.x) {
      const bool active = k < n;
      int l[3] = {0, 0, 0};
      float t[3] = {0.f, 0.f, 0.f};
      if (active) bad |= !particle_local<false>(dx, N, sorted[k], g, o, l, t);
      deposit_warp(lo, hi, active, l, t);
    }
  } else {
    for (int k = threadIdx.x; k < nw; k += blockDim.x) {
      const bool active = k < n;
      int l[3] = {0, 0, 0};
      float t[3] = {0.f, 0.f, 0.f};
      if (active) bad |= !particle_local<false>(dx, N, items[s0 + k], g, o, l, t);
      deposit_warp(lo, hi, active, l, t);
    }
  }
  if (bad) atomicOr(err, ERR_RANGE);
  __syncthreads();
  paint_writeout(lo, hi, o, tile, g, rho, halo);
}

// Stable order of one oversized tile for the permutation output: counting
// sort by local cell with a global cursor table, then the index tie-fix.
// One CTA per tile; tiles within PCAP return at once.
__global__ void k_perm_big(const uint32_t* __restrict__ items, const uint32_t* __restrict__ keys,
                           const uint32_t* __restrict__ tile_start, uint32_t* __restrict__ perm) {
  __shared__ uint32_t cur[TILE3];
  const int tile = blockIdx.x;
  const uint32_t s0 = tile_start[tile], s1 = tile_start[tile + 1];
  if ((int)(s1 - s0) <= PCAP) return;
  for (int k = threadIdx.x; k < TILE3; k += blockDim.x) cur[k] = 0;
  __syncthreads();
  for (uint32_t k = s0 + threadIdx.x; k < s1; k += blockDim.x) atomicAdd(cur + (keys[items[k]] & 4095u), 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = s0;
    for (int c = 0; c < TILE3; ++c) {
      const uint32_t v = cur[c];
      cur[c] = run;
      run += v;
    }
  }
  __syncthreads();
  for (uint32_t k = s0 + threadIdx.x; k < s1; k += blockDim.x) {
    const uint32_t i = items[k];
    perm[atomicAdd(cur + (keys[i] & 4095u), 1u)] = i;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < TILE3; c += blockDim.x) {
    const uint32_t lo = c ? cur[c - 1] : s0, hi = cur[c];
    for (uint32_t a = lo + 1; a < hi; ++a) {
      const uint32_t v = perm[a];
      uint32_t b = a;
      while (b > lo && perm[b - 1] > v) {
        perm[b] = perm[b - 1];
        --b;
      }
      perm[b] = v;
    }
  }
}

// The KDK readout walks compact Lagrangian bricks (k_kdk_brick) where the
// lattice allows it.
constexpr bool KDK_BRICK = true;

// Chunks per CTA for the readout: long chunks at scale, at least ~8 CTAs per SM.
static int readout_iters(size_t N) {
  const size_t per = N / (256 * 152 * 8);
  return (int)(per < 1 ? 1 : (per > 8 ? 8 : per));
}

// ---------------------------------------------------------------- host side
static int grid_of(size_t n, int threads) { return (int)((n + threads - 1) / threads); }

int paint_setup() {
  FPM_CUDA_TRY(cudaFuncSetAttribute(k_paint_sorted, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)SORTED_SMEM));
  return FPM_OK;
}

Geom make_geom(int np, int nc) {
  Geom g;
  g.np = np;
  g.nc = nc;
  g.ratio = nc / np;
  g.nt = nc / TILE;
  g.mass = (float)((double)(nc / np) * (nc / np) * (nc / np));
  g.div_np = make_fastdiv((uint32_t)np);
  g.div_np2 = make_fastdiv((uint32_t)np * (uint32_t)np);
  return g;
}

size_t paint_halo_elems(int ntiles) { return (size_t)ntiles * SHELL; }

int launch_keys(const PaintCtx& c, const float* dx, cudaStream_t s) {
  FPM_CUDA_TRY(cudaMemsetAsync(c.tile_count, 0, sizeof(uint32_t) * c.ntiles, s));
  k_keys<<<grid_of(c.N, 256), 256, 0, s>>>(dx, c.g, c.N, c.keys, c.tile_count, c.err);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_scan(const PaintCtx& c, cudaStream_t s) {
  k_scan_tiles<<<1, SCAN_THREADS, 0, s>>>(c.tile_count, c.ntiles, c.tile_start, c.tile_cursor);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_scatter(const PaintCtx& c, cudaStream_t s) {
  if (c.g.np % SC_CUBE != 0) return FPM_EINVAL;   // every supported lattice size is a multiple of 16
  k_scatter_cube<<<scatter_cube_items(c.g.np, SC_THREADS), SC_THREADS, 0, s>>>(c.keys, c.g.np, c.tile_cursor,
                                                                             c.items, cells_of(c), c.err);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_paint_tiles(const PaintCtx& c, const float* dx, float* rho, uint32_t* perm, cudaStream_t s) {
  if (perm) {
    k_paint_sorted<<<c.ntiles, PS_THREADS, SORTED_SMEM, s>>>(dx, c.N, c.items, c.keys, c.tile_start, c.g, rho,
                                                              c.halo, perm, c.err);
  } else if (c.tile_done) {
    k_paint_bucket_faces<<<c.ntiles, PB_THREADS, 0, s>>>(dx, c.N, c.items, c.tile_start, c.g, rho, c.halo,
                                                          c.tile_done, c.err, cells_of(c));
  } else {
    k_paint_bucket<<<c.ntiles, PB_THREADS, 0, s>>>(dx, c.N, c.items, c.tile_start, c.g, rho, c.halo, c.err);
  }
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_perm_big(const PaintCtx& c, uint32_t* perm, cudaStream_t s) {
  k_perm_big<<<c.ntiles, 256, 0, s>>>(c.items, c.keys, c.tile_start, perm);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_halo(const PaintCtx& c, float* rho, cudaStream_t s) {
  k_paint_halo<<<c.ntiles, 768, 0, s>>>(c.halo, c.g, rho);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_readout(const PaintCtx& c, const float* F, const float* dx, float* f_out, cudaStream_t s) {
  const int it = readout_iters(c.N);
  k_readout<false, false><<<grid_of(c.N, 256 * it), 256, 0, s>>>(const_cast<float*>(dx), nullptr, F, c.g, c.N,
                                                                 c.M, nullptr, -1, -1, -1, f_out, nullptr,
                                                                 nullptr, c.err, it);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

// F is [3][M] (f4 = false) or interleaved float4 [M] (f4 = true).
int launch_kdk(const PaintCtx& c, float* dx, float* p, const float* F, bool f4, const double* fac, int ik1,
               int ik2, int idr, bool emit_keys, cudaStream_t s, float* dx_out) {
  if (emit_keys) FPM_CUDA_TRY(cudaMemsetAsync(c.tile_count, 0, sizeof(uint32_t) * c.ntiles, s));
  const int it = readout_iters(c.N);
  uint32_t* keys = emit_keys ? c.keys : nullptr;
  if (f4 && KDK_BRICK && KdkBrick::fits(c.g.np))
    return launch_kdk_brick(c, dx, dx_out ? dx_out : dx, p, reinterpret_cast<const float4*>(F), fac, ik1, ik2, idr,
                            keys, s);
  if (dx_out && dx_out != dx) return FPM_EINVAL;
  if (f4)
    k_readout<true, true><<<grid_of(c.N, 256 * it), 256, 0, s>>>(dx, p, F, c.g, c.N, c.M, fac, ik1, ik2, idr,
                                                                 nullptr, keys, c.tile_count, c.err, it);
  else
    k_readout<true, false><<<grid_of(c.N, 256 * it), 256, 0, s>>>(dx, p, F, c.g, c.N, c.M, fac, ik1, ik2, idr,
                                                                  nullptr, keys, c.tile_count, c.err, it);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

// ================================================================ adjoints
// Transposed Jacobians of paint and readout at fixed particle positions.

// g_dx_i (+)= sum_c grad W(x_i - c) (mass g_rho_c + v_i . F_c): the paint
// transpose (first term) and the readout's position term (second) share the
// CIC gradient weights dW/dt_d = (b_d ? +1 : -1) prod_{e != d} w_e (the
// right derivative at integer t, matching the floor-based cell).
template <bool F4>
__global__ void __launch_bounds__(256) k_gather_adj(const float* __restrict__ dx, Geom g, size_t N, size_t M,
                                                    const float* __restrict__ g_rho, const float* __restrict__ F,
                                                    const float* __restrict__ v, float* __restrict__ g_dx,
                                                    int accumulate, int iters) {
  // each block walks a contiguous chunk of iters*256 particles (the mesh
  // rows its lattice rows share stay in L1) and fetches the next particle's
  // dx and v while it gathers; per-particle arrays are streamed so that L2
  // keeps the meshes
  const int nc = g.nc;
  const size_t c0 = (size_t)blockIdx.x * iters * blockDim.x;
  float dn[3] = {0.f, 0.f, 0.f}, vn[3] = {0.f, 0.f, 0.f};
  {
    const size_t i = c0 + threadIdx.x;
    if (i < N)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        dn[a] = __ldcs(dx + a * N + i);
        if (v) vn[a] = __ldcs(v + a * N + i);
      }
  }
  for (int it = 0; it < iters; ++it) {
    if (c0 + (size_t)it * blockDim.x >= N) break;
    const size_t i = c0 + (size_t)it * blockDim.x + threadIdx.x;
    const float d[3] = {dn[0], dn[1], dn[2]}, vi[3] = {vn[0], vn[1], vn[2]};
    const size_t inext = i + blockDim.x;
    if (it + 1 < iters && inext < N)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        dn[a] = __ldcs(dx + a * N + inext);
        if (v) vn[a] = __ldcs(v + a * N + inext);
      }
    if (i >= N) continue;
    int q[3], c[3];
    float t[3];
    lattice_node((uint32_t)i, g, q);
#pragma unroll
    for (int a = 0; a < 3; ++a) cic_cell(d[a], q[a], nc, &c[a], &t[a]);
    const int c1[3] = {c[0] + 1 == nc ? 0 : c[0] + 1, c[1] + 1 == nc ? 0 : c[1] + 1, c[2] + 1 == nc ? 0 : c[2] + 1};
    float gsum[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int bx = b >> 2, by = (b >> 1) & 1, bz = b & 1;
      const size_t idx = ((size_t)(bx ? c1[0] : c[0]) * nc + (by ? c1[1] : c[1])) * nc + (bz ? c1[2] : c[2]);
      float s = 0.f;
      if (g_rho) s = g.mass * __ldg(g_rho + idx);
      if (v) {
        if (F4) {
          const float4 f = __ldg(reinterpret_cast<const float4*>(F) + idx);
          s = fmaf(vi[0], f.x, fmaf(vi[1], f.y, fmaf(vi[2], f.z, s)));
        } else {
          for (int a = 0; a < 3; ++a) s = fmaf(vi[a], __ldg(F + a * M + idx), s);
        }
      }
      const float wx = bx ? t[0] : 1.f - t[0], wy = by ? t[1] : 1.f - t[1], wz = bz ? t[2] : 1.f - t[2];
      gsum[0] = fmaf((bx ? 1.f : -1.f) * wy * wz, s, gsum[0]);
      gsum[1] = fmaf((by ? 1.f : -1.f) * wx * wz, s, gsum[1]);
      gsum[2] = fmaf((bz ? 1.f : -1.f) * wx * wy, s, gsum[2]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) __stcs(g_dx + a * N + i, accumulate ? __ldcs(g_dx + a * N + i) + gsum[a] : gsum[a]);
  }
}

// The same transposed gather over the Lagrangian bricks of the fused
// readout (KdkBrick): the mesh corners a CTA's particles touch stay in L1
// while it marches through its brick.  Identical arithmetic per particle.
//
// With a drift-kick tail (dk.gp non-null) each particle then applies the
// next reverse step's drift and kick transposes to its new cotangent, as
// k_adj_drift_kick does (gp += D g_dx; v = K gp, v overwritten in place),
// and the block records max |v| for the next vector paint.  In this form
// the cotangent velocities are not stored: v holds the momentum cotangents
// gp themselves, the kernel takes v_i = K gp_i with the current kick factor
// (vk), updates gp in place and records max |K' gp'| for the next step.
struct DriftKickTail {
  bool on = false;
  const double* fac = nullptr;
  int idr = -1, ik1 = -1, ik2 = -1;
  unsigned* vmax = nullptr;        // zeroed by the launcher
};

template <bool F4>
__global__ void __launch_bounds__(KB_THREADS) k_gather_adj_brick(const float* __restrict__ dx, Geom g, size_t N,
                                                                 size_t M, const float* __restrict__ g_rho,
                                                                 const float* __restrict__ F, float* v, KScale vk,
                                                                 float* __restrict__ g_dx, int accumulate,
                                                                 DriftKickTail dk) {
  using BS = KdkBrick;
  __shared__ unsigned s_max[KB_THREADS / 32];
  const float Kc = kscale(vk);
  float Dn = 0.f, Kn = 0.f;
  if (dk.on) {
    Dn = (float)dk.fac[dk.idr];
    Kn = (float)(dk.fac[dk.ik1] + (dk.ik2 >= 0 ? dk.fac[dk.ik2] : 0.0));
  }
  unsigned vm = 0;
  const int np = g.np, nc = g.nc;
  const int nbz = np / BS::Z, nby = np / BS::Y;
  const int blk = blockIdx.x;
  const int bz = blk % nbz, by = (blk / nbz) % nby, bx = blk / (nbz * nby);
  float dn[3], vn[3] = {0.f, 0.f, 0.f};
  {
    const uint32_t i = brick_particle<BS>(0, bx, by, bz, np);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dn[a] = __ldcs(dx + a * N + i);
      if (v) vn[a] = __ldcs(v + a * N + i);
    }
  }
#pragma unroll 1
  for (int it = 0; it < BS::ITERS; ++it) {
    const uint32_t i = brick_particle<BS>(it, bx, by, bz, np);
    const float d[3] = {dn[0], dn[1], dn[2]}, vr[3] = {vn[0], vn[1], vn[2]};
    const float vi[3] = {Kc * vr[0], Kc * vr[1], Kc * vr[2]};
    if (it + 1 < BS::ITERS) {
      const uint32_t inext = brick_particle<BS>(it + 1, bx, by, bz, np);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        dn[a] = __ldcs(dx + a * N + inext);
        if (v) vn[a] = __ldcs(v + a * N + inext);
      }
    }
    int q[3], c[3];
    float t[3];
    lattice_node(i, g, q);
#pragma unroll
    for (int a = 0; a < 3; ++a) cic_cell(d[a], q[a], nc, &c[a], &t[a]);
    const int c1[3] = {c[0] + 1 == nc ? 0 : c[0] + 1, c[1] + 1 == nc ? 0 : c[1] + 1, c[2] + 1 == nc ? 0 : c[2] + 1};
    float gsum[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int bx_ = b >> 2, by_ = (b >> 1) & 1, bz_ = b & 1;
      const size_t idx = ((size_t)(bx_ ? c1[0] : c[0]) * nc + (by_ ? c1[1] : c[1])) * nc + (bz_ ? c1[2] : c[2]);
      float s = 0.f;
      if (g_rho) s = g.mass * __ldg(g_rho + idx);
      if (v) {
        if (F4) {
          const float4 f = __ldg(reinterpret_cast<const float4*>(F) + idx);
          s = fmaf(vi[0], f.x, fmaf(vi[1], f.y, fmaf(vi[2], f.z, s)));
        } else {
          for (int a = 0; a < 3; ++a) s = fmaf(vi[a], __ldg(F + a * M + idx), s);
        }
      }
      const float wx = bx_ ? t[0] : 1.f - t[0], wy = by_ ? t[1] : 1.f - t[1], wz = bz_ ? t[2] : 1.f - t[2];
      gsum[0] = fmaf((bx_ ? 1.f : -1.f) * wy * wz, s, gsum[0]);
      gsum[1] = fmaf((by_ ? 1.f : -1.f) * wx * wz, s, gsum[1]);
      gsum[2] = fmaf((bz_ ? 1.f : -1.f) * wx * wy, s, gsum[2]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float gx = accumulate ? __ldcs(g_dx + a * N + i) + gsum[a] : gsum[a];
      __stcs(g_dx + a * N + i, gx);
      if (dk.on) {
        const float gq = fmaf(Dn, gx, vr[a]);
        __stcs(v + a * N + i, gq);
        vm = max(vm, __float_as_uint(fabsf(Kn * gq)));
      }
    }
  }
  if (dk.on) {
    for (int off = 16; off; off >>= 1) vm = max(vm, __shfl_xor_sync(0xffffffffu, vm, off));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = vm;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned m = 0;
      for (int w = 0; w < KB_THREADS / 32; ++w) m = max(m, s_max[w]);
      atomicMax(dk.vmax, m);
    }
  }
}

// max |v| over n values as the bit pattern of a non-negative float (the
// integer order of such patterns is their numeric order): order-independent.
__global__ void k_maxabs(const float* __restrict__ v, KScale vk, size_t n, unsigned* __restrict__ out) {
  const float K = kscale(vk);
  unsigned m = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(fabsf(K * v[i])));
  for (int off = 16; off; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Fixed-point unit 2^S for signed deposits: |w v| 2^S < 2^29 for every
// deposit (weights <= 1), built from the exponent bits of max |v| so that it
// is exactly a power of two.
__device__ __forceinline__ float signed_scale(unsigned maxbits) {
  // m < 2^(e+1) with e the unbiased exponent of m: S = 28 - e gives m 2^S < 2^29
  const int e = (int)((maxbits >> 23) & 0xffu) - 127;
  if (maxbits == 0u || e < -100 || e > 100) return 1.f;
  return __int_as_float((127 + 28 - e) << 23);
}

// 64-bit two's-complement accumulation of a signed 32-bit value with 32-bit
// shared atomics: low word with carry out, high word with carry minus sign.
__device__ __forceinline__ void acc_add_signed(uint32_t* lo, uint32_t* hi, int c, int w) {
  const uint32_t old = atomicAdd(lo + c, (uint32_t)w);
  const int delta = ((old + (uint32_t)w) < old ? 1 : 0) - (w < 0 ? 1 : 0);
  if (delta) atomicAdd(hi + c, (uint32_t)delta);
}

__device__ __forceinline__ float from_fix_signed(long long v, float inv_scale) {
  return __ll2float_rn(v) * inv_scale;     // one rounding of the exact sum; the scale is a power of two
}

// Face cells of tile bx from the shells of the up to 8 tiles covering them
// (signed fixed point, unit 1/inv); nb: 8 words of shared memory.
__device__ __forceinline__ void body_halo_vec(const unsigned long long* __restrict__ halo, const Geom& g, float inv,
                                              float* __restrict__ out, uint32_t* nb, int bx) {
  tile_face_sums(halo, g, out, nb, bx, [inv](unsigned long long v) { return from_fix_signed((long long)v, inv); });
}

// Readout transpose for one channel: out_c = sum_i W(x_i - c) v_i (no
// mass), v_i = K vch_i (vk), deterministic signed fixed point in units set
// by max |v|.
// With nch = 3 one launch paints the three channels: block b takes tile
// b / 3 and channel b % 3 (the three blocks of a tile run side by side and
// share the tile's items, cells and dx gathers through L2), each channel
// with its own output, shell buffer and face counters (strides M, hstride,
// ntiles); with nch = 1 the block paints channel 0 of the given pointers.
__global__ void __launch_bounds__(PB_THREADS) k_paint_vec(const float* __restrict__ dx, size_t N,
                                                          const uint32_t* __restrict__ items,
                                                          const uint32_t* __restrict__ tile_start, Geom g,
                                                          const float* __restrict__ v, KScale vk,
                                                          const unsigned* __restrict__ vmax,
                                                          float* __restrict__ out_all,
                                                          unsigned long long* __restrict__ halo_all,
                                                          const uint16_t* __restrict__ cells,
                                                          uint32_t* __restrict__ done_all, int nch, size_t M,
                                                          size_t hstride) {
  __shared__ uint32_t lo[ACC], hi[ACC];
  __shared__ uint32_t sm[24];
  const int nt = g.nt;
  const int tile = nch == 1 ? (int)blockIdx.x : (int)blockIdx.x / 3;
  const float* __restrict__ vch = v + (blockIdx.x - tile * nch) * N;
  const int o[3] = {(tile / (nt * nt)) * TILE, ((tile / nt) % nt) * TILE, (tile % nt) * TILE};
  const uint32_t s0 = tile_start[tile], s1 = tile_start[tile + 1];
  const float scale = signed_scale(*vmax), inv = 1.f / scale;
  const float K = kscale(vk);
  for (int k = threadIdx.x; k < ACC; k += blockDim.x) lo[k] = hi[k] = 0u;
  __syncthreads();
  auto deposit = [&](const int* l, const float* t, float vi) {
    const float vs = (K * vi) * scale;
    const int base = (l[0] * TILE1 + l[1]) * TILE1 + l[2];
    const float wx[2] = {1.f - t[0], t[0]}, wy[2] = {1.f - t[1], t[1]}, wz[2] = {1.f - t[2], t[2]};
#pragma unroll
    for (int c = 0; c < 8; ++c)
      acc_add_signed(lo, hi, base + (c >> 2) * TILE1 * TILE1 + ((c >> 1) & 1) * TILE1 + (c & 1),
                     __float2int_rn(wx[c >> 2] * wy[(c >> 1) & 1] * wz[c & 1] * vs));
  };
  if (cells) {
    // two particles per thread and pass, their loads in flight together
    const uint32_t B = blockDim.x;
    for (uint32_t k0 = s0 + threadIdx.x; k0 < s1; k0 += 2 * B) {
      const bool a1 = k0 + B < s1;
      const uint32_t i0 = __ldg(items + k0), i1 = a1 ? __ldg(items + k0 + B) : 0u;
      const uint32_t c0 = __ldg(cells + k0), c1 = a1 ? __ldg(cells + k0 + B) : 0u;
      float d0[3], d1[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        d0[a] = __ldg(dx + a * N + i0);
        if (a1) d1[a] = __ldg(dx + a * N + i1);
      }
      const float v0 = __ldg(vch + i0), v1 = a1 ? __ldg(vch + i1) : 0.f;
      {
        const int l[3] = {(int)(c0 >> 8), (int)(c0 >> 4) & (TILE - 1), (int)c0 & (TILE - 1)};
        const float t[3] = {d0[0] - floorf(d0[0]), d0[1] - floorf(d0[1]), d0[2] - floorf(d0[2])};
        deposit(l, t, v0);
      }
      if (a1) {
        const int l[3] = {(int)(c1 >> 8), (int)(c1 >> 4) & (TILE - 1), (int)c1 & (TILE - 1)};
        const float t[3] = {d1[0] - floorf(d1[0]), d1[1] - floorf(d1[1]), d1[2] - floorf(d1[2])};
        deposit(l, t, v1);
      }
    }
  } else {
    for (uint32_t k = s0 + threadIdx.x; k < s1; k += blockDim.x) {
      const uint32_t i = __ldg(items + k);
      int l[3];
      float t[3];
      if (!particle_local<false>(dx, N, i, g, o, l, t)) continue;
      deposit(l, t, __ldg(vch + i));
    }
  }
  __syncthreads();
  // this block's channel's output, shell buffer and face counters
  const int ch = blockIdx.x - tile * nch;
  float* out = out_all + ch * M;
  unsigned long long* halo = halo_all + ch * hstride;
  uint32_t* done = done_all ? done_all + (size_t)ch * nt * nt * nt : nullptr;
  paint_writeout_conv(Acc32{lo, hi}, o, tile, g, out, halo,
                      [inv](unsigned long long v) { return from_fix_signed((long long)v, inv); });
  if (done) faces_last(done, halo, g, tile, sm, [&](int u) { body_halo_vec(halo, g, inv, out, sm, u); });
}

// Face cells of the vector paint: signed sums of the covering tiles' shells.
__global__ void __launch_bounds__(768) k_halo_vec(const unsigned long long* __restrict__ halo, Geom g,
                                                  const unsigned* __restrict__ vmax, float* __restrict__ out) {
  __shared__ uint32_t nb[8];
  const int nt = g.nt, nc = g.nc;
  const int tile = blockIdx.x;
  const int tc[3] = {tile / (nt * nt), (tile / nt) % nt, tile % nt};
  if (threadIdx.x < 8) {
    const int b = threadIdx.x;
    const int x = tc[0] - (b >> 2), y = tc[1] - ((b >> 1) & 1), z = tc[2] - (b & 1);
    nb[b] = ((x < 0 ? x + nt : x) * nt + (y < 0 ? y + nt : y)) * nt + (z < 0 ? z + nt : z);
  }
  __syncthreads();
  const int k = threadIdx.x;
  if (k >= NFACE) return;
  int l[3];
  if (k < TILE * TILE) {
    l[0] = 0; l[1] = k >> 4; l[2] = k & 15;
  } else if (k < TILE * TILE + (TILE - 1) * TILE) {
    const int r = k - TILE * TILE;
    l[0] = 1 + (r >> 4); l[1] = 0; l[2] = r & 15;
  } else {
    const int r = k - TILE * TILE - (TILE - 1) * TILE;
    l[0] = 1 + r / (TILE - 1); l[1] = 1 + r % (TILE - 1); l[2] = 0;
  }
  unsigned long long sum = 0;
  for (int b = 0; b < 8; ++b) {
    const int bx = b >> 2, by = (b >> 1) & 1, bz = b & 1;
    if ((bx && l[0]) || (by && l[1]) || (bz && l[2])) continue;
    sum += halo[(size_t)nb[b] * SHELL + shell_index(l[0] + TILE * bx, l[1] + TILE * by, l[2] + TILE * bz)];
  }
  out[((size_t)(tc[0] * TILE + l[0]) * nc + tc[1] * TILE + l[1]) * nc + tc[2] * TILE + l[2]] =
      from_fix_signed((long long)sum, 1.f / signed_scale(*vmax));
}

int launch_gather_adj(const PaintCtx& c, const float* dx, const float* g_rho, const float* F, bool f4,
                      const float* v, float* g_dx, bool accumulate, cudaStream_t s, KScale vk) {
  const int it = readout_iters(c.N);
  if (KDK_BRICK && KdkBrick::fits(c.g.np)) {
    float* vv = const_cast<float*>(v);     // read only without a drift-kick tail
    if (f4)
      k_gather_adj_brick<true><<<KdkBrick::blocks(c.g.np), KB_THREADS, 0, s>>>(dx, c.g, c.N, c.M, g_rho, F, vv,
                                                                              vk, g_dx, accumulate,
                                                                              DriftKickTail{});
    else
      k_gather_adj_brick<false><<<KdkBrick::blocks(c.g.np), KB_THREADS, 0, s>>>(dx, c.g, c.N, c.M, g_rho, F, vv,
                                                                               vk, g_dx, accumulate,
                                                                               DriftKickTail{});
  } else if (vk.fac) {
    return FPM_EINVAL;     // scaled cotangents need the brick gather
  } else if (f4)
    k_gather_adj<true><<<grid_of(c.N, 256 * it), 256, 0, s>>>(dx, c.g, c.N, c.M, g_rho, F, v, g_dx, accumulate, it);
  else
    k_gather_adj<false><<<grid_of(c.N, 256 * it), 256, 0, s>>>(dx, c.g, c.N, c.M, g_rho, F, v, g_dx, accumulate,
                                                               it);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

// Readout transpose of the 3 channels of v into meshes out[3][M]; the tile
// buckets must hold the positions dx (a paint of dx ran last on this ctx).
int launch_gather_adj_dk(const PaintCtx& c, const float* dx, const float* g_rho, const float* F, bool f4, float* gp,
                         KScale vk, float* g_dx, const double* fac, int idr, int ik1, int ik2, unsigned* vmax,
                         cudaStream_t s) {
  if (!(KDK_BRICK && KdkBrick::fits(c.g.np) && f4)) return FPM_ENOTIMPL;
  FPM_CUDA_TRY(cudaMemsetAsync(vmax, 0, sizeof(unsigned), s));
  DriftKickTail dk;
  dk.on = true;
  dk.fac = fac;
  dk.idr = idr;
  dk.ik1 = ik1;
  dk.ik2 = ik2;
  dk.vmax = vmax;
  k_gather_adj_brick<true><<<KdkBrick::blocks(c.g.np), KB_THREADS, 0, s>>>(dx, c.g, c.N, c.M, g_rho, F, gp, vk, g_dx,
                                                                          1, dk);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_paint_vec(const PaintCtx& c, const float* dx, const float* v, KScale vk, unsigned* vmax, float* out,
                     cudaStream_t s, bool vmax_ready, unsigned long long* halo3, uint32_t* done3) {
  if (!vmax_ready) {
    FPM_CUDA_TRY(cudaMemsetAsync(vmax, 0, sizeof(unsigned), s));
    k_maxabs<<<1024, 256, 0, s>>>(v, vk, 3 * c.N, vmax);
    FPM_CUDA_TRY(cudaGetLastError());
  }
  if (halo3 && done3 && c.tile_done && c.ntiles <= VEC3_MAX_TILES) {
    k_paint_vec<<<3 * c.ntiles, PB_THREADS, 0, s>>>(dx, c.N, c.items, c.tile_start, c.g, v, vk, vmax, out, halo3,
                                                    cells_of(c), done3, 3, c.M, paint_halo_elems(c.ntiles));
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  }
  for (int ch = 0; ch < 3; ++ch) {
    k_paint_vec<<<c.ntiles, PB_THREADS, 0, s>>>(dx, c.N, c.items, c.tile_start, c.g, v + ch * c.N, vk, vmax,
                                                out + ch * c.M, c.halo, cells_of(c), c.tile_done, 1, 0, 0);
    FPM_CUDA_TRY(cudaGetLastError());
    if (!c.tile_done) {
      k_halo_vec<<<c.ntiles, 768, 0, s>>>(c.halo, c.g, vmax, out + ch * c.M);
      FPM_CUDA_TRY(cudaGetLastError());
    }
  }
  return FPM_OK;
}

}  // namespace fpm
