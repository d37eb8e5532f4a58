// paint.cu -- cell keys, counting sort, deterministic CIC paint, CIC readout
// fused with the KDK kick and drift (Sec. 2 and Eqs. 1-2).
//
// Sort.  The mesh is cut into 16^3-cell tiles.  Each particle's tile-major
// cell key is computed from its float32 displacement (cell = wrap(q +
// floor(dx)), exact in float), tile counts are histogrammed with
// warp-aggregated atomics into an L2-resident table, scanned, and the
// particles are bucketed by tile.  Inside a tile, a shared-memory counting
// sort by local cell puts them in cell order (with the index tie-fix when
// the caller asks for the permutation).
//
// Paint.  One CTA per tile accumulates the CIC weights of its particles into
// a 17^3 shared-memory block (the tile plus its upper halo) in 2^-40 fixed
// point with int64 atomics, after summing equal-cell runs of a warp with a
// segmented shuffle reduction.  Integer addition is associative, so the
// density does not depend on the order of anything: it is deterministic.
// Cells that only this tile touches are written directly; the shell of the
// 17^3 block goes to a per-tile halo buffer that a second kernel sums over
// the (up to 8) tiles that overlap each lower-face cell.
#include "internal.h"

namespace fpm {

constexpr int PT_THREADS = 256;
constexpr int PCAP = 8192;      // particles per tile sorted in shared memory
constexpr int ACC = TILE1 * TILE1 * TILE1;
constexpr size_t PAINT_SMEM = ACC * sizeof(long long) + TILE3 * sizeof(uint32_t) + PCAP * sizeof(uint32_t);

__device__ __forceinline__ int wrapi(int c, int n) {
  c %= n;
  return c < 0 ? c + n : c;
}

__device__ __forceinline__ void lattice_node(uint32_t i, const Geom& g, int* q) {
  const uint32_t np = g.np;
  const uint32_t ix = i / (np * np);
  const uint32_t rem = i - ix * np * np;
  const uint32_t iy = rem / np;
  const uint32_t iz = rem - iy * np;
  q[0] = ix * g.ratio;
  q[1] = iy * g.ratio;
  q[2] = iz * g.ratio;
}

// Base cell and fraction from a float32 displacement.  Returns false (and
// the cell 0) for a non-finite or absurdly large displacement.
__device__ __forceinline__ bool cic_cell(float d, int q, int nc, int* c, float* t) {
  if (!(fabsf(d) < 1.0e7f)) {
    *c = 0;
    *t = 0.f;
    return false;
  }
  const float fl = floorf(d);
  *c = wrapi(q + (int)fl, nc);
  *t = d - fl;
  return true;
}

__device__ __forceinline__ uint32_t tile_key(const int* c, int nt) {
  const uint32_t tile = ((uint32_t)(c[0] >> 4) * nt + (c[1] >> 4)) * nt + (c[2] >> 4);
  const uint32_t local = ((c[0] & 15) * TILE + (c[1] & 15)) * TILE + (c[2] & 15);
  return tile * TILE3 + local;
}

// Warp-aggregated increment of counter[bucket] for every active lane.
__device__ __forceinline__ void warp_count(uint32_t* counter, int bucket, bool active) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int key = active ? bucket : -1 - lane;
  const unsigned grp = __match_any_sync(full, key);
  if (active && lane == __ffs(grp) - 1) atomicAdd(counter + bucket, (uint32_t)__popc(grp));
}

// ---------------------------------------------------------------- keys + tile histogram
__global__ void k_keys(const float* __restrict__ dx, Geom g, size_t N, uint32_t* __restrict__ keys,
                       uint32_t* __restrict__ tile_count, int* __restrict__ err) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i < N;
  int tile = 0;
  if (active) {
    int q[3], c[3];
    float t;
    lattice_node((uint32_t)i, g, q);
    bool ok = true;
    for (int d = 0; d < 3; ++d) ok &= cic_cell(dx[d * N + i], q[d], g.nc, &c[d], &t);
    if (!ok) atomicOr(err, ERR_NAN);
    const uint32_t key = tile_key(c, g.nt);
    keys[i] = key;
    tile = key >> 12;
  }
  warp_count(tile_count, tile, active);
}

// ---------------------------------------------------------------- scan of tile counts
constexpr int SCAN_THREADS = 1024;
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const uint32_t* __restrict__ count, int ntiles,
                                                             uint32_t* __restrict__ start,
                                                             uint32_t* __restrict__ cursor) {
  __shared__ uint32_t part[SCAN_THREADS];
  const int per = (ntiles + SCAN_THREADS - 1) / SCAN_THREADS;
  const int b = threadIdx.x * per;
  uint32_t s = 0;
  for (int k = 0; k < per && b + k < ntiles; ++k) s += count[b + k];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < SCAN_THREADS; off <<= 1) {      // Hillis-Steele inclusive scan
    const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (int k = 0; k < per && b + k < ntiles; ++k) {
    start[b + k] = run;
    cursor[b + k] = run;
    run += count[b + k];
  }
  if (threadIdx.x == SCAN_THREADS - 1) start[ntiles] = part[SCAN_THREADS - 1];
}

// ---------------------------------------------------------------- bucket by tile
__global__ void k_scatter(const uint32_t* __restrict__ keys, size_t N, uint32_t* __restrict__ cursor,
                          uint2* __restrict__ items) {
  const unsigned full = 0xffffffffu;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool active = i < N;
  const uint32_t key = active ? keys[i] : 0u;
  const int tile = active ? (int)(key >> 12) : -1 - lane;
  const unsigned grp = __match_any_sync(full, tile);
  const int leader = __ffs(grp) - 1;
  uint32_t base = 0;
  if (active && lane == leader) base = atomicAdd(cursor + tile, (uint32_t)__popc(grp));
  base = __shfl_sync(full, base, leader);
  if (active) items[base + __popc(grp & ((1u << lane) - 1u))] = make_uint2((uint32_t)i, key & 4095u);
}

// ---------------------------------------------------------------- fixed point helpers
// w >= 0 float -> round-toward-zero of w * 2^40 as int64, using 32-bit
// conversions only (exact split of the float into high and low words).
__device__ __forceinline__ long long to_fix(float w) {
  const float s = w * 1099511627776.0f;                 // * 2^40, exact
  const float hi_f = floorf(s * 2.3283064365386963e-10f);  // / 2^32, exact
  const float lo_f = s - hi_f * 4294967296.0f;            // exact
  return ((long long)(int)hi_f << 32) + (long long)(unsigned)lo_f;
}

__device__ __forceinline__ float from_fix(long long v) {
  const int hi = (int)(v >> 32);
  const unsigned lo = (unsigned)(v & 0xffffffffll);
  return fmaf((float)hi, 0.00390625f, (float)lo * 9.094947017729282e-13f);   // 2^-8, 2^-40
}

__device__ __forceinline__ int shell_index(int lx, int ly, int lz) {
  // cells of the 17^3 block with a coordinate in {0, 16}
  if (lx == 0 || lx == TILE) return (lx == TILE) * TILE1 * TILE1 + ly * TILE1 + lz;
  if (ly == 0 || ly == TILE) return 2 * TILE1 * TILE1 + (ly == TILE) * (TILE - 1) * TILE1 + (lx - 1) * TILE1 + lz;
  return 2 * TILE1 * TILE1 + 2 * (TILE - 1) * TILE1 + (lz == TILE) * (TILE - 1) * (TILE - 1) +
         (lx - 1) * (TILE - 1) + (ly - 1);
}

__device__ __forceinline__ void shell_decode(int s, int* l) {
  if (s < 2 * TILE1 * TILE1) {
    l[0] = (s >= TILE1 * TILE1) ? TILE : 0;
    s %= TILE1 * TILE1;
    l[1] = s / TILE1;
    l[2] = s % TILE1;
    return;
  }
  s -= 2 * TILE1 * TILE1;
  if (s < 2 * (TILE - 1) * TILE1) {
    l[1] = (s >= (TILE - 1) * TILE1) ? TILE : 0;
    s %= (TILE - 1) * TILE1;
    l[0] = 1 + s / TILE1;
    l[2] = s % TILE1;
    return;
  }
  s -= 2 * (TILE - 1) * TILE1;
  l[2] = (s >= (TILE - 1) * (TILE - 1)) ? TILE : 0;
  s %= (TILE - 1) * (TILE - 1);
  l[0] = 1 + s / (TILE - 1);
  l[1] = 1 + s % (TILE - 1);
}

// Deposit one warp's particles.  `sorted_run` says equal local cells form
// contiguous lane runs, so a segmented shuffle sum can merge them first.
__device__ __forceinline__ void deposit_warp(long long* acc, bool active, int lkey, const int* l,
                                             const float* t, float mass, bool sorted_run) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  long long w[8];
  {
    const float wx[2] = {1.f - t[0], t[0]}, wy[2] = {1.f - t[1], t[1]}, wz[2] = {1.f - t[2], t[2]};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float v = mass * wx[c >> 2] * wy[(c >> 1) & 1] * wz[c & 1];
      w[c] = active ? to_fix(v) : 0ll;
    }
  }
  bool lead = active;
  if (sorted_run) {
    const unsigned grp = __match_any_sync(full, active ? lkey : -1 - lane);
    if (__any_sync(full, __popc(grp) > 1)) {
      const int last = 31 - __clz(grp);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        long long v = w[c];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const long long o = __shfl_down_sync(full, v, off);
          if (lane + off <= last) v += o;
        }
        w[c] = v;
      }
    }
    lead = active && (lane == __ffs(grp) - 1);
  }
  if (lead) {
    const int base = (l[0] * TILE1 + l[1]) * TILE1 + l[2];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int off = (c >> 2) * TILE1 * TILE1 + ((c >> 1) & 1) * TILE1 + (c & 1);
      atomicAdd(reinterpret_cast<unsigned long long*>(acc + base + off), (unsigned long long)w[c]);
    }
  }
}

// Local cell (relative to tile origin o) and fraction of particle i.
__device__ __forceinline__ bool particle_local(const float* __restrict__ dx, size_t N, uint32_t i,
                                               const Geom& g, const int* o, int* l, float* t) {
  int q[3], c[3];
  lattice_node(i, g, q);
  bool ok = true;
  for (int d = 0; d < 3; ++d) ok &= cic_cell(__ldg(dx + d * N + i), q[d], g.nc, &c[d], &t[d]);
  for (int d = 0; d < 3; ++d) {
    l[d] = c[d] - o[d];
    if (l[d] < 0 || l[d] >= TILE) {   // cannot happen for a consistent key; guard anyway
      ok = false;
      l[d] = 0;
    }
  }
  return ok;
}

template <bool PERM>
__global__ void __launch_bounds__(PT_THREADS) k_paint_tiles(const float* __restrict__ dx, size_t N,
                                                            const uint2* __restrict__ items,
                                                            const uint32_t* __restrict__ tile_start, Geom g,
                                                            float* __restrict__ rho, long long* __restrict__ halo,
                                                            uint32_t* __restrict__ perm, int* __restrict__ err,
                                                            int* __restrict__ big_flag) {
  extern __shared__ unsigned char smraw[];
  long long* acc = reinterpret_cast<long long*>(smraw);
  uint32_t* hist = reinterpret_cast<uint32_t*>(acc + ACC);
  uint32_t* sorted = hist + TILE3;
  const int nt = g.nt;
  const int tid = blockIdx.x;
  const int o[3] = {(tid / (nt * nt)) * TILE, ((tid / nt) % nt) * TILE, (tid % nt) * TILE};
  const uint32_t s0 = tile_start[tid], s1 = tile_start[tid + 1];
  const int n = (int)(s1 - s0);
  for (int k = threadIdx.x; k < ACC; k += blockDim.x) acc[k] = 0;
  for (int k = threadIdx.x; k < TILE3; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  bool bad = false;
  if (n <= PCAP) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) atomicAdd(hist + items[s0 + k].y, 1u);
    __syncthreads();
    {   // exclusive scan of the 4096 local-cell counts: 16 per thread
      constexpr int PER = TILE3 / PT_THREADS;
      __shared__ uint32_t part[PT_THREADS];
      uint32_t loc[PER];
      uint32_t s = 0;
      for (int k = 0; k < PER; ++k) {
        loc[k] = hist[threadIdx.x * PER + k];
        s += loc[k];
      }
      part[threadIdx.x] = s;
      __syncthreads();
      for (int off = 1; off < PT_THREADS; off <<= 1) {
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
      const uint2 it = items[s0 + k];
      sorted[atomicAdd(hist + it.y, 1u)] = it.x;
    }
    __syncthreads();
    if (PERM) {   // order equal cells by particle index (hist[c] is now the end of cell c)
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
    }
    const int nw = (n + 31) & ~31;
    for (int k = threadIdx.x; k < nw; k += blockDim.x) {
      const bool active = k < n;
      int l[3] = {0, 0, 0};
      float t[3] = {0.f, 0.f, 0.f};
      if (active) bad |= !particle_local(dx, N, sorted[k], g, o, l, t);
      const int lkey = (l[0] * TILE + l[1]) * TILE + l[2];
      deposit_warp(acc, active, lkey, l, t, g.mass, true);
    }
  } else {
    if (PERM && threadIdx.x == 0) atomicOr(big_flag, 1);
    const int nw = (n + 31) & ~31;
    for (int k = threadIdx.x; k < nw; k += blockDim.x) {
      const bool active = k < n;
      int l[3] = {0, 0, 0};
      float t[3] = {0.f, 0.f, 0.f};
      if (active) bad |= !particle_local(dx, N, items[s0 + k].x, g, o, l, t);
      deposit_warp(acc, active, 0, l, t, g.mass, false);
    }
  }
  if (bad) atomicOr(err, ERR_RANGE);
  __syncthreads();
  // interior cells: final
  const int nc = g.nc;
  for (int k = threadIdx.x; k < (TILE - 1) * (TILE - 1) * (TILE - 1); k += blockDim.x) {
    const int lx = 1 + k / ((TILE - 1) * (TILE - 1));
    const int ly = 1 + (k / (TILE - 1)) % (TILE - 1);
    const int lz = 1 + k % (TILE - 1);
    rho[((size_t)(o[0] + lx) * nc + (o[1] + ly)) * nc + o[2] + lz] =
        from_fix(acc[(lx * TILE1 + ly) * TILE1 + lz]);
  }
  long long* hb = halo + (size_t)tid * SHELL;
  for (int s = threadIdx.x; s < SHELL; s += blockDim.x) {
    int l[3];
    shell_decode(s, l);
    hb[s] = acc[(l[0] * TILE1 + l[1]) * TILE1 + l[2]];
  }
}

// Lower-face cells of every tile: sum the shell partials of the up to 8
// tiles whose 17^3 blocks cover the cell.
__global__ void k_paint_halo(const long long* __restrict__ halo, Geom g, float* __restrict__ rho) {
  const int nt = g.nt, nc = g.nc;
  const int tid = blockIdx.x;
  const int tc[3] = {tid / (nt * nt), (tid / nt) % nt, tid % nt};
  for (int k = threadIdx.x; k < TILE3; k += blockDim.x) {
    const int l[3] = {k >> 8, (k >> 4) & 15, k & 15};
    if (l[0] && l[1] && l[2]) continue;
    long long sum = 0;
    for (int b = 0; b < 8; ++b) {
      const int bb[3] = {b >> 2, (b >> 1) & 1, b & 1};
      bool ok = true;
      for (int d = 0; d < 3; ++d) ok &= !(bb[d] && l[d]);
      if (!ok) continue;
      const int st = ((wrapi(tc[0] - bb[0], nt)) * nt + wrapi(tc[1] - bb[1], nt)) * nt + wrapi(tc[2] - bb[2], nt);
      sum += halo[(size_t)st * SHELL + shell_index(l[0] + TILE * bb[0], l[1] + TILE * bb[1], l[2] + TILE * bb[2])];
    }
    rho[((size_t)(tc[0] * TILE + l[0]) * nc + tc[1] * TILE + l[1]) * nc + tc[2] * TILE + l[2]] = from_fix(sum);
  }
}

// Stable order of one oversized tile for the permutation output: counting
// sort by local cell with a global cursor table, then the index tie-fix.
// One CTA per tile; only launched when some tile exceeded PCAP.
__global__ void k_perm_big(const uint2* __restrict__ items, const uint32_t* __restrict__ tile_start,
                           uint32_t* __restrict__ perm) {
  __shared__ uint32_t cur[TILE3];
  const int tid = blockIdx.x;
  const uint32_t s0 = tile_start[tid], s1 = tile_start[tid + 1];
  if ((int)(s1 - s0) <= PCAP) return;
  for (int k = threadIdx.x; k < TILE3; k += blockDim.x) cur[k] = 0;
  __syncthreads();
  for (uint32_t k = s0 + threadIdx.x; k < s1; k += blockDim.x) atomicAdd(cur + items[k].y, 1u);
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
    const uint2 it = items[k];
    perm[atomicAdd(cur + it.y, 1u)] = it.x;
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

// ---------------------------------------------------------------- readout (+ kick, drift)
// f_i = sum_c W(x_i - c) F_c.  With KDK: p += K f, dx += D p, then the new
// cell key and tile histogram of the drifted particle.
template <bool KDK>
__global__ void k_readout(float* __restrict__ dx, float* __restrict__ p, const float* __restrict__ F, Geom g,
                          size_t N, size_t M, const double* __restrict__ fac, int ik1, int ik2, int idr,
                          float* __restrict__ f_out, uint32_t* __restrict__ keys,
                          uint32_t* __restrict__ tile_count, int* __restrict__ err) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i < N;
  const int nc = g.nc;
  int tile = 0;
  if (active) {
    int q[3], c[3];
    float t[3], d[3];
    lattice_node((uint32_t)i, g, q);
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      d[a] = dx[a * N + i];
      ok &= cic_cell(d[a], q[a], nc, &c[a], &t[a]);
    }
    int c1[3];
    for (int a = 0; a < 3; ++a) c1[a] = (c[a] + 1 == nc) ? 0 : c[a] + 1;
    float f[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int cx = (b & 4) ? c1[0] : c[0], cy = (b & 2) ? c1[1] : c[1], cz = (b & 1) ? c1[2] : c[2];
      const float w = ((b & 4) ? t[0] : 1.f - t[0]) * ((b & 2) ? t[1] : 1.f - t[1]) * ((b & 1) ? t[2] : 1.f - t[2]);
      const size_t idx = ((size_t)cx * nc + cy) * nc + cz;
#pragma unroll
      for (int a = 0; a < 3; ++a) f[a] = fmaf(w, __ldg(F + a * M + idx), f[a]);
    }
    if (!KDK) {
      for (int a = 0; a < 3; ++a) f_out[a * N + i] = f[a];
      if (!ok) atomicOr(err, ERR_NAN);
    } else {
      const float K = (float)((ik1 >= 0 ? fac[ik1] : 0.0) + (ik2 >= 0 ? fac[ik2] : 0.0));
      const float D = idr >= 0 ? (float)fac[idr] : 0.f;
      for (int a = 0; a < 3; ++a) {
        const float pa = fmaf(K, f[a], p[a * N + i]);
        p[a * N + i] = pa;
        d[a] = fmaf(D, pa, d[a]);
        dx[a * N + i] = d[a];
      }
      if (keys) {
        for (int a = 0; a < 3; ++a) ok &= cic_cell(d[a], q[a], nc, &c[a], &t[a]);
        const uint32_t key = tile_key(c, g.nt);
        keys[i] = key;
        tile = key >> 12;
      }
      if (!ok) atomicOr(err, ERR_NAN);
    }
  }
  if (KDK && keys) warp_count(tile_count, tile, active);
}

// ---------------------------------------------------------------- host side
static int grid_of(size_t n, int threads) { return (int)((n + threads - 1) / threads); }

int paint_setup() {
  FPM_CUDA_TRY(cudaFuncSetAttribute(k_paint_tiles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)PAINT_SMEM));
  FPM_CUDA_TRY(cudaFuncSetAttribute(k_paint_tiles<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)PAINT_SMEM));
  return FPM_OK;
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
  k_scatter<<<grid_of(c.N, 256), 256, 0, s>>>(c.keys, c.N, c.tile_cursor, c.items);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_paint_tiles(const PaintCtx& c, const float* dx, float* rho, uint32_t* perm, cudaStream_t s) {
  if (perm) {
    FPM_CUDA_TRY(cudaMemsetAsync(c.big_flag, 0, sizeof(int), s));
    k_paint_tiles<true><<<c.ntiles, PT_THREADS, PAINT_SMEM, s>>>(dx, c.N, c.items, c.tile_start, c.g, rho,
                                                                  c.halo, perm, c.err, c.big_flag);
  } else {
    k_paint_tiles<false><<<c.ntiles, PT_THREADS, PAINT_SMEM, s>>>(dx, c.N, c.items, c.tile_start, c.g, rho,
                                                                   c.halo, nullptr, c.err, c.big_flag);
  }
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_perm_big(const PaintCtx& c, uint32_t* perm, cudaStream_t s) {
  k_perm_big<<<c.ntiles, 256, 0, s>>>(c.items, c.tile_start, perm);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_halo(const PaintCtx& c, float* rho, cudaStream_t s) {
  k_paint_halo<<<c.ntiles, 256, 0, s>>>(c.halo, c.g, rho);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_readout(const PaintCtx& c, const float* F, const float* dx, float* f_out, cudaStream_t s) {
  k_readout<false><<<grid_of(c.N, 256), 256, 0, s>>>(const_cast<float*>(dx), nullptr, F, c.g, c.N, c.M,
                                                     nullptr, -1, -1, -1, f_out, nullptr, nullptr, c.err);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

int launch_kdk(const PaintCtx& c, float* dx, float* p, const float* F, const double* fac, int ik1, int ik2,
               int idr, bool emit_keys, cudaStream_t s) {
  if (emit_keys) FPM_CUDA_TRY(cudaMemsetAsync(c.tile_count, 0, sizeof(uint32_t) * c.ntiles, s));
  k_readout<true><<<grid_of(c.N, 256), 256, 0, s>>>(dx, p, F, c.g, c.N, c.M, fac, ik1, ik2, idr, nullptr,
                                                    emit_keys ? c.keys : nullptr, c.tile_count, c.err);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

}  // namespace fpm
