// paint_dev.cuh -- device bodies of the cell keys, tile sort, deterministic
// CIC paint and fused readout-kick-drift (internal).  Each body takes its
// block index (and any shared memory) explicitly, so that the same code runs
// as its own kernel or as a phase of the batched persistent kernel.  The
// cell and key helpers are in cells.cuh, the brick traversal of the fused
// readout in readout_dev.cuh.
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
#pragma once
#include "cells.cuh"
#include "internal.h"

namespace fpm {

constexpr int PB_THREADS = 512;     // paint CTA (bucket order)
constexpr int PS_THREADS = 256;     // paint CTA (sorted order, permutation output)
constexpr int PCAP = 8192;          // particles per tile sorted in shared memory
constexpr int ACC = TILE1 * TILE1 * TILE1;
constexpr size_t SORTED_SMEM = 2 * ACC * sizeof(uint32_t) + TILE3 * sizeof(uint32_t) + PCAP * sizeof(uint32_t);
constexpr float W_ONE = 16777216.0f;              // 2^24: fixed-point unit of a CIC weight
constexpr float W_INV = 5.9604644775390625e-08f;  // 2^-24
constexpr int NFACE = TILE * TILE + (TILE - 1) * TILE + (TILE - 1) * (TILE - 1);   // 721 lower-face cells

static_assert(TileC<16>::ACC == ACC && TileC<16>::SHELL == SHELL && TileC<16>::NFACE == NFACE, "16^3 tiles");

// ---------------------------------------------------------------- keys + tile histogram
template <int TE = 16>
__device__ __forceinline__ void body_keys(const float* __restrict__ dx, Geom g, size_t N, uint32_t* __restrict__ keys,
                                          uint32_t* __restrict__ tile_count, int* __restrict__ err, int bx) {
  const size_t i = (size_t)bx * blockDim.x + threadIdx.x;
  const bool active = i < N;
  int tile = 0;
  if (active) {
    int q[3], c[3];
    float t;
    lattice_node((uint32_t)i, g, q);
    bool ok = true;
    for (int d = 0; d < 3; ++d) ok &= cic_cell(dx[d * N + i], q[d], g.nc, &c[d], &t);
    if (!ok) atomicOr(err, ERR_NAN);
    const uint32_t key = tile_key<TE>(c, g.nc / TE);
    keys[i] = key;
    tile = key >> (3 * TileC<TE>::LG);
  }
  warp_count(tile_count, tile, active);
}

// ---------------------------------------------------------------- scan of tile counts
// Each warp scans a contiguous segment of the counts in coalesced rounds of
// 32 (shuffle scan with a running carry), the warp totals are scanned in
// shared memory, and a second pass adds each warp's offset.  part: blockDim/32
// + 1 words of shared memory.  With zero_counts the consumed counts are
// cleared for the next histogram.
__device__ __forceinline__ void body_scan_tiles(uint32_t* __restrict__ count, int ntiles, uint32_t* __restrict__ start,
                                                uint32_t* __restrict__ cursor, uint32_t* part, int zero_counts) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int seg = ((ntiles + nw - 1) / nw + 31) & ~31;
  const int b0 = warp * seg, b1 = min(b0 + seg, ntiles);
  uint32_t carry = 0;
  for (int b = b0; b < b1; b += 32) {
    const int i = b + lane;
    const uint32_t v = i < b1 ? __ldcg(count + i) : 0u;
    uint32_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(full, x, off);
      if (lane >= off) x += y;
    }
    if (i < b1) start[i] = carry + x - v;
    carry += __shfl_sync(full, x, 31);
  }
  if (lane == 0) part[warp] = carry;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < nw; ++w) {
      const uint32_t t = part[w];
      part[w] = run;
      run += t;
    }
    part[nw] = run;
  }
  __syncthreads();
  const uint32_t off = part[warp];
  for (int i = b0 + lane; i < b1; i += 32) {
    const uint32_t v = start[i] + off;
    start[i] = v;
    cursor[i] = v;
    if (zero_counts) count[i] = 0u;
  }
  if (threadIdx.x == 0) start[ntiles] = part[nw];
}

// ---------------------------------------------------------------- bucket by tile
// Bucketing by tile, aggregated per Lagrangian cube: work item `item` takes
// the 16 x 16 x CX particles of one lattice block (CX = 8 NT / 256: 8
// per thread), whose cells fall in few tiles.  Each warp groups its 32 keys
// by tile (match_any); the group leader registers the tile in a shared
// open-addressing table and reserves the group's places in that tile's
// shared count; then one global cursor atomic per (block, tile) reserves the
// block's range of the bucket.  A tile that finds the table full takes its
// places with a global atomic per warp group instead.  Beside each item the
// in-tile cell (the key's low 12 bits) goes to cells (if not null).  Order
// inside a bucket is not fixed: the paint's integer sums and the stable sort
// of the permutation output do not depend on it.  NT: the block's threads;
// tbl: 3 SC_TBL words of shared memory.  np must be a multiple of 16.
constexpr int SC_CUBE = 16;
constexpr int SC_PER = 8;
constexpr int SC_TBL = 256;

__host__ __device__ inline int scatter_cube_items(int np, int threads) {
  const int cx = SC_PER * threads / (SC_CUBE * SC_CUBE);
  return (np / cx) * (np / SC_CUBE) * (np / SC_CUBE);
}

// A place at or past np^3 (tile counts that do not match the keys, which
// the callers never produce) is not written: it raises ERR_RANGE instead.
template <int NT, int TE = 16>
__device__ __forceinline__ void body_scatter_cube(const uint32_t* __restrict__ keys, int np,
                                                  uint32_t* __restrict__ cursor, uint32_t* __restrict__ items,
                                                  uint16_t* __restrict__ cells, int item, uint32_t* tbl,
                                                  int* __restrict__ err) {
  const uint32_t nall = (uint32_t)np * np * np;
  uint32_t* t_tile = tbl;
  uint32_t* t_cnt = tbl + SC_TBL;
  uint32_t* t_base = tbl + 2 * SC_TBL;
  const unsigned full = 0xffffffffu;
  const int t = threadIdx.x, lane = t & 31;
  constexpr int nt = NT, cxw = SC_PER * NT / (SC_CUBE * SC_CUBE);   // x extent of the block of particles
  const int nq = np / SC_CUBE;
  const int cz = item % nq, cy = (item / nq) % nq, cx = item / (nq * nq);
  auto index_of = [&](int e) -> uint32_t {
    const int l = e * nt + t;
    const int lx = l >> 8, ly = (l >> 4) & 15, lz = l & 15;
    return ((uint32_t)(cx * cxw + lx) * np + (uint32_t)(cy * SC_CUBE + ly)) * np + (uint32_t)(cz * SC_CUBE + lz);
  };
  uint32_t key[SC_PER];
#pragma unroll
  for (int e = 0; e < SC_PER; ++e) key[e] = __ldcg(keys + index_of(e));
  for (int k = t; k < SC_TBL; k += nt) {
    t_tile[k] = 0xffffffffu;
    t_cnt[k] = 0;
  }
  __syncthreads();
  uint32_t packed[SC_PER];   // slot << 16 | place in the block's range; ~0 once written directly
#pragma unroll
  for (int e = 0; e < SC_PER; ++e) {
    const uint32_t tile = key[e] >> (3 * TileC<TE>::LG);
    const unsigned grp = __match_any_sync(full, tile);
    const int leader = __ffs(grp) - 1;
    int sl = -1;
    uint32_t off = 0;
    if (lane == leader) {
      uint32_t h = (tile * 2654435761u) >> 24;
      for (int probe = 0; probe < SC_TBL; ++probe, h = (h + 1) & (SC_TBL - 1)) {
        const uint32_t prev = atomicCAS(&t_tile[h], 0xffffffffu, tile);
        if (prev == 0xffffffffu || prev == tile) {
          sl = (int)h;
          break;
        }
      }
      off = sl >= 0 ? atomicAdd(&t_cnt[sl], (uint32_t)__popc(grp))
                    : atomicAdd(cursor + tile, (uint32_t)__popc(grp));   // table full: direct
    }
    sl = __shfl_sync(full, sl, leader);
    const uint32_t place = __shfl_sync(full, off, leader) + __popc(grp & ((1u << lane) - 1u));
    if (sl < 0) {
      if (place < nall) {
        items[place] = index_of(e);
        if (cells) cells[place] = (uint16_t)(key[e] & (TileC<TE>::E3 - 1));
      } else {
        atomicOr(err, ERR_RANGE);
      }
      packed[e] = 0xffffffffu;
    } else {
      packed[e] = ((uint32_t)sl << 16) | place;
    }
  }
  __syncthreads();
  for (int k = t; k < SC_TBL; k += nt)
    if (t_tile[k] != 0xffffffffu) t_base[k] = atomicAdd(cursor + t_tile[k], t_cnt[k]);
  __syncthreads();
#pragma unroll
  for (int e = 0; e < SC_PER; ++e)
    if (packed[e] != 0xffffffffu) {
      const uint32_t place = t_base[packed[e] >> 16] + (packed[e] & 0xffffu);
      if (place >= nall) {
        atomicOr(err, ERR_RANGE);
        continue;
      }
      items[place] = index_of(e);
      if (cells) cells[place] = (uint16_t)(key[e] & (TileC<TE>::E3 - 1));
    }
}

// ---------------------------------------------------------------- fixed point
__device__ __forceinline__ float from_fix(unsigned long long v, float mass) {
  const float hi = (float)(uint32_t)(v >> 32);
  const float lo = (float)(uint32_t)(v & 0xffffffffull);
  return fmaf(hi, 256.0f, lo * W_INV) * mass;                // (hi 2^32 + lo) 2^-24
}

// Exact 64-bit accumulation with 32-bit shared atomics: the thread whose
// add wraps the low word carries into the high word.
__device__ __forceinline__ void acc_add(uint32_t* lo, uint32_t* hi, int c, uint32_t w) {
  const uint32_t old = atomicAdd(lo + c, w);
  if (old + w < old) atomicAdd(hi + c, 1u);
}

__device__ __forceinline__ unsigned long long acc_get(const uint32_t* lo, const uint32_t* hi, int c) {
  return ((unsigned long long)hi[c] << 32) | lo[c];
}

// A tile block's shared accumulator of 64-bit fixed-point sums as two
// 32-bit words with an explicit carry (64-bit shared atomic adds measured
// 2.7x slower for the paint on the GB300).
struct Acc32 {
  uint32_t* lo;
  uint32_t* hi;
  __device__ __forceinline__ void add(int c, uint32_t w) const { acc_add(lo, hi, c, w); }
  __device__ __forceinline__ unsigned long long get(int c) const { return acc_get(lo, hi, c); }
  __device__ __forceinline__ void zero(int c) const { lo[c] = hi[c] = 0u; }
};

template <int TE = 16>
__device__ __forceinline__ int shell_index(int lx, int ly, int lz) {
  // cells of the (TE+1)^3 block with a coordinate in {0, TE}
  constexpr int E = TE, E1 = TE + 1;
  if (lx == 0 || lx == E) return (lx == E) * E1 * E1 + ly * E1 + lz;
  if (ly == 0 || ly == E) return 2 * E1 * E1 + (ly == E) * (E - 1) * E1 + (lx - 1) * E1 + lz;
  return 2 * E1 * E1 + 2 * (E - 1) * E1 + (lz == E) * (E - 1) * (E - 1) + (lx - 1) * (E - 1) + (ly - 1);
}

template <int TE = 16>
__device__ __forceinline__ void shell_decode(int s, int* l) {
  constexpr int E = TE, E1 = TE + 1;
  if (s < 2 * E1 * E1) {
    l[0] = (s >= E1 * E1) ? E : 0;
    s %= E1 * E1;
    l[1] = s / E1;
    l[2] = s % E1;
    return;
  }
  s -= 2 * E1 * E1;
  if (s < 2 * (E - 1) * E1) {
    l[1] = (s >= (E - 1) * E1) ? E : 0;
    s %= (E - 1) * E1;
    l[0] = 1 + s / E1;
    l[2] = s % E1;
    return;
  }
  s -= 2 * (E - 1) * E1;
  l[2] = (s >= (E - 1) * (E - 1)) ? E : 0;
  s %= (E - 1) * (E - 1);
  l[0] = 1 + s / (E - 1);
  l[1] = 1 + s % (E - 1);
}

// Deposit one warp's particles.  When the warp holds long runs of the same
// local cell in adjacent lanes (at most MERGE_RUNS distinct runs: dense
// clumps, where same-address atomics would serialise), each run is summed
// first (one redux.sync per corner over the run's lanes; a run of <= 32
// weights of <= 2^24 fits 32 bits) and its head lane adds the 8 corner sums;
// otherwise every lane adds its own.
constexpr int MERGE_RUNS = 8;
template <class A, int TE = 16>
__device__ __forceinline__ void deposit_warp(const A& acc, bool active, const int* l, const float* t) {
  constexpr int E = TE, E1 = TE + 1;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  uint32_t w[8];
  {
    const float wx[2] = {1.f - t[0], t[0]}, wy[2] = {1.f - t[1], t[1]}, wz[2] = {1.f - t[2], t[2]};
#pragma unroll
    for (int c = 0; c < 8; ++c)
      w[c] = active ? __float2uint_rn(wx[c >> 2] * wy[(c >> 1) & 1] * wz[c & 1] * W_ONE) : 0u;
  }
  const int key = active ? (l[0] * E + l[1]) * E + l[2] : -1 - lane;
  const int prev = __shfl_up_sync(full, key, 1);
  const bool head = (lane == 0) || (prev != key);
  const unsigned heads = __ballot_sync(full, head);
  const int base = (l[0] * E1 + l[1]) * E1 + l[2];
  if (__popc(heads) > MERGE_RUNS) {
    if (active) {
#pragma unroll
      for (int c = 0; c < 8; ++c) acc.add(base + (c >> 2) * E1 * E1 + ((c >> 1) & 1) * E1 + (c & 1), w[c]);
    }
    return;
  }
  // the lane's run is lanes [first, end): first = its head, end = next head
  const unsigned after = heads & ~((2u << lane) - 1u);
  const int end = after ? __ffs(after) - 1 : 32;
  const int first = 31 - __clz(heads & ((2u << lane) - 1u));
  const unsigned run = (end == 32 ? full : ((1u << end) - 1u)) & ~((1u << first) - 1u);
#pragma unroll
  for (int c = 0; c < 8; ++c) w[c] = __reduce_add_sync(run, w[c]);
  if (active && head) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc.add(base + (c >> 2) * E1 * E1 + ((c >> 1) & 1) * E1 + (c & 1), w[c]);
  }
}

__device__ __forceinline__ void deposit_warp(uint32_t* lo, uint32_t* hi, bool active, const int* l,
                                             const float* t) {
  deposit_warp(Acc32{lo, hi}, active, l, t);
}

// Load of particle data: through the read-only path (COH = false), or
// L2-coherent when another block of the same launch wrote it (COH = true).
template <bool COH, typename T>
__device__ __forceinline__ T ld_part(const T* p) {
  if (COH) return __ldcg(p);
  return __ldg(p);
}

// Local cell (relative to tile origin o) and fraction of particle i at
// displacement d.
template <int TE = 16>
__device__ __forceinline__ bool local_cell(const float* d, uint32_t i, const Geom& g, const int* o, int* l,
                                           float* t) {
  int q[3], c[3];
  lattice_node(i, g, q);
  bool ok = true;
  for (int a = 0; a < 3; ++a) ok &= cic_cell(d[a], q[a], g.nc, &c[a], &t[a]);
  for (int a = 0; a < 3; ++a) {
    l[a] = c[a] - o[a];
    if (l[a] < 0 || l[a] >= TE) {     // cannot happen for a consistent key; guard anyway
      ok = false;
      l[a] = 0;
    }
  }
  return ok;
}

template <bool COH, int TE = 16>
__device__ __forceinline__ bool particle_local(const float* __restrict__ dx, size_t N, uint32_t i,
                                               const Geom& g, const int* o, int* l, float* t) {
  float d[3];   // the three gathers are issued back to back
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = ld_part<COH>(dx + a * N + i);
  return local_cell<TE>(d, i, g, o, l, t);
}

// Write the tile's interior cells (final) and its (TE+1)^3 shell (partials).
// The tile's own TE^3 cells go one z row per TE lanes (blockDim.x a multiple
// of TE): interior cells to rho, lower-face cells to the shell; then the
// cells of the block with a coordinate equal to TE (the upper halo).
template <class A, int TE = 16, class Conv>
__device__ __forceinline__ void paint_writeout_conv(const A& acc, const int* o, int tile, const Geom& g,
                                                    float* __restrict__ rho, unsigned long long* __restrict__ halo,
                                                    Conv conv) {
  constexpr int E = TE, E1 = TE + 1, LG = TileC<TE>::LG;
  const int nc = g.nc;
  unsigned long long* hb = halo + (size_t)tile * TileC<TE>::SHELL;
  const int lz = threadIdx.x & (E - 1);
  float* rb = rho + ((size_t)o[0] * nc + o[1]) * nc + o[2] + lz;
  for (int r = threadIdx.x >> LG; r < E * E; r += blockDim.x >> LG) {
    const int lx = r >> LG, ly = r & (E - 1);
    const unsigned long long v = acc.get((lx * E1 + ly) * E1 + lz);
    if (lx && ly && lz)
      rb[(lx * nc + ly) * nc] = conv(v);
    else
      hb[shell_index<TE>(lx, ly, lz)] = v;
  }
  constexpr int UP = E1 * E1 + E * E1 + E * E;     // cells with a coordinate equal to E
  for (int k = threadIdx.x; k < UP; k += blockDim.x) {
    int l[3];
    if (k < E1 * E1) {
      l[0] = E;
      l[1] = k / E1;
      l[2] = k - l[1] * E1;
    } else if (k < E1 * E1 + E * E1) {
      const int r = k - E1 * E1;
      l[0] = r / E1;
      l[1] = E;
      l[2] = r - l[0] * E1;
    } else {
      const int r = k - E1 * E1 - E * E1;
      l[0] = r >> LG;
      l[1] = r & (E - 1);
      l[2] = E;
    }
    hb[shell_index<TE>(l[0], l[1], l[2])] = acc.get((l[0] * E1 + l[1]) * E1 + l[2]);
  }
}

template <class A, int TE = 16>
__device__ __forceinline__ void paint_writeout(const A& acc, const int* o, int tile, const Geom& g,
                                               float* __restrict__ rho, unsigned long long* __restrict__ halo) {
  const float mass = g.mass;
  paint_writeout_conv<A, TE>(acc, o, tile, g, rho, halo, [mass](unsigned long long v) { return from_fix(v, mass); });
}

__device__ __forceinline__ void paint_writeout(const uint32_t* lo, const uint32_t* hi, const int* o, int tile,
                                               const Geom& g, float* __restrict__ rho,
                                               unsigned long long* __restrict__ halo) {
  paint_writeout(Acc32{const_cast<uint32_t*>(lo), const_cast<uint32_t*>(hi)}, o, tile, g, rho, halo);
}

// Hot-path paint: one CTA per tile of edge TE, particles in bucket order.
template <bool COH, class A, int TE = 16>
__device__ __forceinline__ void body_paint_bucket_acc(const float* __restrict__ dx, size_t N,
                                                      const uint32_t* __restrict__ items,
                                                      const uint32_t* __restrict__ tile_start, Geom g,
                                                      float* __restrict__ rho, unsigned long long* __restrict__ halo,
                                                      int* __restrict__ err, const A& acc, int bx,
                                                      const uint16_t* __restrict__ cells = nullptr) {
  using C = TileC<TE>;
  const int nt = g.nc / TE;
  const int tile = bx;
  const int o[3] = {(tile / (nt * nt)) * TE, ((tile / nt) % nt) * TE, (tile % nt) * TE};
  const uint32_t s0 = tile_start[tile], s1 = tile_start[tile + 1];
  const int n = (int)(s1 - s0);
  for (int k = threadIdx.x; k < C::ACC; k += blockDim.x) acc.zero(k);
  __syncthreads();
  bool bad = false;
  const int nw = (n + 31) & ~31;
  if (cells) {
    // two particles per thread and pass: both items' loads, then both
    // particles' dx gathers, are in flight together
    for (int k0 = threadIdx.x; k0 < nw; k0 += 2 * blockDim.x) {
      const int k1 = k0 + blockDim.x;          // k1 < nw is uniform over the warp
      const bool a0 = k0 < n, a1 = k1 < n;
      const uint32_t i0 = a0 ? ld_part<COH>(items + s0 + k0) : 0u, i1 = a1 ? ld_part<COH>(items + s0 + k1) : 0u;
      const uint32_t c0 = a0 ? ld_part<COH>(cells + s0 + k0) : 0u, c1 = a1 ? ld_part<COH>(cells + s0 + k1) : 0u;
      float d0[3] = {0.f, 0.f, 0.f}, d1[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a0) d0[a] = ld_part<COH>(dx + a * N + i0);
        if (a1) d1[a] = ld_part<COH>(dx + a * N + i1);
      }
      {
        const int l[3] = {(int)(c0 >> (2 * C::LG)), (int)(c0 >> C::LG) & (TE - 1), (int)c0 & (TE - 1)};
        const float t[3] = {d0[0] - floorf(d0[0]), d0[1] - floorf(d0[1]), d0[2] - floorf(d0[2])};
        deposit_warp<A, TE>(acc, a0, l, t);
      }
      if (k1 < nw) {
        const int l[3] = {(int)(c1 >> (2 * C::LG)), (int)(c1 >> C::LG) & (TE - 1), (int)c1 & (TE - 1)};
        const float t[3] = {d1[0] - floorf(d1[0]), d1[1] - floorf(d1[1]), d1[2] - floorf(d1[2])};
        deposit_warp<A, TE>(acc, a1, l, t);
      }
    }
  } else {
    for (int k = threadIdx.x; k < nw; k += blockDim.x) {
      const bool active = k < n;
      int l[3] = {0, 0, 0};
      float t[3] = {0.f, 0.f, 0.f};
      if (active) bad |= !particle_local<COH, TE>(dx, N, ld_part<COH>(items + s0 + k), g, o, l, t);
      deposit_warp<A, TE>(acc, active, l, t);
    }
  }
  if (bad) atomicOr(err, ERR_RANGE);
  __syncthreads();
  paint_writeout<A, TE>(acc, o, tile, g, rho, halo);
}

template <bool COH = false>
__device__ __forceinline__ void body_paint_bucket(const float* __restrict__ dx, size_t N,
                                                  const uint32_t* __restrict__ items,
                                                  const uint32_t* __restrict__ tile_start, Geom g,
                                                  float* __restrict__ rho, unsigned long long* __restrict__ halo,
                                                  int* __restrict__ err, uint32_t* lo, uint32_t* hi, int bx) {
  body_paint_bucket_acc<COH>(dx, N, items, tile_start, g, rho, halo, err, Acc32{lo, hi}, bx);
}

// Lower-face cells of every tile: sum the shell partials of the up to 8
// tiles whose (TE+1)^3 blocks cover the cell.  One thread per face cell.
// nb: 8 words of shared memory.
// In-tile coordinates of lower-face cell k < NFACE: the x = 0 face, then
// y = 0 (x >= 1), then z = 0 (x, y >= 1).
template <int TE = 16>
__device__ __forceinline__ void face_cell(int k, int* l) {
  constexpr int E = TE, LG = TileC<TE>::LG;
  if (k < E * E) {
    l[0] = 0;
    l[1] = k >> LG;
    l[2] = k & (E - 1);
  } else if (k < E * E + (E - 1) * E) {
    const int r = k - E * E;
    l[0] = 1 + (r >> LG);
    l[1] = 0;
    l[2] = r & (E - 1);
  } else {
    const int r = k - E * E - (E - 1) * E;
    l[0] = 1 + r / (E - 1);
    l[1] = 1 + r % (E - 1);
    l[2] = 0;
  }
}

template <int TE = 16, class Conv>
__device__ __forceinline__ void tile_face_sums(const unsigned long long* __restrict__ halo, const Geom& g,
                                               float* __restrict__ rho, uint32_t* nb, int bx, Conv conv) {
  using C = TileC<TE>;
  constexpr int E = TE, E1 = TE + 1, LG = C::LG;
  // shell offsets: x faces (lx = 0, E), y faces (lx in [1, E)), z faces (lx, ly in [1, E))
  constexpr int SX = E1 * E1, SY = 2 * E1 * E1, SYE = SY + (E - 1) * E1, SZ = SY + 2 * (E - 1) * E1,
                SZE = SZ + (E - 1) * (E - 1);
  const int nc = g.nc, nt = nc / TE;
  const int tile = bx;
  const int tc[3] = {tile / (nt * nt), (tile / nt) % nt, tile % nt};
  if (threadIdx.x < 8) {
    const int b = threadIdx.x;
    const int x = tc[0] - (b >> 2), y = tc[1] - ((b >> 1) & 1), z = tc[2] - (b & 1);
    nb[b] = ((x < 0 ? x + nt : x) * nt + (y < 0 ? y + nt : y)) * nt + (z < 0 ? z + nt : z);
  }
  __syncthreads();
  // partial of cell s of the shell of lower neighbour b (bit 2: -x, bit 1: -y, bit 0: -z)
  auto H = [&](int b, int s) { return __ldcg(halo + (size_t)nb[b] * C::SHELL + s); };
  float* rt = rho + ((size_t)tc[0] * E * nc + tc[1] * E) * nc + tc[2] * E;
  for (int k = threadIdx.x; k < C::NFACE; k += blockDim.x) {
    unsigned long long sum;
    int l0, l1, l2;
    if (k < E * E) {                       // x = 0 face
      l0 = 0;
      l1 = k >> LG;
      l2 = k & (E - 1);
      sum = H(0, l1 * E1 + l2) + H(4, SX + l1 * E1 + l2);
      if (l1 == 0) sum += H(2, E * E1 + l2) + H(6, SX + E * E1 + l2);
      if (l2 == 0) sum += H(1, l1 * E1 + E) + H(5, SX + l1 * E1 + E);
      if (l1 == 0 && l2 == 0) sum += H(3, E * E1 + E) + H(7, SX + E * E1 + E);
    } else if (k < E * E + (E - 1) * E) {  // y = 0 face, lx >= 1
      const int r = k - E * E;
      l0 = 1 + (r >> LG);
      l1 = 0;
      l2 = r & (E - 1);
      sum = H(0, SY + (l0 - 1) * E1 + l2) + H(2, SYE + (l0 - 1) * E1 + l2);
      if (l2 == 0) sum += H(1, SY + (l0 - 1) * E1 + E) + H(3, SYE + (l0 - 1) * E1 + E);
    } else {                               // z = 0 face, lx, ly >= 1
      const int r = k - E * E - (E - 1) * E;
      l0 = 1 + r / (E - 1);
      l1 = 1 + r % (E - 1);
      l2 = 0;
      sum = H(0, SZ + (l0 - 1) * (E - 1) + (l1 - 1)) + H(1, SZE + (l0 - 1) * (E - 1) + (l1 - 1));
    }
    rt[(l0 * nc + l1) * nc + l2] = conv(sum);
  }
}

template <int TE = 16>
__device__ __forceinline__ void body_paint_halo(const unsigned long long* __restrict__ halo, Geom g,
                                                float* __restrict__ rho, uint32_t* nb, int bx) {
  const float mass = g.mass;
  tile_face_sums<TE>(halo, g, rho, nb, bx, [mass](unsigned long long v) { return from_fix(v, mass); });
}

// Faces summed by the last contributor.  A tile's lower-face cells receive
// the shells of the tile and of its 7 lower neighbours; after a block has
// written its shell it counts it toward the 8 tiles T + {0,1}^3 its 17^3
// block overlaps, and the block whose count completes a tile (the 8th)
// sums that tile's faces at once, while the partials are still in L2 --
// no separate launch and no waiting.  Release: every thread's stores, block
// barrier, fence, count; acquire: count seen at 7, fence, block barrier.
// The finisher resets the count for the next paint.  sm: 24 words of
// shared memory.
template <class Fn>
__device__ __forceinline__ void faces_last(uint32_t* __restrict__ done, const unsigned long long* halo,
                                           const Geom& g, int tile, uint32_t* sm, Fn sum_faces) {
  const int nt = g.nt;
  uint32_t* list = sm + 8;           // up to 8 completed tiles (sm[0..7]: the face sum's neighbours)
  __syncthreads();
  if (threadIdx.x < 32) {
    // lanes 0..7 count the block toward the 8 tiles T + {0,1}^3 at once
    const int b = threadIdx.x;
    bool last = false;
    uint32_t u = 0;
    if (b < 8) {
      const int tc[3] = {tile / (nt * nt), (tile / nt) % nt, tile % nt};
      const int x = tc[0] + (b >> 2), y = tc[1] + ((b >> 1) & 1), z = tc[2] + (b & 1);
      u = (uint32_t)(((x == nt ? 0 : x) * nt + (y == nt ? 0 : y)) * nt + (z == nt ? 0 : z));
      __threadfence();
      last = atomicAdd(done + u, 1u) == 7u;
      __threadfence();
    }
    const unsigned m = __ballot_sync(0xffffffffu, last);
    if (last) list[__popc(m & ((1u << b) - 1u))] = u;
    if (b == 0) sm[16] = __popc(m);
  }
  __syncthreads();
  const uint32_t nl = sm[16];
  for (uint32_t k = 0; k < nl; ++k) {
    const int u = (int)list[k];
    sum_faces(u);
    __syncthreads();
    if (threadIdx.x == 0) done[u] = 0u;
  }
}

__device__ __forceinline__ void paint_faces_last(uint32_t* __restrict__ done, const unsigned long long* halo,
                                                 const Geom& g, float* __restrict__ rho, int tile, uint32_t* sm) {
  faces_last(done, halo, g, tile, sm, [&](int u) { body_paint_halo(halo, g, rho, sm, u); });
}

// ---------------------------------------------------------------- readout (+ kick, drift)
// f_i = sum_c W(x_i - c) F_c.  With KDK: p += K f, dx += D p, then the new
// cell key and tile histogram of the drifted particle.
// Force at CIC corner `idx`: three separate meshes, or interleaved float4.
template <bool F4, bool COH>
__device__ __forceinline__ void corner_force(const float* __restrict__ F, size_t M, size_t idx, float w,
                                             float* f) {
  if (F4) {
    const float4 v = ld_part<COH>(reinterpret_cast<const float4*>(F) + idx);
    f[0] = fmaf(w, v.x, f[0]);
    f[1] = fmaf(w, v.y, f[1]);
    f[2] = fmaf(w, v.z, f[2]);
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) f[a] = fmaf(w, ld_part<COH>(F + a * M + idx), f[a]);
  }
}

template <bool KDK, bool F4, bool COH = false, int TE = 16>
__device__ __forceinline__ void body_readout(float* __restrict__ dx, float* __restrict__ p,
                                                 const float* __restrict__ F, Geom g, size_t N, size_t M,
                                                 const double* __restrict__ fac, int ik1, int ik2, int idr,
                                                 float* __restrict__ f_out, uint32_t* __restrict__ keys,
                                                 uint32_t* __restrict__ tile_count, int* __restrict__ err,
                                                 int iters, int bx) {
  // each CTA walks a contiguous chunk of iters*256 particles, so that the
  // force rows its neighbouring lattice rows share stay in its L1; the next
  // chunk's dx and p are fetched while the current one gathers its forces.
  // The particle arrays are streamed (evict-first) so that L2 keeps the
  // force mesh.
  const int nc = g.nc;
  float K = 0.f, D = 0.f;
  if (KDK) {
    K = (float)((ik1 >= 0 ? fac[ik1] : 0.0) + (ik2 >= 0 ? fac[ik2] : 0.0));
    D = idr >= 0 ? (float)fac[idr] : 0.f;
  }
  const size_t c0 = (size_t)bx * iters * blockDim.x;
  float dn[3] = {0.f, 0.f, 0.f}, pn[3] = {0.f, 0.f, 0.f};
  {
    const size_t i = c0 + threadIdx.x;
    if (i < N) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        dn[a] = __ldcs(dx + a * N + i);
        if (KDK) pn[a] = __ldcs(p + a * N + i);
      }
    }
  }
  for (int it = 0; it < iters; ++it) {
    if (c0 + (size_t)it * blockDim.x >= N) break;
    const size_t i = c0 + (size_t)it * blockDim.x + threadIdx.x;
    const bool active = i < N;
    float d[3] = {dn[0], dn[1], dn[2]}, pp[3] = {pn[0], pn[1], pn[2]};
    const size_t inext = i + blockDim.x;
    if (it + 1 < iters && inext < N) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        dn[a] = __ldcs(dx + a * N + inext);
        if (KDK) pn[a] = __ldcs(p + a * N + inext);
      }
    }
    int tile = 0;
    if (active) {
      int q[3], c[3];
      float t[3];
      lattice_node((uint32_t)i, g, q);
      bool ok = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) ok &= cic_cell(d[a], q[a], nc, &c[a], &t[a]);
      const int cx1 = (c[0] + 1 == nc) ? 0 : c[0] + 1;
      const int cy1 = (c[1] + 1 == nc) ? 0 : c[1] + 1;
      const int cz1 = (c[2] + 1 == nc) ? 0 : c[2] + 1;
      const size_t rx[2] = {(size_t)c[0] * nc * nc, (size_t)cx1 * nc * nc};
      const int ry[2] = {c[1] * nc, cy1 * nc};
      const int rz[2] = {c[2], cz1};
      const float wx[2] = {1.f - t[0], t[0]}, wy[2] = {1.f - t[1], t[1]}, wz[2] = {1.f - t[2], t[2]};
      float f[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int b = 0; b < 8; ++b)
        corner_force<F4, COH>(F, M, rx[b >> 2] + ry[(b >> 1) & 1] + rz[b & 1],
                         wx[b >> 2] * wy[(b >> 1) & 1] * wz[b & 1], f);
      if (!KDK) {
#pragma unroll
        for (int a = 0; a < 3; ++a) f_out[a * N + i] = f[a];
      } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float pa = fmaf(K, f[a], pp[a]);
          __stcs(p + a * N + i, pa);
          d[a] = fmaf(D, pa, d[a]);
          __stcs(dx + a * N + i, d[a]);
        }
        if (keys) {
#pragma unroll
          for (int a = 0; a < 3; ++a) ok &= cic_cell(d[a], q[a], nc, &c[a], &t[a]);
          const uint32_t key = tile_key<TE>(c, g.nc / TE);
          keys[i] = key;
          tile = key >> (3 * TileC<TE>::LG);
        }
      }
      if (!ok) atomicOr(err, ERR_NAN);
    }
    if (KDK && keys) warp_count(tile_count, tile, active);
  }
}


}  // namespace fpm
