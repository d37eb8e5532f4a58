// readout_dev.cuh -- device body of the fused readout + kick + drift over
// Lagrangian bricks (internal), used by the single-simulation kernel and the
// batched persistent step.
#pragma once
#include "cells.cuh"

namespace fpm {

// ---------------------------------------------------------------- readout over Lagrangian bricks
// Readout + kick + drift + next key over compact Lagrangian bricks.  A CTA
// of KB_THREADS takes a brick of X x Y x Z lattice particles (x slowest)
// and walks it IPX iterations per x plane, each warp a 32-particle z
// segment: the force corners its particles gather lie in two x planes of
// about (Y + 1) x (Z + 1) cells at a time, a window that stays in L1 (a
// 16-byte float4 per cell) while the CTA marches through the brick, so each
// force cell is fetched from L2 about once per brick rather than once per z
// line.  The next iteration's dx and p are fetched (streamed, evict-first)
// while the current one gathers.  Arithmetic and outputs are those of
// body_readout<true, true>.  The force mesh is read through the read-only
// path: it must not be written earlier in the same launch.  The drifted
// displacements go to dx_out, which may be dx itself (each particle is read
// before it is written, by the same thread).
constexpr int KB_THREADS = 256;

template <int Z_, int IPX_, int X_>
struct BrickShape {
  static constexpr int Z = Z_;                          // z extent: Z / 32 warps per row
  static constexpr int IPX = IPX_;                      // iterations per x plane
  static constexpr int X = X_;                          // x planes per brick
  static constexpr int RPI = (KB_THREADS / 32) / (Z / 32);   // y rows per iteration
  static constexpr int Y = RPI * IPX;
  static constexpr int ITERS = X * IPX;
  static_assert(Z % 32 == 0 && (KB_THREADS / 32) % (Z / 32) == 0, "brick z extent");
  static __host__ __device__ bool fits(int np) { return np % Z == 0 && np % Y == 0 && np % X == 0; }
  static __host__ __device__ int blocks(int np) { return (np / X) * (np / Y) * (np / Z); }
};

template <class BS>
__device__ __forceinline__ uint32_t brick_particle(int it, int bx, int by, int bz, int np) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int z = bz * BS::Z + (w % (BS::Z / 32)) * 32 + lane;
  const int y = by * BS::Y + (it % BS::IPX) * BS::RPI + w / (BS::Z / 32);
  const int x = bx * BS::X + it / BS::IPX;
  return ((uint32_t)x * np + y) * np + z;
}

template <class BS, int TE = 16>
__device__ __forceinline__ void body_kdk_brick(const float* dx, float* dx_out, float* __restrict__ p,
                                               const float4* __restrict__ F, const Geom& g, size_t N,
                                               const double* __restrict__ fac, int ik1, int ik2, int idr,
                                               uint32_t* __restrict__ keys, uint32_t* __restrict__ tile_count,
                                               int* __restrict__ err, int blk) {
  const int np = g.np, nc = g.nc;
  const int nbz = np / BS::Z, nby = np / BS::Y;
  const int bz = blk % nbz, by = (blk / nbz) % nby, bx = blk / (nbz * nby);
  const float K = (float)((ik1 >= 0 ? fac[ik1] : 0.0) + (ik2 >= 0 ? fac[ik2] : 0.0));
  const float D = idr >= 0 ? (float)fac[idr] : 0.f;
  float dn[3], pn[3];
  {
    const uint32_t i = brick_particle<BS>(0, bx, by, bz, np);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dn[a] = __ldcs(dx + a * N + i);
      pn[a] = __ldcs(p + a * N + i);
    }
  }
#pragma unroll 1
  for (int it = 0; it < BS::ITERS; ++it) {
    const uint32_t i = brick_particle<BS>(it, bx, by, bz, np);
    float d[3] = {dn[0], dn[1], dn[2]}, pp[3] = {pn[0], pn[1], pn[2]};
    if (it + 1 < BS::ITERS) {
      const uint32_t inext = brick_particle<BS>(it + 1, bx, by, bz, np);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        dn[a] = __ldcs(dx + a * N + inext);
        pn[a] = __ldcs(p + a * N + inext);
      }
    }
    int q[3], c[3];
    float t[3];
    lattice_node(i, g, q);
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
    for (int b = 0; b < 8; ++b) {
      const float4 v = __ldg(F + rx[b >> 2] + ry[(b >> 1) & 1] + rz[b & 1]);
      const float wt = wx[b >> 2] * wy[(b >> 1) & 1] * wz[b & 1];
      f[0] = fmaf(wt, v.x, f[0]);
      f[1] = fmaf(wt, v.y, f[1]);
      f[2] = fmaf(wt, v.z, f[2]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float pa = fmaf(K, f[a], pp[a]);
      __stcs(p + a * N + i, pa);
      d[a] = fmaf(D, pa, d[a]);
      __stcs(dx_out + a * N + i, d[a]);
    }
    int tile = 0;
    if (keys) {
#pragma unroll
      for (int a = 0; a < 3; ++a) ok &= cic_cell(d[a], q[a], nc, &c[a], &t[a]);
      const uint32_t key = tile_key<TE>(c, g.nc / TE);
      keys[i] = key;
      tile = key >> (3 * TileC<TE>::LG);
    }
    if (!ok) atomicOr(err, ERR_NAN);
    if (keys) warp_count(tile_count, tile, true);
  }
}

// The single-simulation brick: 4 x 16 x 64 particles per CTA, x slowest.
using KdkBrick = BrickShape<64, 4, 4>;

}  // namespace fpm
