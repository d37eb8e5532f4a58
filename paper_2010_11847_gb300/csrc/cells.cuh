// cells.cuh -- the cell of a particle and its tile-major key (internal):
// lattice node of a particle index, base cell and fraction of a float32
// displacement (cell = wrap(q + floor(dx)), exact in float), the tile-major
// key with TE^3 tiles, and the warp-aggregated tile histogram.  Shared by the
// sort, the paint and the fused readout.
#pragma once
#include "common.cuh"

namespace fpm {

// Geometry of a paint tile of edge TE (16: the cell key's tiles; 8: the
// batched step may bucket and paint small meshes by 8^3 tiles).
template <int TE>
struct TileC {
  static_assert(TE == 8 || TE == 16, "paint tile edge");
  static constexpr int E = TE, E1 = TE + 1, E3 = TE * TE * TE, LG = TE == 8 ? 3 : 4;
  static constexpr int ACC = E1 * E1 * E1;                                        // accumulator cells
  static constexpr int SHELL = 2 * E1 * E1 + 2 * (E - 1) * E1 + 2 * (E - 1) * (E - 1);   // its shell
  static constexpr int NFACE = E * E + (E - 1) * E + (E - 1) * (E - 1);            // lower-face cells
};

// Wrap c into [0, n) for |c| < 2^31 - n (one correction in the common case).
__device__ __forceinline__ int wrapi(int c, int n) {
  if (c < 0) c += n;
  if (c >= n) c -= n;
  if ((unsigned)c >= (unsigned)n) {
    c %= n;
    if (c < 0) c += n;
  }
  return c;
}

__device__ __forceinline__ void lattice_node(uint32_t i, const Geom& g, int* q) {
  const uint32_t ix = fdiv(i, g.div_np2);
  const uint32_t rem = i - ix * g.div_np2.d;
  const uint32_t iy = fdiv(rem, g.div_np);
  const uint32_t iz = rem - iy * g.div_np.d;
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

// Tile-major key of cell c with TE^3 tiles, nt = nc / TE tiles per side.
template <int TE = 16>
__device__ __forceinline__ uint32_t tile_key(const int* c, int nt) {
  using C = TileC<TE>;
  const uint32_t tile = ((uint32_t)(c[0] >> C::LG) * nt + (c[1] >> C::LG)) * nt + (c[2] >> C::LG);
  const uint32_t local = ((c[0] & (TE - 1)) * TE + (c[1] & (TE - 1))) * TE + (c[2] & (TE - 1));
  return tile * C::E3 + local;
}

// Warp-aggregated increment of counter[bucket] for every active lane.
__device__ __forceinline__ void warp_count(uint32_t* counter, int bucket, bool active) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int key = active ? bucket : -1 - lane;
  const unsigned grp = __match_any_sync(full, key);
  if (active && lane == __ffs(grp) - 1) atomicAdd(counter + bucket, (uint32_t)__popc(grp));
}

}  // namespace fpm
