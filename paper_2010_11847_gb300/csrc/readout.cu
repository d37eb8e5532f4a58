// readout.cu -- CIC readout of the force mesh fused with the KDK kick and
// drift and the next step's cell key (Eqs. 1-2 and the CIC interpolation of
// Sec. 2), over compact Lagrangian bricks of 4 x 16 x 64 particles per CTA.
// The device body lives in readout_dev.cuh so that the batched persistent
// step runs the same code.
#include "internal.h"
#include "readout_dev.cuh"

namespace fpm {

__global__ void __launch_bounds__(KB_THREADS) k_kdk_brick(const float* dx, float* dx_out, float* __restrict__ p,
                                                          const float4* __restrict__ F, Geom g, size_t N,
                                                          const double* __restrict__ fac, int ik1, int ik2, int idr,
                                                          uint32_t* __restrict__ keys,
                                                          uint32_t* __restrict__ tile_count, int* __restrict__ err) {
  body_kdk_brick<KdkBrick>(dx, dx_out, p, F, g, N, fac, ik1, ik2, idr, keys, tile_count, err, blockIdx.x);
}

bool kdk_brick_fits(const PaintCtx& c, bool f4) { return f4 && KdkBrick::fits(c.g.np); }

int launch_kdk_brick(const PaintCtx& c, const float* dx, float* dx_out, float* p, const float4* F, const double* fac,
                     int ik1, int ik2, int idr, uint32_t* keys, cudaStream_t s) {
  if (!KdkBrick::fits(c.g.np)) return FPM_EINVAL;
  k_kdk_brick<<<KdkBrick::blocks(c.g.np), KB_THREADS, 0, s>>>(dx, dx_out, p, F, c.g, c.N, fac, ik1, ik2, idr, keys,
                                                              c.tile_count, c.err);
  FPM_CUDA_TRY(cudaGetLastError());
  return FPM_OK;
}

}  // namespace fpm
