// pyramid.cu -- the multi-grid pyramid force (Sec. 3.1 Eqs. 6-9,
// Algorithms 2-3) on one GPU.
//
// Long-range force: the density contrast is REDUCEd `levels` times (stride-2
// convolutions with the order-6 discrete B-spline, binomial weights
// C(6, j)/64) and its force computed on the coarse mesh, in fine-cell units:
// by default with the fine mesh's operator at the same wavenumber (the
// gradient symbol s g(w/s) of Eq. 5 at the fine frequency, s = 2^levels,
// through the three-field spectral passes), or with Eq. 5 in coarse-cell
// units times s.  Short-range force: the fine mesh is cut into split^3 cubic
// blocks, each padded by `halo` cells of its periodic neighbours and treated
// as periodic by its own (local) FFTs.  Algorithm 3 combines
//   F = EXPAND(F_L) + F_S - EXPAND(REDUCE(F_S)).
// By default the band-pass F_S - EXPAND(REDUCE(F_S)) acts on each padded
// block (REDUCE and EXPAND periodic on the block) before its interior is
// kept, and F = EXPAND(F_L) + F_S; otherwise it acts on the assembled F_S,
// evaluated as F = F_S + EXPAND(F_L - REDUCE(F_S)) (EXPAND is linear), one
// EXPAND instead of two.  The last EXPAND pass adds F_S and writes the force
// meshes (planar or float4-interleaved).
//
// Every resampling step is one separable pass along one axis: each output
// element reads 7 (REDUCE) or 3-4 (EXPAND) inputs along that axis, with
// threads running along the contiguous z axis, so the passes are HBM-bound
// streams with the taps served from L1.
#include "internal.h"

namespace fpm {

namespace {

// Order-6 discrete B-spline, C(6, j) / 64 (exact in float).
__constant__ float c_bs[7] = {1.f / 64, 6.f / 64, 15.f / 64, 20.f / 64, 15.f / 64, 6.f / 64, 1.f / 64};

constexpr int RS_THREADS = 256;

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// One REDUCE pass along axis AX over fields of shape [a0][a1][a2] (a2
// fastest; the field index is blockIdx.y): that axis is halved,
//   out[i] = sum_t w_t in[2i + t] - bias   (t = -3..3, periodic),
// or, when `minus_from` is set, out[i] = minus_from[i] - sum_t w_t in[2i + t].
// (minus_from may alias out: each element is read and then written by one thread.)
template <int AX>
__global__ void __launch_bounds__(RS_THREADS) k_reduce_axis(const float* __restrict__ in, float* out,
                                                            const float* minus_from, int a0, int a1,
                                                            int a2, size_t in_fs, size_t out_fs, float bias) {
  const int o0 = AX == 0 ? a0 / 2 : a0, o1 = AX == 1 ? a1 / 2 : a1, o2 = AX == 2 ? a2 / 2 : a2;
  const size_t total = (size_t)o0 * o1 * o2;
  const float* src = in + blockIdx.y * in_fs;
  float* dst = out + blockIdx.y * out_fs;
  const float* sub = minus_from ? minus_from + blockIdx.y * out_fs : nullptr;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % o2);
    const size_t r = e / o2;
    const int j = (int)(r % o1);
    const int i = (int)(r / o1);
    float acc = 0.f;
#pragma unroll
    for (int t = -3; t <= 3; ++t) {
      const int ii = AX == 0 ? wrap(2 * i + t, a0) : i;
      const int jj = AX == 1 ? wrap(2 * j + t, a1) : j;
      const int kk = AX == 2 ? wrap(2 * k + t, a2) : k;
      acc = fmaf(c_bs[t + 3], __ldg(src + ((size_t)ii * a1 + jj) * a2 + kk), acc);
    }
    dst[e] = sub ? sub[e] - acc : acc - bias;
  }
}

// Transposed-convolution tap of output index x (along the doubled axis):
// out[x] = sum_i 2 w_{x - 2i} in[i], |x - 2i| <= 3.  Even x: i = x/2 - 1,
// x/2, x/2 + 1 (w_2, w_0, w_-2); odd x: i = (x-3)/2 .. (x+3)/2 (w_3, w_1,
// w_-1, w_-3).  The factor 2 per axis is Algorithm 2's 8 in 3-D.
template <typename Ld>
__device__ __forceinline__ float expand_taps(int x, int n_in, Ld ld) {
  if ((x & 1) == 0) {
    const int c = x >> 1;
    return 2.f * (c_bs[5] * ld(wrap(c - 1, n_in)) + c_bs[3] * ld(c) + c_bs[1] * ld(wrap(c + 1, n_in)));
  }
  const int c = (x - 3) >> 1;
  return 2.f * (c_bs[6] * ld(wrap(c, n_in)) + c_bs[4] * ld(wrap(c + 1, n_in)) + c_bs[2] * ld(wrap(c + 2, n_in)) +
                c_bs[0] * ld(wrap(c + 3, n_in)));
}

// One EXPAND pass along axis AX over fields [a0][a1][a2] (input shape):
// that axis is doubled.
template <int AX>
__global__ void __launch_bounds__(RS_THREADS) k_expand_axis(const float* __restrict__ in, float* __restrict__ out,
                                                            int a0, int a1, int a2, size_t in_fs, size_t out_fs) {
  const int o0 = AX == 0 ? 2 * a0 : a0, o1 = AX == 1 ? 2 * a1 : a1, o2 = AX == 2 ? 2 * a2 : a2;
  const size_t total = (size_t)o0 * o1 * o2;
  const float* src = in + blockIdx.y * in_fs;
  float* dst = out + blockIdx.y * out_fs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % o2);
    const size_t r = e / o2;
    const int j = (int)(r % o1);
    const int i = (int)(r / o1);
    float v;
    if (AX == 0)
      v = expand_taps(i, a0, [&](int c) { return __ldg(src + ((size_t)c * a1 + j) * a2 + k); });
    else if (AX == 1)
      v = expand_taps(j, a1, [&](int c) { return __ldg(src + ((size_t)i * a1 + c) * a2 + k); });
    else
      v = expand_taps(k, a2, [&](int c) { return __ldg(src + ((size_t)i * a1 + j) * a2 + c); });
    dst[e] = v;
  }
}

// Last EXPAND pass (along z) fused with the sum: F_d = F_S,d + EXPAND(...)_d
// for the three components of every cell, written planar (F[3][n^3]) or as
// float4 (F_x, F_y, F_z, 0).  Input: 3 fields [n][n][n/2].
template <bool F4>
__global__ void __launch_bounds__(RS_THREADS) k_expand_z_final(const float* __restrict__ in, size_t in_fs,
                                                               const float* __restrict__ FS, float* __restrict__ F,
                                                               int n) {
  const size_t M = (size_t)n * n * n;
  const int h = n / 2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < M; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % n);
    const size_t row = e / n;
    float f[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float* src = in + d * in_fs + row * h;
      f[d] = __ldg(FS + d * M + e) + expand_taps(k, h, [&](int c) { return __ldg(src + c); });
    }
    if (F4)
      reinterpret_cast<float4*>(F)[e] = make_float4(f[0], f[1], f[2], 0.f);
    else
      for (int d = 0; d < 3; ++d) F[d * M + e] = f[d];
  }
}

// Last EXPAND pass (along z) of a padded block's band, fused with the
// band-pass and the crop: for the m^3 interior cells of the block (offset
// `halo`), F_S,d = F_b,d - EXPAND(...)_d, written into F_S at (x0, y0, z0).
// in: 3 fields [B][B][B/2]; Fb: 3 fields B^3.
__global__ void __launch_bounds__(RS_THREADS) k_expand_z_bandpass_crop(const float* __restrict__ in, size_t in_fs,
                                                                       const float* __restrict__ Fb,
                                                                       float* __restrict__ FS, int n, int B, int m,
                                                                       int halo, int x0, int y0, int z0) {
  const size_t total = (size_t)m * m * m;
  const size_t MB = (size_t)B * B * B, M = (size_t)n * n * n;
  const int h = B / 2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % m);
    const size_t r = e / m;
    const int b = (int)(r % m);
    const int a = (int)(r / m);
    const size_t row = (size_t)(halo + a) * B + (halo + b);
    const int kz = halo + c;
    const size_t out = ((size_t)(x0 + a) * n + (y0 + b)) * n + (z0 + c);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float* src = in + d * in_fs + row * h;
      FS[d * M + out] = __ldg(Fb + d * MB + row * B + kz) - expand_taps(kz, h, [&](int q) { return __ldg(src + q); });
    }
  }
}

// Padded block: blk[a][b][c] = rho[ox + a][oy + b][oz + c] (periodic), B^3.
__global__ void __launch_bounds__(RS_THREADS) k_block_gather(const float* __restrict__ rho, float* __restrict__ blk,
                                                             int n, int B, int ox, int oy, int oz) {
  const size_t total = (size_t)B * B * B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % B);
    const size_t r = e / B;
    const int b = (int)(r % B);
    const int a = (int)(r / B);
    blk[e] = __ldg(rho + ((size_t)wrap(ox + a, n) * n + wrap(oy + b, n)) * n + wrap(oz + c, n));
  }
}

// Interior m^3 of a block's force (offset `halo`) into F_S at (x0, y0, z0);
// field index = blockIdx.y.
__global__ void __launch_bounds__(RS_THREADS) k_block_scatter(const float* __restrict__ Fb, float* __restrict__ FS,
                                                              int n, int B, int m, int halo, int x0, int y0, int z0) {
  const size_t total = (size_t)m * m * m;
  const float* src = Fb + blockIdx.y * (size_t)B * B * B;
  float* dst = FS + blockIdx.y * (size_t)n * n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % m);
    const size_t r = e / m;
    const int b = (int)(r % m);
    const int a = (int)(r / m);
    dst[((size_t)(x0 + a) * n + (y0 + b)) * n + (z0 + c)] =
        __ldg(src + ((size_t)(halo + a) * B + (halo + b)) * B + (halo + c));
  }
}

int grid_for(size_t total) {
  size_t g = (total + RS_THREADS - 1) / RS_THREADS;
  return (int)(g < 152 * 16 ? (g ? g : 1) : 152 * 16);
}

// Force meshes F[3][n^3] (planar, cell units of this mesh) of density `in`
// with the kernel of tables t (naive Green's function and Eq. 5 gradient:
// through the potential on power-of-two meshes unless `spectral`; the
// three-field spectral passes use t's gradient symbol as it is); coef
// = scale * 1.5 omega_m / n^3 folds the inverse-DFT normalisation and a
// unit scale into the Green's function.
int mesh_force(const FftTables& t, const float* in, float* F, float2* spec, size_t specmax, float coef,
               unsigned* ctr, int* err, cudaStream_t s, int* launches, bool spectral = false) {
  const size_t M = (size_t)t.n * t.n * t.n;
  if (fft_has_potential(t.n) && !spectral) {
    float* phi = reinterpret_cast<float*>(spec + specmax);
    FPM_TRY(fft_pot_forward(t, in, spec, ctr, err, s));
    FPM_TRY(fft_pot_xgreen(t, spec, coef, ctr, err, s));
    FPM_TRY(fft_pot_inverse(t, spec, phi, ctr, err, s));
    *launches += t.n >= 128 ? 4 : 6;
    return fft_pot_gradient(t, phi, F, false, M, s);
  }
  FPM_TRY(fft_zfwd(t, in, spec, 1, 0, 0, s));
  FPM_TRY(fft_y(t, spec, 1, 0, false, s));
  FPM_TRY(fft_xforce(t, spec, spec, specmax, coef, s));
  FPM_TRY(fft_y(t, spec, 3, specmax, true, s));
  *launches += 5;
  return fft_zinv(t, spec, F, 3, specmax, M, s);
}

// `levels` REDUCEs of nf fields of n^3 (stride in_fs) into out (stride
// out_fs, (n >> levels)^3 per field); the first pass subtracts `bias`, the
// last one computes minus_from - result when minus_from is set.
int reduce_levels(const float* in, size_t in_fs, float* out, size_t out_fs, const float* minus_from, int nf, int n,
                  int levels, float bias, float* ping, float* pong, cudaStream_t s, int* launches) {
  int d[3] = {n, n, n};
  const float* cur = in;
  size_t cur_fs = in_fs;
  float* bufs[2] = {ping, pong};
  int which = 0;
  for (int l = 0; l < levels; ++l) {
    for (int ax = 0; ax < 3; ++ax) {
      const bool last = (l == levels - 1) && ax == 2;
      int o[3] = {d[0], d[1], d[2]};
      o[ax] /= 2;
      const size_t ototal = (size_t)o[0] * o[1] * o[2];
      float* dst = last ? out : bufs[which];
      const size_t dst_fs = last ? out_fs : ototal;
      const float b = (l == 0 && ax == 0) ? bias : 0.f;
      const float* sub = last ? minus_from : nullptr;
      dim3 grid(grid_for(ototal), nf);
      if (ax == 0)
        k_reduce_axis<0><<<grid, RS_THREADS, 0, s>>>(cur, dst, sub, d[0], d[1], d[2], cur_fs, dst_fs, b);
      else if (ax == 1)
        k_reduce_axis<1><<<grid, RS_THREADS, 0, s>>>(cur, dst, sub, d[0], d[1], d[2], cur_fs, dst_fs, b);
      else
        k_reduce_axis<2><<<grid, RS_THREADS, 0, s>>>(cur, dst, sub, d[0], d[1], d[2], cur_fs, dst_fs, b);
      FPM_CUDA_TRY(cudaGetLastError());
      ++*launches;
      cur = dst;
      cur_fs = dst_fs;
      which ^= 1;
      d[ax] = o[ax];
    }
  }
  return FPM_OK;
}

// `levels` EXPANDs of 3 fields of n^3 (stride in_fs) but the last pass
// (along z), which `last(cur, cur_fs)` enqueues on the [N][N][N/2] fields.
template <typename Last>
int expand_levels(const float* in, size_t in_fs, int n, int levels, float* ping, float* pong, cudaStream_t s,
                  int* launches, Last last) {
  int d[3] = {n, n, n};
  const float* cur = in;
  size_t cur_fs = in_fs;
  float* bufs[2] = {ping, pong};
  int which = 0;
  for (int l = 0; l < levels; ++l) {
    for (int ax = 0; ax < 3; ++ax) {
      if (l == levels - 1 && ax == 2) {
        FPM_TRY(last(cur, cur_fs));
        ++*launches;
        return FPM_OK;
      }
      int o[3] = {d[0], d[1], d[2]};
      o[ax] *= 2;
      const size_t ototal = (size_t)o[0] * o[1] * o[2];
      float* dst = bufs[which];
      dim3 grid(grid_for(ototal), 3);
      if (ax == 0)
        k_expand_axis<0><<<grid, RS_THREADS, 0, s>>>(cur, dst, d[0], d[1], d[2], cur_fs, ototal);
      else if (ax == 1)
        k_expand_axis<1><<<grid, RS_THREADS, 0, s>>>(cur, dst, d[0], d[1], d[2], cur_fs, ototal);
      else
        k_expand_axis<2><<<grid, RS_THREADS, 0, s>>>(cur, dst, d[0], d[1], d[2], cur_fs, ototal);
      FPM_CUDA_TRY(cudaGetLastError());
      ++*launches;
      cur = dst;
      cur_fs = ototal;
      which ^= 1;
      d[ax] = o[ax];
    }
  }
  return FPM_OK;
}

}  // namespace

int pyramid_create(Pyramid* y, int nc, int levels, int split, int halo, int block_bandpass, int matched) {
  if (levels < 1 || levels > 2 || split < 1 || halo < 0 || nc % split != 0 || (nc >> levels) << levels != nc)
    return FPM_EINVAL;
  const int nco = nc >> levels, m = nc / split, B = m + 2 * halo;
  if (!fft_size_ok(nco) || !fft_size_ok(B)) return FPM_EINVAL;
  if (block_bandpass && (B % (1 << levels) != 0)) return FPM_EINVAL;
  y->block_bandpass = block_bandpass ? 1 : 0;
  y->matched = matched ? 1 : 0;
  y->nc = nc;
  y->levels = levels;
  y->split = split;
  y->halo = halo;
  y->nco = nco;
  y->m = m;
  y->B = B;
  y->spec_co = (size_t)nco * nco * (nco / 2 + 1);
  y->spec_b = (size_t)B * B * (B / 2 + 1);
  const size_t M = (size_t)nc * nc * nc, Mco = (size_t)nco * nco * nco, MB = (size_t)B * B * B;
  FPM_TRY(fft_tables_create(&y->tco, nco, 0, 0, matched ? (double)(1 << levels) : 1.0));
  FPM_TRY(fft_tables_create(&y->tb, B));
  FPM_CUDA_TRY(cudaMalloc(&y->dco, Mco * sizeof(float)));
  FPM_CUDA_TRY(cudaMalloc(&y->sco, 3 * y->spec_co * sizeof(float2)));
  FPM_CUDA_TRY(cudaMalloc(&y->FL, 3 * Mco * sizeof(float)));
  FPM_CUDA_TRY(cudaMalloc(&y->blk, MB * sizeof(float)));
  FPM_CUDA_TRY(cudaMalloc(&y->sb, 3 * y->spec_b * sizeof(float2)));
  FPM_CUDA_TRY(cudaMalloc(&y->Fb, 3 * MB * sizeof(float)));
  FPM_CUDA_TRY(cudaMalloc(&y->FS, 3 * M * sizeof(float)));
  const size_t half = (M > MB ? M : MB) / 2;
  const int Bco = B >> levels;
  const size_t MBco = block_bandpass ? (size_t)Bco * Bco * Bco : 0;
  FPM_CUDA_TRY(cudaMalloc(&y->ping, 3 * half * sizeof(float)));
  FPM_CUDA_TRY(cudaMalloc(&y->pong, 3 * half * sizeof(float)));
  if (block_bandpass) FPM_CUDA_TRY(cudaMalloc(&y->bco, 3 * MBco * sizeof(float)));
  y->bytes = (int64_t)((Mco + 3 * Mco + MB + 3 * MB + 3 * M + 6 * half + 3 * MBco) * sizeof(float) +
                       3 * (y->spec_co + y->spec_b) * sizeof(float2));
  return FPM_OK;
}

void pyramid_destroy(Pyramid* y) {
  if (y->tco.tw) fft_tables_destroy(&y->tco);
  if (y->tb.tw) fft_tables_destroy(&y->tb);
  cudaFree(y->dco);
  cudaFree(y->sco);
  cudaFree(y->FL);
  cudaFree(y->blk);
  cudaFree(y->sb);
  cudaFree(y->Fb);
  cudaFree(y->FS);
  cudaFree(y->ping);
  cudaFree(y->pong);
  cudaFree(y->bco);
  *y = Pyramid();
}

int pyramid_force(const Pyramid& y, const float* rho, float* F, bool f4, double omega_m, unsigned* ctr, int* err,
                  cudaStream_t s, int* launches) {
  const int n = y.nc, nco = y.nco, B = y.B, m = y.m;
  const size_t M = (size_t)n * n * n, Mco = (size_t)nco * nco * nco, MB = (size_t)B * B * B;
  const int Bco = B >> y.levels;
  const size_t MBco = (size_t)Bco * Bco * Bco;
  // long range: F_L = force(REDUCE(rho - 1)) on the coarse mesh, in fine-cell
  // units (the 2^levels of coarse-cell units folded into coef; with matched
  // tables it pairs with their s g(w/s) to give the fine operator)
  FPM_TRY(reduce_levels(rho, M, y.dco, Mco, nullptr, 1, n, y.levels, 1.f, y.ping, y.pong, s, launches));
  const float coef_co = (float)((double)(1 << y.levels) * 1.5 * omega_m / (double)Mco);
  FPM_TRY(mesh_force(y.tco, y.dco, y.FL, y.sco, y.spec_co, coef_co, ctr, err, s, launches, y.matched != 0));
  // short range: local FFTs of the padded blocks, interiors into F_S
  const float coef_b = (float)(1.5 * omega_m / (double)MB);
  for (int bx = 0; bx < y.split; ++bx)
    for (int by = 0; by < y.split; ++by)
      for (int bz = 0; bz < y.split; ++bz) {
        k_block_gather<<<grid_for(MB), RS_THREADS, 0, s>>>(rho, y.blk, n, B, bx * m - y.halo, by * m - y.halo,
                                                           bz * m - y.halo);
        FPM_CUDA_TRY(cudaGetLastError());
        ++*launches;
        FPM_TRY(mesh_force(y.tb, y.blk, y.Fb, y.sb, y.spec_b, coef_b, ctr, err, s, launches));
        if (y.block_bandpass) {
          // F_b - EXPAND(REDUCE(F_b)) on the periodic padded block, interior into F_S
          FPM_TRY(reduce_levels(y.Fb, MB, y.bco, MBco, nullptr, 3, B, y.levels, 0.f, y.ping, y.pong, s, launches));
          FPM_TRY(expand_levels(y.bco, MBco, Bco, y.levels, y.ping, y.pong, s, launches,
                                [&](const float* cur, size_t cur_fs) {
                                  k_expand_z_bandpass_crop<<<grid_for((size_t)m * m * m), RS_THREADS, 0, s>>>(
                                      cur, cur_fs, y.Fb, y.FS, n, B, m, y.halo, bx * m, by * m, bz * m);
                                  FPM_CUDA_TRY(cudaGetLastError());
                                  return FPM_OK;
                                }));
        } else {
          k_block_scatter<<<dim3(grid_for((size_t)m * m * m), 3), RS_THREADS, 0, s>>>(y.Fb, y.FS, n, B, m, y.halo,
                                                                                      bx * m, by * m, bz * m);
          FPM_CUDA_TRY(cudaGetLastError());
          ++*launches;
        }
      }
  // band-pass of the assembled F_S: coarse difference F_L - REDUCE(F_S), written over F_L
  if (!y.block_bandpass)
    FPM_TRY(reduce_levels(y.FS, M, y.FL, Mco, y.FL, 3, n, y.levels, 0.f, y.ping, y.pong, s, launches));
  // EXPAND the coarse field back; the last pass adds F_S and writes F
  return expand_levels(y.FL, Mco, nco, y.levels, y.ping, y.pong, s, launches, [&](const float* cur, size_t cur_fs) {
    if (f4)
      k_expand_z_final<true><<<grid_for(M), RS_THREADS, 0, s>>>(cur, cur_fs, y.FS, F, n);
    else
      k_expand_z_final<false><<<grid_for(M), RS_THREADS, 0, s>>>(cur, cur_fs, y.FS, F, n);
    FPM_CUDA_TRY(cudaGetLastError());
    return FPM_OK;
  });
}

}  // namespace fpm
