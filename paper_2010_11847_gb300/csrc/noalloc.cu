// noalloc.cu -- a CIC paint that allocates no device memory.
//
// Some callers cannot call cudaMalloc: host applications or plugins that
// hand out every byte of device memory themselves (a fixed budget or their
// own pool), and latency-critical loops in which cudaMalloc's implicit
// device synchronisation is not acceptable.  fpm_paint_noalloc serves them:
// it runs the same deterministic sort-and-paint kernels as fpm_paint, but
// its scratch (cell keys, tile buckets, tile counters, the paint's
// tile-face partial sums and the error flag) lives in one file-scope
// __device__ array of fixed size, NOALLOC_SCRATCH_BYTES, that every GPU
// which loads the library holds until the process exits.
//
// In host code the array's name is only a host-side stand-in, not a device
// address: each call looks the device address up with cudaGetSymbolAddress
// (a lookup that allocates nothing) with the caller's device current, so the
// address is right on every device and after a device reset.  The first
// call on a device may load the library's device code there.
#include "internal.h"

namespace fpm {

constexpr int NOALLOC_MAX_N = 64;                         // np <= 64 and nc <= 64
constexpr size_t NOALLOC_MAX_PARTICLES = (size_t)NOALLOC_MAX_N * NOALLOC_MAX_N * NOALLOC_MAX_N;
constexpr int NOALLOC_MAX_TILES = (NOALLOC_MAX_N / TILE) * (NOALLOC_MAX_N / TILE) * (NOALLOC_MAX_N / TILE);

// byte offsets of the scratch pieces (each 256-byte aligned)
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t OFF_KEYS = 0;
constexpr size_t OFF_ITEMS = OFF_KEYS + align256(NOALLOC_MAX_PARTICLES * sizeof(uint32_t));
constexpr size_t OFF_COUNT = OFF_ITEMS + align256(NOALLOC_MAX_PARTICLES * sizeof(uint32_t));
constexpr size_t OFF_START = OFF_COUNT + align256(NOALLOC_MAX_TILES * sizeof(uint32_t));
constexpr size_t OFF_CURSOR = OFF_START + align256((NOALLOC_MAX_TILES + 1) * sizeof(uint32_t));
constexpr size_t OFF_HALO = OFF_CURSOR + align256(NOALLOC_MAX_TILES * sizeof(uint32_t));
constexpr size_t OFF_FLAGS = OFF_HALO + align256((size_t)NOALLOC_MAX_TILES * SHELL * sizeof(unsigned long long));
constexpr size_t NOALLOC_SCRATCH_BYTES = OFF_FLAGS + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
// Device address of the scratch array on the current device.
int scratch_address(unsigned char** out) {
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return FPM_ECUDA;
  }
  *out = static_cast<unsigned char*>(ptr);
  return FPM_OK;
}
}  // namespace

}  // namespace fpm

using namespace fpm;

extern "C" int fpm_paint_noalloc(int np, int nc, const float* dx, float* rho, void* stream) {
  if (!dx || !rho) return FPM_EINVAL;
  if (!fft_size_ok(np) || !fft_size_ok(nc) || nc % np != 0 || nc / np > 4 || nc % TILE != 0 ||
      np > NOALLOC_MAX_N || nc > NOALLOC_MAX_N)
    return FPM_EINVAL;
  unsigned char* base = nullptr;
  FPM_TRY(scratch_address(&base));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  PaintCtx c;
  c.g = make_geom(np, nc);
  c.N = (size_t)np * np * np;
  c.M = (size_t)nc * nc * nc;
  c.ntiles = c.g.nt * c.g.nt * c.g.nt;
  c.keys = reinterpret_cast<uint32_t*>(base + OFF_KEYS);
  c.items = reinterpret_cast<uint32_t*>(base + OFF_ITEMS);
  c.tile_count = reinterpret_cast<uint32_t*>(base + OFF_COUNT);
  c.tile_start = reinterpret_cast<uint32_t*>(base + OFF_START);
  c.tile_cursor = reinterpret_cast<uint32_t*>(base + OFF_CURSOR);
  c.halo = reinterpret_cast<unsigned long long*>(base + OFF_HALO);
  c.err = reinterpret_cast<int*>(base + OFF_FLAGS);
  c.big_flag = c.err + 1;
  FPM_CUDA_TRY(cudaMemsetAsync(c.err, 0, 2 * sizeof(int), s));
  FPM_TRY(launch_keys(c, dx, s));   // also clears the tile counters
  FPM_TRY(launch_scan(c, s));
  FPM_TRY(launch_scatter(c, s));
  FPM_TRY(launch_paint_tiles(c, dx, rho, nullptr, s));
  FPM_TRY(launch_halo(c, rho, s));
  return FPM_OK;
}
