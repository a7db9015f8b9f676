// Complex transform along y of length 512 in FP32 with the data in
// registers (pp_r512.cuh): the y step of the eigenexpansion solve
// (Sec. 3.3.1) for the periodic 512-point lines of mixed plans.  Thread b
// of a line loads x[64 a + b] from global memory straight into registers
// and stores X[b + 64 h] straight back: two shared-memory round trips per
// value (the Stockham passes of the generic kernel make three, plus the
// staging copy).  A block holds TX consecutive kx columns of one z plane
// (TX lanes cover one row segment of TX * 8 bytes) and walks the (plane,
// kx tile) tiles with stride gridDim.x, loading the next tile's values
// while it transforms the current one.
#include "pp_r512.cuh"
#include "pp_stages.cuh"

namespace pp {

template <int DIR, int TX>
__global__ void __launch_bounds__(64 * TX) k_ffty512(Geo g, const float2* __restrict__ twy,
                                                     float2* __restrict__ spec, long long ntiles,
                                                     const DevStatus* __restrict__ st) {
  if (stopped(st)) return;
  using L = R512<TX>;
  float2* sm = smem_f2();
  float2* tw = sm;
  float2* s1 = sm + L::TW;
  float2* s2 = s1 + L::S1;
  r512_load_twiddles(tw, twy);
  const int nxh = g.nxh;
  const int ntx = (nxh + TX - 1) / TX;
  const int x = threadIdx.x % TX, j = threadIdx.x / TX;  // column in the tile, line thread 0..63
  const size_t rstride = (size_t)nxh;
  const size_t plane = (size_t)L::N * nxh;
  float2 v[8];
  auto load = [&](long long tile) {
    const int bz = (int)(tile / ntx), kx = (int)(tile - (long long)bz * ntx) * TX + x;
    const bool ok = kx < nxh;
    const float2* src = spec + (size_t)bz * plane + kx + (size_t)j * rstride;
#pragma unroll
    for (int a = 0; a < 8; ++a) v[a] = ok ? src[(size_t)(64 * a) * rstride] : make_float2(0.f, 0.f);
  };
  long long tile = blockIdx.x;
  if (tile < ntiles) load(tile);
  __syncthreads();  // twiddle table
  for (; tile < ntiles; tile += gridDim.x) {
    const long long next = tile + gridDim.x;
    // the next tile's loads are issued once this tile's values sit in s1
    float2 u[8];
    r512_transform<DIR, TX>(v, u, s1, s2, tw, x, j, [&]() {
      if (next < ntiles) load(next);
    });
    const int bz = (int)(tile / ntx), kx = (int)(tile - (long long)bz * ntx) * TX + x;
    if (kx < nxh) {
      float2* dst = spec + (size_t)bz * plane + kx + (size_t)j * rstride;
#pragma unroll
      for (int h = 0; h < 8; ++h) dst[(size_t)(64 * h) * rstride] = u[h];
    }
  }
}

// Columns per tile: 8 (64-byte row segments, 512 threads per block).
constexpr int kFfty512Tx = 8;

cudaError_t launch_ffty512(const Geo& g, const float2* twy, float2* spec, int inverse, const DevStatus* st,
                           cudaStream_t s) {
  constexpr int TX = kFfty512Tx;
  const size_t smem = R512<TX>::smem_bytes();
  auto kern = inverse ? k_ffty512<1, TX> : k_ffty512<-1, TX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long ntiles = (long long)((g.nxh + TX - 1) / TX) * g.nz;
  int per_sm = 0, dev = 0, nsm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 64 * TX, smem)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  long long nblk = (long long)nsm * per_sm;
  if (nblk > ntiles) nblk = ntiles;
  kern<<<(int)nblk, 64 * TX, smem, s>>>(g, twy, spec, ntiles, st);
  return cudaGetLastError();
}

}  // namespace pp
