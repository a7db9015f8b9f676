// Complex transform along y of length 512 in FP32 with the data in
// registers: the y step of the eigenexpansion solve (Sec. 3.3.1) for the
// periodic 512-point lines of mixed plans.
//
// A line is split 512 = 8 x 8 x 8 (n = 64 a + b, k = c + 8 d, then
// b = 8 e + f, d = g + 8 h; w = exp(DIR 2 pi i / 512)):
//   X[c + 8 g + 64 h] = sum_f W8^{f h} w^{8 f g} sum_e W8^{e g} y_{8 e + f}[c],
//   y_b[c] = w^{b c} sum_a W8^{a c} x[64 a + b].
// 64 threads hold one line, 8 values each: thread b loads x[64 a + b] from
// global memory straight into registers, does the first 8-point DFT and its
// twiddles, then two exchanges through shared memory feed the second and
// third 8-point DFTs, and thread (c, g) stores X[c + 8 g + 64 h] straight to
// global memory.  Two shared-memory round trips per value (the Stockham
// passes of the generic kernel make four, plus the staging copy).  A block
// holds TX consecutive kx columns of one z plane (TX lanes cover one row
// segment of TX * 8 bytes) and walks the (plane, kx tile) tiles with stride
// gridDim.x, loading the next tile's values while it transforms the current
// one.
#include "pp_stages.cuh"

namespace pp {

namespace {

template <int TX>
struct R512 {
  static constexpr int N = 512;
  static constexpr int S1 = N * TX;        // first exchange buffer [c][b][x]
  static constexpr int CS2 = 64 * TX + TX;  // second buffer: slab of one c, padded
  static constexpr int S2 = 8 * CS2;       // [c][g][f][x]
  static constexpr int TW = N;             // twiddle table (cos, sin)(2 pi m / 512)
  static constexpr size_t smem_bytes() { return (size_t)(TW + S1 + S2) * sizeof(float2); }
};

// v[r] *= w^{r q} for r = 1..7, with w^q, w^{2q}, w^{4q} read from the
// table (index in units of 2 pi / 512) and the other powers formed by
// products.
template <int DIR>
__device__ __forceinline__ void twiddle8(float2* v, const float2* __restrict__ tw, int q) {
  const float2 w1 = tw_dir<DIR>(tw[q & 511]);
  const float2 w2 = tw_dir<DIR>(tw[(2 * q) & 511]);
  const float2 w4 = tw_dir<DIR>(tw[(4 * q) & 511]);
  const float2 w3 = cmul<float>(w1, w2);
  v[1] = cmul<float>(v[1], w1);
  v[2] = cmul<float>(v[2], w2);
  v[3] = cmul<float>(v[3], w3);
  v[4] = cmul<float>(v[4], w4);
  v[5] = cmul<float>(v[5], cmul<float>(w1, w4));
  v[6] = cmul<float>(v[6], cmul<float>(w2, w4));
  v[7] = cmul<float>(v[7], cmul<float>(w3, w4));
}

}  // namespace

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
  for (int i = threadIdx.x; i < L::N; i += blockDim.x) tw[i] = twy[i];
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
    // first 8-point DFT over a, twiddles w^{b c} (b = j)
    Dft<float, DIR, 8>::run(v);
    twiddle8<DIR>(v, tw, j);
#pragma unroll
    for (int c = 0; c < 8; ++c) s1[(c * 64 + j) * TX + x] = v[c];
    const long long next = tile + gridDim.x;
    if (next < ntiles) load(next);  // in flight during the exchanges below
    __syncthreads();
    // second 8-point DFT over e, for (c, f); twiddles w^{8 f g}
    float2 u[8];
    {
      const int c = j >> 3, f = j & 7;
#pragma unroll
      for (int e = 0; e < 8; ++e) u[e] = s1[(c * 64 + 8 * e + f) * TX + x];
      Dft<float, DIR, 8>::run(u);
      twiddle8<DIR>(u, tw, 8 * f);
#pragma unroll
      for (int gg = 0; gg < 8; ++gg) s2[c * L::CS2 + (gg * 8 + f) * TX + x] = u[gg];
    }
    __syncthreads();
    // third 8-point DFT over f, for (c, g); X[c + 8 g + 64 h] = X[j + 64 h]
    {
      const int c = j & 7, gg = j >> 3;
#pragma unroll
      for (int f = 0; f < 8; ++f) u[f] = s2[c * L::CS2 + (gg * 8 + f) * TX + x];
      Dft<float, DIR, 8>::run(u);
      const int bz = (int)(tile / ntx), kx = (int)(tile - (long long)bz * ntx) * TX + x;
      if (kx < nxh) {
        float2* dst = spec + (size_t)bz * plane + kx + (size_t)j * rstride;
#pragma unroll
        for (int h = 0; h < 8; ++h) dst[(size_t)(64 * h) * rstride] = u[h];
      }
    }
    // the next tile's first exchange writes s1 only after every thread of
    // this block has passed the barrier above, i.e. finished reading s1
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
