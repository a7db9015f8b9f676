// y step of the eigenexpansion solve of FP64 plans on a stretched y between
// walls (Sec. 3.3.1): the y part of L is W^{-1} T with W = diag(dyf), and
// its W-orthonormal eigenvectors V are dense, so the transform is a matrix
// product per z plane, here on the FP64 pipe (the mixed plans run it on the
// tensor cores, pp_dense_tc.cu).  The spectrum of plane k is X[j][kx] (complex, kx
// fastest); the forward step writes (V^T W) X, the inverse step V X, in
// place.
//
// A block holds TX consecutive kx columns of one plane, all ny rows, in
// shared memory; thread t computes output rows t, t + 256, ... (R of them)
// for the TX columns, with the matrix read transposed (mt[j][m] = M[m][j])
// so that the 32 lanes of a warp load 32 consecutive entries.  The tile's
// values are shared-memory broadcasts (every thread reads the same entry).
#include "pp_stages.cuh"

namespace pp {

template <typename T, int TX, int R>
__global__ void __launch_bounds__(256) k_ydense(Geo g, const T* __restrict__ mt, C2<T>* spec,
                                                const DevStatus* __restrict__ st) {
  if (stopped(st)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tile = reinterpret_cast<C2<T>*>(smem_raw);  // [ny][TX]
  const int ny = g.ny, nxh = g.nxh;
  const int ntx = (nxh + TX - 1) / TX;
  const int bz = (int)(blockIdx.x / ntx);
  const int kx0 = (int)(blockIdx.x - (unsigned)bz * ntx) * TX;
  const int wdt = min(TX, nxh - kx0);
  C2<T>* base = spec + (size_t)bz * ny * nxh + kx0;
  for (int e = threadIdx.x; e < ny * TX; e += blockDim.x) {
    const int j = e / TX, x = e - j * TX;
    C2<T> v;
    v.x = (T)0;
    v.y = (T)0;
    if (x < wdt) v = base[(size_t)j * nxh + x];
    tile[e] = v;
  }
  __syncthreads();
  T ar[R][TX], ai[R][TX];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int x = 0; x < TX; ++x) ar[r][x] = ai[r][x] = (T)0;
  int mrow[R];
#pragma unroll
  for (int r = 0; r < R; ++r) mrow[r] = min((int)threadIdx.x + 256 * r, ny - 1);
  for (int j = 0; j < ny; ++j) {
    T a[R];
    const T* col = mt + (size_t)j * ny;
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = col[mrow[r]];
#pragma unroll
    for (int x = 0; x < TX; ++x) {
      const C2<T> v = tile[j * TX + x];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        ar[r][x] = fma(a[r], v.x, ar[r][x]);
        ai[r][x] = fma(a[r], v.y, ai[r][x]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int m = (int)threadIdx.x + 256 * r;
    if (m >= ny) continue;
#pragma unroll
    for (int x = 0; x < TX; ++x) {
      if (x < wdt) {
        C2<T> o;
        o.x = ar[r][x];
        o.y = ai[r][x];
        base[(size_t)m * nxh + x] = o;
      }
    }
  }
}

template <typename T, int TX, int R>
static cudaError_t launch_ydense_r(const Geo& g, const T* mt, C2<T>* spec, const DevStatus* st, cudaStream_t s) {
  const size_t smem = (size_t)g.ny * TX * sizeof(C2<T>);
  cudaError_t e = cudaFuncSetAttribute(k_ydense<T, TX, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long nblk = (long long)((g.nxh + TX - 1) / TX) * g.nz;
  k_ydense<T, TX, R><<<(unsigned)nblk, 256, smem, s>>>(g, mt, spec, st);
  return cudaGetLastError();
}

// Columns per block: 4 complex FP64 values of a row, 64 bytes.
cudaError_t launch_ydense(const Geo& g, const double* mt, double2* spec, const DevStatus* st, cudaStream_t s) {
  constexpr int TX = 4;
  switch ((g.ny + 255) / 256) {
    case 1: return launch_ydense_r<double, TX, 1>(g, mt, spec, st, s);
    case 2: return launch_ydense_r<double, TX, 2>(g, mt, spec, st, s);
    case 3: return launch_ydense_r<double, TX, 3>(g, mt, spec, st, s);
    case 4: return launch_ydense_r<double, TX, 4>(g, mt, spec, st, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pp
