// Single-grid kernels of the eigenexpansion solve and Algorithm 1's pass;
// each is a thin wrapper around a stage of pp_stages.cuh.
#include <cmath>

#include "pp_stages.cuh"

namespace pp {

// YS: stretched y between walls (row factors of Geo::ym).
template <typename T, bool YS>
__global__ void __launch_bounds__(256, 4) k_resid_fftx(Geo g, Faces fc, FftDesc fx,
                                                    const C2<T>* __restrict__ twx,
                                                    const double* __restrict__ b,
                                                    const double* __restrict__ rho,
                                                    const double* __restrict__ p, int mode, int p_zero,
                                                    int scale_rho, C2<T>* __restrict__ spec,
                                                    double* __restrict__ red, int rpb,
                                                    const DevStatus* __restrict__ st,
                                                    float* __restrict__ E,
                                                    const float* __restrict__ delta) {
  if (stopped(st)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const bool need_exact = (st == nullptr) || st->need_exact;
  stage_resid_fftx<T, YS>(g, fc, fx, twx, b, rho, p, mode, p_zero, scale_rho, spec, red, rpb, blockIdx.x,
                      need_exact, E, delta, smem_raw);
}

// DCT: the cosine transform of walls in y instead of the periodic DFT.
template <typename T, int DIR, bool DCT>
// Three blocks per SM (FP32: 52 KB of buffers each at ny = 512) measured
// faster than four; the bound also keeps the register count from deciding it.
__global__ void __launch_bounds__(256, sizeof(T) == sizeof(float) ? 3 : 2) k_ffty(Geo g, FftDesc fy, const C2<T>* __restrict__ twy,
                                              C2<T>* __restrict__ spec, int tx, long long ntiles,
                                              const DevStatus* __restrict__ st,
                                              const C2<T>* __restrict__ dct) {
  if (stopped(st)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  stage_ffty_persistent<T, DIR, DCT>(g, fy, twy, spec, tx, ntiles, blockIdx.x, gridDim.x, smem_raw, dct);
}

// z solve for uniform walls in z: cosine transform along z with the
// eigenvalue divide (DIR = -1), then the inverse cosine transform (DIR = +1).
template <typename T, int DIR>
__global__ void __launch_bounds__(256, 2) k_fftz(Geo g, FftDesc fz, const C2<T>* __restrict__ twz,
                                                 C2<T>* __restrict__ spec, int tx, long long ntiles,
                                                 const DevStatus* __restrict__ st,
                                                 const C2<T>* __restrict__ dct, ZDivide zd) {
  if (stopped(st)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  stage_ffty_persistent<T, DIR, true, 1>(g, fz, twz, spec, tx, ntiles, blockIdx.x, gridDim.x, smem_raw, dct, zd);
}

template <typename T>
__global__ void __launch_bounds__(128) k_tridiag(Geo g, const double* __restrict__ invd,
                                                 C2<T>* spec, double2* ybuf,  // ybuf may alias spec
                                                 const DevStatus* __restrict__ st) {
  if (stopped(st)) return;
  const size_t ncol = (size_t)g.ny * g.nxh;
  const size_t col = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  if (col == 0) thomas_column<T, true>(g, invd, spec, ybuf, col, ncol);
  else thomas_column<T, false>(g, invd, spec, ybuf, col, ncol);
}

template <typename T>
__global__ void __launch_bounds__(128, 16) k_tridiag_split(Geo g, const double* __restrict__ mtab,
                                                           const double* __restrict__ invd, T* spec,
                                                           const DevStatus* __restrict__ st) {
  if (stopped(st)) return;
  __shared__ double shm[34];
  double m0 = 0.0;
  if (blockIdx.x == 0) {  // holds column 0 (scalars 0 and 1)
    zero_column_means<T>(g, spec, 2 * (size_t)g.ny * g.nxh, shm);
    if (threadIdx.x < 2) m0 = shm[32 + threadIdx.x];
  }
  stage_tridiag_split<T>(g, mtab, invd, spec, (size_t)blockIdx.x * blockDim.x + threadIdx.x, m0);
}

// PP_MIXED_Z64 z solve: one thread per (kx, ky) column, all FP64
// recurrences (stage_tridiag_z64).  The grid is persistent-sized (every
// block resident at once) and the columns are dealt out a warp at a time,
// round robin over the blocks (work warp = warp-in-block x gridDim +
// block), so every SM gets the same number of FP64 chains whatever the
// block scheduler's placement; a warp still takes 32 consecutive columns.
// Work warp 0 (warp 0 of block 0) holds the singular column 0 alone, so no
// warp runs both variants of the sweep one after the other; work warp w > 0
// holds columns 1 + 32 (w - 1) + lane.  Block 0 first reduces column 0's
// dzf-weighted z means.
__global__ void __launch_bounds__(128, 8) k_tridiag_z64(Geo g, TriZ64 t, float2* spec,
                                                        const DevStatus* __restrict__ st) {
  if (stopped(st)) return;
  __shared__ double shm[34];
  const unsigned ncol = (unsigned)g.ny * g.nxh;
  const unsigned ntc = (unsigned)t.nyt * g.nxh;
  if (blockIdx.x == 0) zero_column_means<float>(g, reinterpret_cast<const float*>(spec), 2 * (size_t)ncol, shm);
  const unsigned wstride = (blockDim.x >> 5) * gridDim.x;
  const unsigned lane = threadIdx.x & 31u;
  for (unsigned wq = (threadIdx.x >> 5) * gridDim.x + blockIdx.x; wq == 0 || (wq - 1) * 32u + 1u < ncol;
       wq += wstride) {
    if (wq == 0) {  // warp 0 of block 0: column 0 on lane 0
      if (lane == 0) stage_tridiag_z64<true>(g, t, spec, 0, ncol, 0, ntc, shm[32], shm[33]);
      continue;
    }
    const unsigned col = 1u + (wq - 1) * 32u + lane;
    if (col >= ncol) continue;
    const int ky = (int)(col / (unsigned)g.nxh);
    const int kx = (int)(col - (unsigned)ky * g.nxh);
    const int kyt = (t.ysym && 2 * ky > g.ny) ? g.ny - ky : ky;
    stage_tridiag_z64<false>(g, t, spec, col, ncol, (unsigned)kyt * g.nxh + kx, ntc, 0.0, 0.0);
  }
}

__global__ void __launch_bounds__(128, 8) k_tridiag_mixed(Geo g, const double* __restrict__ mtab,
                                                         const double* __restrict__ invd, TriF32 f,
                                                         float2* spec, const DevStatus* __restrict__ st) {
  if (stopped(st)) return;
  stage_tridiag_mixed(g, mtab, invd, f, spec, blockIdx.x);
}

// p += sdelta when the last residual of the loop was an updated one (the
// increments since the last exact residual are still pending).
__global__ void k_fold_pending(size_t n, double* __restrict__ p, const float* __restrict__ sdelta,
                               const DevStatus* __restrict__ st) {
  if (st->last_exact) return;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    p[c] += widen_f32(sdelta[c]);
}

__global__ void k_narrow(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

template <typename T>
__global__ void __launch_bounds__(256) k_fftx_inv(Geo g, FftDesc fx, const C2<T>* __restrict__ twx,
                                                  const C2<T>* __restrict__ spec, double scale,
                                                  double* __restrict__ p, int p_zero, int rpb,
                                                  const DevStatus* __restrict__ st,
                                                  T* __restrict__ delta, float* __restrict__ sdelta) {
  if (stopped(st)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const bool lazy = sdelta != nullptr && st != nullptr;
  const bool fold = lazy && st->need_exact != 0;
  const bool fresh = lazy && st->since_exact <= 1;
  stage_fftx_inv<T>(g, fx, twx, spec, scale, p, p_zero, rpb, blockIdx.x, delta, lazy ? sdelta : nullptr,
                    fold, fresh, smem_raw);
}

// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_resid_fftx(const Geo& g, const Faces& fc, const FftDesc& fx, const C2<T>* twx,
                              const double* b, double inv_dt, const double* rho, const double* p,
                              int p_zero, int scale_rho, C2<T>* spec, double* red, int* nblk_out,
                              const DevStatus* st, cudaStream_t s, float* E, const float* delta) {
  const int rpb = rows_per_block(g.nx, kEpt);
  const long nrows = (long)g.nz * g.ny;
  const int nblk = (int)((nrows + rpb - 1) / rpb);
  // two transform buffers, then (FP32) the padding of the second buffer and
  // the twiddle table of the fast path
  const size_t nbuf = (size_t)(rpb / 2) * g.nx;
  const size_t smem = (sizeof(T) == sizeof(float))
                          ? (nbuf + fft_pad_elems((int)nbuf) + g.nx) * sizeof(float2)
                          : 2 * nbuf * sizeof(C2<T>);
  auto kern = (g.ym != nullptr) ? k_resid_fftx<T, true> : k_resid_fftx<T, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int mode = (red == nullptr) ? 0 : 1;
  (void)inv_dt;
  kern<<<nblk, kThreads, smem, s>>>(g, fc, fx, twx, b, rho, p, mode, p_zero, scale_rho, spec, red, rpb, st, E,
                                    delta);
  if (nblk_out) *nblk_out = nblk;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ffty(const Geo& g, const FftDesc& fy, const C2<T>* twy, C2<T>* spec, int inverse,
                        const DevStatus* st, cudaStream_t s, const C2<T>* dct) {
  if constexpr (std::is_same<T, float>::value) {
    if (g.ny == 512 && dct == nullptr)
      return launch_ffty512(g, reinterpret_cast<const float2*>(twy), reinterpret_cast<float2*>(spec), inverse, st, s);
  }
  const int tx = ffty_tile(g.ny, sizeof(C2<T>), kEpt);
  const int tsz = g.ny * tx;
  const size_t smem = (sizeof(T) == sizeof(float))
                          ? ((size_t)2 * tsz + fft_pad_elems(tsz) + g.ny) * sizeof(float2)
                          : (size_t)3 * tsz * sizeof(C2<T>);
  const long long ntiles = (long long)((g.nxh + tx - 1) / tx) * g.nz;
  // persistent grid: exactly the blocks that are resident at once (shared
  // memory and registers both counted), so no block waits for a second wave
  auto kern = dct ? (inverse ? k_ffty<T, 1, true> : k_ffty<T, -1, true>)
                  : (inverse ? k_ffty<T, 1, false> : k_ffty<T, -1, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, nsm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  long long nblk = (long long)nsm * per_sm;
  if (nblk > ntiles) nblk = ntiles;
  kern<<<(int)nblk, kThreads, smem, s>>>(g, fy, twy, spec, tx, ntiles, st, dct);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zdct(const Geo& g, const FftDesc& fz, const C2<T>* twz, C2<T>* spec, int inverse,
                        const DevStatus* st, cudaStream_t s, const C2<T>* dct, const ZDivide& zd) {
  const int tx = ffty_tile(g.nz, sizeof(C2<T>), kEpt);
  const int tsz = g.nz * tx;
  const size_t smem = (sizeof(T) == sizeof(float))
                          ? ((size_t)2 * tsz + fft_pad_elems(tsz) + g.nz) * sizeof(float2)
                          : (size_t)3 * tsz * sizeof(C2<T>);
  const long long ntiles = (long long)((g.nxh + tx - 1) / tx) * g.ny;
  auto kern = inverse ? k_fftz<T, 1> : k_fftz<T, -1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, nsm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  long long nblk = (long long)nsm * per_sm;
  if (nblk > ntiles) nblk = ntiles;
  kern<<<(int)nblk, kThreads, smem, s>>>(g, fz, twz, spec, tx, ntiles, st, dct, zd);
  return cudaGetLastError();
}
template cudaError_t launch_zdct<double>(const Geo&, const FftDesc&, const double2*, double2*, int,
                                         const DevStatus*, cudaStream_t, const double2*, const ZDivide&);

template <typename T>
cudaError_t launch_tridiag(const Geo& g, const double* invd, C2<T>* spec, double2* ybuf,
                           const DevStatus* st, cudaStream_t s, const double* mtab, const TriF32* f32) {
  const size_t ncol = (size_t)g.ny * g.nxh;
  if (mtab != nullptr && f32 != nullptr && sizeof(T) == sizeof(float)) {
    k_tridiag_mixed<<<tri_mixed_blocks(ncol, f32->nlow), 128, 0, s>>>(g, mtab, invd, *f32,
                                                                     reinterpret_cast<float2*>(spec), st);
  } else if (mtab != nullptr) {
    const int nblk = (int)((2 * ncol + 127) / 128);
    k_tridiag_split<T><<<nblk, 128, 0, s>>>(g, mtab, invd, reinterpret_cast<T*>(spec), st);
  } else {
    const int nblk = (int)((ncol + 127) / 128);
    k_tridiag<T><<<nblk, 128, 0, s>>>(g, invd, spec, ybuf, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_tridiag_z64(const Geo& g, const TriZ64& t, float2* spec, const DevStatus* st,
                               cudaStream_t s) {
  const size_t ncol = (size_t)g.ny * g.nxh;
  const long long nwarps = 1 + (long long)((ncol - 1 + 31) / 32);  // column 0 alone, then 32 per warp
  int per_sm = 0, dev = 0, nsm = 0;
  cudaError_t e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tridiag_z64, 128, 0)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  // all blocks resident at once; no more blocks than warps of work (each
  // block then still holds at least one column in its first warp)
  long long nblk = (long long)nsm * per_sm;
  if (nblk > nwarps) nblk = nwarps;
  if (nblk < 1) nblk = 1;
  k_tridiag_z64<<<(int)nblk, 128, 0, s>>>(g, t, spec, st);
  return cudaGetLastError();
}

std::vector<int> tri_low_columns(const std::vector<double>& lamx, const std::vector<double>& lamy,
                                 double thr) {
  std::vector<int> low{0};
  const int nxh = (int)lamx.size(), ny = (int)lamy.size();
  for (int j = 0; j < ny; ++j)
    for (int kx = 0; kx < nxh; ++kx)
      if ((j != 0 || kx != 0) && std::fabs(lamx[kx] + lamy[j]) < thr) low.push_back(j * nxh + kx);
  return low;
}

cudaError_t launch_fold_pending(const Geo& g, double* p, const float* sdelta, const DevStatus* st,
                                cudaStream_t s) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  size_t nb = (n + 255) / 256;
  if (nb > (size_t)152 * 32) nb = (size_t)152 * 32;
  k_fold_pending<<<(int)(nb == 0 ? 1 : nb), 256, 0, s>>>(n, p, sdelta, st);
  return cudaGetLastError();
}

cudaError_t launch_narrow(const double* src, float* dst, size_t n, cudaStream_t s) {
  size_t nb = (n + 255) / 256;
  if (nb > (size_t)152 * 32) nb = (size_t)152 * 32;
  k_narrow<<<(int)(nb == 0 ? 1 : nb), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fftx_inv(const Geo& g, const FftDesc& fx, const C2<T>* twx, const C2<T>* spec,
                            double scale, double* p, int p_zero, const DevStatus* st, cudaStream_t s,
                            T* delta, float* sdelta) {
  if constexpr (std::is_same<T, float>::value) {
    if (g.nx == 512)
      return launch_fftx512_inv(g, reinterpret_cast<const float2*>(twx), reinterpret_cast<const float2*>(spec),
                                scale, p, p_zero, st, s, delta, sdelta);
  }
  const int rpb = rows_per_block(g.nx, kEpt);
  const long nrows = (long)g.nz * g.ny;
  const int nblk = (int)((nrows + rpb - 1) / rpb);
  // two transform buffers, then (FP32) the padding of the second buffer and
  // the twiddle table of the fast path
  const size_t nbuf = (size_t)(rpb / 2) * g.nx;
  const size_t smem = (sizeof(T) == sizeof(float))
                          ? (nbuf + fft_pad_elems((int)nbuf) + g.nx) * sizeof(float2)
                          : 2 * nbuf * sizeof(C2<T>);
  cudaError_t e = cudaFuncSetAttribute(k_fftx_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_fftx_inv<T><<<nblk, kThreads, smem, s>>>(g, fx, twx, spec, scale, p, p_zero, rpb, st, delta, sdelta);
  return cudaGetLastError();
}

#define PP_INST(T)                                                                                   \
  template cudaError_t launch_resid_fftx<T>(const Geo&, const Faces&, const FftDesc&, const C2<T>*,  \
                                            const double*, double, const double*, const double*,     \
                                            int, int, C2<T>*, double*, int*, const DevStatus*,       \
                                            cudaStream_t, float*, const float*);                    \
  template cudaError_t launch_ffty<T>(const Geo&, const FftDesc&, const C2<T>*, C2<T>*, int,         \
                                      const DevStatus*, cudaStream_t, const C2<T>*);                 \
  template cudaError_t launch_tridiag<T>(const Geo&, const double*, C2<T>*, double2*,                \
                                         const DevStatus*, cudaStream_t, const double*,              \
                                         const TriF32*);                                             \
  template cudaError_t launch_fftx_inv<T>(const Geo&, const FftDesc&, const C2<T>*, const C2<T>*,    \
                                          double, double*, int, const DevStatus*, cudaStream_t,      \
                                          T*, float*);
PP_INST(double)
PP_INST(float)
#undef PP_INST

}  // namespace pp
