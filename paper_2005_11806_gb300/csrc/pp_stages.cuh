// Device-side stages of one constant-coefficient eigenexpansion solve
// (Sec. 3.3.1: the pressure equation with homogeneous boundary conditions
// solved exactly by the eigenexpansion method) and of Algorithm 1's pass:
// residual + forward x transform, y transforms, the per-(kx, ky) tridiagonal
// solve along z, and the inverse x transform fused with the pressure update.
// The single-grid kernels (pp_kernels_fft.cu) and the grouped multi-grid
// kernels (pp_batch.cu) both call these.
#pragma once
#include "pp_fft.cuh"

namespace pp {

constexpr int kThreads = 256;
// FFT elements per block = kEpt * kThreads (two shared buffers of that many
// complex values).  8 was the fastest of {2, 4, 8, 16} for every kernel in a
// 512^3 sweep on GB300.
constexpr int kEpt = 8;
constexpr int kPrefetchInv = 8;  // p values prefetched per thread in the inverse x kernel

// Rows per block of the x kernels: (rows/2) complex sequences of length nx
// with at most ept * kThreads elements in the shared buffer.
inline int rows_per_block(int nx, int ept) {
  int nseq = (ept * kThreads) / nx;
  if (nseq > 32) nseq = 32;
  if (nseq < 1) nseq = 1;
  return 2 * nseq;
}

// kx columns per y tile: a power of two with tx * ny <= ept * kThreads.
inline int ffty_tile(int ny, size_t csize, int ept) {
  int tx = (int)(128 / csize);  // 128-byte row segments
  while (tx > 1 && ny * tx > ept * kThreads) tx >>= 1;
  return tx;
}

__device__ __forceinline__ bool stopped(const DevStatus* st) { return st != nullptr && st->done; }

// Transform dispatch: compile-time passes for the power-of-two lengths and
// batch shapes the default block sizes produce, the generic mixed-radix
// passes otherwise (same passes in the same order, so the same results).
#define PP_TRY_FIXED(NN, NBB)                                                                       \
  if (n == NN && nbatch == NBB) {                                                                   \
    if (BATCH_FAST) return fft_block_fixed<T, DIR, true, NN, NBB, NBB, 1>(a, b, tw, tid, nth);      \
    return fft_block_fixed<T, DIR, false, NN, NBB, 1, NN>(a, b, tw, tid, nth);                      \
  }

template <typename T, int DIR, bool BATCH_FAST>
__device__ __forceinline__ C2<T>* fft_dispatch(C2<T>* a, C2<T>* b, const FftDesc& d, int nbatch, int es, int bs,
                                               const C2<T>* __restrict__ tw, int tid, int nth) {
  const int n = d.n;
  const bool shape_ok = BATCH_FAST ? (es == nbatch && bs == 1) : (es == 1 && bs == n);
  if (shape_ok) {
    if (BATCH_FAST) {
      PP_TRY_FIXED(512, 4)
      PP_TRY_FIXED(256, 8)
      PP_TRY_FIXED(128, 16)
      PP_TRY_FIXED(128, 8)
      PP_TRY_FIXED(64, 16)
      PP_TRY_FIXED(64, 8)
    } else {
      PP_TRY_FIXED(512, 4)
      PP_TRY_FIXED(256, 8)
      PP_TRY_FIXED(128, 16)
      PP_TRY_FIXED(64, 32)
      PP_TRY_FIXED(32, 32)
    }
  }
  return fft_block<T, DIR, BATCH_FAST>(a, b, d, nbatch, es, bs, tw, tid, nth);
}
#undef PP_TRY_FIXED

// ---------------------------------------------------------------------------
// Residual of the variable-coefficient equation and forward real x transform.
//   mode 0: r = f (constant-coefficient solve)
//   mode 1: e = (D u^s - S_c)/dt, evaluated in FP64 in the row-scaled form
//           dzf_k e = b_s - (sum_nb c_nb p_nb - diag p_c), b_s = dzf_k b / dt;
//           r = rho e (or e).  The mixed path narrows dzf_k e to FP32 and
//           finishes (scaling, norms, rho) in FP32.
// Two real rows are packed into one complex sequence (re = even row,
// im = odd row), transformed together and separated afterwards.
template <typename T>
__device__ __forceinline__ void stage_resid_fftx(const Geo& g, const Faces& fc, const FftDesc& fx,
                                                 const C2<T>* __restrict__ twx,
                                                 const double* __restrict__ b,
                                                 const double* __restrict__ rho,
                                                 const double* __restrict__ p, int mode, int p_zero,
                                                 int scale_rho, C2<T>* __restrict__ spec,
                                                 double* __restrict__ red, int rpb, int blk,
                                                 bool need_exact, double* __restrict__ E,
                                                 const float* __restrict__ delta,
                                                 unsigned char* smem_raw) {
  __shared__ double shred[32];
  const int nx = g.nx, ny = g.ny, nz = g.nz, nxh = g.nxh;
  const bool update = (E != nullptr) && !p_zero && !need_exact;
  const int nseq = rpb >> 1;
  C2<T>* bufA = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* bufB = bufA + (size_t)nseq * nx;
  const int nrows = nz * ny;
  const long row0 = (long)blk * rpb;
  const size_t plane = (size_t)ny * nx;
  T s2 = (T)0, s1 = (T)0;
  // constant scaling of Methods I and II (one device scalar for all cells)
  const bool const_scale = fc.rho_tilde != nullptr;
  const double rt = (const_scale && mode != 0) ? *fc.rho_tilde : 0.0;
  const float rt_f = (float)rt;
  // thread -> (row offset, first column); index math is done once per row
  const int tpr = nx < (int)blockDim.x ? nx : (int)blockDim.x;
  const int rows_par = blockDim.x / tpr;
  const int qoff = threadIdx.x / tpr, i0 = threadIdx.x - qoff * tpr;
  for (int q = qoff; q < rpb && qoff < rows_par; q += rows_par) {
    const int row = (int)row0 + q;
    const bool valid = row < nrows;
    const int k = valid ? row / ny : 0, j = valid ? row - k * ny : 0;
    const int jp = (j + 1 == ny) ? 0 : j + 1, jm = (j == 0) ? ny - 1 : j - 1;
    const size_t rowoff = (size_t)row * nx;
    const size_t kp = (size_t)k * plane;
    const size_t rowp = kp + (size_t)jp * nx, rowm = kp + (size_t)jm * nx;
    const float idzf_f = (mode != 0 && sizeof(T) == sizeof(float)) ? g.inv_dzf_f[k] : 0.f;
    const double idzf = (mode != 0 && sizeof(T) == sizeof(double)) ? g.inv_dzf[k] : 0.0;
    for (int i = i0; i < nx; i += tpr) {
      T r = (T)0;
      if (valid) {
        const size_t c = rowoff + i;
        if (mode == 0) {
          r = (T)b[c];
        } else {
          const int ip = (i + 1 == nx) ? 0 : i + 1, im = (i == 0) ? nx - 1 : i - 1;
          double ep;
          if (update) {
            // E^s = E^{s-1} - A delta, A delta in FP32
            float t = -fc.diagf[c] * delta[c];
            t = fmaf(fc.cxf[rowoff + ip], delta[rowoff + ip], t);
            t = fmaf(fc.cxf[c], delta[rowoff + im], t);
            t = fmaf(fc.cyf[rowp + i], delta[rowp + i], t);
            t = fmaf(fc.cyf[c], delta[rowm + i], t);
            if (k + 1 < nz) t = fmaf(fc.czf[c + plane], delta[c + plane], t);
            if (k > 0) t = fmaf(fc.czf[c], delta[c - plane], t);
            ep = E[c] - widen_f32(t);
            E[c] = ep;
          } else {
            ep = b[c];
            if (!p_zero) {
              double t = -fc.diag[c] * p[c];
              t = fma(fc.cx[rowoff + ip], p[rowoff + ip], t);
              t = fma(fc.cx[c], p[rowoff + im], t);
              t = fma(fc.cy[rowp + i], p[rowp + i], t);
              t = fma(fc.cy[c], p[rowm + i], t);
              if (k + 1 < nz) t = fma(fc.cz[c + plane], p[c + plane], t);
              if (k > 0) t = fma(fc.cz[c], p[c - plane], t);
              ep -= t;
            }
            if (E != nullptr) E[c] = ep;
          }
          if (sizeof(T) == sizeof(float)) {
            const float e = narrow_f64(ep) * idzf_f;
            s2 = fmaf(e, e, (float)s2);
            s1 += fabsf(e);
            r = (T)(scale_rho ? (const_scale ? rt_f : fc.rhof[c]) * e : e);
          } else {
            const double e = ep * idzf;
            s2 = (T)fma(e, e, (double)s2);
            s1 += (T)fabs(e);
            r = (T)(scale_rho ? (const_scale ? rt : rho[c]) * e : e);
          }
        }
      }
      C2<T>& z = bufA[(size_t)(q >> 1) * nx + i];
      if (q & 1) z.y = r; else z.x = r;
    }
  }
  if (mode != 0) {
    const double a2 = block_sum<double>((double)s2, shred);
    const double a1 = block_sum<double>((double)s1, shred);
    if (threadIdx.x == 0) {
      red[2 * (size_t)blk] = a2;
      red[2 * (size_t)blk + 1] = a1;
    }
  }
  __syncthreads();
  const C2<T>* res = fft_dispatch<T, -1, false>(bufA, bufB, fx, nseq, 1, nx, twx, threadIdx.x, blockDim.x);
  for (int t = threadIdx.x; t < nseq * nxh; t += blockDim.x) {
    const int q = t / nxh, kx = t - q * nxh;
    const C2<T> Z = res[(size_t)q * nx + kx];
    const int km = (kx == 0) ? 0 : nx - kx;
    const C2<T> W = res[(size_t)q * nx + km];
    // A = (Z + conj W)/2, B = (Z - conj W)/(2i)
    C2<T> A, B;
    A.x = (T)0.5 * (Z.x + W.x); A.y = (T)0.5 * (Z.y - W.y);
    B.x = (T)0.5 * (Z.y + W.y); B.y = (T)-0.5 * (Z.x - W.x);
    const long ra = row0 + 2 * q;
    if (ra < nrows) spec[(size_t)ra * nxh + kx] = A;
    if (ra + 1 < nrows) spec[(size_t)(ra + 1) * nxh + kx] = B;
  }
}

// Complex transform along y of one z-plane tile of tx consecutive kx.
template <typename T, int DIR>
__device__ __forceinline__ void stage_ffty(const Geo& g, const FftDesc& fy, const C2<T>* __restrict__ twy,
                                           C2<T>* __restrict__ spec, int tx, int bx, int bz,
                                           unsigned char* smem_raw) {
  const int ny = g.ny, nxh = g.nxh;
  C2<T>* bufA = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* bufB = bufA + (size_t)ny * tx;
  const int kx0 = bx * tx;
  const size_t base = (size_t)bz * ny * nxh;
  for (int t = threadIdx.x; t < ny * tx; t += blockDim.x) {
    const int y = t / tx, x = t - y * tx;
    C2<T> v; v.x = (T)0; v.y = (T)0;
    if (kx0 + x < nxh) v = spec[base + (size_t)y * nxh + kx0 + x];
    bufA[t] = v;
  }
  __syncthreads();
  const C2<T>* res = fft_dispatch<T, DIR, true>(bufA, bufB, fy, tx, tx, 1, twy, threadIdx.x, blockDim.x);
  for (int t = threadIdx.x; t < ny * tx; t += blockDim.x) {
    const int y = t / tx, x = t - y * tx;
    if (kx0 + x < nxh) spec[base + (size_t)y * nxh + kx0 + x] = res[t];
  }
}

// Persistent y transform: each block walks the (kx tile, z plane) tiles
// with stride gridDim.x over three rotating shared buffers: while the
// current tile is transformed in two of them, the next tile is copied into
// the third by cp.async.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;"
               :: "r"((uint32_t)__cvta_generic_to_shared(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ void ffty_issue_tile(const Geo& g, const C2<T>* __restrict__ spec, int tx, int ntx,
                                                long long tile, C2<T>* buf) {
  const int ny = g.ny, nxh = g.nxh;
  const int bz = (int)(tile / ntx), bx = (int)(tile - (long long)bz * ntx);
  const int kx0 = bx * tx;
  const size_t base = (size_t)bz * ny * nxh;
  for (int t = threadIdx.x; t < ny * tx; t += blockDim.x) {
    const int y = t / tx, x = t - y * tx;
    if (kx0 + x < nxh) {
      if (sizeof(C2<T>) == 8) cp_async8(&buf[t], &spec[base + (size_t)y * nxh + kx0 + x]);
      else {
        cp_async8(&buf[t], &spec[base + (size_t)y * nxh + kx0 + x]);
        cp_async8(reinterpret_cast<char*>(&buf[t]) + 8,
                  reinterpret_cast<const char*>(&spec[base + (size_t)y * nxh + kx0 + x]) + 8);
      }
    } else {
      buf[t].x = (T)0;
      buf[t].y = (T)0;
    }
  }
  cp_async_commit();
}

template <typename T, int DIR>
__device__ __forceinline__ void stage_ffty_persistent(const Geo& g, const FftDesc& fy,
                                                      const C2<T>* __restrict__ twy, C2<T>* spec, int tx,
                                                      long long ntiles, long long first, long long stride,
                                                      unsigned char* smem_raw) {
  const int ny = g.ny, nxh = g.nxh;
  const int ntx = (nxh + tx - 1) / tx;
  const size_t tsz = (size_t)ny * tx;
  C2<T>* X[3] = {reinterpret_cast<C2<T>*>(smem_raw), reinterpret_cast<C2<T>*>(smem_raw) + tsz,
                 reinterpret_cast<C2<T>*>(smem_raw) + 2 * tsz};
  int L = 0, Q = 1, F = 2;
  if (first < ntiles) ffty_issue_tile<T>(g, spec, tx, ntx, first, X[L]);
  for (long long tile = first; tile < ntiles; tile += stride) {
    cp_async_wait_all();
    __syncthreads();
    const long long next = tile + stride;
    if (next < ntiles) ffty_issue_tile<T>(g, spec, tx, ntx, next, X[F]);
    const C2<T>* res = fft_dispatch<T, DIR, true>(X[L], X[Q], fy, tx, tx, 1, twy, threadIdx.x, blockDim.x);
    const int bz = (int)(tile / ntx), bx = (int)(tile - (long long)bz * ntx);
    const int kx0 = bx * tx;
    const size_t base = (size_t)bz * ny * nxh;
    for (int t = threadIdx.x; t < ny * tx; t += blockDim.x) {
      const int y = t / tx, x = t - y * tx;
      if (kx0 + x < nxh) spec[base + (size_t)y * nxh + kx0 + x] = res[t];
    }
    __syncthreads();
    // rotate: the prefetched buffer holds the next tile; the other two are free
    const int nl = F;
    F = L;
    L = nl;
  }
}

// Per-column Thomas solve of (L_z + lambda_x + lambda_y) x = f with the
// inverse pivots precomputed at plan time.  Column (0, 0) is singular: its
// right-hand side loses its dzf-weighted mean (compatibility) and its last
// unknown is pinned (inverse pivot 0); the pressure gauge is fixed later.
// Loads run PF levels ahead of the recurrence; FP32 spectra are widened and
// narrowed on the integer pipe.
template <typename T> __device__ __forceinline__ double2 to_d2(C2<T> v);
template <> __device__ __forceinline__ double2 to_d2<double>(double2 v) { return v; }
template <> __device__ __forceinline__ double2 to_d2<float>(float2 v) {
  return make_double2(widen_f32(v.x), widen_f32(v.y));
}
template <typename T> __device__ __forceinline__ C2<T> from_d(double x, double y);
template <> __device__ __forceinline__ double2 from_d<double>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 from_d<float>(double x, double y) {
  return make_float2(narrow_f64(x), narrow_f64(y));
}

template <typename T, bool ZERO_MODE>
__device__ __forceinline__ void thomas_column(const Geo& g, const double* __restrict__ invd,
                                              C2<T>* spec, double2* ybuf, size_t col, size_t stride) {
  constexpr int PF = 4;
  const int nz = g.nz;
  double mr = 0.0, mi = 0.0;
  if (ZERO_MODE) {
    for (int k = 0; k < nz; ++k) {
      const double2 f = to_d2<T>(spec[(size_t)k * stride + col]);
      mr += g.dzf[k] * f.x;
      mi += g.dzf[k] * f.y;
    }
    mr /= g.lz;
    mi /= g.lz;
  }
  // forward sweep: y_k = f_k - (a_k / d_{k-1}) y_{k-1}
  C2<T> fq[PF];
  double dq[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const int k = u < nz ? u : nz - 1;
    fq[u] = spec[(size_t)k * stride + col];
    dq[u] = invd[(size_t)k * stride + col];
  }
  double yr = 0.0, yi = 0.0, dprev = 0.0;
  for (int k0 = 0; k0 < nz; k0 += PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int k = k0 + u;
      if (k < nz) {
        const double2 f = to_d2<T>(fq[u]);
        const double d = dq[u];
        const int kn = k + PF < nz ? k + PF : nz - 1;
        fq[u] = spec[(size_t)kn * stride + col];
        dq[u] = invd[(size_t)kn * stride + col];
        const double m = (k == 0) ? 0.0 : g.za[k] * dprev;
        yr = (f.x - mr) - m * yr;
        yi = (f.y - mi) - m * yi;
        ybuf[(size_t)k * stride + col] = make_double2(yr, yi);
        dprev = d;
      }
    }
  }
  // back substitution: x_k = (y_k - c_k x_{k+1}) / d_k
  double xr = yr * dprev, xi = yi * dprev;
  spec[(size_t)(nz - 1) * stride + col] = from_d<T>(xr, xi);
  double2 yq[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const int k = nz - 2 - u >= 0 ? nz - 2 - u : 0;
    yq[u] = ybuf[(size_t)k * stride + col];
    dq[u] = invd[(size_t)k * stride + col];
  }
  for (int k0 = nz - 2; k0 >= 0; k0 -= PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int k = k0 - u;
      if (k >= 0) {
        const double2 y = yq[u];
        const double d = dq[u];
        const int kn = k - PF >= 0 ? k - PF : 0;
        yq[u] = ybuf[(size_t)kn * stride + col];
        dq[u] = invd[(size_t)kn * stride + col];
        const double c = g.zc[k];
        xr = (y.x - c * xr) * d;
        xi = (y.y - c * xi) * d;
        spec[(size_t)k * stride + col] = from_d<T>(xr, xi);
      }
    }
  }
}

// The same solve with the real and imaginary parts of a column in two
// threads (twice the parallelism) and the elimination multipliers
// m_k = a_k / d_{k-1} read from a table: per scalar one FP64 FMA forward and
// one FMA + one multiply backward.  The recurrences run in FP64 registers;
// the forward-sweep values are stored in place in the spectrum's own
// precision (FP32 on mixed plans, like the spectrum the solve reads and
// writes).  Scalar view: spec as T[nz][2 ncol].
template <typename T>
__device__ __forceinline__ void stage_tridiag_split(const Geo& g, const double* __restrict__ mtab,
                                                    const double* __restrict__ invd, T* spec,
                                                    size_t sid) {
  constexpr int PF = 4;
  const size_t ncol = (size_t)g.ny * g.nxh;
  if (sid >= 2 * ncol) return;
  const size_t col = sid >> 1;
  const size_t stride = 2 * ncol;
  const int nz = g.nz;
  auto ld = [&](size_t o) -> double {
    if (sizeof(T) == sizeof(float)) return widen_f32((float)spec[o]);
    return (double)spec[o];
  };
  auto stv = [&](size_t o, double v) {
    if (sizeof(T) == sizeof(float)) spec[o] = (T)narrow_f64(v);
    else spec[o] = (T)v;
  };
  if (col == 0) {  // singular (0, 0) column: remove the dzf-weighted mean first
    double mean = 0.0;
    for (int k = 0; k < nz; ++k) mean += g.dzf[k] * ld((size_t)k * stride + sid);
    mean /= g.lz;
    for (int k = 0; k < nz; ++k) stv((size_t)k * stride + sid, ld((size_t)k * stride + sid) - mean);
  }
  double fq[PF], mq[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const int k = u < nz ? u : nz - 1;
    fq[u] = ld((size_t)k * stride + sid);
    mq[u] = mtab[(size_t)k * ncol + col];
  }
  double y = 0.0;
  for (int k0 = 0; k0 < nz; k0 += PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int k = k0 + u;
      if (k < nz) {
        const double f = fq[u], m = mq[u];
        const int kn = k + PF < nz ? k + PF : nz - 1;
        fq[u] = ld((size_t)kn * stride + sid);
        mq[u] = mtab[(size_t)kn * ncol + col];
        y = fma(-m, y, f);
        if (k < nz - 1) stv((size_t)k * stride + sid, y);
      }
    }
  }
  double x = y * invd[(size_t)(nz - 1) * ncol + col];
  stv((size_t)(nz - 1) * stride + sid, x);
  double yq[PF], dq[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const int k = nz - 2 - u >= 0 ? nz - 2 - u : 0;
    yq[u] = ld((size_t)k * stride + sid);
    dq[u] = invd[(size_t)k * ncol + col];
  }
  for (int k0 = nz - 2; k0 >= 0; k0 -= PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int k = k0 - u;
      if (k >= 0) {
        const double yy = yq[u], d = dq[u];
        const int kn = k - PF >= 0 ? k - PF : 0;
        yq[u] = ld((size_t)kn * stride + sid);
        dq[u] = invd[(size_t)kn * ncol + col];
        x = fma(-g.zc[k], x, yy) * d;
        stv((size_t)k * stride + sid, x);
      }
    }
  }
}

// Inverse x transform of two half spectra per complex sequence, then
// p = scale * z (p_zero) or p += scale * z.  The p values a thread updates
// are loaded before the transform so their latency overlaps it.
template <typename T>
__device__ __forceinline__ void stage_fftx_inv(const Geo& g, const FftDesc& fx,
                                               const C2<T>* __restrict__ twx,
                                               const C2<T>* __restrict__ spec, double scale,
                                               double* __restrict__ p, int p_zero, int rpb, int blk,
                                               T* __restrict__ delta, unsigned char* smem_raw) {
  const int nx = g.nx, ny = g.ny, nz = g.nz, nxh = g.nxh;
  const int nseq = rpb >> 1;
  const float scale_f = (float)scale;
  C2<T>* bufA = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* bufB = bufA + (size_t)nseq * nx;
  const long nrows = (long)nz * ny;
  const long row0 = (long)blk * rpb;
  const bool even = (nx & 1) == 0;
  const int nout = rpb * nx;
  const int lgx = ((nx & (nx - 1)) == 0) ? 31 - __clz(nx) : -1;
  auto split = [&](int t, int& q, int& i) {
    if (lgx >= 0) { q = t >> lgx; i = t & (nx - 1); }
    else { q = t / nx; i = t - q * nx; }
  };
  constexpr int NP = kPrefetchInv;
  double pv[NP];
#pragma unroll
  for (int u = 0; u < NP; ++u) {
    const int t = threadIdx.x + u * blockDim.x;
    int q, i;
    split(t, q, i);
    pv[u] = 0.0;
    if (!p_zero && t < nout && row0 + q < nrows) pv[u] = p[(size_t)(row0 + q) * nx + i];
  }
  for (int t = threadIdx.x; t < nseq * nx; t += blockDim.x) {
    int q, kx;
    split(t, q, kx);
    const long ra = row0 + 2 * q;
    const bool upper = kx >= nxh;
    const int m = upper ? nx - kx : kx;
    C2<T> A, B;
    A.x = A.y = B.x = B.y = (T)0;
    if (ra < nrows) A = spec[(size_t)ra * nxh + m];
    if (ra + 1 < nrows) B = spec[(size_t)(ra + 1) * nxh + m];
    if (m == 0 || (even && m == nx / 2)) { A.y = (T)0; B.y = (T)0; }
    if (upper) { A.y = -A.y; B.y = -B.y; }
    C2<T> Z;
    Z.x = A.x - B.y;
    Z.y = A.y + B.x;
    bufA[t] = Z;
  }
  __syncthreads();
  const C2<T>* res = fft_dispatch<T, 1, false>(bufA, bufB, fx, nseq, 1, nx, twx, threadIdx.x, blockDim.x);
#pragma unroll
  for (int u = 0; u < NP; ++u) {
    const int t = threadIdx.x + u * blockDim.x;
    int q, i;
    split(t, q, i);
    const long row = row0 + q;
    if (t < nout && row < nrows) {
      const C2<T> z = res[(size_t)(q >> 1) * nx + i];
      const T zv = (q & 1) ? z.y : z.x;
      const double zd = (sizeof(T) == sizeof(float)) ? widen_f32((float)zv) : (double)zv;
      p[(size_t)row * nx + i] = fma(scale, zd, pv[u]);
      if (delta != nullptr)
        delta[(size_t)row * nx + i] = (sizeof(T) == sizeof(float)) ? (T)(scale_f * (float)zv) : (T)(scale * zd);
    }
  }
  for (int t = threadIdx.x + NP * blockDim.x; t < nout; t += blockDim.x) {  // beyond the prefetch
    int q, i;
    split(t, q, i);
    const long row = row0 + q;
    if (row < nrows) {
      const C2<T> z = res[(size_t)(q >> 1) * nx + i];
      const T zv = (q & 1) ? z.y : z.x;
      const double zd = (sizeof(T) == sizeof(float)) ? widen_f32((float)zv) : (double)zv;
      const size_t c = (size_t)row * nx + i;
      p[c] = p_zero ? scale * zd : fma(scale, zd, p[c]);
      if (delta != nullptr) delta[c] = scale_f * (float)zv;
    }
  }
}


}  // namespace pp
