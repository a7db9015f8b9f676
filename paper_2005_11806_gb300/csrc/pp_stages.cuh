// Device-side stages of one constant-coefficient eigenexpansion solve
// (Sec. 3.3.1: the pressure equation with homogeneous boundary conditions
// solved exactly by the eigenexpansion method) and of Algorithm 1's pass:
// residual + forward x transform, y transforms, the per-(kx, ky) tridiagonal
// solve along z, and the inverse x transform fused with the pressure update.
// The single-grid kernels (pp_kernels_fft.cu) and the grouped multi-grid
// kernels (pp_batch.cu) both call these.
#pragma once
#include <type_traits>

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

// FP32 fast path (fft_block_smem) for the same shapes; returns the element
// offset of the result buffer, or -1 when the shape has no fast path (the
// caller then runs fft_dispatch).  twb: offset of the N-entry twiddle table.
#define PP_TRY_SMEM(NN, NBB)                                                                        \
  if (n == NN && nbatch == NBB) {                                                                   \
    if (BATCH_FAST) return fft_block_smem<DIR, true, NN, NBB, NBB, 1>(a, b, twb, tid, nth);         \
    return fft_block_smem<DIR, false, NN, NBB, 1, NN>(a, b, twb, tid, nth);                         \
  }

template <int DIR, bool BATCH_FAST>
__device__ __forceinline__ int fft_dispatch_smem(int a, int b, int twb, const FftDesc& d, int nbatch, int es,
                                                 int bs, int tid, int nth) {
  const int n = d.n;
  const bool shape_ok = BATCH_FAST ? (es == nbatch && bs == 1) : (es == 1 && bs == n);
  if (!shape_ok) return -1;
  if (BATCH_FAST) {
    PP_TRY_SMEM(512, 4)
    PP_TRY_SMEM(256, 8)
    PP_TRY_SMEM(128, 16)
    PP_TRY_SMEM(128, 8)
    PP_TRY_SMEM(64, 16)
    PP_TRY_SMEM(64, 8)
  } else {
    PP_TRY_SMEM(512, 4)
    PP_TRY_SMEM(256, 8)
    PP_TRY_SMEM(128, 16)
    PP_TRY_SMEM(64, 32)
    PP_TRY_SMEM(32, 32)
  }
  return -1;
}
#undef PP_TRY_SMEM

// Whether fft_dispatch_smem has a fast path for this shape (host and device).
__host__ __device__ inline bool fft_smem_shape(int n, int nbatch, bool batch_fast) {
  if (batch_fast)
    return (n == 512 && nbatch == 4) || (n == 256 && nbatch == 8) || (n == 128 && (nbatch == 16 || nbatch == 8)) ||
           (n == 64 && (nbatch == 16 || nbatch == 8));
  return (n == 512 && nbatch == 4) || (n == 256 && nbatch == 8) || (n == 128 && nbatch == 16) ||
         (n == 64 && nbatch == 32) || (n == 32 && nbatch == 32);
}

// Copies the N-entry twiddle table into shared memory at element offset twb.
__device__ __forceinline__ void load_twiddles_smem(const float2* __restrict__ tw, int n, int twb) {
  float2* S = smem_f2();
  for (int i = threadIdx.x; i < n; i += blockDim.x) S[twb + i] = tw[i];
}

// ---------------------------------------------------------------------------
// Update pass of the mixed residual for nx % 4 == 0, vectorised: each thread
// takes the two rows of one complex sequence and four consecutive cells of
// each (16-byte loads of E, delta and the FP32 coefficients, all issued
// before the arithmetic), subtracts A delta = sum_nb c_nb (delta_nb -
// delta_c) from E, and writes the scaled residual of both rows as two
// interleaved complex pairs.  Same per-cell arithmetic as the scalar path.
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

template <bool YS>
__device__ __forceinline__ void resid_update_vec4(const Geo& g, const Faces& fc, float* __restrict__ E,
                                                  const float* __restrict__ delta, int scale_rho,
                                                  bool const_scale, float rt_f, long row0, int rpb,
                                                  float2* bufA, int seq_stride, float& s2, float& s1) {
  // 32-bit cell offsets (grids keep nx ny (nz + 1) below 2^31); the block's
  // first row is split into (layer, row in layer) once, the others step
  // from it (no 64-bit division per cell group)
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int nrows = nz * ny;
  const unsigned plane = (unsigned)nx * ny;
  const int t4 = nx >> 2;
  const int npairs = rpb >> 1;
  const int lg4 = ((t4 & (t4 - 1)) == 0) ? 31 - __clz(t4) : -1;
  const int r0 = (int)row0;
  const int k0 = r0 / ny, j0 = r0 - k0 * ny;
  for (int w = threadIdx.x; w < npairs * t4; w += blockDim.x) {
    const int qp = lg4 >= 0 ? (w >> lg4) : w / t4;
    const int i = (w - qp * t4) << 2;
    float4 rr[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = r0 + 2 * qp + h;
      float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < nrows) {
        int k = k0, j = j0 + 2 * qp + h;
        while (j >= ny) { j -= ny; ++k; }
        const int jp = (j + 1 == ny) ? 0 : j + 1, jm = (j == 0) ? ny - 1 : j - 1;
        const unsigned rowoff = (unsigned)row * nx;
        const unsigned kp = (unsigned)k * plane;
        const unsigned c = rowoff + i;
        const unsigned cyp = kp + (unsigned)jp * nx + i, cym = kp + (unsigned)jm * nx + i;
        const int il = (i == 0) ? nx - 1 : i - 1, ir = (i + 4 == nx) ? 0 : i + 4;
        const float4 d = ld4(delta + c);
        const float dl = delta[rowoff + il], dr = delta[rowoff + ir];
        const float4 dyp = ld4(delta + cyp), dym = ld4(delta + cym);
        const bool up = k + 1 < nz, dn = k > 0;
        float4 dzp = d, dzm = d;
        if (up) dzp = ld4(delta + c + plane);
        if (dn) dzm = ld4(delta + c - plane);
        // FP32 face coefficients from the FP32 density of the cell and its
        // six neighbours and the layer factors (z walls: factor 0; y walls:
        // the wall faces of rows 0 and ny - 1 are 0)
        const float4 rc = ld4(fc.rhof + c);
        const float rl = fc.rhof[rowoff + il], rr = fc.rhof[rowoff + ir];
        const float4 ryp = ld4(fc.rhof + cyp), rym = ld4(fc.rhof + cym);
        float4 rzp = rc, rzm = rc;
        if (up) rzp = ld4(fc.rhof + c + plane);
        if (dn) rzm = ld4(fc.rhof + c - plane);
        const int nz1 = nz + 1;
        // stretched y: row factor s_j on the x and z faces, t_j and t_{j+1}
        // on the y faces below and above, 1 / s_j on the cell's value
        // (a separate instantiation: the uniform one keeps its registers)
        float wx = g.cw_f[k];
        float wyl = (g.ywall && j == 0) ? 0.f : g.cw_f[nz1 + k];
        float wyh = (g.ywall && j + 1 == ny) ? 0.f : g.cw_f[nz1 + k];
        float wzp = g.cw_f[2 * nz1 + k + 1], wzm = g.cw_f[2 * nz1 + k];
        if constexpr (YS) {
          const float sj = g.ym_f[j];
          wx *= sj;
          wzp *= sj;
          wzm *= sj;
          wyl *= g.ym_f[ny + j];
          wyh = (j + 1 < ny) ? wyh * g.ym_f[ny + j + 1] : 0.f;
        }
        const float4 cx = make_float4(wx * face_beta_f(rl, rc.x), wx * face_beta_f(rc.x, rc.y),
                                      wx * face_beta_f(rc.y, rc.z), wx * face_beta_f(rc.z, rc.w));
        const float cxr = wx * face_beta_f(rc.w, rr);
        const float4 cyp4 = make_float4(wyh * face_beta_f(rc.x, ryp.x), wyh * face_beta_f(rc.y, ryp.y),
                                        wyh * face_beta_f(rc.z, ryp.z), wyh * face_beta_f(rc.w, ryp.w));
        const float4 cym4 = make_float4(wyl * face_beta_f(rc.x, rym.x), wyl * face_beta_f(rc.y, rym.y),
                                        wyl * face_beta_f(rc.z, rym.z), wyl * face_beta_f(rc.w, rym.w));
        const float4 czp = make_float4(wzp * face_beta_f(rc.x, rzp.x), wzp * face_beta_f(rc.y, rzp.y),
                                       wzp * face_beta_f(rc.z, rzp.z), wzp * face_beta_f(rc.w, rzp.w));
        const float4 czm = make_float4(wzm * face_beta_f(rc.x, rzm.x), wzm * face_beta_f(rc.y, rzm.y),
                                       wzm * face_beta_f(rc.z, rzm.z), wzm * face_beta_f(rc.w, rzm.w));
        float4 e = ld4(E + c);
        const float4 rh = scale_rho && !const_scale ? rc : make_float4(rt_f, rt_f, rt_f, rt_f);
        float idzf = g.inv_dzf_f[k];
        if constexpr (YS) idzf *= g.ym_f[2 * ny + j];
        auto cell = [&](float dc, float dxm, float dxp, float cxm, float cxp, float dypv, float cypv,
                        float dymv, float cymv, float dzpv, float czpv, float dzmv, float czmv, float& ev,
                        float rhv) -> float {
          float t = cxp * (dxp - dc);
          t = fmaf(cxm, dxm - dc, t);
          t = fmaf(cypv, dypv - dc, t);
          t = fmaf(cymv, dymv - dc, t);
          t = fmaf(czpv, dzpv - dc, t);
          t = fmaf(czmv, dzmv - dc, t);
          ev = ev - t;
          const float ee = ev * idzf;
          s2 = fmaf(ee, ee, s2);
          s1 += fabsf(ee);
          return scale_rho ? rhv * ee : ee;
        };
        r.x = cell(d.x, dl, d.y, cx.x, cx.y, dyp.x, cyp4.x, dym.x, cym4.x, dzp.x, czp.x, dzm.x, czm.x, e.x, rh.x);
        r.y = cell(d.y, d.x, d.z, cx.y, cx.z, dyp.y, cyp4.y, dym.y, cym4.y, dzp.y, czp.y, dzm.y, czm.y, e.y, rh.y);
        r.z = cell(d.z, d.y, d.w, cx.z, cx.w, dyp.z, cyp4.z, dym.z, cym4.z, dzp.z, czp.z, dzm.z, czm.z, e.z, rh.z);
        r.w = cell(d.w, d.z, dr, cx.w, cxr, dyp.w, cyp4.w, dym.w, cym4.w, dzp.w, czp.w, dzm.w, czm.w, e.w, rh.w);
        *reinterpret_cast<float4*>(E + c) = e;
      }
      rr[h] = r;
    }
    float4* dst = reinterpret_cast<float4*>(bufA + qp * seq_stride + i);
    dst[0] = make_float4(rr[0].x, rr[1].x, rr[0].y, rr[1].y);
    dst[1] = make_float4(rr[0].z, rr[1].z, rr[0].w, rr[1].w);
  }
}

// The same update with the two rows of a sequence taken together.  With ny
// even, rows 2q and 2q + 1 of a block (its first row is even) lie in one
// layer and are y neighbours of each other: the rows j - 1 .. j + 2 of delta
// and of the density are loaded once each (four float4 loads fewer per
// pair) and the face between the two rows is formed once (four reciprocals
// fewer).  Same per-cell arithmetic as resid_update_vec4.
template <bool YS>
__device__ __forceinline__ void resid_update_pair4(const Geo& g, const Faces& fc, float* __restrict__ E,
                                                   const float* __restrict__ delta, int scale_rho,
                                                   bool const_scale, float rt_f, long row0, int rpb,
                                                   float2* bufA, int seq_stride, float& s2, float& s1) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int nrows = nz * ny;
  const unsigned plane = (unsigned)nx * ny;
  const int t4 = nx >> 2;
  const int npairs = rpb >> 1;
  const int lg4 = ((t4 & (t4 - 1)) == 0) ? 31 - __clz(t4) : -1;
  const int r0 = (int)row0;
  const int k0 = r0 / ny, j0 = r0 - k0 * ny;
  const int nz1 = nz + 1;
  for (int w = threadIdx.x; w < npairs * t4; w += blockDim.x) {
    const int qp = lg4 >= 0 ? (w >> lg4) : w / t4;
    const int i = (w - qp * t4) << 2;
    const int row = r0 + 2 * qp;  // row A; row B = row + 1, same layer
    float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra;
    if (row < nrows) {
      int k = k0, j = j0 + 2 * qp;
      while (j >= ny) { j -= ny; ++k; }
      const int jm = (j == 0) ? ny - 1 : j - 1;
      const int jpp = (j + 2 == ny) ? 0 : j + 2;
      const unsigned oa = (unsigned)row * nx, ob = oa + nx;
      const unsigned kp = (unsigned)k * plane;
      const unsigned ca = oa + i, cb = ob + i;
      const unsigned cm = kp + (unsigned)jm * nx + i, cp = kp + (unsigned)jpp * nx + i;
      const int il = (i == 0) ? nx - 1 : i - 1, ir = (i + 4 == nx) ? 0 : i + 4;
      const bool up = k + 1 < nz, dn = k > 0;
      const bool own = scale_rho && !const_scale;
      // layer factors; the y faces below A (face j), between A and B (face
      // j + 1) and above B (face j + 2); walls in y zero the faces of rows
      // 0 and ny - 1
      float wxA = g.cw_f[k], wxB = wxA;
      const float wy = g.cw_f[nz1 + k];
      float wlo = (g.ywall && j == 0) ? 0.f : wy, wmid = wy, whi = (g.ywall && j + 2 == ny) ? 0.f : wy;
      float wuA = g.cw_f[2 * nz1 + k + 1], wdA = g.cw_f[2 * nz1 + k], wuB = wuA, wdB = wdA;
      float idA = g.inv_dzf_f[k], idB = idA;
      if constexpr (YS) {
        const float sA = g.ym_f[j], sB = g.ym_f[j + 1];
        wxA *= sA; wuA *= sA; wdA *= sA;
        wxB *= sB; wuB *= sB; wdB *= sB;
        wlo *= g.ym_f[ny + j];
        wmid *= g.ym_f[ny + j + 1];
        whi = (j + 2 < ny) ? whi * g.ym_f[ny + j + 2] : 0.f;
        idA *= g.ym_f[2 * ny + j];
        idB *= g.ym_f[2 * ny + j + 1];
      }
      auto cell = [&](float dc, float dxm, float dxp, float cxm, float cxp, float dypv, float cypv,
                      float dymv, float cymv, float dzpv, float czpv, float dzmv, float czmv, float& ev,
                      float rhv, float idzf) -> float {
        float t = cxp * (dxp - dc);
        t = fmaf(cxm, dxm - dc, t);
        t = fmaf(cypv, dypv - dc, t);
        t = fmaf(cymv, dymv - dc, t);
        t = fmaf(czpv, dzpv - dc, t);
        t = fmaf(czmv, dzmv - dc, t);
        ev = ev - t;
        const float ee = ev * idzf;
        s2 = fmaf(ee, ee, s2);
        s1 += fabsf(ee);
        return scale_rho ? (own ? rhv : rt_f) * ee : ee;
      };
      // the two centre rows (A's y+ neighbour is B, B's y- neighbour is A)
      const float4 dA = ld4(delta + ca), dB = ld4(delta + cb);
      const float4 hA = ld4(fc.rhof + ca), hB = ld4(fc.rhof + cb);
      const float4 cym = make_float4(wmid * face_beta_f(hA.x, hB.x), wmid * face_beta_f(hA.y, hB.y),
                                     wmid * face_beta_f(hA.z, hB.z), wmid * face_beta_f(hA.w, hB.w));
      {  // row A: y- neighbour row j - 1 (face j)
        const float4 dM = ld4(delta + cm), hM = ld4(fc.rhof + cm);
        const float dAl = delta[oa + il], dAr = delta[oa + ir];
        const float hAl = fc.rhof[oa + il], hAr = fc.rhof[oa + ir];
        float4 dAu = dA, dAd = dA, hAu = hA, hAd = hA;
        if (up) { dAu = ld4(delta + ca + plane); hAu = ld4(fc.rhof + ca + plane); }
        if (dn) { dAd = ld4(delta + ca - plane); hAd = ld4(fc.rhof + ca - plane); }
        float4 eA = ld4(E + ca);
        const float4 cxA = make_float4(wxA * face_beta_f(hAl, hA.x), wxA * face_beta_f(hA.x, hA.y),
                                       wxA * face_beta_f(hA.y, hA.z), wxA * face_beta_f(hA.z, hA.w));
        const float cxAr = wxA * face_beta_f(hA.w, hAr);
        const float4 cyl = make_float4(wlo * face_beta_f(hA.x, hM.x), wlo * face_beta_f(hA.y, hM.y),
                                       wlo * face_beta_f(hA.z, hM.z), wlo * face_beta_f(hA.w, hM.w));
        const float4 cuA = make_float4(wuA * face_beta_f(hA.x, hAu.x), wuA * face_beta_f(hA.y, hAu.y),
                                       wuA * face_beta_f(hA.z, hAu.z), wuA * face_beta_f(hA.w, hAu.w));
        const float4 cdA = make_float4(wdA * face_beta_f(hA.x, hAd.x), wdA * face_beta_f(hA.y, hAd.y),
                                       wdA * face_beta_f(hA.z, hAd.z), wdA * face_beta_f(hA.w, hAd.w));
        ra.x = cell(dA.x, dAl, dA.y, cxA.x, cxA.y, dB.x, cym.x, dM.x, cyl.x, dAu.x, cuA.x, dAd.x, cdA.x, eA.x, hA.x, idA);
        ra.y = cell(dA.y, dA.x, dA.z, cxA.y, cxA.z, dB.y, cym.y, dM.y, cyl.y, dAu.y, cuA.y, dAd.y, cdA.y, eA.y, hA.y, idA);
        ra.z = cell(dA.z, dA.y, dA.w, cxA.z, cxA.w, dB.z, cym.z, dM.z, cyl.z, dAu.z, cuA.z, dAd.z, cdA.z, eA.z, hA.z, idA);
        ra.w = cell(dA.w, dA.z, dAr, cxA.w, cxAr, dB.w, cym.w, dM.w, cyl.w, dAu.w, cuA.w, dAd.w, cdA.w, eA.w, hA.w, idA);
        *reinterpret_cast<float4*>(E + ca) = eA;
      }
      {  // row B: y+ neighbour row j + 2 (face j + 2)
        const float4 dP = ld4(delta + cp), hP = ld4(fc.rhof + cp);
        const float dBl = delta[ob + il], dBr = delta[ob + ir];
        const float hBl = fc.rhof[ob + il], hBr = fc.rhof[ob + ir];
        float4 dBu = dB, dBd = dB, hBu = hB, hBd = hB;
        if (up) { dBu = ld4(delta + cb + plane); hBu = ld4(fc.rhof + cb + plane); }
        if (dn) { dBd = ld4(delta + cb - plane); hBd = ld4(fc.rhof + cb - plane); }
        float4 eB = ld4(E + cb);
        const float4 cxB = make_float4(wxB * face_beta_f(hBl, hB.x), wxB * face_beta_f(hB.x, hB.y),
                                       wxB * face_beta_f(hB.y, hB.z), wxB * face_beta_f(hB.z, hB.w));
        const float cxBr = wxB * face_beta_f(hB.w, hBr);
        const float4 cyh = make_float4(whi * face_beta_f(hB.x, hP.x), whi * face_beta_f(hB.y, hP.y),
                                       whi * face_beta_f(hB.z, hP.z), whi * face_beta_f(hB.w, hP.w));
        const float4 cuB = make_float4(wuB * face_beta_f(hB.x, hBu.x), wuB * face_beta_f(hB.y, hBu.y),
                                       wuB * face_beta_f(hB.z, hBu.z), wuB * face_beta_f(hB.w, hBu.w));
        const float4 cdB = make_float4(wdB * face_beta_f(hB.x, hBd.x), wdB * face_beta_f(hB.y, hBd.y),
                                       wdB * face_beta_f(hB.z, hBd.z), wdB * face_beta_f(hB.w, hBd.w));
        rb.x = cell(dB.x, dBl, dB.y, cxB.x, cxB.y, dP.x, cyh.x, dA.x, cym.x, dBu.x, cuB.x, dBd.x, cdB.x, eB.x, hB.x, idB);
        rb.y = cell(dB.y, dB.x, dB.z, cxB.y, cxB.z, dP.y, cyh.y, dA.y, cym.y, dBu.y, cuB.y, dBd.y, cdB.y, eB.y, hB.y, idB);
        rb.z = cell(dB.z, dB.y, dB.w, cxB.z, cxB.w, dP.z, cyh.z, dA.z, cym.z, dBu.z, cuB.z, dBd.z, cdB.z, eB.z, hB.z, idB);
        rb.w = cell(dB.w, dB.z, dBr, cxB.w, cxBr, dP.w, cyh.w, dA.w, cym.w, dBu.w, cuB.w, dBd.w, cdB.w, eB.w, hB.w, idB);
        *reinterpret_cast<float4*>(E + cb) = eB;
      }
    }
    float4* dst = reinterpret_cast<float4*>(bufA + qp * seq_stride + i);
    dst[0] = make_float4(ra.x, rb.x, ra.y, rb.y);
    dst[1] = make_float4(ra.z, rb.z, ra.w, rb.w);
  }
}

// ---------------------------------------------------------------------------
// Residual of the variable-coefficient equation and forward real x transform.
//   mode 0: r = f (constant-coefficient solve)
//   mode 1: e = (D u^s - S_c)/dt, evaluated in FP64 in the row-scaled form
//           dzf_k e = b_s - (sum_nb c_nb p_nb - diag p_c), b_s = dzf_k b / dt;
//           r = rho e (or e).  The mixed path narrows dzf_k e to FP32 and
//           finishes (scaling, norms, rho) in FP32.
//   Mixed path with E: E = dzf_k e is kept in FP32.  An exact pass stores
//   the FP64 value narrowed; an update pass subtracts A delta, evaluated in
//   FP32 as sum_nb c_nb (delta_nb - delta_c) (no diagonal needed).
// Two real rows are packed into one complex sequence (re = even row,
// im = odd row), transformed together and separated afterwards.
// The rows [row0, row0 + rpb) of the residual (the first step of the stage
// below) into bufA: complex sequence q = (row - row0) / 2 at element offset
// q * seq_stride (re = even row, im = odd row); s2, s1 accumulate e^2 and
// |e| of the thread's cells.  Every thread of the block calls it.
template <typename T, bool YS>
__device__ __forceinline__ void resid_rows(const Geo& g, const Faces& fc, const double* __restrict__ b,
                                           const double* __restrict__ rho, const double* __restrict__ p, int mode,
                                           int p_zero, int scale_rho, long row0, int rpb, bool need_exact,
                                           float* __restrict__ E, const float* __restrict__ delta, C2<T>* bufA,
                                           int seq_stride, T& s2, T& s1) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const bool update = (E != nullptr) && !p_zero && !need_exact;
  const int nrows = nz * ny;
  const size_t plane = (size_t)ny * nx;
  // constant scaling of Methods I and II (one device scalar for all cells)
  const bool const_scale = fc.rho_tilde != nullptr;
  const double rt = (const_scale && mode != 0) ? *fc.rho_tilde : 0.0;
  const float rt_f = (float)rt;
  // thread -> (row offset, first column); index math is done once per row
  const int tpr = nx < (int)blockDim.x ? nx : (int)blockDim.x;
  const int rows_par = blockDim.x / tpr;
  const int qoff = threadIdx.x / tpr, i0 = threadIdx.x - qoff * tpr;
  const bool vec = update && sizeof(T) == sizeof(float) && (nx & 3) == 0;
  if (vec) {
    float a2 = 0.f, a1 = 0.f;
    if ((ny & 1) == 0)  // the two rows of a sequence share a layer
      resid_update_pair4<YS>(g, fc, E, delta, scale_rho, const_scale, rt_f, row0, rpb,
                             reinterpret_cast<float2*>(bufA), seq_stride, a2, a1);
    else
      resid_update_vec4<YS>(g, fc, E, delta, scale_rho, const_scale, rt_f, row0, rpb,
                            reinterpret_cast<float2*>(bufA), seq_stride, a2, a1);
    s2 += (T)a2;
    s1 += (T)a1;
  }
  for (int q = qoff; !vec && q < rpb && qoff < rows_par; q += rows_par) {
    const int row = (int)row0 + q;
    const bool valid = row < nrows;
    const int k = valid ? row / ny : 0, j = valid ? row - k * ny : 0;
    const int jp = (j + 1 == ny) ? 0 : j + 1, jm = (j == 0) ? ny - 1 : j - 1;
    const size_t rowoff = (size_t)row * nx;
    const size_t kp = (size_t)k * plane;
    const size_t rowp = kp + (size_t)jp * nx, rowm = kp + (size_t)jm * nx;
    // stretched y: the row is scaled by dzf_k s_j (Geo::ym)
    const bool ys = YS && valid;
    const float idzf_f =
        (mode != 0 && sizeof(T) == sizeof(float)) ? g.inv_dzf_f[k] * (ys ? g.ym_f[2 * ny + j] : 1.f) : 0.f;
    const double idzf =
        (mode != 0 && sizeof(T) == sizeof(double)) ? g.inv_dzf[k] * (ys ? g.ym[2 * ny + j] : 1.0) : 0.0;
    const float ysj = ys ? g.ym_f[j] : 1.f, ytlo = ys ? g.ym_f[ny + j] : 1.f;
    const float ythi = ys ? ((j + 1 < ny) ? g.ym_f[ny + j + 1] : 0.f) : 1.f;
    for (int i = i0; i < nx; i += tpr) {
      T r = (T)0;
      if (valid) {
        const size_t c = rowoff + i;
        if (mode == 0) {
          r = (T)b[c];
        } else {
          const int ip = (i + 1 == nx) ? 0 : i + 1, im = (i == 0) ? nx - 1 : i - 1;
          double ep = 0.0;
          float ev = 0.f;  // FP32 dzf_k e of the mixed path
          if (update) {
            // E^s = E^{s-1} - A delta, A delta in FP32 with the FP32
            // coefficients formed from rhof (as in resid_update_vec4)
            const float dc = delta[c];
            const float rcc = fc.rhof[c];
            const int nz1 = nz + 1;
            const float wx = g.cw_f[k] * ysj, wy = g.cw_f[nz1 + k];
            const float wyl = (g.ywall && j == 0) ? 0.f : wy * ytlo;
            const float wyh = (g.ywall && j + 1 == ny) ? 0.f : wy * ythi;
            float t = wx * face_beta_f(rcc, fc.rhof[rowoff + ip]) * (delta[rowoff + ip] - dc);
            t = fmaf(wx * face_beta_f(fc.rhof[rowoff + im], rcc), delta[rowoff + im] - dc, t);
            t = fmaf(wyh * face_beta_f(rcc, fc.rhof[rowp + i]), delta[rowp + i] - dc, t);
            t = fmaf(wyl * face_beta_f(rcc, fc.rhof[rowm + i]), delta[rowm + i] - dc, t);
            if (k + 1 < nz)
              t = fmaf(g.cw_f[2 * nz1 + k + 1] * ysj * face_beta_f(rcc, fc.rhof[c + plane]), delta[c + plane] - dc, t);
            if (k > 0)
              t = fmaf(g.cw_f[2 * nz1 + k] * ysj * face_beta_f(rcc, fc.rhof[c - plane]), delta[c - plane] - dc, t);
            ev = E[c] - t;
            E[c] = ev;
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
            if (sizeof(T) == sizeof(float)) {
              ev = narrow_f64(ep);
              if (E != nullptr) E[c] = ev;
            }
          }
          if (sizeof(T) == sizeof(float)) {
            const float e = ev * idzf_f;
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
      C2<T>& z = bufA[(size_t)(q >> 1) * seq_stride + i];
      if (q & 1) z.y = r; else z.x = r;
    }
  }
}

template <typename T, bool YS = false>
__device__ __forceinline__ void stage_resid_fftx(const Geo& g, const Faces& fc, const FftDesc& fx,
                                                 const C2<T>* __restrict__ twx,
                                                 const double* __restrict__ b,
                                                 const double* __restrict__ rho,
                                                 const double* __restrict__ p, int mode, int p_zero,
                                                 int scale_rho, C2<T>* __restrict__ spec,
                                                 double* __restrict__ red, int rpb, int blk,
                                                 bool need_exact, float* __restrict__ E,
                                                 const float* __restrict__ delta,
                                                 unsigned char* smem_raw) {
  __shared__ double shred[64];
  const int nx = g.nx, ny = g.ny, nz = g.nz, nxh = g.nxh;
  const int nseq = rpb >> 1;
  C2<T>* bufA = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* bufB = bufA + (size_t)nseq * nx;
  const int nrows = nz * ny;
  const long row0 = (long)blk * rpb;
  T s2 = (T)0, s1 = (T)0;
  // FP32 fast transform: buffer A, buffer B (written padded by the first
  // pass: fft_pad_elems), then the twiddle table
  constexpr bool F32 = std::is_same<T, float>::value;
  const int twb = nseq * nx + fft_pad_elems(nseq * nx);
  const bool fast = F32 && fft_smem_shape(nx, nseq, false);
  if constexpr (F32) {
    if (fast) load_twiddles_smem(twx, nx, twb);
  }
  resid_rows<T, YS>(g, fc, b, rho, p, mode, p_zero, scale_rho, row0, rpb, need_exact, E, delta, bufA, nx, s2, s1);
  if (mode != 0) {
    // block partial sums of e^2 and |e|: in the arithmetic's own precision
    // (FP32 shuffles on mixed plans: the FP64 pipe is the scarce one)
    block_sum2<T>(s2, s1, reinterpret_cast<T*>(shred));
    if (threadIdx.x == 0) {
      red[2 * (size_t)blk] = (double)s2;
      red[2 * (size_t)blk + 1] = (double)s1;
    }
  }
  __syncthreads();
  const C2<T>* res = nullptr;
  if constexpr (F32) {
    if (fast)
      res = smem_f2() + fft_dispatch_smem<-1, false>(0, nseq * nx, twb, fx, nseq, 1, nx, threadIdx.x, blockDim.x);
  }
  if (!fast) res = fft_dispatch<T, -1, false>(bufA, bufB, fx, nseq, 1, nx, twx, threadIdx.x, blockDim.x);
  // (q, kx) walked incrementally: no division by the odd nxh per element
  int q = threadIdx.x / nxh, kx = threadIdx.x - q * nxh;
  const int dq = blockDim.x / nxh, dkx = blockDim.x - dq * nxh;
  for (; q < nseq; q += dq, kx += dkx) {
    if (kx >= nxh) { kx -= nxh; ++q; if (q >= nseq) break; }
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

// Row order of the cosine transform through a complex FFT (Makhoul): the
// sequence v_r = x_{2r} (r < n/2), v_r = x_{2(n-1-r)+1} (r >= n/2), n even.
__device__ __forceinline__ int dct_row(int r, int n) { return (r < (n >> 1)) ? 2 * r : 2 * (n - 1 - r) + 1; }

template <typename T> __device__ __forceinline__ C2<T> cmulc(C2<T> a, C2<T> b) {  // a * conj(b)
  C2<T> r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}

// Complex transform along y of one z-plane tile of tx consecutive kx.  DCT:
// the cosine transform of walls in y (dct = exp(-i pi m / (2 ny))), in the
// steps of the persistent kernel below: the forward pass loads the rows in
// the order dct_row and finishes with X_r = (w_r Z_r + conj(w_r)
// Z_{ny-r}) / 2, the inverse pass pairs (Y_m, Y_{ny-m}) before its FFT and
// stores the rows back in the order dct_row.
template <typename T, int DIR, bool DCT = false>
__device__ __forceinline__ void stage_ffty(const Geo& g, const FftDesc& fy, const C2<T>* __restrict__ twy,
                                           C2<T>* __restrict__ spec, int tx, int bx, int bz,
                                           unsigned char* smem_raw, const C2<T>* __restrict__ dct = nullptr) {
  constexpr bool REORDER_IN = DCT && DIR < 0;
  constexpr bool REORDER_OUT = DCT && DIR > 0;
  const int ny = g.ny, nxh = g.nxh;
  C2<T>* bufA = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* bufB = bufA + (size_t)ny * tx;
  const int kx0 = bx * tx;
  const size_t base = (size_t)bz * ny * nxh;
  const int lg_tx = 31 - __clz(tx);  // tx is a power of two (ffty_tile)
  constexpr bool F32 = std::is_same<T, float>::value;
  const int twb = ny * tx + fft_pad_elems(ny * tx);  // buffer B is written padded
  const bool fast = F32 && fft_smem_shape(ny, tx, true);
  if constexpr (F32) {
    if (fast) load_twiddles_smem(twy, ny, twb);
  }
  for (int t = threadIdx.x; t < ny * tx; t += blockDim.x) {
    const int r = t >> lg_tx, x = t & (tx - 1);
    const int y = REORDER_IN ? dct_row(r, ny) : r;
    C2<T> v; v.x = (T)0; v.y = (T)0;
    if (kx0 + x < nxh) v = spec[base + (size_t)y * nxh + kx0 + x];
    bufA[t] = v;
  }
  __syncthreads();
  if constexpr (REORDER_OUT) {
    // V_m and V_{ny-m} from the pair (Y_m, Y_{ny-m}), in place; V_0 = Y_0
    const int half = ny >> 1;
    for (int t = threadIdx.x; t < half * tx; t += blockDim.x) {
      const int m = 1 + (t >> lg_tx), x = t & (tx - 1);
      const C2<T> w = dct[m];
      const C2<T> a = bufA[m * tx + x], b = bufA[(ny - m) * tx + x];
      C2<T> d, e;  // a - i b, a + i b
      d.x = a.x + b.y; d.y = a.y - b.x;
      e.x = a.x - b.y; e.y = a.y + b.x;
      bufA[m * tx + x] = cmulc<T>(d, w);
      if (m != ny - m) bufA[(ny - m) * tx + x] = cmul<T>(e, w);
    }
    __syncthreads();
  }
  const C2<T>* res = nullptr;
  if constexpr (F32) {
    if (fast) res = smem_f2() + fft_dispatch_smem<DIR, true>(0, ny * tx, twb, fy, tx, tx, 1, threadIdx.x, blockDim.x);
  }
  if (!fast) res = fft_dispatch<T, DIR, true>(bufA, bufB, fy, tx, tx, 1, twy, threadIdx.x, blockDim.x);
  for (int t = threadIdx.x; t < ny * tx; t += blockDim.x) {
    const int r = t >> lg_tx, x = t & (tx - 1);
    if (kx0 + x >= nxh) continue;
    if constexpr (REORDER_IN) {
      // X_r = (w_r Z_r + conj(w_r) Z_{ny-r}) / 2
      const C2<T> w = dct[r];
      const C2<T> a = cmul<T>(res[t], w);
      const C2<T> b = cmulc<T>(res[(r == 0 ? 0 : ny - r) * tx + x], w);
      C2<T> o;
      o.x = (T)0.5 * (a.x + b.x);
      o.y = (T)0.5 * (a.y + b.y);
      spec[base + (size_t)r * nxh + kx0 + x] = o;
    } else {
      const int y = REORDER_OUT ? dct_row(r, ny) : r;
      spec[base + (size_t)y * nxh + kx0 + x] = res[t];
    }
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

// Lines of the spectrum [nz][ny][nxh] that a persistent transform walks.
// AXIS = 0: along y (length ny, element stride nxh), one tile per (z plane,
// kx tile).  AXIS = 1: along z (length nz, stride ny nxh), one tile per
// (ky, kx tile).
template <int AXIS> struct Lines {
  int n;             // transform length
  size_t rstride;    // elements between consecutive entries of a line
  size_t ostride;    // elements between consecutive outer indices
  __device__ __forceinline__ explicit Lines(const Geo& g)
      : n(AXIS ? g.nz : g.ny), rstride(AXIS ? (size_t)g.ny * g.nxh : (size_t)g.nxh),
        ostride(AXIS ? (size_t)g.nxh : (size_t)g.ny * g.nxh) {}
};

// REORDER: shared row r receives global row dct_row(r) (forward cosine
// transform); otherwise row r receives row r.
template <typename T, bool REORDER = false, int AXIS = 0>
__device__ __forceinline__ void ffty_issue_tile(const Geo& g, const C2<T>* __restrict__ spec, int tx, int ntx,
                                                long long tile, C2<T>* buf) {
  const Lines<AXIS> ln(g);
  const int n = ln.n, nxh = g.nxh;
  const int bz = (int)(tile / ntx), bx = (int)(tile - (long long)bz * ntx);
  const int kx0 = bx * tx;
  const size_t base = (size_t)bz * ln.ostride;
  const int lg_tx = 31 - __clz(tx);  // tx is a power of two (ffty_tile)
  for (int t = threadIdx.x; t < n * tx; t += blockDim.x) {
    const int r = t >> lg_tx, x = t & (tx - 1);
    const int y = REORDER ? dct_row(r, n) : r;
    if (kx0 + x < nxh) {
      const size_t at = base + (size_t)y * ln.rstride + kx0 + x;
      if (sizeof(C2<T>) == 8) cp_async8(&buf[t], &spec[at]);
      else {
        cp_async8(&buf[t], &spec[at]);
        cp_async8(reinterpret_cast<char*>(&buf[t]) + 8, reinterpret_cast<const char*>(&spec[at]) + 8);
      }
    } else {
      buf[t].x = (T)0;
      buf[t].y = (T)0;
    }
  }
  cp_async_commit();
}


// Persistent y transform.  DCT = false: complex DFT along y (periodic y).
// DCT = true (walls in y): the eigenbasis of the Neumann second difference
// on cell centres, X_m = sum_j x_j cos(pi m (2j + 1) / (2 ny)), computed
// with one complex FFT of length ny (Makhoul's reordering) and the twiddles
// w_m = exp(-i pi m / (2 ny)) of `dct`:
//   forward:  Z = FFT(x reordered by dct_row);
//             X_m = (w_m Z_m + conj(w_m) Z_{ny-m}) / 2   (Z_ny = Z_0);
//   inverse:  V_m = conj(w_m) (Y_m - i Y_{ny-m})          (Y_ny = 0);
//             x_{dct_row(r)} = (IFFT(V))_r, unnormalised like the periodic
//             inverse (the caller's 1/(nx ny) completes both).
// The transform acts on real and imaginary parts alike, so the complex
// x-spectrum goes through unchanged.
// AXIS = 1 runs the same transforms along z (uniform walls in z: the z
// eigenbasis is the same cosine basis).  Its forward pass also divides by
// the eigenvalue: X / (nz (lambda_x + lambda_y + lambda_z)), with the
// singular (0, 0, 0) mode set to 0 (zero mean), so forward + inverse is the
// whole z solve.
template <typename T, int DIR, bool DCT = false, int AXIS = 0>
__device__ __forceinline__ void stage_ffty_persistent(const Geo& g, const FftDesc& fy,
                                                      const C2<T>* __restrict__ twy, C2<T>* spec, int tx,
                                                      long long ntiles, long long first, long long stride,
                                                      unsigned char* smem_raw,
                                                      const C2<T>* __restrict__ dct = nullptr,
                                                      ZDivide zd = ZDivide{}) {
  constexpr bool REORDER_IN = DCT && DIR < 0;
  constexpr bool REORDER_OUT = DCT && DIR > 0;
  const Lines<AXIS> ln(g);
  const int ny = ln.n, nxh = g.nxh;  // ny: the transform length (ny, or nz for AXIS = 1)
  const int ntx = (nxh + tx - 1) / tx;
  const int tsz = ny * tx;
  const int lg_tx = 31 - __clz(tx);  // tx is a power of two (ffty_tile)
  C2<T>* X0 = reinterpret_cast<C2<T>*>(smem_raw);
  // element offsets of the three buffers, rotated (no pointer array: the
  // transforms then address shared memory directly)
  // FP32 fast path: Q, the scratch buffer of the transform, is written
  // padded by its first pass and holds fft_pad_elems(tsz) elements, then the
  // twiddle table follows; otherwise three plain buffers.  L and F (tsz
  // each) rotate.  The launcher sizes shared memory for the same layout.
  constexpr bool F32 = std::is_same<T, float>::value;
  const int qsz = F32 ? fft_pad_elems(tsz) : tsz;
  int L = 0, Q = tsz, F = tsz + qsz;
  const int twb = 2 * tsz + qsz;
  const bool fast = F32 && fft_smem_shape(ny, tx, true);
  if constexpr (F32) {
    if (fast) load_twiddles_smem(twy, ny, twb);
  }
  if (first < ntiles) ffty_issue_tile<T, REORDER_IN, AXIS>(g, spec, tx, ntx, first, X0 + L);
  for (long long tile = first; tile < ntiles; tile += stride) {
    cp_async_wait_all();
    __syncthreads();
    const long long next = tile + stride;
    if (next < ntiles) ffty_issue_tile<T, REORDER_IN, AXIS>(g, spec, tx, ntx, next, X0 + F);
    if constexpr (REORDER_OUT) {
      // V_m and V_{ny-m} from the pair (Y_m, Y_{ny-m}), in place; V_0 = Y_0.
      C2<T>* Y = X0 + L;
      const int half = ny >> 1;
      for (int t = threadIdx.x; t < half * tx; t += blockDim.x) {
        const int m = 1 + (t >> lg_tx), x = t & (tx - 1);
        const C2<T> w = dct[m];
        const C2<T> a = Y[m * tx + x], b = Y[(ny - m) * tx + x];
        C2<T> d, e;  // a - i b, a + i b
        d.x = a.x + b.y; d.y = a.y - b.x;
        e.x = a.x - b.y; e.y = a.y + b.x;
        if (m == ny - m) {
          Y[m * tx + x] = cmulc<T>(d, w);
        } else {
          Y[m * tx + x] = cmulc<T>(d, w);
          Y[(ny - m) * tx + x] = cmul<T>(e, w);
        }
      }
      __syncthreads();
    }
    const C2<T>* res = nullptr;
    if constexpr (F32) {
      if (fast) res = smem_f2() + fft_dispatch_smem<DIR, true>(L, Q, twb, fy, tx, tx, 1, threadIdx.x, blockDim.x);
    }
    if (!fast) res = fft_dispatch<T, DIR, true>(X0 + L, X0 + Q, fy, tx, tx, 1, twy, threadIdx.x, blockDim.x);
    const int bz = (int)(tile / ntx), bx = (int)(tile - (long long)bz * ntx);
    const int kx0 = bx * tx;
    const size_t base = (size_t)bz * ln.ostride;
    for (int t = threadIdx.x; t < ny * tx; t += blockDim.x) {
      const int r = t >> lg_tx, x = t & (tx - 1);
      if (kx0 + x >= nxh) continue;
      if constexpr (REORDER_IN) {
        // X_r = (w_r Z_r + conj(w_r) Z_{ny-r}) / 2
        const C2<T> w = dct[r];
        const C2<T> a = cmul<T>(res[t], w);
        const C2<T> b = cmulc<T>(res[(r == 0 ? 0 : ny - r) * tx + x], w);
        T h = (T)0.5;
        if constexpr (AXIS == 1) {
          // bz is ky here; the (0, 0, 0) mode is the pinned mean
          const double lam = zd.lamx[kx0 + x] + zd.lamy[bz] + zd.lamz[r];
          h = (kx0 + x == 0 && bz == 0 && r == 0) ? (T)0 : (T)(0.5 / ((double)ny * lam));
        }
        C2<T> o;
        o.x = h * (a.x + b.x);
        o.y = h * (a.y + b.y);
        spec[base + (size_t)r * ln.rstride + kx0 + x] = o;
      } else {
        const int y = REORDER_OUT ? dct_row(r, ny) : r;
        spec[base + (size_t)y * ln.rstride + kx0 + x] = res[t];
      }
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

// dzf-weighted z means of the real and imaginary parts of column 0 (scalar
// view T[nz][2 ncol]), reduced by the whole block; returned in sh[0], sh[1]
// (sh: at least 34 entries) after a barrier.  Every thread must call it.
template <typename T>
__device__ __forceinline__ void zero_column_means(const Geo& g, const T* spec, size_t stride, double* sh) {
  double sx = 0.0, sy = 0.0;
  for (int k = threadIdx.x; k < g.nz; k += blockDim.x) {
    sx += g.dzf[k] * (double)spec[(size_t)k * stride];
    sy += g.dzf[k] * (double)spec[(size_t)k * stride + 1];
  }
  sx = block_sum<double>(sx, sh);
  __syncthreads();
  sy = block_sum<double>(sy, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    sh[32] = sx / g.lz;
    sh[33] = sy / g.lz;
  }
  __syncthreads();
}

// The same solve with the real and imaginary parts of a column in two
// threads (twice the parallelism) and the elimination multipliers
// m_k = a_k / d_{k-1} read from a table: per scalar one FP64 FMA forward and
// one FMA + one multiply backward.  The recurrences run in FP64 registers;
// the forward-sweep values are stored in place in the spectrum's own
// precision (FP32 on mixed plans, like the spectrum the solve reads and
// writes).  Scalar view: spec as T[nz][2 ncol].  m0 is subtracted from every
// right-hand-side value: the dzf-weighted z mean of the singular (0, 0)
// column, 0 for every other column.
template <typename T>
__device__ __forceinline__ void stage_tridiag_split(const Geo& g, const double* __restrict__ mtab,
                                                    const double* __restrict__ invd, T* spec,
                                                    size_t sid, double m0 = 0.0) {
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
        y = fma(-m, y, f - m0);
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

// One column of a PP_MIXED_Z64 plan (TriZ64), both components in one thread
// (two independent FP64 chains sharing the table loads): both sweeps are
// FP64 recurrences with one FMA per row and component; the spectrum keeps
// its FP32 storage, so the forward values are stored as s_k = (1/d_k) y_k,
// rounded to FP32 and multiplied by the FP32 inverse pivot (the same 2^-24
// relative perturbation per value as storing y_k itself).  ZERO: the
// singular column 0, whose right-hand side first loses its dzf-weighted z
// mean (m0x, m0y).  Loads run PF rows ahead.  32-bit offsets: the plan keeps
// nx ny (nz + 1) below 2^31.
template <bool ZERO>
__device__ __forceinline__ void stage_tridiag_z64(const Geo& g, const TriZ64& t, float2* __restrict__ spec,
                                                  unsigned col, unsigned ncol, unsigned tc, unsigned ntc,
                                                  double m0x, double m0y) {
  constexpr int PF = 4;
  const int nz = g.nz;
  const double* __restrict__ tm = t.m;
  const double* __restrict__ te = t.e;
  const float* __restrict__ td = t.d;
  float2 fq[PF];
  float dq[PF];
  double mq[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const unsigned k = u < nz ? u : nz - 1;
    fq[u] = spec[k * ncol + col];
    mq[u] = tm[k * ntc + tc];
    dq[u] = td[k * ntc + tc];
  }
  double yx = 0.0, yy = 0.0;
  float2 s = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < nz; k0 += PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int k = k0 + u;
      if (k < nz) {
        const double fx = widen_f32(fq[u].x), fy = widen_f32(fq[u].y);
        const double m = mq[u];
        const float dk = dq[u];
        const unsigned kn = k + PF < nz ? k + PF : nz - 1;
        fq[u] = spec[kn * ncol + col];
        mq[u] = tm[kn * ntc + tc];
        dq[u] = td[kn * ntc + tc];
        yx = fma(-m, yx, ZERO ? fx - m0x : fx);
        yy = fma(-m, yy, ZERO ? fy - m0y : fy);
        s = make_float2(narrow_f64(yx) * dk, narrow_f64(yy) * dk);
        spec[(unsigned)k * ncol + col] = s;
      }
    }
  }
  // x_{nz-1} = s_{nz-1} (already stored); backward from row nz - 2
  double xx = widen_f32(s.x), xy = widen_f32(s.y);
  float2 sq[PF];
  double eq[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const unsigned k = nz - 2 - u >= 0 ? nz - 2 - u : 0;
    sq[u] = spec[k * ncol + col];
    eq[u] = te[k * ntc + tc];
  }
  for (int k0 = nz - 2; k0 >= 0; k0 -= PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int k = k0 - u;
      if (k >= 0) {
        const double sx = widen_f32(sq[u].x), sy = widen_f32(sq[u].y);
        const double e = eq[u];
        const unsigned kn = k - PF >= 0 ? k - PF : 0;
        sq[u] = spec[kn * ncol + col];
        eq[u] = te[kn * ntc + tc];
        xx = fma(-e, xx, sx);
        xy = fma(-e, xy, sy);
        spec[(unsigned)k * ncol + col] = make_float2(narrow_f64(xx), narrow_f64(xy));
      }
    }
  }
}

// One ill-conditioned column of a mixed plan, solved by a whole warp in
// FP64.  Both sweeps of the Thomas elimination are first-order affine
// recurrences,
//   forward   y_k = -m_k y_{k-1} + f_k                (y_{-1} = 0),
//   backward  x_k = -c_k d_k x_{k+1} + d_k y_k        (x_{nz-1} = d_{nz-1} y_{nz-1}),
// so each lane composes the maps of its R = ceil(nz/32) consecutive rows, a
// shuffle scan combines the lanes' maps, and each lane replays its rows from
// the value entering its segment.  The values stay FP32 in memory (the
// intermediate y too, as in stage_tridiag_split); the recurrences run in
// FP64.  Column 0 (the singular (0, 0) system, its last pivot pinned) first
// loses its dzf-weighted z mean.
__device__ __forceinline__ void tridiag_col_warp64(const Geo& g, const double* __restrict__ mtab,
                                                   const double* __restrict__ invd, float2* spec,
                                                   size_t col, size_t ncol) {
  const int lane = threadIdx.x & 31;
  const int nz = g.nz;
  const int R = (nz + 31) >> 5;
  const int k0 = lane * R < nz ? lane * R : nz;
  const int k1 = k0 + R < nz ? k0 + R : nz;
  auto at = [&](int k) { return (size_t)k * ncol + col; };
  double m0x = 0.0, m0y = 0.0;
  if (col == 0) {
    double sx = 0.0, sy = 0.0;
    for (int k = k0; k < k1; ++k) {
      const float2 v = spec[at(k)];
      sx += g.dzf[k] * widen_f32(v.x);
      sy += g.dzf[k] * widen_f32(v.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    m0x = sx / g.lz;
    m0y = sy / g.lz;
  }
  // forward: compose y -> a y + b over the lane's rows, then scan the lanes
  double A = 1.0, Bx = 0.0, By = 0.0;
  for (int k = k0; k < k1; ++k) {
    const double a = -mtab[at(k)];
    const float2 f = spec[at(k)];
    Bx = fma(a, Bx, widen_f32(f.x) - m0x);
    By = fma(a, By, widen_f32(f.y) - m0y);
    A *= a;
  }
  for (int d = 1; d < 32; d <<= 1) {  // inclusive scan, earlier lanes' maps applied first
    const double Ap = __shfl_up_sync(0xffffffffu, A, d);
    const double Bxp = __shfl_up_sync(0xffffffffu, Bx, d);
    const double Byp = __shfl_up_sync(0xffffffffu, By, d);
    if (lane >= d) {
      Bx = fma(A, Bxp, Bx);
      By = fma(A, Byp, By);
      A *= Ap;
    }
  }
  double yx = __shfl_up_sync(0xffffffffu, Bx, 1), yy = __shfl_up_sync(0xffffffffu, By, 1);
  if (lane == 0) { yx = 0.0; yy = 0.0; }
  for (int k = k0; k < k1; ++k) {
    const double a = -mtab[at(k)];
    const float2 f = spec[at(k)];
    yx = fma(a, yx, widen_f32(f.x) - m0x);
    yy = fma(a, yy, widen_f32(f.y) - m0y);
    spec[at(k)] = make_float2(narrow_f64(yx), narrow_f64(yy));
  }
  __syncwarp();
  // backward: maps x_{k+1} -> x_k over the lane's rows from the top down
  auto row_map = [&](int k, double& a, double& bx, double& by) {
    const float2 yv = spec[at(k)];
    const double d = invd[at(k)];
    a = (k == nz - 1) ? 0.0 : -g.zc[k] * d;
    bx = d * widen_f32(yv.x);
    by = d * widen_f32(yv.y);
  };
  A = 1.0; Bx = 0.0; By = 0.0;
  for (int k = k1 - 1; k >= k0; --k) {
    double a, bx, by;
    row_map(k, a, bx, by);
    Bx = fma(a, Bx, bx);
    By = fma(a, By, by);
    A *= a;
  }
  for (int d = 1; d < 32; d <<= 1) {  // inclusive scan, later lanes' maps applied first
    const double Ap = __shfl_down_sync(0xffffffffu, A, d);
    const double Bxp = __shfl_down_sync(0xffffffffu, Bx, d);
    const double Byp = __shfl_down_sync(0xffffffffu, By, d);
    if (lane + d < 32) {
      Bx = fma(A, Bxp, Bx);
      By = fma(A, Byp, By);
      A *= Ap;
    }
  }
  double xx = __shfl_down_sync(0xffffffffu, Bx, 1), xy = __shfl_down_sync(0xffffffffu, By, 1);
  if (lane == 31) { xx = 0.0; xy = 0.0; }
  // every lane reads its own rows' y before any lane overwrites them
  for (int k = k1 - 1; k >= k0; --k) {
    double a, bx, by;
    row_map(k, a, bx, by);
    xx = fma(a, xx, bx);
    xy = fma(a, xy, by);
    spec[at(k)] = make_float2(narrow_f64(xx), narrow_f64(xy));
  }
}

// Mixed plans, one thread per (kx, ky) column holding both components, in
// FP32 with FP32 tables (float2 loads and stores of the spectrum).  Only the well-conditioned columns (TriF32) take this path;
// column 0 and the other ill-conditioned columns are left to
// tridiag_col_warp64.
__device__ __forceinline__ void stage_tridiag_col32(const Geo& g, const TriF32& f, float2* spec, size_t col) {
  constexpr int PF = 1;  // deeper register prefetch (2-16 rows) measured slower at 512^3
  const size_t ncol = (size_t)g.ny * g.nxh;
  if (col >= ncol) return;
  const int j = (int)(col / (size_t)g.nxh);
  const int kx = (int)(col - (size_t)j * g.nxh);
  if (col == 0 || fabs(f.lamx[kx] + f.lamy[j]) < f.thr) return;
  const int nz = g.nz;
  float2 fq[PF];
  float mq[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const int k = u < nz ? u : nz - 1;
    fq[u] = spec[(size_t)k * ncol + col];
    mq[u] = f.mtab[(size_t)k * ncol + col];
  }
  float2 y = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < nz; k0 += PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int k = k0 + u;
      if (k < nz) {
        const float2 fv = fq[u];
        const float m = mq[u];
        const int kn = k + PF < nz ? k + PF : nz - 1;
        fq[u] = spec[(size_t)kn * ncol + col];
        mq[u] = f.mtab[(size_t)kn * ncol + col];
        y.x = fmaf(-m, y.x, fv.x);
        y.y = fmaf(-m, y.y, fv.y);
        if (k < nz - 1) spec[(size_t)k * ncol + col] = y;
      }
    }
  }
  const float dl = f.invd[(size_t)(nz - 1) * ncol + col];
  float2 x = make_float2(y.x * dl, y.y * dl);
  spec[(size_t)(nz - 1) * ncol + col] = x;
  float2 yq[PF];
  float dq[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    const int k = nz - 2 - u >= 0 ? nz - 2 - u : 0;
    yq[u] = spec[(size_t)k * ncol + col];
    dq[u] = f.invd[(size_t)k * ncol + col];
  }
  for (int k0 = nz - 2; k0 >= 0; k0 -= PF) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int k = k0 - u;
      if (k >= 0) {
        const float2 yy = yq[u];
        const float d = dq[u], c = f.zc[k];
        const int kn = k - PF >= 0 ? k - PF : 0;
        yq[u] = spec[(size_t)kn * ncol + col];
        dq[u] = f.invd[(size_t)kn * ncol + col];
        x.x = fmaf(-c, x.x, yy.x) * d;
        x.y = fmaf(-c, x.y, yy.y) * d;
        spec[(size_t)k * ncol + col] = x;
      }
    }
  }
}

// Block b of the mixed z solve: the first nblk_low blocks give one warp to
// each ill-conditioned column of the list (scheduled first: their chains are
// the longest), the rest one thread to each column.  Block-uniform branch.
__device__ __forceinline__ void stage_tridiag_mixed(const Geo& g, const double* __restrict__ mtab,
                                                    const double* __restrict__ invd, const TriF32& f,
                                                    float2* spec, int b) {
  const int nblk_low = (f.nlow + 3) >> 2;
  if (b < nblk_low) {
    const int w = b * 4 + (threadIdx.x >> 5);
    if (w < f.nlow) tridiag_col_warp64(g, mtab, invd, spec, (size_t)f.low[w], (size_t)g.ny * g.nxh);
    return;
  }
  stage_tridiag_col32(g, f, spec, (size_t)(b - nblk_low) * blockDim.x + threadIdx.x);
}

// Inverse x transform of two half spectra per complex sequence, then
// p = scale * z (p_zero) or p += scale * z.  The p values a thread updates
// are loaded before the transform so their latency overlaps it.  delta (if
// not null) receives the increment scale * z in the precision T.
//
// Mixed path (sdelta not null): p is only brought up to date where an
// exact residual needs it.  sdelta holds the FP32 sum of the increments
// since p was last updated:
//   fold  (the next residual is exact): p += sdelta + increment (FP64);
//   else: sdelta = increment (fresh: p was updated last pass) or
//         sdelta += increment.
// With fresh set, fold ignores sdelta.
// Update modes of the inverse x stage (compile-time, so each pass runs only
// its own arithmetic).
enum InvMode { kInvPlain = 0, kInvFold = 1, kInvFoldFresh = 2, kInvFresh = 3, kInvAccum = 4 };

template <typename T, int MODE>
__device__ __forceinline__ void stage_fftx_inv_m(const Geo& g, const FftDesc& fx,
                                                 const C2<T>* __restrict__ twx,
                                                 const C2<T>* __restrict__ spec, double scale,
                                                 double* __restrict__ p, int p_zero, int rpb, int blk,
                                                 T* __restrict__ delta, float* __restrict__ sdelta,
                                                 unsigned char* smem_raw) {
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
  const bool need_p = !p_zero && MODE <= kInvFoldFresh;            // p is read
  constexpr bool need_s = MODE == kInvFold || MODE == kInvAccum;  // sdelta is read
  // p is prefetched in the plain mode of FP64 plans (every pass); the fold
  // passes of mixed plans (one in forty) read it where it is used, which keeps
  // their registers within the other modes' budget
  const bool pre_p = need_p && MODE == kInvPlain && sizeof(T) == sizeof(double);
  constexpr bool F32 = std::is_same<T, float>::value;
  const int twb = nseq * nx + fft_pad_elems(nseq * nx);  // buffer B is written padded
  const bool fast = F32 && fft_smem_shape(nx, nseq, false);
  if constexpr (F32) {
    if (fast) load_twiddles_smem(twx, nx, twb);
  }
  auto split = [&](int t, int& q, int& i) {
    if (lgx >= 0) { q = t >> lgx; i = t & (nx - 1); }
    else { q = t / nx; i = t - q * nx; }
  };
  // one output value: zv = unscaled inverse transform at cell c
  auto emit = [&](size_t c, T zv, double pv, float sv) {
    const float inc_f = scale_f * (float)zv;
    if constexpr (MODE <= kInvFoldFresh) {
      const double zd = (sizeof(T) == sizeof(float)) ? widen_f32((float)zv) : (double)zv;
      if constexpr (MODE == kInvFold) p[c] = fma(scale, zd, pv + widen_f32(sv));
      else p[c] = fma(scale, zd, pv);
      if (delta != nullptr) delta[c] = (sizeof(T) == sizeof(float)) ? (T)inc_f : (T)(scale * zd);
    } else {
      sdelta[c] = (MODE == kInvAccum) ? sv + inc_f : inc_f;
      if (delta != nullptr) delta[c] = (T)inc_f;
    }
  };
  constexpr int NP = kPrefetchInv;
  double pv[NP];
  float sv[NP];
#pragma unroll
  for (int u = 0; u < NP; ++u) {
    const int t = threadIdx.x + u * blockDim.x;
    int q, i;
    split(t, q, i);
    pv[u] = 0.0;
    sv[u] = 0.f;
    const bool in = t < nout && row0 + q < nrows;
    if (pre_p && in) pv[u] = p[(size_t)(row0 + q) * nx + i];
    if (need_s && in) sv[u] = sdelta[(size_t)(row0 + q) * nx + i];
  }
  // Z = A + i B from the two half spectra; each stored coefficient m also
  // gives its mirror nx - m (conjugates), so it is loaded once.  (q, m) is
  // walked incrementally over the nseq x nxh stored coefficients.
  {
    int q = threadIdx.x / nxh, m = threadIdx.x - q * nxh;
    const int dq = blockDim.x / nxh, dm = blockDim.x - dq * nxh;
    for (; q < nseq; q += dq, m += dm) {
      if (m >= nxh) { m -= nxh; ++q; if (q >= nseq) break; }
      const long ra = row0 + 2 * q;
      C2<T> A, B;
      A.x = A.y = B.x = B.y = (T)0;
      if (ra < nrows) A = spec[(size_t)ra * nxh + m];
      if (ra + 1 < nrows) B = spec[(size_t)(ra + 1) * nxh + m];
      C2<T>* row = bufA + (size_t)q * nx;
      if (m == 0 || (even && m == nx / 2)) {
        C2<T> Z;
        Z.x = A.x;
        Z.y = B.x;
        row[m] = Z;
      } else {
        C2<T> Z, Zm;
        Z.x = A.x - B.y;
        Z.y = A.y + B.x;
        Zm.x = A.x + B.y;   // mirror: A, B conjugated
        Zm.y = B.x - A.y;
        row[m] = Z;
        if (m < nx - m) row[nx - m] = Zm;
      }
    }
  }
  __syncthreads();
  const C2<T>* res = nullptr;
  if constexpr (F32) {
    if (fast) res = smem_f2() + fft_dispatch_smem<1, false>(0, nseq * nx, twb, fx, nseq, 1, nx, threadIdx.x, blockDim.x);
  }
  if (!fast) res = fft_dispatch<T, 1, false>(bufA, bufB, fx, nseq, 1, nx, twx, threadIdx.x, blockDim.x);
#pragma unroll
  for (int u = 0; u < NP; ++u) {
    const int t = threadIdx.x + u * blockDim.x;
    int q, i;
    split(t, q, i);
    const long row = row0 + q;
    if (t < nout && row < nrows) {
      const C2<T> z = res[(size_t)(q >> 1) * nx + i];
      const size_t c = (size_t)row * nx + i;
      emit(c, (q & 1) ? z.y : z.x, pre_p ? pv[u] : (need_p ? p[c] : 0.0), sv[u]);
    }
  }
  for (int t = threadIdx.x + NP * blockDim.x; t < nout; t += blockDim.x) {  // beyond the prefetch
    int q, i;
    split(t, q, i);
    const long row = row0 + q;
    if (row < nrows) {
      const C2<T> z = res[(size_t)(q >> 1) * nx + i];
      const size_t c = (size_t)row * nx + i;
      emit(c, (q & 1) ? z.y : z.x, need_p ? p[c] : 0.0, need_s ? sdelta[c] : 0.f);
    }
  }
}

// Mode dispatch (block-uniform): sdelta null -> plain update of p.
template <typename T>
__device__ __forceinline__ void stage_fftx_inv(const Geo& g, const FftDesc& fx, const C2<T>* __restrict__ twx,
                                               const C2<T>* __restrict__ spec, double scale,
                                               double* __restrict__ p, int p_zero, int rpb, int blk,
                                               T* __restrict__ delta, float* __restrict__ sdelta,
                                               bool fold, bool fresh, unsigned char* smem_raw) {
  if (sizeof(T) == sizeof(double) || sdelta == nullptr) {  // FP64 plans: plain only
    stage_fftx_inv_m<T, kInvPlain>(g, fx, twx, spec, scale, p, p_zero, rpb, blk, delta, sdelta, smem_raw);
    return;
  }
  if constexpr (sizeof(T) == sizeof(double)) return;
  if (fold && !fresh)
    stage_fftx_inv_m<T, kInvFold>(g, fx, twx, spec, scale, p, p_zero, rpb, blk, delta, sdelta, smem_raw);
  else if (fold)
    stage_fftx_inv_m<T, kInvFoldFresh>(g, fx, twx, spec, scale, p, p_zero, rpb, blk, delta, sdelta, smem_raw);
  else if (fresh)
    stage_fftx_inv_m<T, kInvFresh>(g, fx, twx, spec, scale, p, p_zero, rpb, blk, delta, sdelta, smem_raw);
  else
    stage_fftx_inv_m<T, kInvAccum>(g, fx, twx, spec, scale, p, p_zero, rpb, blk, delta, sdelta, smem_raw);
}

}  // namespace pp
