// Dense transform of strided real lines on the tensor cores, out of place:
// for every column g of a real view (slab s = g / ncs, offset c = g % ncs)
// the n entries x_k = X[s * slab + k * ld + c] become
//   y_m = f(m, g) * sum_k M[m][k] x_k,   m < n,
// stored at Y[s * slab + m * ld + c].  It is the dense eigenvector step of
// the eigenexpansion solve (Sec. 3.3.1) along a direction whose eigenbasis
// has no fast transform: a stretched y between walls (M = V^T W forward,
// M = V back; f = 1), or z (the forward product with the eigenvalue divide
// f = 1 / (mu_m + lambda_x + lambda_y), zero on the pinned mode).
//
// Products: BF16 x3 split (hi*hi + hi*lo + lo*hi, FP32 accumulation in
// tensor memory).  Orientation: D[g][m] = sum_k X^T[g][k] M^T[k][m], so the
// MMA's M dimension is 128 data columns (TMEM lanes) and its N dimension 256
// outputs (TMEM columns): the epilogue thread of a lane owns one column g
// and writes 32 consecutive g per warp instruction.  A work item is a tile of
// 128 columns times one block of 256 outputs; a persistent CTA walks items
// with stride gridDim.x.  Warp roles (320 threads):
//   warp 0     bulk-copies the pre-split M tiles (256 x 32 per chunk) into a
//              kStagesM-deep ring;
//   warp 1     allocates TMEM (2 x 256 columns, double-buffered D) and one
//              thread issues the MMAs;
//   warps 2-5  load 32 rows of X for the 128 columns, split them into BF16
//              hi/lo with 16-byte shared stores in the core-matrix layout
//              (kStagesD-deep ring);
//   warps 6-9  read D from TMEM (lane quarter = warp % 4), scale, store.
// Every wait is bounded; a wait that runs out sets DevStatus::pad, the other
// roles stop at their next wait, and the CTA drains its copies and MMAs
// before it frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "pp_internal.cuh"
#include "pp_tc.cuh"

namespace pp {

using namespace tc;

namespace {

constexpr int kCols = 128;                    // data columns per tile (MMA M)
constexpr int kOut = 256;                     // outputs per item (MMA N)
constexpr int kKC = 32;                       // K per chunk
constexpr uint32_t kSbo = (kKC / 8) * 128;    // 8-row group stride of a chunk
constexpr int kHalfD = kCols * kKC * 2;       // bytes of one BF16 half of a data chunk (8 KB)
constexpr int kHalfM = kOut * kKC * 2;        // bytes of one BF16 half of a matrix chunk (16 KB)
constexpr int kStagesM = 4;
constexpr int kBytesF = kCols * kKC * 4;      // FP32 data chunk brought by TMA (16 KB)
constexpr int kThreadsTC = 320;

// Stage counts: with TMA (one slab, 16-byte aligned rows: the z expansion)
// the copy thread also brings each 32 x 128 FP32 data chunk into a staging
// ring, and the BF16 ring shrinks to fit 224 KB; without it the convert
// warps load the columns themselves.
template <bool TMA> struct Cfg {
  static constexpr int SD = TMA ? 2 : 4;   // BF16 data stages
  static constexpr int SF = TMA ? 4 : 0;   // FP32 staging stages
  static constexpr size_t smem =
      (size_t)kStagesM * 2 * kHalfM + (size_t)SD * 2 * kHalfD + (size_t)SF * kBytesF + 1024;
};

struct Bars {
  uint64_t dfull[4], dempty[4], mfull[kStagesM], mempty[kStagesM], ffull[4], fempty[4], tfull[2], tempty[2],
      drain;
};

__device__ __forceinline__ void tma_load_2d(void* dst_smem, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                            uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      :: "r"(smem_u32(dst_smem)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace

template <bool TMA>
__global__ void __launch_bounds__(kThreadsTC, 1) k_dense_tc(DenseTcArgs a, const __grid_constant__ CUtensorMap tmap,
                                                          DevStatus* st) {
  if (st != nullptr && st->done) return;
  constexpr int kStagesD = Cfg<TMA>::SD, kStagesF = Cfg<TMA>::SF;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  unsigned char* sM = smem;                                   // kStagesM x (hi | lo)
  unsigned char* sD = smem + (size_t)kStagesM * 2 * kHalfM;   // kStagesD x (hi | lo)
  unsigned char* sF = sD + (size_t)kStagesD * 2 * kHalfD;     // kStagesF x FP32 [32][128]
  __shared__ __align__(8) Bars bars;
  __shared__ uint32_t taddr_s;
  __shared__ volatile int fail_s;
  __shared__ int consumed_s, consumed_f;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long total_cols = a.ncs * a.nslab;
  const long long ntiles = (total_cols + kCols - 1) / kCols;
  const long long nitems = ntiles * a.nt;
  if (tid == 0) {
    for (int i = 0; i < kStagesD; ++i) { mbar_init(&bars.dfull[i], 128); mbar_init(&bars.dempty[i], 1); }
    for (int i = 0; i < kStagesM; ++i) { mbar_init(&bars.mfull[i], 1); mbar_init(&bars.mempty[i], 1); }
    for (int i = 0; i < kStagesF; ++i) { mbar_init(&bars.ffull[i], 1); mbar_init(&bars.fempty[i], 128); }
    for (int i = 0; i < 2; ++i) { mbar_init(&bars.tfull[i], 1); mbar_init(&bars.tempty[i], 128); }
    mbar_init(&bars.drain, 1);
    mbar_init_fence();
    fail_s = 0;
    consumed_s = 0;
    consumed_f = 0;
  }
  if (warp == 1) tmem_alloc(&taddr_s, 2 * kOut);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = taddr_s;
  auto fail = [&]() { fail_s = 1; };
  long long issued = 0, issued_f = 0;  // chunks copied (warp 0, lane 0)

  if (warp == 0) {
    // ---- matrix producer (and, with TMA, the data chunks) ----------------
    if (lane == 0) {
      long long q = 0;
      for (long long it = blockIdx.x; it < nitems && !fail_s; it += gridDim.x) {
        const int h = (int)(it % a.nt);
        for (int kc = 0; kc < a.nkc && !fail_s; ++kc, ++q) {
          if constexpr (TMA) {
            const int f = (int)(q % kStagesF);
            if (!mbar_wait(&bars.fempty[f], (uint32_t)(((q / kStagesF) & 1) ^ 1))) { fail(); break; }
            // rows past n and columns past the view read as zeros
            tma_load_2d(sF + (size_t)f * kBytesF, &tmap, (int)((it / a.nt) * kCols), kc * kKC, &bars.ffull[f],
                        kBytesF);
            ++issued_f;
          }
          const int s = (int)(q % kStagesM);
          if (!mbar_wait(&bars.mempty[s], (uint32_t)(((q / kStagesM) & 1) ^ 1))) { fail(); break; }
          bulk_copy(sM + (size_t)s * 2 * kHalfM, a.mat + ((size_t)h * a.nkc + kc) * 2 * kHalfM, 2 * kHalfM,
                    &bars.mfull[s]);
          ++issued;
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer -------------------------------------------------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kCols, kOut);
      long long q = 0, j = 0;
      for (long long it = blockIdx.x; it < nitems && !fail_s; it += gridDim.x, ++j) {
        const int b = (int)(j & 1);
        if (!mbar_wait(&bars.tempty[b], (uint32_t)(((j >> 1) & 1) ^ 1))) { fail(); break; }
        tc_fence_after();
        const uint32_t dt = tbase + (uint32_t)(b * kOut);
        for (int kc = 0; kc < a.nkc; ++kc, ++q) {
          const int sd = (int)(q % kStagesD), sm = (int)(q % kStagesM);
          if (!mbar_wait(&bars.dfull[sd], (uint32_t)((q / kStagesD) & 1)) ||
              !mbar_wait(&bars.mfull[sm], (uint32_t)((q / kStagesM) & 1))) { fail(); break; }
          tc_fence_after();
          const uint32_t d_hi = smem_u32(sD + (size_t)sd * 2 * kHalfD), d_lo = d_hi + kHalfD;
          const uint32_t m_hi = smem_u32(sM + (size_t)sm * 2 * kHalfM), m_lo = m_hi + kHalfM;
#pragma unroll
          for (int kk = 0; kk < kKC / 16; ++kk) {
            const uint32_t o = (uint32_t)kk * 256u;  // two core matrices along K
            const uint32_t acc = (kc == 0 && kk == 0) ? 0u : 1u;
            mma_bf16(dt, smem_desc(d_hi + o, 128, kSbo), smem_desc(m_hi + o, 128, kSbo), idesc, acc);
            mma_bf16(dt, smem_desc(d_hi + o, 128, kSbo), smem_desc(m_lo + o, 128, kSbo), idesc, 1u);
            mma_bf16(dt, smem_desc(d_lo + o, 128, kSbo), smem_desc(m_hi + o, 128, kSbo), idesc, 1u);
          }
          mma_commit(&bars.dempty[sd]);
          mma_commit(&bars.mempty[sm]);
          consumed_s = (int)(q + 1);
        }
        if (fail_s) break;
        mma_commit(&bars.tfull[b]);
      }
      // every MMA issued has completed once this arrives
      mma_commit(&bars.drain);
      if (!mbar_wait(&bars.drain, 0)) fail();
    }
  } else if (warp < 6) {
   if constexpr (TMA) {
    // ---- data converters, TMA-fed: thread = column n of the staged chunk ----
    const int n = tid - 64;
    long long q = 0;
    for (long long it = blockIdx.x; it < nitems && !fail_s; it += gridDim.x) {
      for (int kc = 0; kc < a.nkc; ++kc, ++q) {
        const int f = (int)(q % kStagesF);
        if (!mbar_wait(&bars.ffull[f], (uint32_t)((q / kStagesF) & 1))) { fail(); break; }
        const float* stg = reinterpret_cast<const float*>(sF + (size_t)f * kBytesF);
        float v[kKC];
#pragma unroll
        for (int e = 0; e < kKC; ++e) v[e] = stg[e * kCols + n];  // a warp reads 128 consecutive bytes
        mbar_arrive(&bars.fempty[f]);
        if (tid == 64) consumed_f = (int)(q + 1);
        const int s = (int)(q % kStagesD);
        if (!mbar_wait(&bars.dempty[s], (uint32_t)(((q / kStagesD) & 1) ^ 1))) { fail(); break; }
        unsigned char* dst = sD + (size_t)s * 2 * kHalfD;
#pragma unroll
        for (int grp = 0; grp < kKC / 8; ++grp) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int e = 0; e < 8; e += 2) split_pack2(v[grp * 8 + e], v[grp * 8 + e + 1], hi[e >> 1], lo[e >> 1]);
          const uint32_t o = core_off(n, grp * 8, kSbo);
          *reinterpret_cast<uint4*>(dst + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(dst + kHalfD + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        fence_async_smem();
        mbar_arrive(&bars.dfull[s]);
      }
    }
   } else {
    // ---- data converters ---------------------------------------------------
    // Converter warp cw = warp - 2 takes columns 64 (cw & 1) + 2 lane and
    // + 1 (a float2: columns come in pairs within a slab, ncs being even) and
    // rows 16 (cw >> 1) .. + 16 of each 32-row chunk, loaded past L1: a warp
    // request moves 256 contiguous bytes (the number of requests in flight,
    // not their bytes, limits this role).  Four chunks in registers: while
    // chunk q is split and stored, chunks q + 1 .. q + 3 are loading.
    const int cw = warp - 2;
    const int n0 = 64 * (cw & 1) + 2 * lane, rb = 16 * (cw >> 1);
    long long q = 0;
    constexpr int kR = kKC / 2;  // rows per thread and chunk
    float2 v0[kR], v1[kR], v2[kR], v3[kR];
    auto load = [&](float2 (&v)[kR], long long it, int kc) {
      const long long g = (it / a.nt) * kCols + n0;
      const bool valid = it < nitems && g < total_cols;
      const long long sl = valid ? g / a.ncs : 0;
      const float* src = a.x + (valid ? sl * a.slab + (g - sl * a.ncs) : 0);
#pragma unroll
      for (int e = 0; e < kR; ++e) {
        const int k = kc * kKC + rb + e;
        v[e] = (valid && k < a.n) ? __ldcg(reinterpret_cast<const float2*>(src + (long long)k * a.ld))
                                  : make_float2(0.f, 0.f);
      }
    };
    auto store = [&](const float2 (&v)[kR]) -> bool {
      const int s = (int)(q % kStagesD);
      if (!mbar_wait(&bars.dempty[s], (uint32_t)(((q / kStagesD) & 1) ^ 1))) return false;
      unsigned char* dst = sD + (size_t)s * 2 * kHalfD;
#pragma unroll
      for (int grp = 0; grp < kR / 8; ++grp) {
        uint32_t h0[4], l0[4], h1[4], l1[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          split_pack2(v[grp * 8 + e].x, v[grp * 8 + e + 1].x, h0[e >> 1], l0[e >> 1]);
          split_pack2(v[grp * 8 + e].y, v[grp * 8 + e + 1].y, h1[e >> 1], l1[e >> 1]);
        }
        const uint32_t o0 = core_off(n0, rb + grp * 8, kSbo), o1 = core_off(n0 + 1, rb + grp * 8, kSbo);
        *reinterpret_cast<uint4*>(dst + o0) = make_uint4(h0[0], h0[1], h0[2], h0[3]);
        *reinterpret_cast<uint4*>(dst + kHalfD + o0) = make_uint4(l0[0], l0[1], l0[2], l0[3]);
        *reinterpret_cast<uint4*>(dst + o1) = make_uint4(h1[0], h1[1], h1[2], h1[3]);
        *reinterpret_cast<uint4*>(dst + kHalfD + o1) = make_uint4(l1[0], l1[1], l1[2], l1[3]);
      }
      fence_async_smem();
      mbar_arrive(&bars.dfull[s]);
      ++q;
      return true;
    };
    // this CTA's chunk sequence: (item, chunk), chunk fastest; c[0] is the
    // oldest chunk held, c[3] the next one to load
    long long cit[4];
    int ckc[4];
    cit[0] = blockIdx.x;
    ckc[0] = 0;
    for (int i = 1; i < 4; ++i) {
      cit[i] = cit[i - 1];
      ckc[i] = ckc[i - 1] + 1;
      if (ckc[i] == a.nkc) { ckc[i] = 0; cit[i] += gridDim.x; }
    }
    auto shift = [&]() {
      cit[0] = cit[1]; ckc[0] = ckc[1];
      cit[1] = cit[2]; ckc[1] = ckc[2];
      cit[2] = cit[3]; ckc[2] = ckc[3];
      ckc[3] = ckc[2] + 1;
      cit[3] = cit[2];
      if (ckc[3] == a.nkc) { ckc[3] = 0; cit[3] += gridDim.x; }
    };
    load(v0, cit[0], ckc[0]);  // zeros past the last item
    load(v1, cit[1], ckc[1]);
    load(v2, cit[2], ckc[2]);
    // one step: load the newest chunk into the buffer freed last, store the
    // oldest; the four buffers rotate through the four steps
#define PP_CONVERT_STEP(OLD, NEW)                   \
    {                                               \
      if (cit[0] >= nitems || fail_s) break;        \
      load(NEW, cit[3], ckc[3]);                    \
      if (!store(OLD)) { fail(); break; }           \
      shift();                                      \
    }
    for (;;) {
      PP_CONVERT_STEP(v0, v3)
      PP_CONVERT_STEP(v1, v0)
      PP_CONVERT_STEP(v2, v1)
      PP_CONVERT_STEP(v3, v2)
    }
#undef PP_CONVERT_STEP
   }
  } else {
    // ---- epilogue: lane quarter = warp % 4, thread = column ---------------
    const int qd = warp & 3;
    const int n = qd * 32 + lane;
    long long j = 0;
    for (long long it = blockIdx.x; it < nitems && !fail_s; it += gridDim.x, ++j) {
      const int b = (int)(j & 1), h = (int)(it % a.nt);
      const long long g = (it / a.nt) * kCols + n;
      const bool valid = g < total_cols;
      const long long sl = valid ? g / a.ncs : 0;
      float* dst = a.y + (valid ? sl * a.slab + (g - sl * a.ncs) : 0);
      float lam = 0.f;
      bool pinned = false;
      if (a.mu != nullptr && valid) {
        const long long cc = g >> 1;
        const int ky = (int)(cc / a.nxh), kx = (int)(cc - (long long)ky * a.nxh);
        lam = (float)(a.lamx[kx] + a.lamy[ky]);
        pinned = (cc == 0);
      }
      // warp-uniform outcome: the TMEM loads below are warp-collective
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars.tfull[b], (uint32_t)((j >> 1) & 1)));
      if (!ok) { fail(); break; }
      tc_fence_after();
      for (int c16 = 0; c16 < kOut / 16; ++c16) {
        const int m0 = h * kOut + c16 * 16;
        // divide epilogue: 16 eigenvalues as four 16-byte loads (mu is padded
        // to whole 256-output blocks); the reciprocal is the fast one (2^-22
        // relative, far inside the 2^-16 of the split products)
        float fac[16];
        if (a.mu != nullptr) {
#pragma unroll
          for (int e4 = 0; e4 < 4; ++e4) {
            const float4 m4 = __ldg(reinterpret_cast<const float4*>(a.mu + m0) + e4);
            fac[4 * e4 + 0] = __fdividef(1.f, m4.x + lam);
            fac[4 * e4 + 1] = __fdividef(1.f, m4.y + lam);
            fac[4 * e4 + 2] = __fdividef(1.f, m4.z + lam);
            fac[4 * e4 + 3] = __fdividef(1.f, m4.w + lam);
          }
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (pinned && m0 + e == a.zero_mode) fac[e] = 0.f;
        }
        float v[16];
        tmem_ld16(tbase + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * kOut + c16 * 16), v);
        if (valid) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int m = m0 + e;
            if (m < a.n) dst[(long long)m * a.ld] = (a.mu != nullptr) ? v[e] * fac[e] : v[e];
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&bars.tempty[b]);
    }
  }

  __syncthreads();
  if (fail_s && tid == 0) {
    // copies still in flight land before the CTA's shared memory goes away
    for (long long q = consumed_s; q < issued; ++q)
      mbar_wait(&bars.mfull[q % kStagesM], (uint32_t)((q / kStagesM) & 1));
    if constexpr (TMA)
      for (long long q = consumed_f; q < issued_f; ++q)
        mbar_wait(&bars.ffull[q % kStagesF], (uint32_t)((q / kStagesF) & 1));
    if (st != nullptr) st->pad = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tbase, 2 * kOut);
}

// ---------------------------------------------------------------------------

int dense_tc_out_tiles(int n) { return (n + kOut - 1) / kOut; }
int dense_tc_k_chunks(int n) { return (n + kKC - 1) / kKC; }

// M (n x n, row-major M[m][k]) -> BF16 hi/lo tiles: chunk (nt, kc) holds
// rows 256 nt .. +256 and k = 32 kc .. +32 in the K-major core layout, hi
// then lo, zero beyond n.
void dense_tc_tiles(const std::vector<double>& M, int n, std::vector<uint16_t>& out) {
  const int nt = dense_tc_out_tiles(n), nkc = dense_tc_k_chunks(n);
  const size_t half = (size_t)kHalfM / 2;  // elements of one half
  out.assign((size_t)nt * nkc * 2 * half, 0);
  for (int t = 0; t < nt; ++t)
    for (int kc = 0; kc < nkc; ++kc) {
      uint16_t* hi = out.data() + ((size_t)t * nkc + kc) * 2 * half;
      uint16_t* lo = hi + half;
      for (int r = 0; r < kOut; ++r)
        for (int k = 0; k < kKC; ++k) {
          const int m = t * kOut + r, kk = kc * kKC + k;
          const float x = (m < n && kk < n) ? (float)M[(size_t)m * n + kk] : 0.f;
          const uint16_t h = bf16_rn_host(x);
          const uint16_t l = bf16_rn_host(x - bf16_to_f_host(h));
          const size_t o = core_off(r, k, kSbo) / 2;
          hi[o] = h;
          lo[o] = l;
        }
    }
}

namespace {

// 2D tensor map of the view for the TMA data path: x = the column (FP32,
// contiguous), y = the line entry k (stride ld), box 128 x 32, zero fill
// outside.  False when the driver entry point or the encoding fails.
bool encode_view_map(const DenseTcArgs& a, CUtensorMap* map) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (encode == nullptr) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || fn == nullptr)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)a.ncs, (cuuint64_t)a.n};
  const cuuint64_t strides[1] = {(cuuint64_t)a.ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kCols, (cuuint32_t)kKC};
  const cuuint32_t estr[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(a.x), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <bool TMA>
cudaError_t launch_dense_tc_t(const DenseTcArgs& a, const CUtensorMap& map, int grid, DevStatus* st,
                              cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_dense_tc<TMA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Cfg<TMA>::smem);
  if (e != cudaSuccess) return e;
  k_dense_tc<TMA><<<grid, kThreadsTC, Cfg<TMA>::smem, s>>>(a, map, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dense_tc(const DenseTcArgs& a, DevStatus* st, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const long long ntiles = (a.ncs * a.nslab + kCols - 1) / kCols;
  const long long nitems = ntiles * a.nt;
  if (nitems <= 0) return cudaSuccess;
  const int grid = (int)(nitems < nsm ? nitems : nsm);
  // TMA data path: one slab, rows 16-byte aligned (the tensor map's stride
  // rule and the x coordinate rule: tiles start at multiples of 128 floats)
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const bool tma = a.nslab == 1 && (a.ld * sizeof(float)) % 16 == 0 && ((uintptr_t)a.x % 16) == 0 &&
                   a.ncs < (1LL << 32) && encode_view_map(a, &map);
  return tma ? launch_dense_tc_t<true>(a, map, grid, st, s) : launch_dense_tc_t<false>(a, map, grid, st, s);
}

}  // namespace pp
