// z solve by the eigenvector expansion on the tensor cores (the
// eigenexpansion method of Sec. 3.3.1 applied along z as well): for every
// (kx, ky) column of the half spectrum,
//   x = V diag(1 / (mu_m + lambda_x + lambda_y)) V^T W f,
// with L_z = W^{-1} T (W = diag(dzf), T symmetric tridiagonal) and
// V = W^{-1/2} Q the W-orthonormal eigenvectors (Q: eigenvectors of the
// symmetric S = W^{-1/2} T W^{-1/2}).  Both products run as BF16 x3 split
// products (hi*hi + hi*lo + lo*hi) on tcgen05.mma with FP32 accumulators in
// tensor memory.  The zero mode of the (0, 0) column is removed (inverse
// eigenvalue 0), which both enforces compatibility and pins the gauge.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "pp_internal.cuh"

namespace pp {

namespace {

constexpr int kTileN = 64;    // real spectral columns per CTA
constexpr int kTileM = 128;   // rows of one MMA (M)
constexpr int kChunkK = 64;   // K per staged chunk
constexpr int kThreadsZ = 128;
constexpr int kChunkBytesA = kTileM * kChunkK * 2 * 2;   // hi + lo bf16: 32 KB
constexpr int kChunkBytesB = kTileN * kChunkK * 2 * 2;   // hi + lo bf16: 16 KB
constexpr long kWaitLimit = 1L << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
               : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
  return ok != 0;
}

// Bounded wait: false when the barrier did not complete within the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  for (long i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: no swizzle, K-major core matrices of
// 8 rows x 16 bytes; lbo = byte step between core matrices along K,
// sbo = byte step between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, M = 128, N = kTileN.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile("{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
               :: "r"(dtmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (row, k) in a K-major no-swizzle tile whose 8-row
// groups are `sbo` bytes apart (core matrices along K are 128 bytes apart)
__device__ __forceinline__ uint32_t core_off(int row, int k, uint32_t sbo) {
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16_raw& hi, __nv_bfloat16_raw& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi = h;
  lo = l;
}

}  // namespace

// One CTA: columns [col0, col0 + kTileN) of the real view F[nz][ncols] of the
// half spectrum (FP32), all nz rows (padded to nzp, a multiple of 128).
//   a1: (V^T W) tiles, a2: V tiles, each [mt][kc] chunk = 128 x 64 bf16 hi
//   then lo in the no-swizzle K-major core layout (32 KB contiguous).
// Pipeline: thread 0 streams the A chunks of both products through a
// kStages-deep shared ring (bulk copies, full/empty mbarriers) and issues
// the MMAs; all threads convert the next B chunk of the first product while
// the current one is in use.  The second product consumes the scaled first
// product one 64-mode chunk at a time (double-buffered), produced from TMEM
// by the two warps that own those lanes.
constexpr int kStages = 5;

__global__ void __launch_bounds__(kThreadsZ, 1) k_zgemm(float* spec, long long ncols, int nz, int nzp, int nxh,
                                                      const float* __restrict__ mu, int zero_mode,
                                                      const double* __restrict__ lamx,
                                                      const double* __restrict__ lamy,
                                                      const unsigned char* __restrict__ a1,
                                                      const unsigned char* __restrict__ a2, DevStatus* st) {
  if (st != nullptr && st->done) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  // barriers: [0, S) full, [S, 2S) empty, 2S+{0,1} B free, 2S+{2,3} G free, 2S+4 D1 done, 2S+5 D2 done
  __shared__ __align__(8) uint64_t bars[2 * kStages + 6];
  __shared__ uint32_t taddr_s;
  __shared__ int fail_s;
  __shared__ float lam_s[kTileN / 2];  // lambda_x + lambda_y per complex column
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* bfree = bars + 2 * kStages;
  uint64_t* gfree = bars + 2 * kStages + 2;
  uint64_t* d1done = bars + 2 * kStages + 4;
  uint64_t* d2done = bars + 2 * kStages + 5;
  unsigned char* sA0 = smem;                                  // kStages x 32 KB ring
  unsigned char* sB0 = smem + kStages * kChunkBytesA;         // 2 x 16 KB (first product B)
  unsigned char* sG0 = sB0 + 2 * kChunkBytesB;                // 2 x 16 KB (second product B)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nmt = nzp / kTileM, nkc = nzp / kChunkK;
  const int nch1 = nkc * nmt;
  const int nch = 2 * nch1;
  const long long col0 = (long long)blockIdx.x * kTileN;
  if (tid < kTileN / 2) {
    const long long cc = (col0 >> 1) + tid;
    float l = 0.f;
    if (2 * cc < ncols) {
      const int jj = (int)(cc / nxh), kx = (int)(cc - (long long)jj * nxh);
      l = (float)(lamx[kx] + lamy[jj]);
    }
    lam_s[tid] = l;
  }
  if (tid == 0) {
    for (int i = 0; i < 2 * kStages + 6; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&bars[i])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fail_s = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&taddr_s)), "r"(512) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = taddr_s;
  const uint32_t d1 = tbase, d2 = tbase + 256;
  const uint32_t idesc = idesc_bf16(kTileM, kTileN);

  // chunk i: first product (i < nch1): kc = i / nmt, mt = i % nmt (A1 tile mt, kc);
  // second product: j = i - nch1, kc = j / nmt, lt = j % nmt (A2 tile lt, kc)
  auto chunk_src = [&](int i) -> const unsigned char* {
    const int j = i < nch1 ? i : i - nch1;
    const int kc = j / nmt, t = j - kc * nmt;
    return (i < nch1 ? a1 : a2) + ((size_t)t * nkc + kc) * kChunkBytesA;
  };
  auto issue_copy = [&](int i) {  // thread 0 only
    const int s = i % kStages;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(&full[s])), "r"(kChunkBytesA) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(sA0 + s * kChunkBytesA)), "l"(chunk_src(i)), "r"(kChunkBytesA),
                    "r"(smem_u32(&full[s])) : "memory");
  };
  // thread 0: wait for chunk i, issue its 12 MMAs, release its stage on
  // completion, and refill the stage of chunk i - 1 (whose MMAs precede these)
  auto run_chunk = [&](int i, uint32_t dtile, uint32_t b_hi, uint32_t b_lo, bool first) {
    if (fail_s) return;
    const int s = i % kStages;
    if (!mbar_wait(&full[s], (uint32_t)((i / kStages) & 1))) { fail_s = 1; return; }
    tc_fence_after();
    const uint32_t a_hi = smem_u32(sA0 + s * kChunkBytesA), a_lo = a_hi + kChunkBytesA / 2;
#pragma unroll
    for (int k = 0; k < kChunkK / 16; ++k) {
      const uint32_t acc = (first && k == 0) ? 0u : 1u;
      const uint32_t o = (uint32_t)k * 256u;
      mma_bf16(dtile, smem_desc(a_hi + o, 128, 1024), smem_desc(b_hi + o, 128, 1024), idesc, acc);
      mma_bf16(dtile, smem_desc(a_hi + o, 128, 1024), smem_desc(b_lo + o, 128, 1024), idesc, 1u);
      mma_bf16(dtile, smem_desc(a_lo + o, 128, 1024), smem_desc(b_hi + o, 128, 1024), idesc, 1u);
    }
    mma_commit(&empty[s]);
    const int r = i - 1 + kStages;  // refill the stage chunk i - 1 used
    if (i >= 1 && r < nch) {
      const int sp = (i - 1) % kStages;
      if (!mbar_wait(&empty[sp], (uint32_t)(((i - 1) / kStages) & 1))) { fail_s = 1; return; }
      issue_copy(r);
    }
  };
  // B chunk kc of the first product: levels kc*64 .. +64 of the tile's
  // columns, split into BF16 hi and lo.  Thread (n, group) takes 8
  // consecutive levels of column n at a time, so each half of the split is
  // one 16-byte shared store into the K-major core layout (8 k-values of a
  // row are contiguous there): a quarter-warp's stores fill one 128-byte
  // line, free of bank conflicts.  Every load is issued before use.
  auto convert_b = [&](int kc) {  // all threads
    constexpr int GROUPS = kChunkK / 8;                 // 8 groups of 8 levels
    constexpr int GPT = GROUPS * kTileN / kThreadsZ;    // groups per thread: 4
    unsigned char* sB = sB0 + (kc & 1) * kChunkBytesB;
    const int n = tid & (kTileN - 1), g0 = tid / kTileN;
    const long long col = col0 + n;
    float x[GPT][8];
#pragma unroll
    for (int m = 0; m < GPT; ++m) {
      const int grp = g0 + m * (kThreadsZ / kTileN);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int lev = kc * kChunkK + grp * 8 + e;
        x[m][e] = (lev < nz && col < ncols) ? spec[(long long)lev * ncols + col] : 0.f;
      }
    }
#pragma unroll
    for (int m = 0; m < GPT; ++m) {
      const int grp = g0 + m * (kThreadsZ / kTileN);
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        __nv_bfloat16_raw h0, l0, h1, l1;
        split_bf16(x[m][e], h0, l0);
        split_bf16(x[m][e + 1], h1, l1);
        hi[e >> 1] = (uint32_t)h0.x | ((uint32_t)h1.x << 16);
        lo[e >> 1] = (uint32_t)l0.x | ((uint32_t)l1.x << 16);
      }
      const uint32_t o = core_off(n, grp * 8, 1024u);
      *reinterpret_cast<uint4*>(sB + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(sB + kChunkBytesB / 2 + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    fence_async_smem();
  };

  if (tid == 0)
    for (int i = 0; i < kStages && i < nch; ++i) issue_copy(i);
  convert_b(0);
  __syncthreads();

  // ---- first product: D1[mode][n] = sum_level (V^T W)[mode][level] F[level][n] ----
  for (int kc = 0; kc < nkc; ++kc) {
    if (tid == 0) {
      const uint32_t b_hi = smem_u32(sB0 + (kc & 1) * kChunkBytesB), b_lo = b_hi + kChunkBytesB / 2;
      for (int mt = 0; mt < nmt; ++mt) run_chunk(kc * nmt + mt, d1 + mt * kTileN, b_hi, b_lo, kc == 0);
      mma_commit(&bfree[kc & 1]);
    }
    if (kc + 1 < nkc) {
      if (kc >= 1 && !mbar_wait(&bfree[(kc + 1) & 1], (uint32_t)(((kc - 1) >> 1) & 1))) fail_s = 1;
      convert_b(kc + 1);
    }
    __syncthreads();
    if (fail_s) break;
  }
  if (tid == 0) mma_commit(d1done);
  if (!fail_s && !mbar_wait(d1done, 0)) fail_s = 1;
  tc_fence_after();
  __syncthreads();

  // ---- second product, one 64-mode chunk of the scaled first product at a time ----
  for (int kc = 0; kc < nkc && !fail_s; ++kc) {
    // modes kc*64 .. +64 are TMEM lanes (kc & 1)*64 .. +64 of D1 tile kc / 2
    const int mt = kc >> 1, wbase = (kc & 1) * 2;
    unsigned char* sG = sG0 + (kc & 1) * kChunkBytesB;
    if (warp == wbase || warp == wbase + 1) {
      if (kc >= 2 && !mbar_wait(&gfree[kc & 1], (uint32_t)(((kc - 2) >> 1) & 1))) fail_s = 1;
      const int ml = (warp - wbase) * 32 + lane;  // mode within the chunk
      const int m = kc * kChunkK + ml;
      const float mum = mu[m < nzp ? m : 0];
      for (int c16 = 0; c16 < kTileN / 16; ++c16) {
        float v[16];
        tmem_ld16(d1 + ((uint32_t)(warp * 32) << 16) + mt * kTileN + c16 * 16, v);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int n = c16 * 16 + q;
          const bool in = (col0 + n) < ncols && m < nz;
          const bool zero = (m == zero_mode) && ((col0 + n) >> 1) == 0;
          const float inv = (in && !zero) ? 1.0f / (mum + lam_s[n >> 1]) : 0.f;
          __nv_bfloat16_raw hi, lo;
          split_bf16(v[q] * inv, hi, lo);
          const uint32_t o = core_off(n, ml, 1024u);
          *reinterpret_cast<__nv_bfloat16_raw*>(sG + o) = hi;
          *reinterpret_cast<__nv_bfloat16_raw*>(sG + kChunkBytesB / 2 + o) = lo;
        }
      }
      fence_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && !fail_s) {
      const uint32_t g_hi = smem_u32(sG), g_lo = g_hi + kChunkBytesB / 2;
      for (int lt = 0; lt < nmt; ++lt) run_chunk(nch1 + kc * nmt + lt, d2 + lt * kTileN, g_hi, g_lo, kc == 0);
      mma_commit(&gfree[kc & 1]);
    }
  }
  if (tid == 0) mma_commit(d2done);
  __syncthreads();
  if (!fail_s && !mbar_wait(d2done, 0)) fail_s = 1;
  tc_fence_after();
  __syncthreads();

  // ---- write x back in place ----------------------------------------------
  if (!fail_s) {
    for (int lt = 0; lt < nmt; ++lt) {
      const int lev = lt * kTileM + warp * 32 + lane;
      for (int c16 = 0; c16 < kTileN / 16; ++c16) {
        float v[16];
        tmem_ld16(d2 + ((uint32_t)(warp * 32) << 16) + lt * kTileN + c16 * 16, v);
        if (lev < nz) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const long long col = col0 + c16 * 16 + q;
            if (col < ncols) spec[(long long)lev * ncols + col] = v[q];
          }
        }
      }
    }
  } else if (tid == 0) {
    // a bounded wait ran out: give in-flight copies and MMAs a bounded chance
    // to finish, report it (the host returns PP_ERR_CUDA), then free TMEM
    mma_commit(d2done);
    mbar_wait(d2done, 1);
    if (st != nullptr) st->pad = 1;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(512) : "memory");
}

size_t zgemm_smem_bytes(int nzp) {
  (void)nzp;
  return (size_t)kStages * kChunkBytesA + 4 * (size_t)kChunkBytesB;
}

cudaError_t launch_zgemm(const Geo& g, const ZEigen& ze, float2* spec, DevStatus* st, cudaStream_t s) {
  const long long ncols = 2LL * g.ny * g.nxh;
  const int nblk = (int)((ncols + kTileN - 1) / kTileN);
  const size_t smem = zgemm_smem_bytes(ze.nzp);
  cudaError_t e = cudaFuncSetAttribute(k_zgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_zgemm<<<nblk, kThreadsZ, smem, s>>>(reinterpret_cast<float*>(spec), ncols, g.nz, ze.nzp, g.nxh, ze.mu,
                                        ze.zero_mode, ze.lamx, ze.lamy, ze.a1, ze.a2, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host: eigenvectors of the symmetric tridiagonal S = W^{-1/2} T W^{-1/2} by
// Sturm-sequence bisection (eigenvalues) and inverse iteration with
// Gram-Schmidt (eigenvectors), then the bf16 hi/lo tiles of V^T W and V.

namespace {

// number of eigenvalues of the symmetric tridiagonal (d, e) below x
int sturm_count(const std::vector<double>& d, const std::vector<double>& e2, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    q = (d[i] - x) - (i > 0 ? e2[i - 1] / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// solve (S - s I) y = b in place (tridiagonal Gaussian elimination with
// partial pivoting; S has diagonal d and off-diagonal e)
void shifted_solve(const std::vector<double>& d, const std::vector<double>& e, double s, std::vector<double>& b) {
  const int n = (int)d.size();
  // band storage after pivoting: row i has entries at columns i, i+1, i+2
  std::vector<double> r0(n), r1(n, 0.0), r2(n, 0.0);
  std::vector<double> sub(n, 0.0);
  for (int i = 0; i < n; ++i) {
    r0[i] = d[i] - s;
    if (i + 1 < n) r1[i] = e[i];
    if (i > 0) sub[i] = e[i - 1];
  }
  const double tiny = 1e-300;
  for (int i = 0; i + 1 < n; ++i) {
    // rows i and i+1; sub[i+1] is row i+1's entry in column i
    if (std::fabs(sub[i + 1]) > std::fabs(r0[i])) {
      std::swap(r0[i], sub[i + 1]);
      std::swap(r1[i], r0[i + 1]);
      std::swap(r2[i], r1[i + 1]);
      std::swap(b[i], b[i + 1]);
    }
    const double piv = (r0[i] == 0.0) ? tiny : r0[i];
    const double f = sub[i + 1] / piv;
    r0[i + 1] -= f * r1[i];
    r1[i + 1] -= f * r2[i];
    b[i + 1] -= f * b[i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = b[i];
    if (i + 1 < n) v -= r1[i] * b[i + 1];
    if (i + 2 < n) v -= r2[i] * b[i + 2];
    b[i] = v / ((r0[i] == 0.0) ? tiny : r0[i]);
  }
}

uint16_t bf16_rn(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x7FFFFFu)) return 0x7FC0;
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

float bf16_to_f(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// matrix M (rows x cols = nzp x nzp, row-major, zero padded) -> tiles
void make_tiles(const std::vector<double>& M, int nzp, std::vector<uint16_t>& out) {
  const int nmt = nzp / kTileM, nkc = nzp / kChunkK;
  const size_t half = (size_t)kTileM * kChunkK;  // elements per hi (or lo) chunk
  out.assign((size_t)nmt * nkc * 2 * half, 0);
  for (int mt = 0; mt < nmt; ++mt)
    for (int kc = 0; kc < nkc; ++kc) {
      uint16_t* hi = out.data() + ((size_t)mt * nkc + kc) * 2 * half;
      uint16_t* lo = hi + half;
      for (int r = 0; r < kTileM; ++r)
        for (int k = 0; k < kChunkK; ++k) {
          const float x = (float)M[(size_t)(mt * kTileM + r) * nzp + kc * kChunkK + k];
          const uint16_t h = bf16_rn(x);
          const uint16_t l = bf16_rn(x - bf16_to_f(h));
          const size_t o = ((size_t)(r >> 3) * 1024 + (size_t)(k >> 3) * 128 + (size_t)(r & 7) * 16 + (size_t)(k & 7) * 2) / 2;
          hi[o] = h;
          lo[o] = l;
        }
    }
}

}  // namespace

// Eigenpairs of the symmetric tridiagonal (d, e), ascending: Sturm-sequence
// bisection for the eigenvalues, inverse iteration with two Gram-Schmidt
// passes for the eigenvectors, and a residual check of every pair.
bool sym_tridiag_eigen(const std::vector<double>& d, const std::vector<double>& e, std::vector<double>& lam,
                       std::vector<double>& Q) {
  const int n = (int)d.size();
  std::vector<double> e2(n, 0.0);
  for (int k = 0; k + 1 < n; ++k) e2[k] = e[k] * e[k];
  double lo = 0.0, hi = 0.0;  // Gershgorin interval
  for (int k = 0; k < n; ++k) {
    const double r = (k > 0 ? std::fabs(e[k - 1]) : 0.0) + (k + 1 < n ? std::fabs(e[k]) : 0.0);
    lo = std::min(lo, d[k] - r);
    hi = std::max(hi, d[k] + r);
  }
  lam.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    double a = lo, b = hi;
    for (int it = 0; it < 200 && b - a > 1e-15 * std::max(1.0, std::max(std::fabs(a), std::fabs(b))); ++it) {
      const double m = 0.5 * (a + b);
      if (sturm_count(d, e2, m) > j) b = m; else a = m;
    }
    lam[j] = 0.5 * (a + b);
  }
  Q.assign((size_t)n * n, 0.0);
  unsigned long long seed = 0x9E3779B97F4A7C15ull;
  for (int j = 0; j < n; ++j) {
    std::vector<double> v(n);
    for (int k = 0; k < n; ++k) {
      seed = seed * 6364136223846793005ull + 1442695040888963407ull;
      v[k] = (double)(seed >> 11) / 9007199254740992.0 - 0.5;
    }
    const double shift = lam[j] + 1e-10 * std::max(1.0, std::fabs(lam[j]));
    for (int it = 0; it < 3; ++it) {
      shifted_solve(d, e, shift, v);
      for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < j; ++i) {
          double dot = 0.0;
          for (int k = 0; k < n; ++k) dot += Q[(size_t)k * n + i] * v[k];
          for (int k = 0; k < n; ++k) v[k] -= dot * Q[(size_t)k * n + i];
        }
      double nrm = 0.0;
      for (int k = 0; k < n; ++k) nrm += v[k] * v[k];
      nrm = std::sqrt(nrm);
      if (!(nrm > 0.0)) return false;
      for (int k = 0; k < n; ++k) v[k] /= nrm;
    }
    for (int k = 0; k < n; ++k) Q[(size_t)k * n + j] = v[k];
  }
  // self-check: residual of S q = lambda q for every pair
  for (int j = 0; j < n; ++j) {
    double res = 0.0;
    for (int k = 0; k < n; ++k) {
      double sq = d[k] * Q[(size_t)k * n + j];
      if (k > 0) sq += e[k - 1] * Q[(size_t)(k - 1) * n + j];
      if (k + 1 < n) sq += e[k] * Q[(size_t)(k + 1) * n + j];
      res = std::max(res, std::fabs(sq - lam[j] * Q[(size_t)k * n + j]));
    }
    if (res > 1e-8 * std::max(1.0, std::fabs(lo))) return false;
  }
  return true;
}

// Builds the eigen tables of L_z on the host; device buffers are allocated
// by the caller-provided allocator (plan memory).  Returns false when the
// eigen decomposition failed its own checks.
bool build_zeigen_host(int nz, const double* dzf, const double* inv_dzc, int* nzp_out, std::vector<float>& mu_out,
                       int* zero_mode, std::vector<uint16_t>& a1, std::vector<uint16_t>& a2) {
  const int nzp = ((nz + kTileM - 1) / kTileM) * kTileM;
  *nzp_out = nzp;
  // S = W^{-1/2} T W^{-1/2}, T_kk = -(1/dzc_k + 1/dzc_{k+1}), T_{k,k+1} = 1/dzc_{k+1}
  std::vector<double> d(nz), e(nz > 1 ? nz - 1 : 1, 0.0);
  for (int k = 0; k < nz; ++k) d[k] = -(inv_dzc[k] + inv_dzc[k + 1]) / dzf[k];
  for (int k = 0; k + 1 < nz; ++k) e[k] = inv_dzc[k + 1] / std::sqrt(dzf[k] * dzf[k + 1]);
  std::vector<double> lam, Q;
  if (!sym_tridiag_eigen(d, e, lam, Q)) return false;
  int zm = 0;
  for (int j = 1; j < nz; ++j)
    if (std::fabs(lam[j]) < std::fabs(lam[zm])) zm = j;
  *zero_mode = zm;
  mu_out.assign(nzp, 0.0f);
  for (int j = 0; j < nz; ++j) mu_out[j] = (float)lam[j];
  std::vector<double> M1((size_t)nzp * nzp, 0.0), M2((size_t)nzp * nzp, 0.0);
  for (int j = 0; j < nz; ++j)
    for (int k = 0; k < nz; ++k) {
      const double q = Q[(size_t)k * nz + j];
      M1[(size_t)j * nzp + k] = q * std::sqrt(dzf[k]);  // (V^T W)[mode j][level k]
      M2[(size_t)k * nzp + j] = q / std::sqrt(dzf[k]);  // V[level k][mode j]
    }
  make_tiles(M1, nzp, a1);
  make_tiles(M2, nzp, a2);
  return true;
}

// The same decomposition for a stretched y between walls, in the order the
// spectrum's rows take (mode 0 = the constant, eigenvalue 0, first).  The
// constant mode is set exactly (q_0 = W^{1/2} 1 / sqrt(ly)) and the others
// are made orthogonal to it once more.
bool build_yeigen_host(int ny, const double* dyf, const double* inv_dyc, std::vector<double>& lam,
                       std::vector<double>& mt_fwd, std::vector<double>& mt_inv) {
  std::vector<double> d(ny), e(ny > 1 ? ny - 1 : 1, 0.0);
  for (int j = 0; j < ny; ++j) d[j] = -(inv_dyc[j] + inv_dyc[j + 1]) / dyf[j];
  for (int j = 0; j + 1 < ny; ++j) e[j] = inv_dyc[j + 1] / std::sqrt(dyf[j] * dyf[j + 1]);
  std::vector<double> asc, Q;
  if (!sym_tridiag_eigen(d, e, asc, Q)) return false;
  double ly = 0.0;
  for (int j = 0; j < ny; ++j) ly += dyf[j];
  // mode m of the spectrum = ascending pair ny - 1 - m
  std::vector<double> q((size_t)ny * ny);  // q[m * ny + j]
  for (int m = 0; m < ny; ++m)
    for (int j = 0; j < ny; ++j) q[(size_t)m * ny + j] = Q[(size_t)j * ny + (ny - 1 - m)];
  for (int j = 0; j < ny; ++j) q[j] = std::sqrt(dyf[j] / ly);
  for (int m = 1; m < ny; ++m) {
    double dot = 0.0, nrm = 0.0;
    for (int j = 0; j < ny; ++j) dot += q[j] * q[(size_t)m * ny + j];
    for (int j = 0; j < ny; ++j) {
      q[(size_t)m * ny + j] -= dot * q[j];
      nrm += q[(size_t)m * ny + j] * q[(size_t)m * ny + j];
    }
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0)) return false;
    for (int j = 0; j < ny; ++j) q[(size_t)m * ny + j] /= nrm;
  }
  lam.assign(ny, 0.0);
  for (int m = 1; m < ny; ++m) lam[m] = asc[ny - 1 - m];
  mt_fwd.assign((size_t)ny * ny, 0.0);
  mt_inv.assign((size_t)ny * ny, 0.0);
  for (int m = 0; m < ny; ++m)
    for (int j = 0; j < ny; ++j) {
      const double v = q[(size_t)m * ny + j];
      mt_fwd[(size_t)j * ny + m] = v * std::sqrt(dyf[j]);  // (V^T W)[m][j], stored [j][m]
      mt_inv[(size_t)m * ny + j] = v / std::sqrt(dyf[j]);  // V[j][m], stored [m][j]
    }
  return true;
}

}  // namespace pp
