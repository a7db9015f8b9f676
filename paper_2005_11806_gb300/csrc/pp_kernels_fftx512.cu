// Inverse real x transform of length 512 in FP32 with the data in registers
// (pp_r512.cuh), fused with the update of p: the last step of a pass of
// Algorithm 1 (Sec. 3.3.1) on mixed plans with nx = 512.  Same arithmetic
// and update modes as stage_fftx_inv (pp_stages.cuh): two rows of half
// spectra A, B form one complex line Z = A + i B (the upper half from the
// conjugate symmetry), its inverse transform gives the two real rows.
// A block walks groups of 2 TX rows with stride gridDim.x.  The rows of a
// group (one contiguous span of the spectrum) are copied into shared memory
// by cp.async while the block transforms the group before it; thread j of a
// line then gathers Z[64 a + j] from the staged half spectra (each
// coefficient below nx/2 is read for itself and for its mirror) and updates
// the cells j + 64 h of both rows from its registers.
#include "pp_r512.cuh"
#include "pp_stages.cuh"

namespace pp {

namespace {
constexpr int kXLines = 4;  // complex lines (row pairs) per block: 256 threads
constexpr int kXNh = 257;   // half-spectrum length of a 512-point row
// Row stride of the staged half spectra, in float2: 258 = 2 (mod 8), so the
// A rows (and the B rows) of the 4 lines start 4 bank pairs apart and a half
// warp's gather (4 lines x 4 consecutive coefficients) is conflict-free.
constexpr int kXStageRow = 258;

template <int MODE>
__device__ __forceinline__ void fftx512_inv_body(const Geo& g, const float2* __restrict__ spec, double scale,
                                                 double* __restrict__ p, int p_zero, float* __restrict__ delta,
                                                 float* __restrict__ sdelta, float2* s1, float2* s2,
                                                 const float2* tw, float2* stage, long long ngroups) {
  constexpr int TX = kXLines;
  constexpr int N = 512;
  constexpr int NH = kXNh;
  const long long nrows = (long long)g.nz * g.ny;
  const int x = threadIdx.x % TX, j = threadIdx.x / TX;
  const float scale_f = (float)scale;
  const bool need_p = !p_zero && MODE <= kInvFoldFresh;
  constexpr bool need_s = MODE == kInvFold || MODE == kInvAccum;
  // the rows of group grp (those below nrows) into stage, one commit group
  auto stage_rows = [&](long long grp) {
    const long long r0 = grp * (2 * TX);
    const int nr = nrows - r0 < 2 * TX ? (int)(nrows - r0) : 2 * TX;
    const int ne = nr * NH;
    const float2* src = spec + (size_t)r0 * NH;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const int r = e / NH;
      cp_async8(stage + r * kXStageRow + (e - r * NH), src + e);
    }
    cp_async_commit();
  };
  if (blockIdx.x < ngroups) stage_rows(blockIdx.x);
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const long long ra = grp * (2 * TX) + 2 * x, rb = ra + 1;
    const bool va = ra < nrows, vb = rb < nrows;
    // this group's rows are in stage once every thread's copies have landed
    cp_async_wait_all();
    __syncthreads();
    const float2* SA = stage + (2 * x) * kXStageRow;
    const float2* SB = SA + kXStageRow;
    float2 v[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int m = 64 * a + j;
      const bool mirror = m > N / 2;
      const int mm = mirror ? N - m : m;
      float2 A = make_float2(0.f, 0.f), B = A;
      if (va) A = SA[mm];
      if (vb) B = SB[mm];
      if (m == 0 || m == N / 2) v[a] = make_float2(A.x, B.x);
      else if (!mirror) v[a] = make_float2(A.x - B.y, A.y + B.x);
      else v[a] = make_float2(A.x + B.y, B.x - A.y);
    }
    // pending sums of the increments, in flight during the transform
    float sva[8], svb[8];
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      sva[h] = 0.f;
      svb[h] = 0.f;
      if (need_s) {
        const int i = j + 64 * h;
        if (va) sva[h] = sdelta[(size_t)ra * N + i];
        if (vb) svb[h] = sdelta[(size_t)rb * N + i];
      }
    }
    float2 z[8];
    // stage is free once every thread has passed the transform's first
    // barrier: the next group's copies run during the rest of this one
    const long long next = grp + gridDim.x;
    r512_transform<1, TX>(v, z, s1, s2, tw, x, j, []() {}, [&]() {
      if (next < ngroups) stage_rows(next);
    });
    auto emit = [&](size_t c, float zv, float sv) {
      const float inc_f = scale_f * zv;
      if constexpr (MODE <= kInvFoldFresh) {
        const double zd = widen_f32(zv);
        const double pv = need_p ? p[c] : 0.0;
        if constexpr (MODE == kInvFold) p[c] = fma(scale, zd, pv + widen_f32(sv));
        else p[c] = fma(scale, zd, pv);
      } else {
        sdelta[c] = (MODE == kInvAccum) ? sv + inc_f : inc_f;
      }
      if (delta != nullptr) delta[c] = inc_f;
    };
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int i = j + 64 * h;
      if (va) emit((size_t)ra * N + i, z[h].x, sva[h]);
      if (vb) emit((size_t)rb * N + i, z[h].y, svb[h]);
    }
  }
}
}  // namespace

// Update modes as k_fftx_inv: sdelta null -> plain update of p.
__global__ void __launch_bounds__(64 * kXLines, 4) k_fftx512_inv(Geo g, const float2* __restrict__ twx,
                                                             const float2* __restrict__ spec, double scale,
                                                             double* __restrict__ p, int p_zero,
                                                             long long ngroups, const DevStatus* __restrict__ st,
                                                             float* __restrict__ delta, float* __restrict__ sdelta) {
  if (stopped(st)) return;
  using L = R512<kXLines>;
  float2* sm = smem_f2();
  float2* tw = sm;
  float2* s1 = sm + L::TW;
  float2* s2 = s1 + L::S1;
  float2* stage = s2 + L::S2;
  r512_load_twiddles(tw, twx);
  __syncthreads();
  const bool lazy = sdelta != nullptr && st != nullptr;
  const bool fold = lazy && st->need_exact != 0;
  const bool fresh = lazy && st->since_exact <= 1;
  if (!lazy)
    fftx512_inv_body<kInvPlain>(g, spec, scale, p, p_zero, delta, sdelta, s1, s2, tw, stage, ngroups);
  else if (fold && !fresh)
    fftx512_inv_body<kInvFold>(g, spec, scale, p, p_zero, delta, sdelta, s1, s2, tw, stage, ngroups);
  else if (fold)
    fftx512_inv_body<kInvFoldFresh>(g, spec, scale, p, p_zero, delta, sdelta, s1, s2, tw, stage, ngroups);
  else if (fresh)
    fftx512_inv_body<kInvFresh>(g, spec, scale, p, p_zero, delta, sdelta, s1, s2, tw, stage, ngroups);
  else
    fftx512_inv_body<kInvAccum>(g, spec, scale, p, p_zero, delta, sdelta, s1, s2, tw, stage, ngroups);
}

cudaError_t launch_fftx512_inv(const Geo& g, const float2* twx, const float2* spec, double scale, double* p,
                               int p_zero, const DevStatus* st, cudaStream_t s, float* delta, float* sdelta) {
  if (g.nxh != kXNh) return cudaErrorInvalidValue;
  const size_t smem = R512<kXLines>::smem_bytes() + (size_t)2 * kXLines * kXStageRow * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_fftx512_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long nrows = (long long)g.nz * g.ny;
  const long long ngroups = (nrows + 2 * kXLines - 1) / (2 * kXLines);
  int per_sm = 0, dev = 0, nsm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fftx512_inv, 64 * kXLines, smem)) != cudaSuccess)
    return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  long long nblk = (long long)nsm * per_sm;
  if (nblk > ngroups) nblk = ngroups;
  k_fftx512_inv<<<(int)nblk, 64 * kXLines, smem, s>>>(g, twx, spec, scale, p, p_zero, ngroups, st, delta, sdelta);
  return cudaGetLastError();
}

}  // namespace pp
