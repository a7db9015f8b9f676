// Register-resident complex transform of length 512 in FP32, the core of
// the 512-point x and y transforms of the eigenexpansion solve (Sec. 3.3.1).
//
// A line is split 512 = 8 x 8 x 8 (n = 64 a + b, k = c + 8 d, then
// b = 8 e + f, d = g + 8 h; w = exp(DIR 2 pi i / 512)):
//   X[c + 8 g + 64 h] = sum_f W8^{f h} w^{8 f g} sum_e W8^{e g} y_{8 e + f}[c],
//   y_b[c] = w^{b c} sum_a W8^{a c} x[64 a + b].
// 64 threads hold one line, 8 values each.  Thread j enters with
// x[64 a + j], a = 0..7, does the first 8-point DFT and its twiddles; two
// exchanges through shared memory feed the second and third 8-point DFTs;
// thread j leaves with X[j + 64 h], h = 0..7.  A block holds TX lines, the
// line index x being the fastest-varying part of the thread index
// (thread = x + TX j), so that every exchange is free of bank conflicts:
// the first buffer is [c][b][x], the second [c][g][f][x] with each c slab
// padded by TX values.
#pragma once
#include "pp_fft.cuh"

namespace pp {

template <int TX>
struct R512 {
  static constexpr int N = 512;
  static constexpr int S1 = N * TX;         // first exchange buffer [c][b][x]
  static constexpr int CS2 = 64 * TX + TX;  // second buffer: slab of one c, padded
  static constexpr int S2 = 8 * CS2;        // [c][g][f][x]
  // twiddles, laid out so that a warp's reads are consecutive: T1[c][b] =
  // w^{b c} (c < 8, b < 64) for the first stage, T2[r][f] = w^{8 f r} for
  // the second; each entry copied from the (cos, sin)(2 pi m / 512) table
  static constexpr int TW = 8 * 64 + 64;
  static constexpr size_t smem_bytes() { return (size_t)(TW + S1 + S2) * sizeof(float2); }
};

// Fills the two twiddle tables of R512 from the 512-entry table `tw512`
// (global memory); every thread of the block calls it, a barrier follows.
__device__ __forceinline__ void r512_load_twiddles(float2* tw, const float2* __restrict__ tw512) {
  for (int i = threadIdx.x; i < 8 * 64 + 64; i += blockDim.x) {
    int m;
    if (i < 512) m = (i >> 6) * (i & 63);               // T1[c][b]: b c
    else m = 8 * ((i - 512) & 7) * ((i - 512) >> 3);    // T2[r][f]: 8 f r
    tw[i] = tw512[m & 511];
  }
}

// v[r] *= tab[r * stride + q] for r = 1..7 (the entry holds w^{r q'}, with
// the direction's sign applied here).
template <int DIR>
__device__ __forceinline__ void r512_twiddle8(float2* v, const float2* __restrict__ tab, int stride, int q) {
#pragma unroll
  for (int r = 1; r < 8; ++r) v[r] = cmul<float>(v[r], tw_dir<DIR>(tab[r * stride + q]));
}

// The transform of the thread's line (see above); every thread of the block
// calls it.  v holds x[64 a + j] on entry and is free once its values are in
// s1: `after_s1` runs right then (e.g. to load the next line into v) and
// before the first barrier; `after_b1` runs right after the first barrier
// (every thread of the block has then finished what it did before the call).
// The result X[j + 64 h] is left in u.  The call holds two barriers; s1 is
// last read before the second, s2 last read after it, so a following call
// (whose first barrier comes after its s1 writes and before its s2 writes)
// needs no barrier in between.
template <int DIR, int TX, class F, class G>
__device__ __forceinline__ void r512_transform(float2 (&v)[8], float2 (&u)[8], float2* s1, float2* s2,
                                               const float2* __restrict__ tw, int x, int j, F&& after_s1,
                                               G&& after_b1) {
  using L = R512<TX>;
  Dft<float, DIR, 8>::run(v);
  r512_twiddle8<DIR>(v, tw, 64, j);
#pragma unroll
  for (int c = 0; c < 8; ++c) s1[(c * 64 + j) * TX + x] = v[c];
  after_s1();
  __syncthreads();
  after_b1();
  {
    const int c = j >> 3, f = j & 7;
#pragma unroll
    for (int e = 0; e < 8; ++e) u[e] = s1[(c * 64 + 8 * e + f) * TX + x];
    Dft<float, DIR, 8>::run(u);
    r512_twiddle8<DIR>(u, tw + 512, 8, f);
#pragma unroll
    for (int gg = 0; gg < 8; ++gg) s2[c * L::CS2 + (gg * 8 + f) * TX + x] = u[gg];
  }
  __syncthreads();
  {
    const int c = j & 7, gg = j >> 3;
#pragma unroll
    for (int f = 0; f < 8; ++f) u[f] = s2[c * L::CS2 + (gg * 8 + f) * TX + x];
    Dft<float, DIR, 8>::run(u);
  }
}

template <int DIR, int TX, class F>
__device__ __forceinline__ void r512_transform(float2 (&v)[8], float2 (&u)[8], float2* s1, float2* s2,
                                               const float2* __restrict__ tw, int x, int j, F&& after_s1) {
  r512_transform<DIR, TX>(v, u, s1, s2, tw, x, j, after_s1, []() {});
}

}  // namespace pp
