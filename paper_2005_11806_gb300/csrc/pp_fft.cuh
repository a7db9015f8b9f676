// Shared-memory mixed-radix Stockham FFT (radices 8, 4, 2, 3, 5) used by the
// x and y transforms of the eigenexpansion solver.  The twiddle table holds
// (cos, sin)(2 pi m / n), m = 0..n-1, computed on the host in FP64.
#pragma once
#include "pp_internal.cuh"

namespace pp {

template <typename T> __device__ __forceinline__ C2<T> mk(T x, T y) { C2<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by DIR * i  (DIR = -1: -i, DIR = +1: +i)
template <typename T, int DIR> __device__ __forceinline__ C2<T> mul_i(C2<T> a) {
  return DIR > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// In-register DFT of size R with kernel exp(DIR * 2 pi i q r / R).
template <typename T, int DIR, int R> struct Dft;

template <typename T, int DIR> struct Dft<T, DIR, 2> {
  static __device__ __forceinline__ void run(C2<T>* v) {
    C2<T> a = v[0], b = v[1];
    v[0] = cadd<T>(a, b);
    v[1] = csub<T>(a, b);
  }
};

template <typename T, int DIR> struct Dft<T, DIR, 4> {
  static __device__ __forceinline__ void run(C2<T>* v) {
    C2<T> s02 = cadd<T>(v[0], v[2]), d02 = csub<T>(v[0], v[2]);
    C2<T> s13 = cadd<T>(v[1], v[3]), d13 = mul_i<T, DIR>(csub<T>(v[1], v[3]));
    v[0] = cadd<T>(s02, s13);
    v[2] = csub<T>(s02, s13);
    v[1] = cadd<T>(d02, d13);
    v[3] = csub<T>(d02, d13);
  }
};

template <typename T, int DIR> struct Dft<T, DIR, 8> {
  static __device__ __forceinline__ void run(C2<T>* v) {
    C2<T> e[4] = {v[0], v[2], v[4], v[6]};
    C2<T> o[4] = {v[1], v[3], v[5], v[7]};
    Dft<T, DIR, 4>::run(e);
    Dft<T, DIR, 4>::run(o);
    const T h = (T)0.70710678118654752440;  // cos(pi/4)
    // o[q] *= exp(DIR * 2 pi i q / 8)
    C2<T> o1 = mk<T>(h * (o[1].x - (T)DIR * o[1].y), h * (o[1].y + (T)DIR * o[1].x));
    C2<T> o2 = mul_i<T, DIR>(o[2]);
    C2<T> o3 = mk<T>(h * (-o[3].x - (T)DIR * o[3].y), h * (-o[3].y + (T)DIR * o[3].x));
    v[0] = cadd<T>(e[0], o[0]); v[4] = csub<T>(e[0], o[0]);
    v[1] = cadd<T>(e[1], o1);   v[5] = csub<T>(e[1], o1);
    v[2] = cadd<T>(e[2], o2);   v[6] = csub<T>(e[2], o2);
    v[3] = cadd<T>(e[3], o3);   v[7] = csub<T>(e[3], o3);
  }
};

template <typename T, int DIR> struct Dft<T, DIR, 3> {
  static __device__ __forceinline__ void run(C2<T>* v) {
    const T c = (T)-0.5, s = (T)0.86602540378443864676;  // cos, sin(2 pi / 3)
    C2<T> t1 = cadd<T>(v[1], v[2]);
    C2<T> t2 = mk<T>(v[0].x + c * t1.x, v[0].y + c * t1.y);
    C2<T> d = csub<T>(v[1], v[2]);
    C2<T> t3 = mul_i<T, DIR>(mk<T>(s * d.x, s * d.y));
    v[0] = cadd<T>(v[0], t1);
    v[1] = cadd<T>(t2, t3);
    v[2] = csub<T>(t2, t3);
  }
};

template <typename T, int DIR> struct Dft<T, DIR, 5> {
  static __device__ __forceinline__ void run(C2<T>* v) {
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;  // cos 2pi/5, 4pi/5
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;   // sin 2pi/5, 4pi/5
    C2<T> a14 = cadd<T>(v[1], v[4]), d14 = csub<T>(v[1], v[4]);
    C2<T> a23 = cadd<T>(v[2], v[3]), d23 = csub<T>(v[2], v[3]);
    C2<T> r1 = mk<T>(v[0].x + c1 * a14.x + c2 * a23.x, v[0].y + c1 * a14.y + c2 * a23.y);
    C2<T> r2 = mk<T>(v[0].x + c2 * a14.x + c1 * a23.x, v[0].y + c2 * a14.y + c1 * a23.y);
    C2<T> i1 = mul_i<T, DIR>(mk<T>(s1 * d14.x + s2 * d23.x, s1 * d14.y + s2 * d23.y));
    C2<T> i2 = mul_i<T, DIR>(mk<T>(s2 * d14.x - s1 * d23.x, s2 * d14.y - s1 * d23.y));
    v[0] = cadd<T>(v[0], cadd<T>(a14, a23));
    v[1] = cadd<T>(r1, i1);
    v[4] = csub<T>(r1, i1);
    v[2] = cadd<T>(r2, i2);
    v[3] = csub<T>(r2, i2);
  }
};

// One Stockham pass of radix R over `nbatch` sequences of length n stored at
// buf[b * bs + m * es].  BATCH_FAST selects which index consecutive threads
// walk (the one that is contiguous in shared memory).  POW2: n, Ns and (for
// BATCH_FAST) nbatch are powers of two, so divisions become shifts
// (lg_* are their base-2 logarithms).
template <typename T, int DIR, int R, bool BATCH_FAST, bool POW2>
__device__ __forceinline__ void fft_pass(const C2<T>* __restrict__ src, C2<T>* __restrict__ dst, int n,
                                         int Ns, int lg_ns, int nbatch, int lg_nbatch, int es, int bs,
                                         const C2<T>* __restrict__ tw, int tid, int nth) {
  const int nb = n / R;
  const int total = nb * nbatch;
  const int tws = n / (Ns * R);
  constexpr int LR = R == 8 ? 3 : R == 4 ? 2 : 1;
  const int lg_nb = POW2 ? (31 - __clz(nb)) : 0;
  for (int t = tid; t < total; t += nth) {
    int bi, j, k, jq;
    if (POW2) {
      if (BATCH_FAST) { j = t >> lg_nbatch; bi = t & (nbatch - 1); }
      else { bi = t >> lg_nb; j = t & (nb - 1); }
      k = j & (Ns - 1);
      jq = j >> lg_ns;
    } else {
      if (BATCH_FAST) { j = t / nbatch; bi = t - j * nbatch; }
      else { bi = t / nb; j = t - bi * nb; }
      jq = j / Ns;
      k = j - jq * Ns;
    }
    C2<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[bi * bs + (j + r * nb) * es];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C2<T> w = __ldg(&tw[r * k * tws]);
        w.y = DIR > 0 ? w.y : -w.y;
        v[r] = cmul<T>(v[r], w);
      }
    }
    Dft<T, DIR, R>::run(v);
    const int base = POW2 ? ((jq << (lg_ns + LR)) + k) : (jq * Ns * R + k);
#pragma unroll
    for (int r = 0; r < R; ++r) dst[bi * bs + (base + r * Ns) * es] = v[r];
  }
}

// Full transform; returns the buffer (a or b) holding the result.  Every
// thread of the block must call it (it synchronises between passes).
template <typename T, int DIR, bool BATCH_FAST>
__device__ C2<T>* fft_block(C2<T>* a, C2<T>* b, const FftDesc& d, int nbatch, int es, int bs,
                            const C2<T>* __restrict__ tw, int tid, int nth) {
  int Ns = 1, lg_ns = 0;
  const bool pow2 = d.pow2 && (!BATCH_FAST || (nbatch & (nbatch - 1)) == 0);
  const int lg_nbatch = 31 - __clz(nbatch);
  C2<T>* src = a;
  C2<T>* dst = b;
  for (int s = 0; s < d.nst; ++s) {
    const int R = d.radix[s];
    if (pow2) {
      switch (R) {
        case 8: fft_pass<T, DIR, 8, BATCH_FAST, true>(src, dst, d.n, Ns, lg_ns, nbatch, lg_nbatch, es, bs, tw, tid, nth); break;
        case 4: fft_pass<T, DIR, 4, BATCH_FAST, true>(src, dst, d.n, Ns, lg_ns, nbatch, lg_nbatch, es, bs, tw, tid, nth); break;
        default: fft_pass<T, DIR, 2, BATCH_FAST, true>(src, dst, d.n, Ns, lg_ns, nbatch, lg_nbatch, es, bs, tw, tid, nth); break;
      }
    } else {
      switch (R) {
        case 8: fft_pass<T, DIR, 8, BATCH_FAST, false>(src, dst, d.n, Ns, 0, nbatch, 0, es, bs, tw, tid, nth); break;
        case 4: fft_pass<T, DIR, 4, BATCH_FAST, false>(src, dst, d.n, Ns, 0, nbatch, 0, es, bs, tw, tid, nth); break;
        case 2: fft_pass<T, DIR, 2, BATCH_FAST, false>(src, dst, d.n, Ns, 0, nbatch, 0, es, bs, tw, tid, nth); break;
        case 3: fft_pass<T, DIR, 3, BATCH_FAST, false>(src, dst, d.n, Ns, 0, nbatch, 0, es, bs, tw, tid, nth); break;
        default: fft_pass<T, DIR, 5, BATCH_FAST, false>(src, dst, d.n, Ns, 0, nbatch, 0, es, bs, tw, tid, nth); break;
      }
    }
    __syncthreads();
    C2<T>* t = src; src = dst; dst = t;
    Ns *= R;
    lg_ns += (R == 8) ? 3 : (R == 4) ? 2 : 1;
  }
  return src;
}

// Compile-time variant for power-of-two N (radices 8, then one 4 or 2):
// every index is a constant shift/mask, strides are template arguments.
template <int N> struct Log2 { static constexpr int value = 1 + Log2<N / 2>::value; };
template <> struct Log2<1> { static constexpr int value = 0; };
template <int N, int S> struct Pow2Radix {  // radix of pass S for length N
  static constexpr int rem = Log2<N>::value - 3 * S;
  static constexpr int value = rem >= 3 ? 8 : (rem == 2 ? 4 : 2);
};
template <int N> struct Pow2Passes { static constexpr int value = (Log2<N>::value + 2) / 3; };

template <typename T, int DIR, int R, bool BATCH_FAST, int N, int NS, int NBATCH, int ES, int BS>
__device__ __forceinline__ void fft_pass_fixed(const C2<T>* __restrict__ src, C2<T>* __restrict__ dst,
                                               const C2<T>* __restrict__ tw, int tid, int nth) {
  constexpr int NB = N / R;
  constexpr int TOTAL = NB * NBATCH;
  constexpr int TWS = N / (NS * R);
  for (int t = tid; t < TOTAL; t += nth) {
    int bi, j;
    if (BATCH_FAST) { j = t / NBATCH; bi = t % NBATCH; }
    else { bi = t / NB; j = t % NB; }
    const int k = j % NS;
    C2<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[bi * BS + (j + r * NB) * ES];
    if (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C2<T> w = __ldg(&tw[r * k * TWS]);
        w.y = DIR > 0 ? w.y : -w.y;
        v[r] = cmul<T>(v[r], w);
      }
    }
    Dft<T, DIR, R>::run(v);
    const int base = (j / NS) * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[bi * BS + (base + r * NS) * ES] = v[r];
  }
}

template <typename T, int DIR, bool BATCH_FAST, int N, int NBATCH, int ES, int BS, int S, int NS>
__device__ __forceinline__ void fft_fixed_from(C2<T>*& src, C2<T>*& dst, const C2<T>* __restrict__ tw,
                                               int tid, int nth) {
  if constexpr (S < Pow2Passes<N>::value) {
    constexpr int R = Pow2Radix<N, S>::value;
    fft_pass_fixed<T, DIR, R, BATCH_FAST, N, NS, NBATCH, ES, BS>(src, dst, tw, tid, nth);
    __syncthreads();
    C2<T>* t = src; src = dst; dst = t;
    fft_fixed_from<T, DIR, BATCH_FAST, N, NBATCH, ES, BS, S + 1, NS * R>(src, dst, tw, tid, nth);
  }
}

// Full compile-time transform; returns the buffer holding the result.
template <typename T, int DIR, bool BATCH_FAST, int N, int NBATCH, int ES, int BS>
__device__ __forceinline__ C2<T>* fft_block_fixed(C2<T>* a, C2<T>* b, const C2<T>* __restrict__ tw, int tid,
                                                  int nth) {
  C2<T>* src = a;
  C2<T>* dst = b;
  fft_fixed_from<T, DIR, BATCH_FAST, N, NBATCH, ES, BS, 0, 1>(src, dst, tw, tid, nth);
  return src;
}

// ---------------------------------------------------------------------------
// FP32 fast path for the compile-time power-of-two shapes.  Buffers and the
// twiddle table are addressed by element offsets into the block's dynamic
// shared memory (one float2 array), so every access is a 32-bit shared
// access whose constant strides fold into immediate offsets; pointers chosen
// at run time (rotating buffers) would leave the compiler generic 64-bit
// addressing.  The twiddle table tw[m] = (cos, sin)(2 pi m / N), m < N,
// sits in shared memory too.  A radix-8 butterfly loads w, w^2 and w^4 from
// it and forms w^3, w^5, w^6, w^7 by complex products.
__device__ __forceinline__ float2* smem_f2() {
  extern __shared__ __align__(16) float2 pp_dyn_smem_f2[];
  return pp_dyn_smem_f2;
}

template <int DIR>
__device__ __forceinline__ float2 tw_dir(float2 w) { return make_float2(w.x, DIR > 0 ? w.y : -w.y); }

// Bank-conflict padding of the first pass's output.  That pass writes each
// butterfly's R = 8 outputs to R consecutive positions (stride R*ES between
// threads), a 16-way (x layout) or 8-way (batched y layout) conflict.  The
// buffer it writes therefore holds one gap of PU elements after every PG
// elements (PG = 8 ES, PU = ES), which spreads those writes over all banks;
// the second pass reads through the same map.  Buffers written padded hold
// 9/8 of their elements (fft_pad_elems).
template <bool BATCH_FAST, int NBATCH>
struct FftPad {
  static constexpr int PG = BATCH_FAST ? 8 * NBATCH : 8;
  static constexpr int PU = BATCH_FAST ? NBATCH : 1;
  static __device__ __forceinline__ int map(int pos) { return pos + (pos / PG) * PU; }
};
__host__ __device__ inline int fft_pad_elems(int n) { return n + n / 8; }

template <int DIR, int R, bool BATCH_FAST, int N, int NS, int NBATCH, int ES, int BS, bool PIN, bool POUT>
__device__ __forceinline__ void fft_pass_smem(int src, int dst, int twb, int tid, int nth) {
  float2* S = smem_f2();
  using Pad = FftPad<BATCH_FAST, NBATCH>;
  constexpr int NB = N / R;
  constexpr int TOTAL = NB * NBATCH;
  constexpr int TWS = N / (NS * R);
  // a padded input is read at stride NB*ES, a multiple of PG: the gaps add a
  // constant per r, so the offsets stay compile-time
  constexpr int IN_STEP = PIN ? NB * ES + (NB * ES / Pad::PG) * Pad::PU : NB * ES;
  static_assert(!PIN || (NB * ES) % Pad::PG == 0, "padded reads need strides that are multiples of PG");
  static_assert(!POUT || NS == 1, "only the first pass writes padded");
  for (int t = tid; t < TOTAL; t += nth) {
    int bi, j;
    if (BATCH_FAST) { j = t / NBATCH; bi = t % NBATCH; }
    else { bi = t / NB; j = t % NB; }
    const int k = j % NS;
    const int rel_in = bi * BS + j * ES;
    const int sb = src + (PIN ? Pad::map(rel_in) : rel_in);
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = S[sb + r * IN_STEP];
    if (NS > 1) {
      const int tk = twb + k * TWS;
      float2 w[R];
      w[1] = tw_dir<DIR>(S[tk]);
      if (R >= 4) {
        w[2] = tw_dir<DIR>(S[tk + k * TWS]);
        w[3] = cmul<float>(w[1], w[2]);
      }
      if (R == 8) {
        w[4] = tw_dir<DIR>(S[tk + 3 * k * TWS]);
        w[5] = cmul<float>(w[1], w[4]);
        w[6] = cmul<float>(w[2], w[4]);
        w[7] = cmul<float>(w[3], w[4]);
      }
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul<float>(v[r], w[r]);
    }
    Dft<float, DIR, R>::run(v);
    const int rel_out = bi * BS + ((j / NS) * NS * R + k) * ES;
    // first pass: the R outputs of a butterfly stay inside one PG group
    const int db = dst + (POUT ? Pad::map(rel_out) : rel_out);
#pragma unroll
    for (int r = 0; r < R; ++r) S[db + r * NS * ES] = v[r];
  }
}

template <int DIR, bool BATCH_FAST, int N, int NBATCH, int ES, int BS, int S_, int NS>
__device__ __forceinline__ void fft_smem_from(int& src, int& dst, int twb, int tid, int nth) {
  if constexpr (S_ < Pow2Passes<N>::value) {
    constexpr int R = Pow2Radix<N, S_>::value;
    constexpr bool PIN = S_ == 1 && Pow2Radix<N, 0>::value == 8;
    constexpr bool POUT = S_ == 0 && Pow2Passes<N>::value > 1 && R == 8;
    fft_pass_smem<DIR, R, BATCH_FAST, N, NS, NBATCH, ES, BS, PIN, POUT>(src, dst, twb, tid, nth);
    __syncthreads();
    const int t = src; src = dst; dst = t;
    fft_smem_from<DIR, BATCH_FAST, N, NBATCH, ES, BS, S_ + 1, NS * R>(src, dst, twb, tid, nth);
  }
}

// Full transform on buffers at element offsets a and b (b holds
// fft_pad_elems(its size) elements: the first pass writes it padded);
// returns the offset of the buffer holding the result, unpadded.  Every
// thread of the block calls it.
template <int DIR, bool BATCH_FAST, int N, int NBATCH, int ES, int BS>
__device__ __forceinline__ int fft_block_smem(int a, int b, int twb, int tid, int nth) {
  int src = a, dst = b;
  fft_smem_from<DIR, BATCH_FAST, N, NBATCH, ES, BS, 0, 1>(src, dst, twb, tid, nth);
  return src;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  // sh: at least 32 entries
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  T r = (threadIdx.x < nw) ? sh[threadIdx.x] : (T)0;
  if (w == 0) {
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

// Two block sums at once, each added in the same order as block_sum (the
// same results), through one pair of barriers.  sh: at least 64 entries.
template <typename T>
__device__ __forceinline__ void block_sum2(T& a, T& b, T* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    sh[w] = a;
    sh[32 + w] = b;
  }
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  a = (threadIdx.x < nw) ? sh[threadIdx.x] : (T)0;
  b = (threadIdx.x < nw) ? sh[32 + threadIdx.x] : (T)0;
  if (w == 0) {
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
  }
  // valid in thread 0
}

}  // namespace pp
