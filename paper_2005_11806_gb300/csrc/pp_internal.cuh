// Internal declarations shared by the CUDA translation units of the
// pressure-projection library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <vector>

#include "pressure_projection.h"

namespace pp {

constexpr int kMaxStages = 16;

// Mixed-radix factorisation of one FFT length (radices 8, 4, 2, 3, 5).
struct FftDesc {
  int n;
  int nst;
  int pow2;      // 1 when n is a power of two (all radices 8, 4, 2)
  int radix[kMaxStages];
};

template <typename T> struct Cx;
template <> struct Cx<double> { using t = double2; };
template <> struct Cx<float> { using t = float2; };
template <typename T> using C2 = typename Cx<T>::t;

// Device-resident iteration state of one projection (Algorithm 1's loop
// control): written by the check kernel, read by every kernel of a pass.
struct DevStatus {
  double e2;        // sum of e^2 of the latest residual (e = (D u^s - S_c)/dt)
  double e1;        // sum of |e|
  double e2_0;      // sum of (b/dt)^2, b = D u* - S_c
  double rel;       // sqrt(e2 / e2_0)
  double mean_S;    // volume-weighted mean of S
  double pmean;     // volume-weighted mean of p (gauge removal)
  int iters;        // constant-coefficient solves started
  int done;         // 1 once the loop has stopped
  int code;         // pp_status of the loop
  int need_exact;   // 1: the next residual is recomputed from p in FP64
  int since_exact;  // passes since the last exact residual
  int last_exact;   // 1: the latest residual was an exact one
  int pad;
};

// Geometry and tables on the device (pointers into plan-owned memory).
struct Geo {
  int nx, ny, nz, nxh;
  double dx, dy, inv_dx2, inv_dy2;
  const double* inv_dzf;  // [nz]   1 / cell width
  const double* inv_dzc;  // [nz+1] 1 / centre distance across z-face k (0 at walls)
  const double* dzf;      // [nz]
  const double* za;       // [nz]   sub-diagonal of L_z
  const double* zc;       // [nz]   super-diagonal of L_z
  const float* inv_dzf_f; // [nz]   1 / cell width (FP32 copy)
  // FP32 layer factors of the face coefficients, [3][nz + 1]: dzf_k / dx^2,
  // dzf_k / dy^2 (k < nz) and 1 / dzc_k (z faces k = 0 .. nz, 0 on the walls).
  // The mixed residual update forms its FP32 coefficients from these and the
  // FP32 density instead of reading stored coefficient fields.
  const float* cw_f;
  double lz;
  int ywall;              // 1: walls at y = 0 and y = ly (v row 0 is the wall face); 0: periodic y
  // Stretched y between walls (null for a uniform y): [3][ny] row factors
  // relative to the mean spacing dy = ly / ny,
  //   ym[j] = s_j = dyf_j / dy, ym[ny + j] = t_j = dy / dyc_j (y-face j below
  //   row j; t_0 = 0: the walls), ym[2 ny + j] = 1 / s_j,
  // and their FP32 copy ym_f.  Every cell row is scaled by dzf_k s_j instead
  // of dzf_k, so with dyf_j = s_j dy and dyc_j = dy / t_j the coefficients
  // become cx = dzf_k s_j beta / dx^2, cy = dzf_k t_j beta / dy^2 and
  // cz = s_j beta / dzc (symmetric, as on a uniform y).
  const double* ym;
  const float* ym_f;
};

// Coefficients of D(beta G .) with each cell's row multiplied by its width
// dzf_k (so the z coefficients need no per-cell scaling):
//   cx = dzf_k beta_x / dx^2, cy = dzf_k beta_y / dy^2 (faces of layer k),
//   cz = beta_z / dzc (z faces, 0 on the walls),
//   diag = sum of the six coefficients of the cell, rhof = rho_c in FP32
//   (the mixed residual update recomputes its FP32 coefficients from rhof:
//   face_beta_f); diagf: FP32 diagonal when not null (unused by the solver's
//   own kernels).
//   rho_tilde: device scalar that replaces rho_c as the scaling of the
//   residual (Methods I and II of Sec. 3.3.1); null selects Method III.
struct Faces {
  double* cx;    // [nz][ny][nx]
  double* cy;    // [nz][ny][nx]
  double* cz;    // [nz+1][ny][nx]
  double* diag;  // [nz][ny][nx]
  float* rhof;   // [nz][ny][nx]
  float* diagf;
  const double* rho_tilde;
};

// Exact FP32 -> FP64 widening done on the integer pipe (the FP64 pipe of this
// part is the scarce resource).  Subnormal inputs become signed zeros.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned m = b & 0x7FFFFFu;
  unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
  unsigned lo = m << 29;
  if (e == 0u) { hi = sign; lo = 0u; }
  if (e == 0xFFu) hi = sign | 0x7FF00000u | (m >> 3);
  return __hiloint2double((int)hi, (int)lo);
}

// 1 / rho_f of a face from its two cells' FP32 densities (arithmetic face
// density, as the FP64 coefficients): 2 / (a + b), fast FP32 division.
__device__ __forceinline__ float face_beta_f(float a, float b) { return __fdividef(2.f, a + b); }

// Host: whether the n + 1 face coordinates f[0..n] are finite and strictly
// increasing (the grid descriptor's zfaces / yfaces).
inline bool faces_ok(const double* f, int n) {
  for (int k = 0; k <= n; ++k)
    if (!std::isfinite(f[k])) return false;
  for (int k = 0; k < n; ++k)
    if (!(f[k + 1] > f[k])) return false;
  return true;
}

// Host: the [3][nz + 1] FP32 layer factors of Geo::cw_f.
inline std::vector<float> layer_factors_f32(int nz, const std::vector<double>& dzf,
                                            const std::vector<double>& inv_dzc, double inv_dx2, double inv_dy2) {
  std::vector<float> cw(3 * (size_t)(nz + 1), 0.f);
  for (int k = 0; k < nz; ++k) {
    cw[k] = (float)(inv_dx2 * dzf[k]);
    cw[(nz + 1) + k] = (float)(inv_dy2 * dzf[k]);
  }
  for (int k = 0; k <= nz; ++k) cw[2 * (nz + 1) + k] = (float)inv_dzc[k];
  return cw;
}

// FP64 -> FP32 narrowing on the integer pipe: round half away from zero on
// the first dropped bit; underflow flushes to zero, overflow/NaN give Inf.
__device__ __forceinline__ float narrow_f64(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 896;
  unsigned bits = ((unsigned)e << 23) + (((hi & 0xFFFFFu) << 3) | (lo >> 29)) + ((lo >> 28) & 1u);
  if (e <= 0) bits = 0u;
  if (e >= 255) bits = 0x7F800000u;
  return __uint_as_float(sign | bits);
}

// ---- launchers (pp_kernels_*.cu) -------------------------------------

// Residual e = b/dt - D(beta G p) (or e = f when f_only), r = rho * e
// (or r = e), forward real x-transform of r into spec; block partial sums
// of e^2 and |e| into red[2*block + {0,1}].  Rows are (k, j) pairs.
//
// Mixed path with E != null: E = dzf (D u^s - S_c)/dt is kept in FP32.  When
// st->need_exact is set it is recomputed from p in FP64 (and stored
// narrowed); otherwise it is updated by E -= A delta with
// delta = p^s - p^{s-1} and the FP32 coefficients.
template <typename T>
cudaError_t launch_resid_fftx(const Geo& g, const Faces& fc, const FftDesc& fx, const C2<T>* twx,
                              const double* b, double inv_dt, const double* rho, const double* p,
                              int p_zero, int scale_rho, C2<T>* spec, double* red, int* nblk_out,
                              const DevStatus* st, cudaStream_t s, float* E = nullptr,
                              const float* delta = nullptr);
// z solve of a uniform walled z by the cosine basis (FP64 plans): forward
// transform with the eigenvalue divide (inverse = 0), then the inverse
// transform (inverse = 1).  dct: exp(-i pi m / (2 nz)); zd: the eigenvalues.
struct ZDivide {
  const double* lamx;  // [nxh]
  const double* lamy;  // [ny]
  const double* lamz;  // [nz] -(4/dz^2) sin^2(pi m / (2 nz))
};
template <typename T>
cudaError_t launch_zdct(const Geo& g, const FftDesc& fz, const C2<T>* twz, C2<T>* spec, int inverse,
                        const DevStatus* st, cudaStream_t s, const C2<T>* dct, const ZDivide& zd);

// dct: the cosine-transform twiddles exp(-i pi m / (2 ny)) for walls in y,
// or null for the periodic DFT.
template <typename T>
cudaError_t launch_ffty(const Geo& g, const FftDesc& fy, const C2<T>* twy, C2<T>* spec, int inverse,
                        const DevStatus* st, cudaStream_t s, const C2<T>* dct = nullptr);
// FP32 y transform of length 512 (periodic y) with the data in registers
// (pp_kernels_ffty512.cu); launch_ffty routes such plans to it.
cudaError_t launch_ffty512(const Geo& g, const float2* twy, float2* spec, int inverse, const DevStatus* st,
                           cudaStream_t s);
// FP32 Thomas tables for the well-conditioned z columns of mixed plans.  A
// column (kx, ky) has the shift lambda = lambda_x(kx) + lambda_y(ky) <= 0;
// the eigenvalues of its system lie in [lambda - 2 Dmax, lambda] with
// Dmax = max_k (za_k + zc_k), so |lambda| >= thr = 2 Dmax / 512 bounds its
// condition number by 513, and such a column runs in FP32.  The others,
// the singular (0, 0) column among them, keep the FP64 recurrences.
struct TriF32 {
  const float* mtab;   // [nz][ny][nxh] multipliers m_k (FP32 copy)
  const float* invd;   // [nz][ny][nxh] inverse pivots (FP32 copy)
  const float* zc;     // [nz] super-diagonal of L_z (FP32 copy)
  const double* lamx;  // [nxh]
  const double* lamy;  // [ny]
  double thr;
  const int* low;      // [nlow] the columns with |lambda| < thr, column 0 first
  int nlow;
};
// Columns (index ky * nxh + kx) that keep FP64: |lambda| < thr, and column 0.
std::vector<int> tri_low_columns(const std::vector<double>& lamx, const std::vector<double>& lamy,
                                 double thr);
// Blocks of 128 threads of the mixed z solve.
inline int tri_mixed_blocks(size_t ncol, int nlow) { return (nlow + 3) / 4 + (int)((ncol + 127) / 128); }

// With mtab (multipliers m_k = a_k / d_{k-1}) the real and imaginary parts
// run in separate threads; without it one thread solves a whole column.
// With f32 (mixed plans) the well-conditioned columns run in FP32.
template <typename T>
cudaError_t launch_tridiag(const Geo& g, const double* invd, C2<T>* spec, double2* ybuf,
                           const DevStatus* st, cudaStream_t s, const double* mtab = nullptr,
                           const TriF32* f32 = nullptr);
// FP64 z solve of PP_MIXED_Z64 plans: FP64 recurrences in every (kx, ky)
// column, values stored in FP32.  Thomas elimination in the form
//   forward   y_k = f_k - m_k y_{k-1},            m_k = a_k / d_{k-1}
//             s_k = (1/d_k) y_k                   (stored, FP32)
//   backward  x_k = s_k - e_k x_{k+1},            e_k = c_k / d_k,
// so each sweep costs one FP64 FMA per scalar.  The tables depend on the
// column only through lambda = lambda_x(kx) + lambda_y(ky); with periodic y
// lambda_y(ky) = lambda_y(ny - ky), so ky and ny - ky share one table column
// (ysym: nyt = ny/2 + 1 table rows of nxh columns per layer, ky' = min(ky,
// ny - ky)); with walls in y nyt = ny.  Table column 0 is the singular
// (0, 0) system: its last inverse pivot is 0 (pinned unknown).
struct TriZ64 {
  const double* m;  // [nz][nyt][nxh]
  const double* e;  // [nz][nyt][nxh]
  const float* d;   // [nz][nyt][nxh] 1 / d_k
  int nyt;
  int ysym;
};
cudaError_t launch_setup_z64(const Geo& g, const double* lamx, const double* lamy, int nyt, int ysym,
                             double* m, double* e, float* d, cudaStream_t s);
cudaError_t launch_tridiag_z64(const Geo& g, const TriZ64& t, float2* spec, const DevStatus* st,
                               cudaStream_t s);
// dst[i] = (float) src[i], i < n.
cudaError_t launch_narrow(const double* src, float* dst, size_t n, cudaStream_t s);
// Inverse x-transform; p = scale * z (p_zero) or p += scale * z; when delta
// is not null it also receives scale * z in the transform's precision T.
// With sdelta (mixed plans) p is updated only before an exact residual and
// the increments in between are summed into sdelta (FP32); see
// stage_fftx_inv.  launch_fold_pending adds a sum still pending when the
// loop has stopped.
template <typename T>
cudaError_t launch_fftx_inv(const Geo& g, const FftDesc& fx, const C2<T>* twx, const C2<T>* spec,
                            double scale, double* p, int p_zero, const DevStatus* st, cudaStream_t s,
                            T* delta = nullptr, float* sdelta = nullptr);
// The same for FP32 spectra of length nx = 512, with the transform in
// registers (pp_kernels_fftx512.cu); launch_fftx_inv routes such plans to it.
cudaError_t launch_fftx512_inv(const Geo& g, const float2* twx, const float2* spec, double scale, double* p,
                               int p_zero, const DevStatus* st, cudaStream_t s, float* delta, float* sdelta);
cudaError_t launch_fold_pending(const Geo& g, double* p, const float* sdelta, const DevStatus* st,
                                cudaStream_t s);

// Inverse Thomas pivots; when mtab is not null also the multipliers
// m_k = a_k / d_{k-1} (m_0 = 0).
cudaError_t launch_setup_pivots(const Geo& g, const double* lamx, const double* lamy, double* invd,
                                cudaStream_t s, double* mtab = nullptr);

cudaError_t launch_mixture(const double* phi, double rho_g, double rho_l, double* rho, size_t n,
                           cudaStream_t s);
cudaError_t launch_prep_faces(const Geo& g, const double* rho, Faces fc, cudaStream_t s);
// Constant density of Methods I and II (Sec. 3.3.1) into *out: the minimum
// of rho (method 1) or the harmonic mean of its minimum and maximum, i.e. of
// the two phase densities (method 2).  red holds at least reduce_blocks()
// pairs of partial sums.
cudaError_t launch_rho_tilde(const Geo& g, const double* rho, int method, double* red, double* out,
                             cudaStream_t s);
// Modified correction of Method I (Eq. poisson_me2) from the last iterate p
// and its last increment delta = p - p^q:
//   u = u* - dt [G p / rho0 + (beta - 1/rho0) G p^q]
//     = u* - dt beta G p + dt (beta - 1/rho0) G delta.
template <typename T>
cudaError_t launch_correct_method1(const Geo& g, const Faces& fc, const double* us, const double* vs,
                                   const double* ws, const double* p, const T* delta, double dt,
                                   double* u, double* v, double* w, cudaStream_t s);
// Sum of dzf * f over cells (block partials) -> st->mean_S = sum / (lz nx ny).
cudaError_t launch_weighted_mean(const Geo& g, const double* f, double* red, double* out_mean,
                                 cudaStream_t s);
// b = D u* - (S - mean_S); partial sums of b^2 -> e2_0.
cudaError_t launch_rhs_b(const Geo& g, const double* us, const double* vs, const double* ws,
                         const double* S, double* b, double* red, DevStatus* st, double inv_dt,
                         cudaStream_t s);
// Loop control of Algorithm 1 (one block).  kexact: recompute the residual
// exactly every kexact passes (<= 1: every pass); convergence is only
// accepted on an exact residual.
cudaError_t launch_check(DevStatus* st, const double* red, int nblk, double rtol, int maxit,
                         int kexact, cudaStream_t s);
cudaError_t launch_init_status(DevStatus* st, cudaStream_t s);
// u = us - dt beta G p on all faces (w walls = 0).
cudaError_t launch_correct(const Geo& g, const Faces& fc, const double* us, const double* vs,
                           const double* ws, const double* p, double dt, double* u, double* v,
                           double* w, cudaStream_t s);
// p -= <p>_V
cudaError_t launch_remove_mean(const Geo& g, double* p, double* red, DevStatus* st, cudaStream_t s);
cudaError_t launch_copy_resid_sums(DevStatus* st, const double* red, int nblk, cudaStream_t s);

// Adjoint helpers.
// y = -dt * beta * W_f^{-1} g on the faces (wall z-faces zero).
cudaError_t launch_adj_rhs(const Geo& g, const double* rho, const double* gu, const double* gv,
                           const double* gw, double dt, double* yu, double* yv, double* yw,
                           cudaStream_t s);
// gus = g + W_f G mu ; grho from -dt (G p) * gus and d beta / d rho.
cudaError_t launch_adj_finish(const Geo& g, const double* rho, const double* p, const double* mu,
                              double dt, const double* gu, const double* gv, const double* gw,
                              double* gus, double* gvs, double* gws, double* tx, double* ty,
                              double* tz, cudaStream_t s);
// Eq. 30: out[0..3] = {sum Phi div(k grad T) dV, sum Phi div(u) dV, V_g, RP}
// (RP = NaN when V_g = 0); red holds at least reduce_blocks() values.
cudaError_t launch_thermo_rate(const Geo& g, const double* phi, const double* kc, const double* T,
                               const double* u, const double* v, const double* w, double p0, double gamma,
                               double* red, double* out, cudaStream_t s);
// Eq. 34: S = (1/p0) [ (gamma - 1)/gamma div(k grad T) - dp0dt / gamma ] Phi.
cudaError_t launch_divergence_source(const Geo& g, const double* phi, const double* kc, const double* T,
                                     double p0, double gamma, double dp0dt, double* S, cudaStream_t s);
// Momentum predictor (Eqs. 29, 32): out = u + dt (a RU - b prev) on the u, v
// and w faces (w wall planes zero); ru (entries may be null) receives RU;
// f and prev entries may be null.  D: a cell-field scratch (the divergence).
cudaError_t launch_predictor(const Geo& g, const double* u, const double* v, const double* w, const double* rho,
                             const double* mu, const double* const f[3], const double* const prev[3],
                             const double grav[3], double dt, double a, double b, double* D, double* const out[3],
                             double* const ru[3], cudaStream_t s);
cudaError_t launch_adj_grho(const Geo& g, const double* tx, const double* ty, const double* tz,
                            double* grho, cudaStream_t s);

int reduce_blocks();  // number of partial sums the reduction kernels write

// y step of FP64 plans on a stretched y between walls (Sec. 3.3.1
// eigenexpansion with a numerical eigenbasis): every z plane of the
// spectrum, X[j][kx], becomes M X in place with M = V^T W (forward) or V
// (back); mt holds M transposed, mt[j * ny + m] = M[m][j]
// (pp_kernels_ydense.cu).  ny <= 1024.  Mixed plans take the tensor-core
// dense transform (launch_dense_tc) instead.
cudaError_t launch_ydense(const Geo& g, const double* mt, double2* spec, const DevStatus* st, cudaStream_t s);

// Host: eigenpairs of a symmetric tridiagonal S (diagonal d, off-diagonal e)
// by Sturm-sequence bisection and inverse iteration with Gram-Schmidt,
// ascending; Q[k * n + j] = component k of eigenvector j.  False when a pair
// fails its residual check.
bool sym_tridiag_eigen(const std::vector<double>& d, const std::vector<double>& e, std::vector<double>& lam,
                       std::vector<double>& Q);
// Host: the y eigenbasis of a stretched y between walls: L_y = W^{-1} T with
// W = diag(dyf), T_{j,j+1} = 1/dyc_{j+1}; eigenvalues lam[m] in descending
// order (lam[0] = 0, the constant mode, exact) and the transposed matrices
// of the forward (V^T W) and inverse (V) products.
bool build_yeigen_host(int ny, const double* dyf, const double* inv_dyc, std::vector<double>& lam,
                       std::vector<double>& mt_fwd, std::vector<double>& mt_inv);

// Dense transform of strided real lines on the tensor cores, out of place
// (pp_dense_tc.cu): column g of the real view (slab s = g / ncs, offset
// c = g % ncs) has entries x_k = x[s * slab + k * ld + c], k < n, and gets
// y_m = f(m, g) sum_k M[m][k] x_k at y[s * slab + m * ld + c]; f = 1, or
// with mu set f = 1 / (mu_m + lamx[kx] + lamy[ky]) for the complex entry
// g / 2 = ky * nxh + kx, 0 for m = zero_mode at g / 2 = 0.  BF16x3 products
// with FP32 accumulation; M comes as dense_tc_tiles.
struct DenseTcArgs {
  const float* x;
  float* y;
  const unsigned char* mat;
  int n, nt, nkc;             // line length; dense_tc_out_tiles(n), dense_tc_k_chunks(n)
  long long ncs, nslab, slab, ld;
  const float* mu;            // null: f = 1
  const double* lamx;
  const double* lamy;
  int nxh;
  int zero_mode;
};
int dense_tc_out_tiles(int n);
int dense_tc_k_chunks(int n);
void dense_tc_tiles(const std::vector<double>& M, int n, std::vector<uint16_t>& out);
cudaError_t launch_dense_tc(const DenseTcArgs& a, DevStatus* st, cudaStream_t s);

// Tables of the tensor-core z expansion (PP_MIXED_TC): two launches of the
// dense transform, V^T W with the eigenvalue divide into the second
// spectrum buffer, then V back.
struct ZEigen {
  int nt, nkc;              // dense_tc_out_tiles(nz), dense_tc_k_chunks(nz)
  const float* mu;          // [nt * 256] eigenvalues of L_z (0 on padded modes)
  int zero_mode;            // index of the zero eigenvalue
  const unsigned char* a1;  // dense_tc_tiles of V^T W
  const unsigned char* a2;  // dense_tc_tiles of V
};
// Host: eigen decomposition of L_z (pp_eigen_host.cu): eigenvalues (FP32,
// zero-padded to `pad`), the zero mode, and the row-major matrices V^T W
// and V.
bool build_zeigen_host(int nz, const double* dzf, const double* inv_dzc, int pad, std::vector<float>& mu_out,
                       int* zero_mode, std::vector<double>& m_fwd, std::vector<double>& m_inv);

}  // namespace pp
