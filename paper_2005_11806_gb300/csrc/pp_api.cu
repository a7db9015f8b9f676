// C ABI of the pressure-projection library: plans, the Method III driver
// (Algorithm 1, Sec. 3.3.1), the constant-coefficient solve, the adjoint and
// host-pointer staging.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "pp_internal.cuh"

using namespace pp;

namespace {
enum KId { K_RESID, K_CHECK, K_FFTY_F, K_TRI, K_FFTY_I, K_FFTX_I, K_INIT, K_PREP, K_MEANS, K_RHSB,
           K_RMEAN, K_CORR, K_MIX, K_ADJ_RHS, K_ADJ_FIN, K_ADJ_GRHO, K_RHOT, K_FOLD, K_THERMO, K_SOURCE,
           K_PRED, K_ZDCT_F, K_ZDCT_I, K_COUNT };
const char* const kNames[K_COUNT] = {
    "resid_fftx", "check", "ffty_fwd", "tridiag_z", "ffty_inv", "fftx_inv_update", "init_status",
    "prep_faces", "mean_S", "rhs_b", "remove_mean", "correct", "mixture_density", "adj_rhs",
    "adj_finish", "adj_grho", "rho_tilde", "fold_pending", "p0_rate", "divergence_source", "predictor",
    "zdct_fwd", "zdct_inv"};
const int kLaunches[K_COUNT] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 3, 1, 1, 1, 1, 1, 2, 1, 2, 1, 2, 1, 1};
struct Rec { int kid; cudaEvent_t a, b; };
struct Prof {
  bool on = false;
  std::vector<Rec> rec;
  std::vector<cudaEvent_t> pool;
  double ms[K_COUNT] = {0};
  long long n[K_COUNT] = {0};
  long long launches = 0;
};
}  // namespace

struct pp_plan_s {
  int nx, ny, nz, nxh;
  double lx, ly, lz, dx, dy;
  pp_precision prec;
  cudaStream_t stream;
  int device;
  FftDesc fx, fy;
  Geo geo;
  Faces faces;
  // device tables
  double *d_inv_dzf = nullptr, *d_inv_dzc = nullptr, *d_dzf = nullptr, *d_za = nullptr, *d_zc = nullptr;
  double *d_lamx = nullptr, *d_lamy = nullptr, *d_invd = nullptr, *d_mtab = nullptr;
  float* d_inv_dzf_f = nullptr;
  float* d_cw_f = nullptr;  // [3][nz + 1] FP32 layer factors of the face coefficients
  void *d_twx = nullptr, *d_twy = nullptr;
  void* d_dcty = nullptr;  // walls in y: exp(-i pi m / (2 ny)), m < ny (C2 of the plan's FFT type)
  // stretched y between walls: row factors (Geo::ym, ym_f) and the transposed
  // forward (V^T W) and inverse (V) eigenvector matrices in the plan's
  // transform precision
  bool ystretch = false;
  double* d_ym = nullptr;
  float* d_ym_f = nullptr;
  void *d_ymt_f = nullptr, *d_ymt_i = nullptr;  // FP64 plans: the CUDA-core dense step
  // mixed plans: the tensor-core dense step (BF16 hi/lo tiles of V^T W and
  // V) runs out of place into d_spec2, where the z solve then works
  unsigned char *d_ytc_f = nullptr, *d_ytc_i = nullptr;
  void* d_spec2 = nullptr;
  // z solve by the cosine basis (uniform z, FP64 plans; pressure_plan_set_zsolve)
  int zsolve = PP_ZSOLVE_TRIDIAG;
  bool z_uniform = false;
  double dz = 0.0;
  FftDesc fz{};
  double2* d_twz = nullptr;
  double2* d_dctz = nullptr;
  double* d_lamz = nullptr;
  // workspaces
  void* d_spec = nullptr;
  double2* d_ybuf = nullptr;
  double* d_b = nullptr;
  float* d_E = nullptr;       // mixed: residual carried between passes (FP32)
  float* d_delta = nullptr;   // mixed: last pressure correction (FP32)
  float* d_sdelta = nullptr;  // mixed: sum of the corrections not yet added to p
  // iteration of Sec. 3.3.1 (pp_method); Methods I and II scale the residual
  // by the device scalar d_rho_tilde, Method I keeps the last increment of p
  // (d_delta on mixed plans, d_delta64 on FP64 plans) for Eq. poisson_me2
  int method = PP_METHOD_III;
  // mixed plans: FP32 Thomas tables of the well-conditioned z columns
  float *d_mtab_f = nullptr, *d_invd_f = nullptr, *d_zc_f = nullptr;
  int* d_low = nullptr;
  TriF32 tri32{};
  bool use_tri32 = false;
  // PP_MIXED_Z64: tables of the FP64-recurrence z solve (TriZ64)
  double *d_z64m = nullptr, *d_z64e = nullptr;
  float* d_z64d = nullptr;
  TriZ64 z64{};
  bool use_z64 = false;
  double* d_rho_tilde = nullptr;
  double* d_delta64 = nullptr;
  double* d_thermo = nullptr;  // [4] sums and rate of Eq. 30
  double* d_red = nullptr;
  size_t red_len = 0;
  DevStatus* d_st = nullptr;
  DevStatus* h_st = nullptr;  // pinned, two slots
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // lazily allocated: host staging (10 face-sized buffers), adjoint scratch
  double* d_stage[10] = {nullptr};
  double* d_adj[4] = {nullptr};
  double last_mean_S = 0.0;
  Prof prof;
  bool z_tc = false;           // tensor-core z expansion (PP_MIXED_TC; uses d_spec2)
  ZEigen ze{};
  float* d_mu = nullptr;
  unsigned char* d_za1 = nullptr;
  unsigned char* d_za2 = nullptr;
};

namespace {

bool factor_len(int n, FftDesc* d) {
  if (n < 1) return false;
  d->n = n;
  d->nst = 0;
  int m = n;
  const int rads[5] = {8, 4, 2, 3, 5};
  for (int r : rads) {
    while (m % r == 0) {
      if (d->nst >= kMaxStages) return false;
      d->radix[d->nst++] = r;
      m /= r;
    }
  }
  if (n == 1) { d->radix[0] = 2; d->nst = 0; }
  d->pow2 = (n & (n - 1)) == 0;
  return m == 1;
}

template <typename T>
std::vector<C2<T>> twiddles(int n) {
  std::vector<C2<T>> t(n);
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < n; ++m) {
    const double a = two_pi * (double)m / (double)n;
    t[m].x = (T)std::cos(a);
    t[m].y = (T)std::sin(a);
  }
  return t;
}

// Twiddles of the cosine transform along a walled direction of n cells:
// exp(-i pi m / (2 n)), m = 0 .. n - 1 (FP64 on the host).
template <typename T>
std::vector<C2<T>> dct_twiddles(int n) {
  std::vector<C2<T>> t(n);
  const double pi = 3.14159265358979323846264338327950288;
  for (int m = 0; m < n; ++m) {
    const double a = pi * (double)m / (2.0 * (double)n);
    t[m].x = (T)std::cos(a);
    t[m].y = (T)(-std::sin(a));
  }
  return t;
}

#define PP_CK(call)                                  \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return PP_ERR_CUDA;       \
  } while (0)

cudaEvent_t get_event(pp_plan_s* P) {
  if (!P->prof.pool.empty()) {
    cudaEvent_t e = P->prof.pool.back();
    P->prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launch through f(); count it and, when profiling, bracket it with events.
template <class F>
cudaError_t timed(pp_plan_s* P, int kid, F&& f) {
  P->prof.launches += kLaunches[kid];
  if (!P->prof.on) return f();
  cudaEvent_t a = get_event(P), b = get_event(P);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaEventRecord(a, P->stream);
  if (e != cudaSuccess) return e;
  e = f();
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(b, P->stream);
  P->prof.rec.push_back({kid, a, b});
  return e;
}

#define PP_K(P, KID, expr) PP_CK(timed((P), (KID), [&]() { return (expr); }))

// Mixed plans recompute the FP64 residual from p every kExactEvery passes and
// update it by the FP32 stencil of the last correction in between.
constexpr int kExactEvery = 40;

template <typename X>
pp_status dalloc(X** p, size_t bytes) {
  if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
    *p = nullptr;
    (void)cudaGetLastError();
    return PP_ERR_OOM;
  }
  return PP_OK;
}

size_t ncell(const pp_plan_s* P) { return (size_t)P->nx * P->ny * P->nz; }
size_t nwface(const pp_plan_s* P) { return (size_t)P->nx * P->ny * (P->nz + 1); }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Stage an input: device pointers pass through, host pointers are copied
// into staging slot `slot` (allocated on first use, sized for a w field).
pp_status stage_in(pp_plan_s* P, const double* src, size_t n, int slot, const double** out) {
  if (src == nullptr) { *out = nullptr; return PP_OK; }
  if (is_device_ptr(src)) { *out = src; return PP_OK; }
  if (!P->d_stage[slot]) {
    pp_status s = dalloc(&P->d_stage[slot], nwface(P) * sizeof(double));
    if (s != PP_OK) return s;
  }
  PP_CK(cudaMemcpyAsync(P->d_stage[slot], src, n * sizeof(double), cudaMemcpyHostToDevice, P->stream));
  *out = P->d_stage[slot];
  return PP_OK;
}

pp_status stage_out(pp_plan_s* P, double* dst, int slot, double** out, bool* staged) {
  *staged = false;
  if (is_device_ptr(dst)) { *out = dst; return PP_OK; }
  if (!P->d_stage[slot]) {
    pp_status s = dalloc(&P->d_stage[slot], nwface(P) * sizeof(double));
    if (s != PP_OK) return s;
  }
  *out = P->d_stage[slot];
  *staged = true;
  return PP_OK;
}

pp_status copy_back(pp_plan_s* P, double* host, const double* dev, size_t n) {
  PP_CK(cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  return PP_OK;
}

pp_status read_info(pp_plan_s* P, pp_info* info) {
  PP_CK(cudaMemcpyAsync(P->h_st, P->d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost, P->stream));
  PP_CK(cudaStreamSynchronize(P->stream));
  const DevStatus& s = P->h_st[0];
  if (s.pad != 0) return PP_ERR_CUDA;  // a device-side bounded wait ran out
  if (info) {
    const double dt_scale = 1.0;  // e is stored in units of 1/dt; res0/res_l1 are rescaled by the caller
    info->iters = s.iters;
    info->res0 = std::sqrt(s.e2_0) * dt_scale;
    info->res_final = s.rel;
    info->res_l1_sum = s.e1;
    info->mean_S_removed = s.mean_S;
    info->status = s.code;
  }
  return (pp_status)s.code;
}

// One pass of Algorithm 1 after the residual: forward y, z solve, inverse y,
// inverse x fused with p += delta.
template <typename T>
pp_status solve_pass(pp_plan_s* P, double* p, int p_zero, T* delta = nullptr, float* sdelta = nullptr) {
  const Geo& g = P->geo;
  C2<T>* spec = (C2<T>*)P->d_spec;
  const C2<T>* twx = (const C2<T>*)P->d_twx;
  const C2<T>* twy = (const C2<T>*)P->d_twy;
  // mixed plans with a stretched y: the tensor-core y step runs out of
  // place, so the z solve works on the second spectrum buffer
  const bool ytc = P->ystretch && std::is_same<T, float>::value;
  C2<T>* zs = ytc ? (C2<T>*)P->d_spec2 : spec;
  // the split solve (mtab present) keeps its intermediate in the spectrum
  double2* ybuf = (double2*)zs;
  // the dense y step of a stretched y is W-orthonormal: no 1/ny on the way back
  const double scale = 1.0 / ((double)P->nx * (P->ystretch ? 1.0 : (double)P->ny));
  const C2<T>* dct = (const C2<T>*)P->d_dcty;  // null: periodic y
  auto ytc_args = [&](const void* x, void* y, const unsigned char* mat) {
    DenseTcArgs a{};
    a.x = (const float*)x;
    a.y = (float*)y;
    a.mat = mat;
    a.n = P->ny;
    a.nt = dense_tc_out_tiles(P->ny);
    a.nkc = dense_tc_k_chunks(P->ny);
    a.ncs = 2LL * P->nxh;
    a.nslab = P->nz;
    a.slab = 2LL * P->nxh * P->ny;
    a.ld = 2LL * P->nxh;
    return a;
  };
  if (ytc) PP_K(P, K_FFTY_F, launch_dense_tc(ytc_args(spec, zs, P->d_ytc_f), P->d_st, P->stream));
  else if (P->ystretch) {
    if constexpr (std::is_same<T, double>::value)
      PP_K(P, K_FFTY_F, launch_ydense(g, (const double*)P->d_ymt_f, spec, P->d_st, P->stream));
  } else PP_K(P, K_FFTY_F, launch_ffty<T>(g, P->fy, twy, spec, 0, P->d_st, P->stream, dct));
  if (P->z_tc) {
    // z expansion on the tensor cores: zs -> the other spectrum buffer with
    // the eigenvalue divide, then back
    float* other = (float*)(zs == (C2<T>*)P->d_spec ? P->d_spec2 : P->d_spec);
    DenseTcArgs a{};
    a.n = P->nz;
    a.nt = P->ze.nt;
    a.nkc = P->ze.nkc;
    a.ncs = 2LL * P->ny * P->nxh;
    a.nslab = 1;
    a.slab = 0;
    a.ld = a.ncs;
    a.x = (const float*)zs;
    a.y = other;
    a.mat = P->ze.a1;
    a.mu = P->ze.mu;
    a.lamx = P->d_lamx;
    a.lamy = P->d_lamy;
    a.nxh = P->nxh;
    a.zero_mode = P->ze.zero_mode;
    PP_K(P, K_TRI, launch_dense_tc(a, P->d_st, P->stream));
    a.x = other;
    a.y = (float*)zs;
    a.mat = P->ze.a2;
    a.mu = nullptr;
    PP_K(P, K_TRI, launch_dense_tc(a, P->d_st, P->stream));
  } else if (P->zsolve == PP_ZSOLVE_COSINE) {
    if constexpr (std::is_same<T, double>::value) {
      const ZDivide zd{P->d_lamx, P->d_lamy, P->d_lamz};
      PP_K(P, K_ZDCT_F, launch_zdct<double>(g, P->fz, P->d_twz, zs, 0, P->d_st, P->stream, P->d_dctz, zd));
      PP_K(P, K_ZDCT_I, launch_zdct<double>(g, P->fz, P->d_twz, zs, 1, P->d_st, P->stream, P->d_dctz, zd));
    } else {
      return PP_ERR_UNSUPPORTED;
    }
  } else if (std::is_same<T, float>::value && P->use_z64) {
    PP_K(P, K_TRI, launch_tridiag_z64(g, P->z64, reinterpret_cast<float2*>(zs), P->d_st, P->stream));
  } else {
    PP_K(P, K_TRI, launch_tridiag<T>(g, P->d_invd, zs, ybuf, P->d_st, P->stream, P->d_mtab,
                                     P->use_tri32 ? &P->tri32 : nullptr));
  }
  if (ytc) PP_K(P, K_FFTY_I, launch_dense_tc(ytc_args(zs, spec, P->d_ytc_i), P->d_st, P->stream));
  else if (P->ystretch) {
    if constexpr (std::is_same<T, double>::value)
      PP_K(P, K_FFTY_I, launch_ydense(g, (const double*)P->d_ymt_i, spec, P->d_st, P->stream));
  } else PP_K(P, K_FFTY_I, launch_ffty<T>(g, P->fy, twy, spec, 1, P->d_st, P->stream, dct));
  PP_K(P, K_FFTX_I, launch_fftx_inv<T>(g, P->fx, twx, spec, scale, p, p_zero, P->d_st, P->stream, delta,
                                       sdelta));
  return PP_OK;
}

// Buffer that receives each pass's increment of p: the FP32 one of the
// mixed residual update, or the FP64 one Method I keeps on FP64 plans.
template <typename T> T* increment_buffer(pp_plan_s* P, bool upd);
template <> float* increment_buffer<float>(pp_plan_s* P, bool upd) {
  return (upd || P->method == PP_METHOD_I) ? P->d_delta : nullptr;
}
template <> double* increment_buffer<double>(pp_plan_s* P, bool) {
  return P->method == PP_METHOD_I ? P->d_delta64 : nullptr;
}

// Method III loop on device fields: b = D u* - S_c has been formed; faces
// hold beta of rho.  p is the iterate (zeroed by the caller unless warm).
// With P->method = I or II the same loop runs with the constant scaling.
template <typename T>
pp_status method3_loop(pp_plan_s* P, const double* rho, double* p, int warm, double dt, double rtol,
                       int maxit) {
  const Geo& g = P->geo;
  C2<T>* spec = (C2<T>*)P->d_spec;
  const C2<T>* twx = (const C2<T>*)P->d_twx;
  const double inv_dt = 1.0 / dt;
  const int chunk = 4;
  const bool upd = std::is_same<T, float>::value && P->d_E != nullptr;
  const int kexact = upd ? kExactEvery : 1;
  T* dl = increment_buffer<T>(P, upd);
  int polled = 0;
  bool pending[2] = {false, false};
  for (int it = 0; it <= maxit; ++it) {
    int nblk = 0;
    PP_K(P, K_RESID, launch_resid_fftx<T>(g, P->faces, P->fx, twx, P->d_b, inv_dt, rho, p,
                                          (it == 0 && !warm) ? 1 : 0, 1, spec, P->d_red, &nblk,
                                          P->d_st, P->stream, upd ? P->d_E : nullptr,
                                          upd ? P->d_delta : nullptr));
    PP_K(P, K_CHECK, launch_check(P->d_st, P->d_red, nblk, rtol, maxit, kexact, P->stream));
    pp_status s = solve_pass<T>(P, p, 0, dl, upd ? P->d_sdelta : nullptr);
    if (s != PP_OK) return s;
    if ((it + 1) % chunk == 0) {
      // Poll the device status without draining the queue: read the slot
      // recorded one chunk ago.
      const int slot = polled & 1;
      PP_CK(cudaMemcpyAsync(&P->h_st[slot], P->d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost, P->stream));
      PP_CK(cudaEventRecord(P->ev[slot], P->stream));
      pending[slot] = true;
      const int prev = slot ^ 1;
      if (pending[prev]) {
        PP_CK(cudaEventSynchronize(P->ev[prev]));
        pending[prev] = false;
        if (P->h_st[prev].done) break;
      }
      ++polled;
    }
  }
  return PP_OK;
}

template <typename T>
pp_status projection(pp_plan_s* P, const double* us, const double* vs, const double* ws,
                     const double* rho, const double* S, double dt, double* p, int warm, double* u,
                     double* v, double* w, double rtol, int maxit) {
  const Geo& g = P->geo;
  PP_K(P, K_INIT, launch_init_status(P->d_st, P->stream));
  PP_K(P, K_PREP, launch_prep_faces(g, rho, P->faces, P->stream));
  if (P->method != PP_METHOD_III) {
    PP_K(P, K_RHOT, launch_rho_tilde(g, rho, P->method, P->d_red, P->d_rho_tilde, P->stream));
    // Method I's correction reads the last increment: zero it in case the
    // loop stops before its first pass
    T* dl = increment_buffer<T>(P, false);
    if (P->method == PP_METHOD_I) PP_CK(cudaMemsetAsync(dl, 0, ncell(P) * sizeof(T), P->stream));
  }
  if (S) PP_K(P, K_MEANS, launch_weighted_mean(g, S, P->d_red, &P->d_st->mean_S, P->stream));
  PP_K(P, K_RHSB, launch_rhs_b(g, us, vs, ws, S, P->d_b, P->d_red, P->d_st, 1.0 / dt, P->stream));
  if (!warm) PP_CK(cudaMemsetAsync(p, 0, ncell(P) * sizeof(double), P->stream));
  pp_status s = method3_loop<T>(P, rho, p, warm, dt, rtol, maxit);
  if (s != PP_OK) return s;
  if (std::is_same<T, float>::value && P->d_E != nullptr)
    PP_K(P, K_FOLD, launch_fold_pending(g, p, P->d_sdelta, P->d_st, P->stream));
  PP_K(P, K_RMEAN, launch_remove_mean(g, p, P->d_red, P->d_st, P->stream));
  if (u && P->method == PP_METHOD_I) {
    PP_K(P, K_CORR, launch_correct_method1<T>(g, P->faces, us, vs, ws, p, increment_buffer<T>(P, false), dt,
                                              u, v, w, P->stream));
  } else if (u) {
    PP_K(P, K_CORR, launch_correct(g, P->faces, us, vs, ws, p, dt, u, v, w, P->stream));
  }
  return PP_OK;
}

pp_status check_plan(pp_plan P) {
  if (P == nullptr) return PP_ERR_INVALID_ARG;
  return PP_OK;
}

void free_plan(pp_plan_s* P) {
  if (!P) return;
  double* dptrs[] = {P->d_inv_dzf, P->d_inv_dzc, P->d_dzf, P->d_za, P->d_zc, P->d_lamx, P->d_lamy,
                     P->d_invd, P->d_mtab, P->d_b, P->d_red, P->faces.cx, P->faces.cy, P->faces.cz,
                     P->faces.diag, P->d_rho_tilde, P->d_delta64, P->d_thermo};
  if (P->faces.rhof) cudaFree(P->faces.rhof);
  if (P->d_low) cudaFree(P->d_low);
  float* fptrs[] = {P->faces.diagf, P->d_delta, P->d_sdelta, P->d_mtab_f, P->d_invd_f, P->d_zc_f,
                    P->d_z64d, P->d_cw_f};
  if (P->d_z64m) cudaFree(P->d_z64m);
  if (P->d_z64e) cudaFree(P->d_z64e);
  for (float* f : fptrs) if (f) cudaFree(f);
  if (P->d_E) cudaFree(P->d_E);
  if (P->d_mu) cudaFree(P->d_mu);
  if (P->d_za1) cudaFree(P->d_za1);
  if (P->d_za2) cudaFree(P->d_za2);
  if (P->d_inv_dzf_f) cudaFree(P->d_inv_dzf_f);
  for (double* d : dptrs) if (d) cudaFree(d);
  if (P->d_twx) cudaFree(P->d_twx);
  if (P->d_twy) cudaFree(P->d_twy);
  if (P->d_dcty) cudaFree(P->d_dcty);
  if (P->d_ym) cudaFree(P->d_ym);
  if (P->d_ym_f) cudaFree(P->d_ym_f);
  if (P->d_ymt_f) cudaFree(P->d_ymt_f);
  if (P->d_ymt_i) cudaFree(P->d_ymt_i);
  if (P->d_ytc_f) cudaFree(P->d_ytc_f);
  if (P->d_ytc_i) cudaFree(P->d_ytc_i);
  if (P->d_spec2) cudaFree(P->d_spec2);
  if (P->d_twz) cudaFree(P->d_twz);
  if (P->d_dctz) cudaFree(P->d_dctz);
  if (P->d_lamz) cudaFree(P->d_lamz);
  if (P->d_spec) cudaFree(P->d_spec);
  if (P->d_ybuf) cudaFree(P->d_ybuf);
  if (P->d_st) cudaFree(P->d_st);
  if (P->h_st) cudaFreeHost(P->h_st);
  for (auto& e : P->ev) if (e) cudaEventDestroy(e);
  for (double* d : P->d_stage) if (d) cudaFree(d);
  for (double* d : P->d_adj) if (d) cudaFree(d);
  for (auto& r : P->prof.rec) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : P->prof.pool) cudaEventDestroy(e);
  delete P;
}

}  // namespace

extern "C" {

const char* pressure_status_string(pp_status s) {
  switch (s) {
    case PP_OK: return "ok";
    case PP_ERR_INVALID_ARG: return "invalid argument";
    case PP_ERR_UNSUPPORTED: return "unsupported grid or boundary condition";
    case PP_ERR_NOT_CONVERGED: return "not converged within maxit";
    case PP_ERR_NUMERIC: return "non-finite residual";
    case PP_ERR_CUDA: return "CUDA runtime error";
    case PP_ERR_OOM: return "device allocation failed";
    case PP_ERR_TOO_LARGE: return "grid too large for the fixed no-allocation scratch (16 MiB)";
  }
  return "unknown status";
}

pp_status pressure_plan_create(const pp_grid* grid, pp_precision prec, void* stream, pp_plan* out) {
  if (!grid || !out) return PP_ERR_INVALID_ARG;
  *out = nullptr;
  const pp_grid& G = *grid;
  if (G.nx < 2 || G.ny < 1 || G.nz < 1 || !(G.lx > 0) || !(G.ly > 0) || !(G.lz > 0))
    return PP_ERR_INVALID_ARG;
  if (prec != PP_FP64 && prec != PP_MIXED_FP32 && prec != PP_MIXED_TC && prec != PP_MIXED_Z64)
    return PP_ERR_INVALID_ARG;
  if (prec == PP_MIXED_TC && G.nz > 512) return PP_ERR_UNSUPPORTED;
  if (G.bc[0] != PP_BC_PERIODIC || (G.bc[1] != PP_BC_PERIODIC && G.bc[1] != PP_BC_WALL) ||
      G.bc[2] != PP_BC_WALL)
    return PP_ERR_UNSUPPORTED;
  const bool ywall = (G.bc[1] == PP_BC_WALL);
  const bool ystretch = G.yfaces != nullptr;
  if ((G.nx & 1) != 0) return PP_ERR_UNSUPPORTED;
  if (ystretch && (!ywall || G.ny < 2 || G.ny > 1024)) return PP_ERR_UNSUPPORTED;  // dense y step
  // uniform walls: cosine transform by an FFT of even length
  if (ywall && !ystretch && (G.ny < 2 || (G.ny & 1) != 0)) return PP_ERR_UNSUPPORTED;
  if (ystretch) {  // finite, increasing faces spanning ly
    if (!faces_ok(G.yfaces, G.ny)) return PP_ERR_INVALID_ARG;
    if (!(std::fabs((G.yfaces[G.ny] - G.yfaces[0]) - G.ly) <= 1e-12 * G.ly)) return PP_ERR_INVALID_ARG;
  }
  if (G.zfaces && !faces_ok(G.zfaces, G.nz)) return PP_ERR_INVALID_ARG;
  if (G.nx > 2048 || G.ny > 2048) return PP_ERR_UNSUPPORTED;  // one line per block in the FFTs
  if ((long)G.nx * G.ny * (G.nz + 1) > (1L << 31)) return PP_ERR_UNSUPPORTED;
  pp_plan_s* P = new (std::nothrow) pp_plan_s();
  if (!P) return PP_ERR_OOM;
  P->nx = G.nx; P->ny = G.ny; P->nz = G.nz; P->nxh = G.nx / 2 + 1;
  P->lx = G.lx; P->ly = G.ly; P->lz = G.lz;
  P->dx = G.lx / G.nx; P->dy = G.ly / G.ny;
  P->prec = prec;
  P->stream = (cudaStream_t)stream;
  P->ystretch = ystretch;
  if (!factor_len(G.nx, &P->fx) || (!factor_len(G.ny, &P->fy) && !ystretch)) { delete P; return PP_ERR_UNSUPPORTED; }
  if (cudaGetDevice(&P->device) != cudaSuccess) { delete P; return PP_ERR_CUDA; }

  // z metrics (Sec. 3 grid; stretched faces allowed)
  const int nz = G.nz;
  std::vector<double> zf(nz + 1);
  if (G.zfaces) {  // checked above
    for (int k = 0; k <= nz; ++k) zf[k] = G.zfaces[k];
  } else {
    for (int k = 0; k <= nz; ++k) zf[k] = G.lz * (double)k / (double)nz;
  }
  std::vector<double> dzf(nz), inv_dzf(nz), zcen(nz), inv_dzc(nz + 1, 0.0), za(nz, 0.0), zc(nz, 0.0);
  for (int k = 0; k < nz; ++k) {
    dzf[k] = zf[k + 1] - zf[k];
    inv_dzf[k] = 1.0 / dzf[k];
    zcen[k] = 0.5 * (zf[k] + zf[k + 1]);
  }
  for (int k = 1; k < nz; ++k) inv_dzc[k] = 1.0 / (zcen[k] - zcen[k - 1]);
  for (int k = 1; k < nz; ++k) za[k] = inv_dzc[k] * inv_dzf[k];
  for (int k = 0; k < nz - 1; ++k) zc[k] = inv_dzc[k + 1] * inv_dzf[k];
  const double lz_sum = zf[nz] - zf[0];
  {
    const double h = lz_sum / nz;
    double dev = 0.0;
    for (int k = 0; k < nz; ++k) dev = std::max(dev, std::fabs(dzf[k] - h));
    P->z_uniform = dev <= 1e-12 * h;
    P->dz = h;
  }
  // modified wavenumbers of the periodic second difference
  std::vector<double> lamx(P->nxh), lamy(G.ny);
  const double pi = 3.14159265358979323846264338327950288;
  for (int k = 0; k < P->nxh; ++k) {
    const double s = std::sin(pi * (double)k / (double)G.nx);
    lamx[k] = -4.0 / (P->dx * P->dx) * s * s;
  }
  // walls in y: eigenvalues of the Neumann second difference on cell
  // centres, for the cosine modes cos(pi k (j + 1/2) / ny)
  for (int k = 0; k < G.ny; ++k) {
    const double s = std::sin(pi * (double)k / (ywall ? 2.0 * (double)G.ny : (double)G.ny));
    lamy[k] = -4.0 / (P->dy * P->dy) * s * s;
  }
  // stretched y between walls: metrics, row factors and the numerical
  // eigenbasis of L_y (its eigenvalues replace the cosine ones)
  std::vector<double> ymet, ymt_f, ymt_i;
  if (ystretch) {
    const int ny = G.ny;
    std::vector<double> yf(G.yfaces, G.yfaces + ny + 1), dyf(ny), yc(ny), inv_dyc(ny + 1, 0.0);
    for (int j = 0; j < ny; ++j) {
      dyf[j] = yf[j + 1] - yf[j];
      yc[j] = 0.5 * (yf[j] + yf[j + 1]);
    }
    for (int j = 1; j < ny; ++j) inv_dyc[j] = 1.0 / (yc[j] - yc[j - 1]);
    if (!build_yeigen_host(ny, dyf.data(), inv_dyc.data(), lamy, ymt_f, ymt_i)) { delete P; return PP_ERR_NUMERIC; }
    ymet.assign(3 * (size_t)ny, 0.0);
    for (int j = 0; j < ny; ++j) {
      ymet[j] = dyf[j] / P->dy;
      ymet[ny + j] = P->dy * inv_dyc[j];
      ymet[2 * ny + j] = P->dy / dyf[j];
    }
  }

  pp_status st = PP_OK;
  const size_t nc = (size_t)G.nx * G.ny * nz;
  const size_t nw = (size_t)G.nx * G.ny * (nz + 1);
  const size_t nsp = (size_t)P->nxh * G.ny * nz;
  const size_t csz = (prec == PP_FP64) ? sizeof(double2) : sizeof(float2);
  auto up = [&](double** d, const std::vector<double>& h) -> pp_status {
    pp_status s = dalloc(d, h.size() * sizeof(double));
    if (s != PP_OK) return s;
    return cudaMemcpy(*d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess
               ? PP_OK : PP_ERR_CUDA;
  };
  if ((st = up(&P->d_inv_dzf, inv_dzf)) != PP_OK || (st = up(&P->d_inv_dzc, inv_dzc)) != PP_OK ||
      (st = up(&P->d_dzf, dzf)) != PP_OK || (st = up(&P->d_za, za)) != PP_OK ||
      (st = up(&P->d_zc, zc)) != PP_OK || (st = up(&P->d_lamx, lamx)) != PP_OK ||
      (st = up(&P->d_lamy, lamy)) != PP_OK) {
    free_plan(P);
    return st;
  }
  if (ystretch) {
    std::vector<float> ymf(ymet.begin(), ymet.end());
    const int ny = G.ny;
    const size_t nm = (size_t)ny * ny;
    if ((st = up(&P->d_ym, ymet)) != PP_OK || (st = dalloc(&P->d_ym_f, ymf.size() * sizeof(float))) != PP_OK) {
      free_plan(P);
      return st;
    }
    bool ok = cudaMemcpy(P->d_ym_f, ymf.data(), ymf.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
    if (prec == PP_FP64) {
      if ((st = up((double**)&P->d_ymt_f, ymt_f)) != PP_OK || (st = up((double**)&P->d_ymt_i, ymt_i)) != PP_OK) {
        free_plan(P);
        return st;
      }
    } else {
      // row-major M[m][k] of both products, then their BF16 hi/lo tiles
      std::vector<double> mf(nm), mi(nm);
      for (int r = 0; r < ny; ++r)
        for (int k = 0; k < ny; ++k) {
          mf[(size_t)r * ny + k] = ymt_f[(size_t)k * ny + r];  // (V^T W)[r][k]
          mi[(size_t)r * ny + k] = ymt_i[(size_t)k * ny + r];  // V[r][k]
        }
      std::vector<uint16_t> tf, ti;
      dense_tc_tiles(mf, ny, tf);
      dense_tc_tiles(mi, ny, ti);
      const size_t nsp2 = (size_t)(G.nx / 2 + 1) * ny * nz;
      if ((st = dalloc(&P->d_ytc_f, tf.size() * sizeof(uint16_t))) != PP_OK ||
          (st = dalloc(&P->d_ytc_i, ti.size() * sizeof(uint16_t))) != PP_OK ||
          (st = dalloc(&P->d_spec2, nsp2 * sizeof(float2))) != PP_OK) {
        free_plan(P);
        return st;
      }
      ok = ok && cudaMemcpy(P->d_ytc_f, tf.data(), tf.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(P->d_ytc_i, ti.data(), ti.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (!ok) { free_plan(P); return PP_ERR_CUDA; }
  }
  if (prec == PP_FP64) {
    auto tx = twiddles<double>(G.nx), ty = twiddles<double>(G.ny);
    if ((st = dalloc(&P->d_twx, tx.size() * sizeof(double2))) != PP_OK ||
        (st = dalloc(&P->d_twy, ty.size() * sizeof(double2))) != PP_OK) { free_plan(P); return st; }
    if (cudaMemcpy(P->d_twx, tx.data(), tx.size() * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->d_twy, ty.data(), ty.size() * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess) {
      free_plan(P);
      return PP_ERR_CUDA;
    }
    if (ywall && !ystretch) {
      auto tc = dct_twiddles<double>(G.ny);
      if ((st = dalloc(&P->d_dcty, tc.size() * sizeof(double2))) != PP_OK) { free_plan(P); return st; }
      if (cudaMemcpy(P->d_dcty, tc.data(), tc.size() * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess) {
        free_plan(P);
        return PP_ERR_CUDA;
      }
    }
  } else {
    auto tx = twiddles<float>(G.nx), ty = twiddles<float>(G.ny);
    if ((st = dalloc(&P->d_twx, tx.size() * sizeof(float2))) != PP_OK ||
        (st = dalloc(&P->d_twy, ty.size() * sizeof(float2))) != PP_OK) { free_plan(P); return st; }
    if (cudaMemcpy(P->d_twx, tx.data(), tx.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->d_twy, ty.data(), ty.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
      free_plan(P);
      return PP_ERR_CUDA;
    }
    if (ywall && !ystretch) {
      auto tc = dct_twiddles<float>(G.ny);
      if ((st = dalloc(&P->d_dcty, tc.size() * sizeof(float2))) != PP_OK) { free_plan(P); return st; }
      if (cudaMemcpy(P->d_dcty, tc.data(), tc.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
        free_plan(P);
        return PP_ERR_CUDA;
      }
    }
  }
  // residual partial sums: 2 per residual block, or the reduction grid
  const size_t rpb_min = 2;
  P->red_len = std::max((size_t)2 * ((size_t)G.ny * nz + rpb_min - 1) / rpb_min + 2,
                        (size_t)reduce_blocks());
  if ((st = dalloc(&P->d_invd, nsp * sizeof(double))) != PP_OK ||
      (st = dalloc(&P->d_mtab, nsp * sizeof(double))) != PP_OK ||
      (st = dalloc(&P->d_spec, nsp * csz)) != PP_OK ||
      (prec != PP_FP64 && (st = dalloc(&P->d_E, nc * sizeof(float))) != PP_OK) ||
      (prec != PP_FP64 && (st = dalloc(&P->d_delta, nc * sizeof(float))) != PP_OK) ||
      (prec != PP_FP64 && (st = dalloc(&P->d_sdelta, nc * sizeof(float))) != PP_OK) ||
      (st = dalloc(&P->d_b, nc * sizeof(double))) != PP_OK ||
      (st = dalloc(&P->d_red, P->red_len * sizeof(double))) != PP_OK ||
      (st = dalloc(&P->faces.cx, nc * sizeof(double))) != PP_OK ||
      (st = dalloc(&P->faces.cy, nc * sizeof(double))) != PP_OK ||
      (st = dalloc(&P->faces.cz, nw * sizeof(double))) != PP_OK ||
      (st = dalloc(&P->faces.diag, nc * sizeof(double))) != PP_OK ||
      (st = dalloc(&P->faces.rhof, nc * sizeof(float))) != PP_OK ||
      (st = dalloc(&P->d_inv_dzf_f, (size_t)nz * sizeof(float))) != PP_OK ||
      (st = dalloc(&P->d_cw_f, 3 * (size_t)(nz + 1) * sizeof(float))) != PP_OK ||
      (st = dalloc(&P->d_st, sizeof(DevStatus))) != PP_OK ||
      (st = dalloc(&P->d_thermo, 4 * sizeof(double))) != PP_OK) {
    free_plan(P);
    return st;
  }
  if (cudaMallocHost((void**)&P->h_st, 2 * sizeof(DevStatus)) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev[1], cudaEventDisableTiming) != cudaSuccess) {
    free_plan(P);
    return PP_ERR_CUDA;
  }
  {
    std::vector<float> f32(nz);
    for (int k = 0; k < nz; ++k) f32[k] = (float)inv_dzf[k];
    const std::vector<float> cw = layer_factors_f32(nz, dzf, inv_dzc, 1.0 / (P->dx * P->dx), 1.0 / (P->dy * P->dy));
    if (cudaMemcpy(P->d_inv_dzf_f, f32.data(), nz * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->d_cw_f, cw.data(), cw.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      free_plan(P);
      return PP_ERR_CUDA;
    }
  }
  Geo& g = P->geo;
  g.nx = G.nx; g.ny = G.ny; g.nz = nz; g.nxh = P->nxh;
  g.inv_dzf_f = P->d_inv_dzf_f;
  g.cw_f = P->d_cw_f;
  g.dx = P->dx; g.dy = P->dy;
  g.inv_dx2 = 1.0 / (P->dx * P->dx);
  g.inv_dy2 = 1.0 / (P->dy * P->dy);
  g.inv_dzf = P->d_inv_dzf; g.inv_dzc = P->d_inv_dzc; g.dzf = P->d_dzf;
  g.za = P->d_za; g.zc = P->d_zc; g.lz = lz_sum;
  g.ywall = (G.bc[1] == PP_BC_WALL) ? 1 : 0;
  g.ym = P->d_ym;
  g.ym_f = P->d_ym_f;
  if (prec == PP_MIXED_TC) {
    int zm = 0;
    const int nt = dense_tc_out_tiles(nz);
    std::vector<float> mu;
    std::vector<double> mf, mi;
    std::vector<uint16_t> a1, a2;
    if (!build_zeigen_host(nz, dzf.data(), inv_dzc.data(), nt * 256, mu, &zm, mf, mi)) {
      free_plan(P);
      return PP_ERR_NUMERIC;
    }
    dense_tc_tiles(mf, nz, a1);
    dense_tc_tiles(mi, nz, a2);
    if ((st = dalloc(&P->d_mu, mu.size() * sizeof(float))) != PP_OK ||
        (st = dalloc(&P->d_za1, a1.size() * sizeof(uint16_t))) != PP_OK ||
        (st = dalloc(&P->d_za2, a2.size() * sizeof(uint16_t))) != PP_OK ||
        (!P->d_spec2 && (st = dalloc(&P->d_spec2, nsp * sizeof(float2))) != PP_OK) ||
        cudaMemcpy(P->d_mu, mu.data(), mu.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->d_za1, a1.data(), a1.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->d_za2, a2.data(), a2.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess) {
      free_plan(P);
      return st != PP_OK ? st : PP_ERR_CUDA;
    }
    P->z_tc = true;
    P->ze.nt = nt;
    P->ze.nkc = dense_tc_k_chunks(nz);
    P->ze.mu = P->d_mu;
    P->ze.zero_mode = zm;
    P->ze.a1 = P->d_za1;
    P->ze.a2 = P->d_za2;
  }
  if (launch_setup_pivots(g, P->d_lamx, P->d_lamy, P->d_invd, P->stream, P->d_mtab) != cudaSuccess ||
      launch_init_status(P->d_st, P->stream) != cudaSuccess ||
      cudaStreamSynchronize(P->stream) != cudaSuccess) {
    free_plan(P);
    return PP_ERR_CUDA;
  }
  if (prec == PP_MIXED_FP32) {
    double dmax = 0.0;
    for (int k = 0; k < nz; ++k) dmax = std::max(dmax, za[k] + zc[k]);
    std::vector<float> zcf(nz);
    for (int k = 0; k < nz; ++k) zcf[k] = (float)zc[k];
    const double thr = 2.0 * dmax / 512.0;
    const std::vector<int> low = tri_low_columns(lamx, lamy, thr);
    if ((st = dalloc(&P->d_low, low.size() * sizeof(int))) != PP_OK ||
        cudaMemcpy(P->d_low, low.data(), low.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        (st = dalloc(&P->d_mtab_f, nsp * sizeof(float))) != PP_OK ||
        (st = dalloc(&P->d_invd_f, nsp * sizeof(float))) != PP_OK ||
        (st = dalloc(&P->d_zc_f, (size_t)nz * sizeof(float))) != PP_OK ||
        cudaMemcpy(P->d_zc_f, zcf.data(), nz * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        launch_narrow(P->d_mtab, P->d_mtab_f, nsp, P->stream) != cudaSuccess ||
        launch_narrow(P->d_invd, P->d_invd_f, nsp, P->stream) != cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess) {
      free_plan(P);
      return st != PP_OK ? st : PP_ERR_CUDA;
    }
    P->tri32.mtab = P->d_mtab_f;
    P->tri32.invd = P->d_invd_f;
    P->tri32.zc = P->d_zc_f;
    P->tri32.lamx = P->d_lamx;
    P->tri32.lamy = P->d_lamy;
    P->tri32.thr = thr;
    P->tri32.low = P->d_low;
    P->tri32.nlow = (int)low.size();
    P->use_tri32 = true;
  }
  if (prec == PP_MIXED_Z64) {
    // periodic y: lambda_y(ky) = lambda_y(ny - ky), one table column for both
    const int ysym = ywall ? 0 : 1;
    const int nyt = ysym ? G.ny / 2 + 1 : G.ny;
    const size_t ntab = (size_t)nz * nyt * P->nxh;
    if ((st = dalloc(&P->d_z64m, ntab * sizeof(double))) != PP_OK ||
        (st = dalloc(&P->d_z64e, ntab * sizeof(double))) != PP_OK ||
        (st = dalloc(&P->d_z64d, ntab * sizeof(float))) != PP_OK ||
        launch_setup_z64(g, P->d_lamx, P->d_lamy, nyt, ysym, P->d_z64m, P->d_z64e, P->d_z64d, P->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess) {
      free_plan(P);
      return st != PP_OK ? st : PP_ERR_CUDA;
    }
    P->z64.m = P->d_z64m;
    P->z64.e = P->d_z64e;
    P->z64.d = P->d_z64d;
    P->z64.nyt = nyt;
    P->z64.ysym = ysym;
    P->use_z64 = true;
  }
  *out = P;
  return PP_OK;
}

pp_status pressure_plan_destroy(pp_plan P) {
  if (!P) return PP_ERR_INVALID_ARG;
  cudaStreamSynchronize(P->stream);
  free_plan(P);
  return PP_OK;
}

pp_status pressure_plan_set_zsolve(pp_plan P, int zsolve) {
  if (check_plan(P) != PP_OK) return PP_ERR_INVALID_ARG;
  if (zsolve == PP_ZSOLVE_TRIDIAG) { P->zsolve = zsolve; return PP_OK; }
  if (zsolve != PP_ZSOLVE_COSINE) return PP_ERR_INVALID_ARG;
  if (P->prec != PP_FP64 || !P->z_uniform || (P->nz & 1) != 0 || P->nz > 2048) return PP_ERR_UNSUPPORTED;
  if (P->d_lamz == nullptr) {  // tables made on first use; d_lamz is allocated last
    if (!factor_len(P->nz, &P->fz)) return PP_ERR_UNSUPPORTED;
    const int nz = P->nz;
    auto tw = twiddles<double>(nz);
    auto tc = dct_twiddles<double>(nz);
    std::vector<double> lamz(nz);
    const double pi = 3.14159265358979323846264338327950288;
    for (int m = 0; m < nz; ++m) {
      const double sn = std::sin(pi * (double)m / (2.0 * (double)nz));
      lamz[m] = -4.0 / (P->dz * P->dz) * sn * sn;
    }
    pp_status st;
    if ((!P->d_twz && (st = dalloc(&P->d_twz, nz * sizeof(double2))) != PP_OK) ||
        (!P->d_dctz && (st = dalloc(&P->d_dctz, nz * sizeof(double2))) != PP_OK) ||
        (st = dalloc(&P->d_lamz, nz * sizeof(double))) != PP_OK)
      return st;
    PP_CK(cudaMemcpy(P->d_twz, tw.data(), nz * sizeof(double2), cudaMemcpyHostToDevice));
    PP_CK(cudaMemcpy(P->d_dctz, tc.data(), nz * sizeof(double2), cudaMemcpyHostToDevice));
    PP_CK(cudaMemcpy(P->d_lamz, lamz.data(), nz * sizeof(double), cudaMemcpyHostToDevice));
  }
  P->zsolve = zsolve;
  return PP_OK;
}

pp_status pressure_plan_set_method(pp_plan P, int method) {
  if (check_plan(P) != PP_OK) return PP_ERR_INVALID_ARG;
  if (method != PP_METHOD_III && method != PP_METHOD_I && method != PP_METHOD_II) return PP_ERR_INVALID_ARG;
  if (method != PP_METHOD_III && P->d_rho_tilde == nullptr) {
    pp_status s = dalloc(&P->d_rho_tilde, sizeof(double));
    if (s != PP_OK) return s;
  }
  if (method == PP_METHOD_I && P->prec == PP_FP64 && P->d_delta64 == nullptr) {
    pp_status s = dalloc(&P->d_delta64, ncell(P) * sizeof(double));
    if (s != PP_OK) return s;
  }
  P->method = method;
  P->faces.rho_tilde = (method == PP_METHOD_III) ? nullptr : P->d_rho_tilde;
  return PP_OK;
}

pp_status pressure_p0_rate(pp_plan P, const double* phi, const double* kc, const double* T, const double* u,
                           const double* v, const double* w, double p0, double gamma, double* rp) {
  if (check_plan(P) != PP_OK || !phi || !kc || !T || !u || !v || !w || !rp) return PP_ERR_INVALID_ARG;
  if (!(gamma > 0.0) || !std::isfinite(p0)) return PP_ERR_INVALID_ARG;
  const size_t nc = ncell(P), nw = nwface(P);
  const double *dphi, *dk, *dT, *du, *dv, *dw;
  pp_status s;
  if ((s = stage_in(P, phi, nc, 0, &dphi)) != PP_OK || (s = stage_in(P, kc, nc, 1, &dk)) != PP_OK ||
      (s = stage_in(P, T, nc, 2, &dT)) != PP_OK || (s = stage_in(P, u, nc, 3, &du)) != PP_OK ||
      (s = stage_in(P, v, nc, 4, &dv)) != PP_OK || (s = stage_in(P, w, nw, 5, &dw)) != PP_OK)
    return s;
  PP_K(P, K_THERMO, launch_thermo_rate(P->geo, dphi, dk, dT, du, dv, dw, p0, gamma, P->d_red, P->d_thermo,
                                       P->stream));
  double out[4];
  PP_CK(cudaMemcpyAsync(out, P->d_thermo, sizeof(out), cudaMemcpyDeviceToHost, P->stream));
  PP_CK(cudaStreamSynchronize(P->stream));
  if (!(out[2] > 0.0) || !std::isfinite(out[3])) return PP_ERR_NUMERIC;
  *rp = out[3];
  return PP_OK;
}

pp_status pressure_predictor(pp_plan P, const double* u, const double* v, const double* w, const double* rho,
                             const double* mu, const double* const force[3], const double gravity[3], double dt_new,
                             double dt_old, const double* const ru_prev[3], double* const u_star[3],
                             double* const ru_out[3]) {
  if (check_plan(P) != PP_OK || !u || !v || !w || !rho || !mu || !gravity || !u_star) return PP_ERR_INVALID_ARG;
  if (P->ystretch) return PP_ERR_UNSUPPORTED;
  if (!u_star[0] || !u_star[1] || !u_star[2] || !(dt_new > 0.0)) return PP_ERR_INVALID_ARG;
  const double* f[3] = {nullptr, nullptr, nullptr};
  const double* prev[3] = {nullptr, nullptr, nullptr};
  double* ru[3] = {nullptr, nullptr, nullptr};
  for (int q = 0; q < 3; ++q) {
    if (force) f[q] = force[q];
    if (ru_prev) prev[q] = ru_prev[q];
    if (ru_out) ru[q] = ru_out[q];
  }
  const bool ab2 = prev[0] || prev[1] || prev[2];
  if (ab2 && (!prev[0] || !prev[1] || !prev[2] || !(dt_old > 0.0))) return PP_ERR_INVALID_ARG;
  // device pointers only: the call takes up to 17 fields
  const void* all[] = {u, v, w, rho, mu, f[0], f[1], f[2], prev[0], prev[1], prev[2],
                       u_star[0], u_star[1], u_star[2], ru[0], ru[1], ru[2]};
  for (const void* q : all)
    if (q != nullptr && !is_device_ptr(q)) return PP_ERR_INVALID_ARG;
  const double r = ab2 ? dt_new / dt_old : 0.0;
  const double a = ab2 ? 1.0 + 0.5 * r : 1.0, b = ab2 ? 0.5 * r : 0.0;
  // the cell divergence goes to the plan's right-hand-side workspace (free
  // between projections)
  PP_K(P, K_PRED, launch_predictor(P->geo, u, v, w, rho, mu, f, prev, gravity, dt_new, a, b, P->d_b, u_star, ru,
                                   P->stream));
  return PP_OK;
}

pp_status pressure_dp0dt_extrapolate(double rp_n, double rp_nm1, double dt_new, double dt_old, double* out) {
  if (!out || !(dt_old > 0.0) || !(dt_new > 0.0)) return PP_ERR_INVALID_ARG;
  const double r = dt_new / dt_old;
  *out = (1.0 + r) * rp_n - r * rp_nm1;
  return PP_OK;
}

pp_status pressure_divergence_source(pp_plan P, const double* phi, const double* kc, const double* T, double p0,
                                     double gamma, double dp0dt, double* S) {
  if (check_plan(P) != PP_OK || !phi || !kc || !T || !S) return PP_ERR_INVALID_ARG;
  if (!(gamma > 0.0) || p0 == 0.0 || !std::isfinite(p0) || !std::isfinite(dp0dt)) return PP_ERR_INVALID_ARG;
  const size_t nc = ncell(P);
  const double *dphi, *dk, *dT;
  double* dS;
  bool staged;
  pp_status s;
  if ((s = stage_in(P, phi, nc, 0, &dphi)) != PP_OK || (s = stage_in(P, kc, nc, 1, &dk)) != PP_OK ||
      (s = stage_in(P, T, nc, 2, &dT)) != PP_OK || (s = stage_out(P, S, 3, &dS, &staged)) != PP_OK)
    return s;
  PP_K(P, K_SOURCE, launch_divergence_source(P->geo, dphi, dk, dT, p0, gamma, dp0dt, dS, P->stream));
  if (staged) {
    if ((s = copy_back(P, S, dS, nc)) != PP_OK) return s;
    PP_CK(cudaStreamSynchronize(P->stream));
  }
  return PP_OK;
}

pp_status pressure_mixture_density(pp_plan P, const double* phi, double rho_g, double rho_l, double* rho) {
  if (check_plan(P) != PP_OK || !phi || !rho) return PP_ERR_INVALID_ARG;
  const size_t n = ncell(P);
  const double* dphi;
  double* drho;
  bool staged;
  pp_status s;
  if ((s = stage_in(P, phi, n, 0, &dphi)) != PP_OK) return s;
  if ((s = stage_out(P, rho, 1, &drho, &staged)) != PP_OK) return s;
  PP_K(P, K_MIX, launch_mixture(dphi, rho_g, rho_l, drho, n, P->stream));
  if (staged) {
    if ((s = copy_back(P, rho, drho, n)) != PP_OK) return s;
    PP_CK(cudaStreamSynchronize(P->stream));
  }
  return PP_OK;
}

pp_status pressure_solve(pp_plan P, const double* f, double* p, pp_info* info) {
  if (check_plan(P) != PP_OK || !f || !p) return PP_ERR_INVALID_ARG;
  const size_t n = ncell(P);
  const double* df;
  double* dp;
  bool staged;
  pp_status s;
  if ((s = stage_in(P, f, n, 0, &df)) != PP_OK) return s;
  if ((s = stage_out(P, p, 1, &dp, &staged)) != PP_OK) return s;
  const Geo& g = P->geo;
  PP_K(P, K_INIT, launch_init_status(P->d_st, P->stream));
  if (P->prec == PP_FP64) {
    PP_K(P, K_RESID, launch_resid_fftx<double>(g, P->faces, P->fx, (const double2*)P->d_twx, df, 1.0, nullptr,
                                    nullptr, 1, 0, (double2*)P->d_spec, nullptr, nullptr, P->d_st,
                                    P->stream));
    if ((s = solve_pass<double>(P, dp, 1)) != PP_OK) return s;
  } else {
    PP_K(P, K_RESID, launch_resid_fftx<float>(g, P->faces, P->fx, (const float2*)P->d_twx, df, 1.0, nullptr,
                                   nullptr, 1, 0, (float2*)P->d_spec, nullptr, nullptr, P->d_st,
                                   P->stream));
    if ((s = solve_pass<float>(P, dp, 1)) != PP_OK) return s;
  }
  PP_K(P, K_RMEAN, launch_remove_mean(g, dp, P->d_red, P->d_st, P->stream));
  if (staged && (s = copy_back(P, p, dp, n)) != PP_OK) return s;
  if (info || staged) {
    PP_CK(cudaStreamSynchronize(P->stream));
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->iters = 1;
      info->status = PP_OK;
    }
  }
  return PP_OK;
}

pp_status pressure_correct(pp_plan P, const double* us, const double* vs, const double* ws,
                           const double* rho, const double* S, double dt, double* p, int warm_start,
                           double* u, double* v, double* w, double rtol, int maxit, pp_info* info) {
  if (check_plan(P) != PP_OK || !us || !vs || !ws || !rho || !p || !u || !v || !w) return PP_ERR_INVALID_ARG;
  if (!(dt > 0.0) || !(rtol >= 0.0) || maxit < 0) return PP_ERR_INVALID_ARG;
  const size_t nc = ncell(P), nw = nwface(P);
  const double *dus, *dvs, *dws, *drho, *dS, *dpin = nullptr;
  double *dp, *du, *dv, *dw;
  bool sp, su, sv, sw;
  pp_status s;
  if ((s = stage_in(P, us, nc, 0, &dus)) != PP_OK || (s = stage_in(P, vs, nc, 1, &dvs)) != PP_OK ||
      (s = stage_in(P, ws, nw, 2, &dws)) != PP_OK || (s = stage_in(P, rho, nc, 3, &drho)) != PP_OK ||
      (s = stage_in(P, S, nc, 4, &dS)) != PP_OK)
    return s;
  if ((s = stage_out(P, p, 5, &dp, &sp)) != PP_OK || (s = stage_out(P, u, 6, &du, &su)) != PP_OK ||
      (s = stage_out(P, v, 7, &dv, &sv)) != PP_OK || (s = stage_out(P, w, 8, &dw, &sw)) != PP_OK)
    return s;
  if (warm_start && sp) {
    if ((s = stage_in(P, p, nc, 9, &dpin)) != PP_OK) return s;
    PP_CK(cudaMemcpyAsync(dp, dpin, nc * sizeof(double), cudaMemcpyDeviceToDevice, P->stream));
  }
  if (P->prec == PP_FP64) s = projection<double>(P, dus, dvs, dws, drho, dS, dt, dp, warm_start, du, dv, dw, rtol, maxit);
  else s = projection<float>(P, dus, dvs, dws, drho, dS, dt, dp, warm_start, du, dv, dw, rtol, maxit);
  if (s != PP_OK) return s;
  if (sp && (s = copy_back(P, p, dp, nc)) != PP_OK) return s;
  if (su && (s = copy_back(P, u, du, nc)) != PP_OK) return s;
  if (sv && (s = copy_back(P, v, dv, nc)) != PP_OK) return s;
  if (sw && (s = copy_back(P, w, dw, nw)) != PP_OK) return s;
  if (info || sp || su || sv || sw) {
    pp_info tmp;
    s = read_info(P, &tmp);
    tmp.res0 *= dt;
    tmp.res_l1_sum *= dt;
    if (info) *info = tmp;
    return s;
  }
  return PP_OK;
}

pp_status pressure_last_info(pp_plan P, pp_info* info) {
  if (check_plan(P) != PP_OK || !info) return PP_ERR_INVALID_ARG;
  return read_info(P, info);
}

pp_status pressure_solve_adjoint(pp_plan P, const double* rho, const double* p, double dt,
                                 const double* gu, const double* gv, const double* gw, double* gus,
                                 double* gvs, double* gws, double* grho, double rtol, int maxit,
                                 pp_info* info) {
  if (check_plan(P) != PP_OK || !rho || !p || !gu || !gv || !gw || !gus || !gvs || !gws || !grho)
    return PP_ERR_INVALID_ARG;
  if (!(dt > 0.0) || !(rtol >= 0.0) || maxit < 0) return PP_ERR_INVALID_ARG;
  const size_t nc = ncell(P), nw = nwface(P);
  pp_status s;
  for (int i = 0; i < 4; ++i) {
    if (!P->d_adj[i] && (s = dalloc(&P->d_adj[i], nw * sizeof(double))) != PP_OK) return s;
  }
  const double *drho, *dp, *dgu, *dgv, *dgw;
  double *dgus, *dgvs, *dgws, *dgrho;
  bool s1, s2, s3, s4;
  if ((s = stage_in(P, rho, nc, 0, &drho)) != PP_OK || (s = stage_in(P, p, nc, 1, &dp)) != PP_OK ||
      (s = stage_in(P, gu, nc, 2, &dgu)) != PP_OK || (s = stage_in(P, gv, nc, 3, &dgv)) != PP_OK ||
      (s = stage_in(P, gw, nw, 4, &dgw)) != PP_OK)
    return s;
  if ((s = stage_out(P, gus, 5, &dgus, &s1)) != PP_OK || (s = stage_out(P, gvs, 6, &dgvs, &s2)) != PP_OK ||
      (s = stage_out(P, gws, 7, &dgws, &s3)) != PP_OK || (s = stage_out(P, grho, 8, &dgrho, &s4)) != PP_OK)
    return s;
  const Geo& g = P->geo;
  double *yu = P->d_adj[0], *yv = P->d_adj[1], *yw = P->d_adj[2], *mu = P->d_adj[3];
  PP_K(P, K_ADJ_RHS, launch_adj_rhs(g, drho, dgu, dgv, dgw, dt, yu, yv, yw, P->stream));
  // mu solves D(beta G mu) = D(y)/dt: the projection loop with u* = y, S = 0
  if (P->prec == PP_FP64) s = projection<double>(P, yu, yv, yw, drho, nullptr, dt, mu, 0, nullptr, nullptr, nullptr, rtol, maxit);
  else s = projection<float>(P, yu, yv, yw, drho, nullptr, dt, mu, 0, nullptr, nullptr, nullptr, rtol, maxit);
  if (s != PP_OK) return s;
  // y buffers are free again: reuse them for the face terms of d rho
  PP_K(P, K_ADJ_FIN, launch_adj_finish(g, drho, dp, mu, dt, dgu, dgv, dgw, dgus, dgvs, dgws, yu, yv, yw, P->stream));
  PP_K(P, K_ADJ_GRHO, launch_adj_grho(g, yu, yv, yw, dgrho, P->stream));
  if (s1 && (s = copy_back(P, gus, dgus, nc)) != PP_OK) return s;
  if (s2 && (s = copy_back(P, gvs, dgvs, nc)) != PP_OK) return s;
  if (s3 && (s = copy_back(P, gws, dgws, nw)) != PP_OK) return s;
  if (s4 && (s = copy_back(P, grho, dgrho, nc)) != PP_OK) return s;
  if (info || s1 || s2 || s3 || s4) {
    pp_info tmp;
    s = read_info(P, &tmp);
    tmp.res0 *= dt;
    tmp.res_l1_sum *= dt;
    if (info) *info = tmp;
    return s;
  }
  return PP_OK;
}

pp_status pressure_profile_enable(pp_plan P, int enable) {
  if (check_plan(P) != PP_OK) return PP_ERR_INVALID_ARG;
  PP_CK(cudaStreamSynchronize(P->stream));
  for (auto& r : P->prof.rec) { P->prof.pool.push_back(r.a); P->prof.pool.push_back(r.b); }
  P->prof.rec.clear();
  for (int k = 0; k < K_COUNT; ++k) { P->prof.ms[k] = 0.0; P->prof.n[k] = 0; }
  P->prof.launches = 0;
  P->prof.on = enable != 0;
  return PP_OK;
}

pp_status pressure_profile_read(pp_plan P, pp_kernel_time* out, int max_entries, int* n,
                                long long* total_launches) {
  if (check_plan(P) != PP_OK || !n) return PP_ERR_INVALID_ARG;
  PP_CK(cudaStreamSynchronize(P->stream));
  for (auto& r : P->prof.rec) {
    float ms = 0.f;
    PP_CK(cudaEventElapsedTime(&ms, r.a, r.b));
    P->prof.ms[r.kid] += ms;
    P->prof.n[r.kid] += 1;
    P->prof.pool.push_back(r.a);
    P->prof.pool.push_back(r.b);
  }
  P->prof.rec.clear();
  int cnt = 0;
  for (int k = 0; k < K_COUNT; ++k) {
    if (P->prof.n[k] == 0) continue;
    if (out && cnt < max_entries) {
      std::memset(out[cnt].name, 0, sizeof(out[cnt].name));
      std::strncpy(out[cnt].name, kNames[k], sizeof(out[cnt].name) - 1);
      out[cnt].launches = P->prof.n[k] * kLaunches[k];
      out[cnt].total_ms = P->prof.ms[k];
    }
    ++cnt;
  }
  *n = cnt;
  if (total_launches) *total_launches = P->prof.launches;
  return PP_OK;
}

}  // extern "C"
