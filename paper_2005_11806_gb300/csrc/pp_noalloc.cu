// pressure_solve_noalloc: the FP64 constant-coefficient eigenexpansion solve
// without any device allocation, for callers that cannot call cudaMalloc
// (code that runs while a stream is being captured, hosts whose memory is
// owned by an external pool or budget, real-time loops that forbid allocator
// calls).  Its working memory is one file-scope device array of fixed size;
// every device that loads this library holds that array until the process
// exits.  The kernels are the ones pressure_solve launches.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "pp_internal.cuh"

using namespace pp;

// Scratch of the allocation-free entry point: spectral array, Thomas pivots,
// twiddles, z metrics, eigenvalues, reduction partials and the status word.
static constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) unsigned char pp_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The host-side
// name of a __device__ array is only a stand-in, so the address is looked up
// once per device with that device current.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, pp_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return cudaSuccess;
}

bool factor(int n, FftDesc* d) {
  d->n = n;
  d->nst = 0;
  int m = n;
  const int rads[5] = {8, 4, 2, 3, 5};
  for (int r : rads)
    while (m % r == 0) {
      if (d->nst >= kMaxStages) return false;
      d->radix[d->nst++] = r;
      m /= r;
    }
  d->pow2 = (n & (n - 1)) == 0;
  return m == 1;
}

std::vector<double2> twiddle_table(int n) {
  std::vector<double2> t(n);
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < n; ++m) {
    const double a = two_pi * (double)m / (double)n;
    t[m] = make_double2(std::cos(a), std::sin(a));
  }
  return t;
}

struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t at = off;
    off = (off + bytes + 255) & ~(size_t)255;
    return at;
  }
};

bool is_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" pp_status pressure_solve_noalloc(const pp_grid* grid, const double* f, double* p,
                                            void* stream_ptr) {
  if (!grid || !f || !p) return PP_ERR_INVALID_ARG;
  const pp_grid& G = *grid;
  if (G.nx < 2 || G.ny < 1 || G.nz < 1 || !(G.lx > 0) || !(G.ly > 0) || !(G.lz > 0))
    return PP_ERR_INVALID_ARG;
  if (G.bc[0] != PP_BC_PERIODIC || G.bc[1] != PP_BC_PERIODIC || G.bc[2] != PP_BC_WALL)
    return PP_ERR_UNSUPPORTED;
  if ((G.nx & 1) != 0) return PP_ERR_UNSUPPORTED;
  FftDesc fx, fy;
  if (!factor(G.nx, &fx) || !factor(G.ny, &fy)) return PP_ERR_UNSUPPORTED;
  if (!is_device(f) || !is_device(p)) return PP_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream_ptr;
  const int nx = G.nx, ny = G.ny, nz = G.nz, nxh = nx / 2 + 1;
  const size_t nsp = (size_t)nxh * ny * nz;

  // Layout of the scratch array for this grid; reject what does not fit.
  Carve c;
  const size_t o_spec = c.take(nsp * sizeof(double2));
  const size_t o_invd = c.take(nsp * sizeof(double));
  const size_t o_twx = c.take((size_t)nx * sizeof(double2));
  const size_t o_twy = c.take((size_t)ny * sizeof(double2));
  const size_t o_dzf = c.take((size_t)nz * sizeof(double));
  const size_t o_idzf = c.take((size_t)nz * sizeof(double));
  const size_t o_idzc = c.take((size_t)(nz + 1) * sizeof(double));
  const size_t o_za = c.take((size_t)nz * sizeof(double));
  const size_t o_zc = c.take((size_t)nz * sizeof(double));
  const size_t o_lamx = c.take((size_t)nxh * sizeof(double));
  const size_t o_lamy = c.take((size_t)ny * sizeof(double));
  const size_t o_red = c.take((size_t)reduce_blocks() * sizeof(double));
  const size_t o_st = c.take(sizeof(DevStatus));
  if (c.off > kNoAllocScratchBytes) return PP_ERR_TOO_LARGE;

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return PP_ERR_CUDA;
  unsigned char* S = (unsigned char*)base;

  // Host tables (z metrics of Sec. 3's grid, modified wavenumbers, twiddles).
  std::vector<double> zf(nz + 1);
  for (int k = 0; k <= nz; ++k) zf[k] = G.zfaces ? G.zfaces[k] : G.lz * (double)k / (double)nz;
  for (int k = 0; k < nz; ++k)
    if (!(zf[k + 1] > zf[k])) return PP_ERR_INVALID_ARG;
  std::vector<double> dzf(nz), idzf(nz), zcen(nz), idzc(nz + 1, 0.0), za(nz, 0.0), zc(nz, 0.0);
  for (int k = 0; k < nz; ++k) {
    dzf[k] = zf[k + 1] - zf[k];
    idzf[k] = 1.0 / dzf[k];
    zcen[k] = 0.5 * (zf[k] + zf[k + 1]);
  }
  for (int k = 1; k < nz; ++k) idzc[k] = 1.0 / (zcen[k] - zcen[k - 1]);
  for (int k = 1; k < nz; ++k) za[k] = idzc[k] * idzf[k];
  for (int k = 0; k < nz - 1; ++k) zc[k] = idzc[k + 1] * idzf[k];
  const double dx = G.lx / nx, dy = G.ly / ny;
  const double pi = 3.14159265358979323846264338327950288;
  std::vector<double> lamx(nxh), lamy(ny);
  for (int k = 0; k < nxh; ++k) {
    const double sn = std::sin(pi * (double)k / (double)nx);
    lamx[k] = -4.0 / (dx * dx) * sn * sn;
  }
  for (int k = 0; k < ny; ++k) {
    const double sn = std::sin(pi * (double)k / (double)ny);
    lamy[k] = -4.0 / (dy * dy) * sn * sn;
  }
  std::vector<double2> twx = twiddle_table(nx), twy = twiddle_table(ny);
  struct Up { size_t off; const void* src; size_t bytes; } ups[] = {
      {o_twx, twx.data(), twx.size() * sizeof(double2)}, {o_twy, twy.data(), twy.size() * sizeof(double2)},
      {o_dzf, dzf.data(), dzf.size() * sizeof(double)},  {o_idzf, idzf.data(), idzf.size() * sizeof(double)},
      {o_idzc, idzc.data(), idzc.size() * sizeof(double)}, {o_za, za.data(), za.size() * sizeof(double)},
      {o_zc, zc.data(), zc.size() * sizeof(double)},     {o_lamx, lamx.data(), lamx.size() * sizeof(double)},
      {o_lamy, lamy.data(), lamy.size() * sizeof(double)}};
  for (const Up& u : ups)
    if (cudaMemcpyAsync(S + u.off, u.src, u.bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return PP_ERR_CUDA;

  Geo g;
  g.nx = nx; g.ny = ny; g.nz = nz; g.nxh = nxh;
  g.dx = dx; g.dy = dy;
  g.inv_dx2 = 1.0 / (dx * dx);
  g.inv_dy2 = 1.0 / (dy * dy);
  g.inv_dzf = (const double*)(S + o_idzf);
  g.inv_dzc = (const double*)(S + o_idzc);
  g.dzf = (const double*)(S + o_dzf);
  g.za = (const double*)(S + o_za);
  g.zc = (const double*)(S + o_zc);
  g.lz = zf[nz] - zf[0];
  g.ywall = 0;
  double2* spec = (double2*)(S + o_spec);
  double* invd = (double*)(S + o_invd);
  const double2* dtwx = (const double2*)(S + o_twx);
  const double2* dtwy = (const double2*)(S + o_twy);
  double* red = (double*)(S + o_red);
  DevStatus* st = (DevStatus*)(S + o_st);
  Faces none{nullptr, nullptr, nullptr};
  const double scale = 1.0 / ((double)nx * (double)ny);
  // The status word starts cleared and the pivots are rebuilt: the array
  // still holds whatever the previous call left in it.
  if (launch_init_status(st, s) != cudaSuccess ||
      launch_setup_pivots(g, (const double*)(S + o_lamx), (const double*)(S + o_lamy), invd, s) != cudaSuccess ||
      launch_resid_fftx<double>(g, none, fx, dtwx, f, 1.0, nullptr, nullptr, 1, 0, spec, nullptr, nullptr, st, s) != cudaSuccess ||
      launch_ffty<double>(g, fy, dtwy, spec, 0, st, s) != cudaSuccess ||
      launch_tridiag<double>(g, invd, spec, spec, st, s) != cudaSuccess ||
      launch_ffty<double>(g, fy, dtwy, spec, 1, st, s) != cudaSuccess ||
      launch_fftx_inv<double>(g, fx, dtwx, spec, scale, p, 1, st, s) != cudaSuccess ||
      launch_remove_mean(g, p, red, st, s) != cudaSuccess)
    return PP_ERR_CUDA;
  return PP_OK;
}
