// pressure_solve_noalloc: the FP64 constant-coefficient eigenexpansion solve
// without any device allocation, for callers that cannot call cudaMalloc
// (hosts whose device memory is owned by an external pool or budget, loops
// that must not enter an allocator).  Its working memory is one file-scope
// device array of fixed size; every device that loads this library holds
// that array until the process exits.  The transform and z-solve kernels are
// the ones pressure_solve launches; the tables (twiddles, wavenumbers, z
// metrics) are computed on the device from scalar arguments, with the z face
// coordinates passed by value in kernel parameters, so the call issues no
// host-to-device copy and does not wait for the GPU.
#include <cmath>
#include <cstring>
#include <mutex>

#include "pp_internal.cuh"

using namespace pp;

// Scratch of the allocation-free entry point: spectral array, Thomas pivots,
// twiddles, z faces and metrics, eigenvalues, reduction partials and the
// status word.
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

// z face coordinates travel to the device by value, in kernel parameters
// (under 4 KB per launch), so no host buffer has to outlive the call.
constexpr int kFaceChunk = 480;
struct FaceChunk {
  double v[kFaceChunk];
  int off, n;
};

__global__ void k_na_store_faces(FaceChunk c, double* __restrict__ zf) {
  for (int i = threadIdx.x; i < c.n; i += blockDim.x) zf[c.off + i] = c.v[i];
}

__global__ void k_na_uniform_faces(double lz, int nz, double* __restrict__ zf) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= nz; k += gridDim.x * blockDim.x)
    zf[k] = lz * (double)k / (double)nz;
}

// The tables of one constant-coefficient solve (Sec. 3 grid, Sec. 3.3.1
// eigenexpansion): FFT twiddles (cos, sin)(2 pi m / n), the modified
// wavenumbers -(4/h^2) sin^2(pi k / n) of the periodic second difference,
// and the z metrics of the faces zf (cell widths, centre distances, the
// sub- and super-diagonal of L_z), each entry computed from zf directly.
// With walls in y (ywall) the y eigenvalues are those of the Neumann second
// difference, -(4/dy^2) sin^2(pi m / (2 ny)), and dcty receives the cosine
// transform's twiddles exp(-i pi m / (2 ny)).
__global__ void k_na_tables(int nx, int ny, int nz, double dx, double dy, const double* __restrict__ zf,
                            double2* __restrict__ twx, double2* __restrict__ twy, double* __restrict__ dzf,
                            double* __restrict__ idzf, double* __restrict__ idzc, double* __restrict__ za,
                            double* __restrict__ zc, double* __restrict__ lamx, double* __restrict__ lamy,
                            int ywall, double2* __restrict__ dcty) {
  const int nxh = nx / 2 + 1;
  int nmax = nx > ny ? nx : ny;
  if (nz + 1 > nmax) nmax = nz + 1;
  auto inv_dzc = [&](int k) {  // 1 / centre distance across z-face k (0 on the walls)
    if (k <= 0 || k >= nz) return 0.0;
    const double c1 = 0.5 * (zf[k] + zf[k + 1]), c0 = 0.5 * (zf[k - 1] + zf[k]);
    return 1.0 / (c1 - c0);
  };
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < nmax; m += gridDim.x * blockDim.x) {
    double sn, cs;
    if (m < nx) {
      sincospi(2.0 * (double)m / (double)nx, &sn, &cs);
      twx[m] = make_double2(cs, sn);
    }
    if (m < ny) {
      sincospi(2.0 * (double)m / (double)ny, &sn, &cs);
      twy[m] = make_double2(cs, sn);
      const double s = sinpi((double)m / (ywall ? 2.0 * (double)ny : (double)ny));
      lamy[m] = -4.0 / (dy * dy) * s * s;
      if (ywall) {
        sincospi((double)m / (2.0 * (double)ny), &sn, &cs);
        dcty[m] = make_double2(cs, -sn);
      }
    }
    if (m < nxh) {
      const double s = sinpi((double)m / (double)nx);
      lamx[m] = -4.0 / (dx * dx) * s * s;
    }
    if (m <= nz) idzc[m] = inv_dzc(m);
    if (m < nz) {
      const double w = zf[m + 1] - zf[m];
      const double iw = 1.0 / w;
      dzf[m] = w;
      idzf[m] = iw;
      za[m] = (m >= 1) ? inv_dzc(m) * iw : 0.0;
      zc[m] = (m + 1 < nz) ? inv_dzc(m + 1) * iw : 0.0;
    }
  }
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
  if (G.bc[0] != PP_BC_PERIODIC || (G.bc[1] != PP_BC_PERIODIC && G.bc[1] != PP_BC_WALL) ||
      G.bc[2] != PP_BC_WALL || G.yfaces != nullptr)
    return PP_ERR_UNSUPPORTED;
  const int ywall = (G.bc[1] == PP_BC_WALL) ? 1 : 0;
  if ((G.nx & 1) != 0) return PP_ERR_UNSUPPORTED;
  // walls in y: the cosine transform runs as one complex FFT of even length
  if (ywall && (G.ny < 2 || (G.ny & 1) != 0)) return PP_ERR_UNSUPPORTED;
  // the limits of pressure_plan_create: one transform line per block in the
  // FFT kernels, 32-bit cell offsets
  if (G.nx > 2048 || G.ny > 2048) return PP_ERR_UNSUPPORTED;
  if ((long long)G.nx * G.ny * (G.nz + 1) > (1LL << 31)) return PP_ERR_UNSUPPORTED;
  FftDesc fx, fy;
  if (!factor(G.nx, &fx) || !factor(G.ny, &fy)) return PP_ERR_UNSUPPORTED;
  if (G.zfaces && !faces_ok(G.zfaces, G.nz)) return PP_ERR_INVALID_ARG;
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
  const size_t o_dcty = c.take(ywall ? (size_t)ny * sizeof(double2) : 0);
  const size_t o_red = c.take((size_t)reduce_blocks() * sizeof(double));
  const size_t o_st = c.take(sizeof(DevStatus));
  const size_t o_zf = c.take((size_t)(nz + 1) * sizeof(double));
  if (c.off > kNoAllocScratchBytes) return PP_ERR_TOO_LARGE;

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return PP_ERR_CUDA;
  unsigned char* S = (unsigned char*)base;

  // Face coordinates (checked above) are sent by value (no host buffer is
  // read after the call returns); every table is then computed on the device.
  const double z0 = G.zfaces ? G.zfaces[0] : 0.0;
  const double zn = G.zfaces ? G.zfaces[nz] : G.lz;
  const double dx = G.lx / nx, dy = G.ly / ny;
  double* dzfaces = (double*)(S + o_zf);
  if (G.zfaces) {
    FaceChunk ch;
    for (int off = 0; off <= nz; off += kFaceChunk) {
      ch.off = off;
      ch.n = (nz + 1 - off) < kFaceChunk ? (nz + 1 - off) : kFaceChunk;
      for (int i = 0; i < ch.n; ++i) ch.v[i] = G.zfaces[off + i];
      k_na_store_faces<<<1, 256, 0, s>>>(ch, dzfaces);
    }
  } else {
    k_na_uniform_faces<<<(nz + 256) / 256, 256, 0, s>>>(G.lz, nz, dzfaces);
  }
  {
    int nmax = nx > ny ? nx : ny;
    if (nz + 1 > nmax) nmax = nz + 1;
    int nb = (nmax + 255) / 256;
    if (nb > 1024) nb = 1024;
    k_na_tables<<<nb, 256, 0, s>>>(nx, ny, nz, dx, dy, dzfaces, (double2*)(S + o_twx), (double2*)(S + o_twy),
                                   (double*)(S + o_dzf), (double*)(S + o_idzf), (double*)(S + o_idzc),
                                   (double*)(S + o_za), (double*)(S + o_zc), (double*)(S + o_lamx),
                                   (double*)(S + o_lamy), ywall, (double2*)(S + o_dcty));
  }
  if (cudaGetLastError() != cudaSuccess) return PP_ERR_CUDA;

  Geo g{};
  g.nx = nx; g.ny = ny; g.nz = nz; g.nxh = nxh;
  g.dx = dx; g.dy = dy;
  g.inv_dx2 = 1.0 / (dx * dx);
  g.inv_dy2 = 1.0 / (dy * dy);
  g.inv_dzf = (const double*)(S + o_idzf);
  g.inv_dzc = (const double*)(S + o_idzc);
  g.dzf = (const double*)(S + o_dzf);
  g.za = (const double*)(S + o_za);
  g.zc = (const double*)(S + o_zc);
  g.lz = zn - z0;
  g.ywall = ywall;
  double2* spec = (double2*)(S + o_spec);
  const double2* dct = ywall ? (const double2*)(S + o_dcty) : nullptr;
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
      launch_ffty<double>(g, fy, dtwy, spec, 0, st, s, dct) != cudaSuccess ||
      launch_tridiag<double>(g, invd, spec, spec, st, s) != cudaSuccess ||
      launch_ffty<double>(g, fy, dtwy, spec, 1, st, s, dct) != cudaSuccess ||
      launch_fftx_inv<double>(g, fx, dtwx, spec, scale, p, 1, st, s) != cudaSuccess ||
      launch_remove_mean(g, p, red, st, s) != cudaSuccess)
    return PP_ERR_CUDA;
  return PP_OK;
}
