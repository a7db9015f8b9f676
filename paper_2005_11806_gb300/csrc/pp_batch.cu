// Batched Method III projections (Algorithm 1, Sec. 3.3.1) of independent
// grids of different sizes: every stage of a pass is one grouped launch over
// the tiles of all grids (a work list maps each block to a grid and a tile),
// and the whole solve - set-up, the device-side while loop over passes and
// the correction - is one CUDA graph launch.  Each grid stops on its own
// tolerance; the loop ends when every grid has stopped.  Mixed precision
// (FP32 transforms; FP64 residual, z solve and pressure).  Tile sizes of the
// transform kernels are chosen by timing candidates on the batch at creation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pp_cells.cuh"
#include "pp_stages.cuh"

using namespace pp;

namespace {

constexpr int kChunk = 2048;  // cells per block of the elementwise grouped kernels
constexpr int kTriThreads = 128;
constexpr int kExactEveryBatch = 40;

struct GridDev {
  Geo g;
  Faces fc;
  FftDesc fx, fy;
  const float2* twx;
  const float2* twy;
  const float2* dcty;  // walls in y: exp(-i pi m / (2 ny)); null: periodic y
  const double* invd;
  const double* mtab;
  TriF32 tri;  // FP32 tables of the well-conditioned z columns
  float2* spec;
  float* E;
  float* delta;
  float* sdelta;  // increments not yet added to p (lazy update, stage_fftx_inv)
  double* b;
  double* red;
  DevStatus* st;
  // per call: this grid's fields inside the caller's packed buffers
  const double *us, *vs, *ws, *rho, *S;
  double *p, *u, *v, *w;
  double dt, inv_dt, scale;
  int rpb, nblk_x;  // x kernels: rows per block, blocks
  int tx, ntx;      // y kernels: kx tile, tiles per plane
  int nchunk;       // elementwise chunks
  long long ncell;
};

struct BatchCtl {
  double rtol;
  int maxit;
  int passes;
  int active;
  int pad;
};

// ---- grouped kernels --------------------------------------------------------
__global__ void kb_init(GridDev* G, int n, BatchCtl* ctl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) status_init(G[i].st);
  if (i == 0) { ctl->passes = 0; ctl->active = 1; }
}

#define PP_CHUNK_LOOP(d, w)                                                   \
  const size_t c0 = (size_t)(w).y * kChunk;                                  \
  const size_t c1 = (c0 + (size_t)kChunk < (size_t)(d).ncell) ? c0 + (size_t)kChunk : (size_t)(d).ncell; \
  for (size_t c = c0 + threadIdx.x; c < c1; c += blockDim.x)

__global__ void kb_prep_faces(GridDev* G, const int2* __restrict__ work) {
  const int2 w = work[blockIdx.x];
  const GridDev& d = G[w.x];
  PP_CHUNK_LOOP(d, w) cell_prep_faces(d.g, d.rho, d.fc, c);
}

__global__ void kb_prep_diag(GridDev* G, const int2* __restrict__ work) {
  const int2 w = work[blockIdx.x];
  const GridDev& d = G[w.x];
  PP_CHUNK_LOOP(d, w) cell_prep_diag(d.g, d.fc, c);
}

// partial sums of dzf_k * f over a chunk (f = S, or p when use_p)
__global__ void kb_weighted_partial(GridDev* G, const int2* __restrict__ work, int use_p) {
  __shared__ double sh[32];
  const int2 w = work[blockIdx.x];
  const GridDev& d = G[w.x];
  const double* f = use_p ? d.p : d.S;
  const size_t plane = (size_t)d.g.nx * d.g.ny;
  double s = 0.0;
  if (f != nullptr) {
    PP_CHUNK_LOOP(d, w) s += d.g.dzf[c / plane] * f[c];
  }
  s = block_sum<double>(s, sh);
  if (threadIdx.x == 0) d.red[w.y] = s;
}

// one block per grid: sum of the chunk partials -> mean_S, pmean or e2_0
__global__ void kb_finalize(GridDev* G, int what) {
  __shared__ double sh[32];
  const GridDev& d = G[blockIdx.x];
  double s = 0.0;
  for (int b = threadIdx.x; b < d.nchunk; b += blockDim.x) s += d.red[b];
  s = block_sum<double>(s, sh);
  if (threadIdx.x != 0) return;
  const double vol = d.g.lz * (double)d.g.nx * d.g.ny;
  if (what == 0) d.st->mean_S = s / vol;
  else if (what == 1) d.st->pmean = s / vol;
  else d.st->e2_0 = s * d.inv_dt * d.inv_dt;
}

__global__ void kb_rhs_b(GridDev* G, const int2* __restrict__ work) {
  __shared__ double sh[32];
  const int2 w = work[blockIdx.x];
  const GridDev& d = G[w.x];
  const double meanS = d.st->mean_S;
  double s2 = 0.0;
  PP_CHUNK_LOOP(d, w) {
    const double v = cell_rhs_b(d.g, d.us, d.vs, d.ws, d.S, meanS, d.b, d.inv_dt, c);
    s2 += v * v;
  }
  s2 = block_sum<double>(s2, sh);
  if (threadIdx.x == 0) d.red[w.y] = s2;
}

__global__ void kb_fill_p(GridDev* G, const int2* __restrict__ work, int sub_mean) {
  const int2 w = work[blockIdx.x];
  const GridDev& d = G[w.x];
  const double m = sub_mean ? d.st->pmean : 0.0;
  PP_CHUNK_LOOP(d, w) d.p[c] = sub_mean ? d.p[c] - m : 0.0;
}

__global__ void kb_correct(GridDev* G, const int2* __restrict__ work) {
  const int2 w = work[blockIdx.x];
  const GridDev& d = G[w.x];
  PP_CHUNK_LOOP(d, w) cell_correct(d.g, d.fc, d.us, d.vs, d.ws, d.p, d.dt, d.u, d.v, d.w, c);
}

__global__ void __launch_bounds__(256, 4) kb_resid(GridDev* G, const int2* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 w = work[blockIdx.x];
  const GridDev& d = G[w.x];
  if (d.st->done) return;
  stage_resid_fftx<float>(d.g, d.fc, d.fx, d.twx, d.b, d.rho, d.p, 1, 0, 1, d.spec, d.red, d.rpb, w.y,
                          d.st->need_exact != 0, d.E, d.delta, smem_raw);
}

// one block per grid: reduce the residual partials, update the status
__global__ void kb_check(GridDev* G, const BatchCtl* __restrict__ ctl, int kexact) {
  __shared__ double sh[32];
  const GridDev& d = G[blockIdx.x];
  if (d.st->done) return;
  double s2 = 0.0, s1 = 0.0;
  for (int b = threadIdx.x; b < d.nblk_x; b += blockDim.x) {
    s2 += d.red[2 * (size_t)b];
    s1 += d.red[2 * (size_t)b + 1];
  }
  s2 = block_sum<double>(s2, sh);
  s1 = block_sum<double>(s1, sh);
  if (threadIdx.x == 0) status_update(d.st, s2, s1, ctl->rtol, ctl->maxit, kexact);
}

template <int DIR>
__global__ void __launch_bounds__(256) kb_ffty(GridDev* G, const int2* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 w = work[blockIdx.x];
  const GridDev& d = G[w.x];
  if (d.st->done) return;
  const int bz = w.y / d.ntx, bx = w.y - bz * d.ntx;
  if (d.dcty != nullptr) stage_ffty<float, DIR, true>(d.g, d.fy, d.twy, d.spec, d.tx, bx, bz, smem_raw, d.dcty);
  else stage_ffty<float, DIR>(d.g, d.fy, d.twy, d.spec, d.tx, bx, bz, smem_raw);
}

__global__ void __launch_bounds__(kTriThreads, 8) kb_tridiag(GridDev* G, const int2* __restrict__ work) {
  const int2 w = work[blockIdx.x];
  const GridDev& d = G[w.x];
  if (d.st->done) return;
  stage_tridiag_mixed(d.g, d.mtab, d.invd, d.tri, d.spec, w.y);
}

__global__ void __launch_bounds__(256) kb_fftx_inv(GridDev* G, const int2* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 w = work[blockIdx.x];
  const GridDev& d = G[w.x];
  if (d.st->done) return;
  stage_fftx_inv<float>(d.g, d.fx, d.twx, d.spec, d.scale, d.p, 0, d.rpb, w.y, d.delta, d.sdelta,
                        d.st->need_exact != 0, d.st->since_exact <= 1, smem_raw);
}

// p += sdelta for the grids whose last residual was an updated one.
__global__ void kb_fold(GridDev* G, const int2* __restrict__ work) {
  const int2 w = work[blockIdx.x];
  const GridDev& d = G[w.x];
  if (d.st->last_exact) return;
  PP_CHUNK_LOOP(d, w) d.p[c] += widen_f32(d.sdelta[c]);
}

// Loop control of the device-side while loop: continue while any grid is
// still iterating (each grid stops itself at its tolerance or at maxit).
__global__ void kb_loopctl(GridDev* G, int n, BatchCtl* ctl, cudaGraphConditionalHandle h) {
  __shared__ int sh[32];
  int a = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += G[i].st->done ? 0 : 1;
  a = block_sum<int>(a, sh);
  if (threadIdx.x != 0) return;
  ctl->passes += 1;
  const int go = (a > 0 && ctl->passes <= ctl->maxit + 1) ? 1 : 0;
  ctl->active = a;
  cudaGraphSetConditional(h, go);
}

#define PP_CK(call)                                  \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return PP_ERR_CUDA;       \
  } while (0)

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

bool is_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct pp_batch_s {
  int n = 0;
  cudaStream_t stream = nullptr;   // caller's stream: graph launches and copies
  cudaStream_t cap = nullptr;      // private stream used for capture and tuning
  std::vector<pp_grid> grids;
  std::vector<long long> cell_off, wface_off;
  long long ncell_tot = 0, nwface_tot = 0;
  unsigned char* pool = nullptr;   // every per-grid buffer and table
  int* d_low = nullptr;            // ill-conditioned z columns of every grid
  GridDev* d_dev = nullptr;
  GridDev* h_dev = nullptr;        // pinned mirror
  BatchCtl* d_ctl = nullptr;
  BatchCtl* h_ctl = nullptr;       // pinned
  DevStatus* h_st = nullptr;       // pinned, n entries
  int2 *w_cells = nullptr, *w_x = nullptr, *w_y = nullptr, *w_z = nullptr;
  int n_cells = 0, n_x = 0, n_y = 0, n_z = 0;
  size_t smem_x = 0, smem_y = 0;
  int ept_x = kEpt, ept_y = kEpt;  // chosen by the tuner
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle handle = 0;
};

namespace {

void free_batch(pp_batch_s* B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  if (B->pool) cudaFree(B->pool);
  if (B->d_low) cudaFree(B->d_low);
  if (B->d_dev) cudaFree(B->d_dev);
  if (B->d_ctl) cudaFree(B->d_ctl);
  int2* ws[] = {B->w_cells, B->w_x, B->w_y, B->w_z};
  for (int2* w : ws) if (w) cudaFree(w);
  if (B->h_dev) cudaFreeHost(B->h_dev);
  if (B->h_ctl) cudaFreeHost(B->h_ctl);
  if (B->h_st) cudaFreeHost(B->h_st);
  if (B->cap) cudaStreamDestroy(B->cap);
  delete B;
}

pp_status upload_list(const std::vector<int2>& h, int2** d, int* n) {
  if (*d) { cudaFree(*d); *d = nullptr; }
  *n = (int)h.size();
  if (h.empty()) return PP_OK;
  if (cudaMalloc((void**)d, h.size() * sizeof(int2)) != cudaSuccess) return PP_ERR_OOM;
  return cudaMemcpy(*d, h.data(), h.size() * sizeof(int2), cudaMemcpyHostToDevice) == cudaSuccess
             ? PP_OK : PP_ERR_CUDA;
}

// Work lists for the x kernels (rows) and y kernels (tiles) for given
// elements-per-thread choices; updates rpb/nblk_x/tx/ntx in the mirror.
pp_status build_fft_lists(pp_batch_s* B, int ept_x, int ept_y) {
  std::vector<int2> wx, wy;
  size_t sx = 0, sy = 0;
  for (int i = 0; i < B->n; ++i) {
    GridDev& d = B->h_dev[i];
    d.rpb = rows_per_block(d.g.nx, ept_x);
    const int nrows = d.g.nz * d.g.ny;
    d.nblk_x = (nrows + d.rpb - 1) / d.rpb;
    for (int b = 0; b < d.nblk_x; ++b) wx.push_back(make_int2(i, b));
    {  // buffer A, buffer B written padded, twiddle table
      const int nbuf = (d.rpb / 2) * d.g.nx;
      sx = std::max(sx, (size_t)(nbuf + fft_pad_elems(nbuf) + d.g.nx) * sizeof(float2));
    }
    d.tx = ffty_tile(d.g.ny, sizeof(float2), ept_y);
    d.ntx = (d.g.nxh + d.tx - 1) / d.tx;
    for (int b = 0; b < d.ntx * d.g.nz; ++b) wy.push_back(make_int2(i, b));
    {
      const int tsz = d.g.ny * d.tx;
      sy = std::max(sy, (size_t)(tsz + fft_pad_elems(tsz) + d.g.ny) * sizeof(float2));
    }
  }
  B->smem_x = sx;
  B->smem_y = sy;
  pp_status s;
  if ((s = upload_list(wx, &B->w_x, &B->n_x)) != PP_OK) return s;
  if ((s = upload_list(wy, &B->w_y, &B->n_y)) != PP_OK) return s;
  return cudaMemcpy(B->d_dev, B->h_dev, B->n * sizeof(GridDev), cudaMemcpyHostToDevice) == cudaSuccess
             ? PP_OK : PP_ERR_CUDA;
}

cudaError_t launch_pass(pp_batch_s* B, cudaStream_t s) {
  kb_resid<<<B->n_x, kThreads, B->smem_x, s>>>(B->d_dev, B->w_x);
  kb_check<<<B->n, 1024, 0, s>>>(B->d_dev, B->d_ctl, kExactEveryBatch);
  kb_ffty<-1><<<B->n_y, kThreads, B->smem_y, s>>>(B->d_dev, B->w_y);
  kb_tridiag<<<B->n_z, kTriThreads, 0, s>>>(B->d_dev, B->w_z);
  kb_ffty<1><<<B->n_y, kThreads, B->smem_y, s>>>(B->d_dev, B->w_y);
  kb_fftx_inv<<<B->n_x, kThreads, B->smem_x, s>>>(B->d_dev, B->w_x);
  return cudaGetLastError();
}

cudaError_t launch_pre(pp_batch_s* B, cudaStream_t s) {
  kb_init<<<(B->n + 127) / 128, 128, 0, s>>>(B->d_dev, B->n, B->d_ctl);
  kb_prep_faces<<<B->n_cells, kThreads, 0, s>>>(B->d_dev, B->w_cells);
  kb_prep_diag<<<B->n_cells, kThreads, 0, s>>>(B->d_dev, B->w_cells);
  kb_weighted_partial<<<B->n_cells, kThreads, 0, s>>>(B->d_dev, B->w_cells, 0);
  kb_finalize<<<B->n, 1024, 0, s>>>(B->d_dev, 0);
  kb_rhs_b<<<B->n_cells, kThreads, 0, s>>>(B->d_dev, B->w_cells);
  kb_finalize<<<B->n, 1024, 0, s>>>(B->d_dev, 2);
  kb_fill_p<<<B->n_cells, kThreads, 0, s>>>(B->d_dev, B->w_cells, 0);
  return cudaGetLastError();
}

cudaError_t launch_post(pp_batch_s* B, cudaStream_t s) {
  kb_fold<<<B->n_cells, kThreads, 0, s>>>(B->d_dev, B->w_cells);
  kb_weighted_partial<<<B->n_cells, kThreads, 0, s>>>(B->d_dev, B->w_cells, 1);
  kb_finalize<<<B->n, 1024, 0, s>>>(B->d_dev, 1);
  kb_fill_p<<<B->n_cells, kThreads, 0, s>>>(B->d_dev, B->w_cells, 1);
  kb_correct<<<B->n_cells, kThreads, 0, s>>>(B->d_dev, B->w_cells);
  return cudaGetLastError();
}

// Time `reps` launches of the transform kernels for each candidate and keep
// the fastest (x kernels and y kernels are chosen independently).
pp_status autotune(pp_batch_s* B) {
  const int cands[3] = {4, 8, 16};
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return PP_ERR_CUDA;
  float best_x = 1e30f, best_y = 1e30f;
  int bx = kEpt, by = kEpt;
  pp_status s = PP_OK;
  for (int ci = 0; ci < 3 && s == PP_OK; ++ci) {
    if ((s = build_fft_lists(B, cands[ci], cands[ci])) != PP_OK) break;
    kb_init<<<(B->n + 127) / 128, 128, 0, B->cap>>>(B->d_dev, B->n, B->d_ctl);
    for (int rep = 0; rep < 2; ++rep) {  // first repetition warms up
      float tx = 0.f, ty = 0.f;
      cudaEventRecord(a, B->cap);
      kb_resid<<<B->n_x, kThreads, B->smem_x, B->cap>>>(B->d_dev, B->w_x);
      kb_fftx_inv<<<B->n_x, kThreads, B->smem_x, B->cap>>>(B->d_dev, B->w_x);
      cudaEventRecord(b, B->cap);
      if (cudaEventSynchronize(b) != cudaSuccess) { s = PP_ERR_CUDA; break; }
      cudaEventElapsedTime(&tx, a, b);
      cudaEventRecord(a, B->cap);
      kb_ffty<-1><<<B->n_y, kThreads, B->smem_y, B->cap>>>(B->d_dev, B->w_y);
      kb_ffty<1><<<B->n_y, kThreads, B->smem_y, B->cap>>>(B->d_dev, B->w_y);
      cudaEventRecord(b, B->cap);
      if (cudaEventSynchronize(b) != cudaSuccess) { s = PP_ERR_CUDA; break; }
      cudaEventElapsedTime(&ty, a, b);
      if (rep == 1) {
        if (tx < best_x) { best_x = tx; bx = cands[ci]; }
        if (ty < best_y) { best_y = ty; by = cands[ci]; }
      }
    }
    if (cudaGetLastError() != cudaSuccess) s = PP_ERR_CUDA;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (s != PP_OK) return s;
  B->ept_x = bx;
  B->ept_y = by;
  return build_fft_lists(B, bx, by);
}

pp_status build_graph(pp_batch_s* B) {
  cudaGraph_t g_pre = nullptr, g_post = nullptr;
  PP_CK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = launch_pre(B, B->cap);
  cudaError_t e2 = cudaStreamEndCapture(B->cap, &g_pre);
  if (e != cudaSuccess || e2 != cudaSuccess) return PP_ERR_CUDA;
  PP_CK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
  e = launch_post(B, B->cap);
  e2 = cudaStreamEndCapture(B->cap, &g_post);
  if (e != cudaSuccess || e2 != cudaSuccess) return PP_ERR_CUDA;

  PP_CK(cudaGraphCreate(&B->graph, 0));
  PP_CK(cudaGraphConditionalHandleCreate(&B->handle, B->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNode_t n_pre, n_while, n_post;
  PP_CK(cudaGraphAddChildGraphNode(&n_pre, B->graph, nullptr, 0, g_pre));
  // cudaGraphNodeParams has no default constructor (union member); zeroed storage
  alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
  std::memset(cp_raw, 0, sizeof(cp_raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = B->handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  PP_CK(cudaGraphAddNode(&n_while, B->graph, &n_pre, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  PP_CK(cudaStreamBeginCaptureToGraph(B->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  e = launch_pass(B, B->cap);
  kb_loopctl<<<1, 1024, 0, B->cap>>>(B->d_dev, B->n, B->d_ctl, B->handle);
  e2 = cudaStreamEndCapture(B->cap, &body);
  if (e != cudaSuccess || e2 != cudaSuccess || cudaGetLastError() != cudaSuccess) return PP_ERR_CUDA;
  PP_CK(cudaGraphAddChildGraphNode(&n_post, B->graph, &n_while, 1, g_post));
  cudaGraphDestroy(g_pre);
  cudaGraphDestroy(g_post);
  PP_CK(cudaGraphInstantiate(&B->exec, B->graph, 0));
  return PP_OK;
}

struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t at = off;
    off = (off + bytes + 255) & ~(size_t)255;
    return at;
  }
};

}  // namespace

extern "C" {

pp_status pressure_batch_create(const pp_grid* grids, int ngrids, pp_precision prec, void* stream,
                                pp_batch* out) {
  if (!grids || ngrids < 1 || !out) return PP_ERR_INVALID_ARG;
  if (prec != PP_MIXED_FP32) return PP_ERR_UNSUPPORTED;
  *out = nullptr;
  for (int i = 0; i < ngrids; ++i) {
    const pp_grid& G = grids[i];
    if (G.nx < 2 || G.ny < 1 || G.nz < 1 || !(G.lx > 0) || !(G.ly > 0) || !(G.lz > 0)) return PP_ERR_INVALID_ARG;
    if (G.bc[0] != PP_BC_PERIODIC || (G.bc[1] != PP_BC_PERIODIC && G.bc[1] != PP_BC_WALL) ||
        G.bc[2] != PP_BC_WALL)
      return PP_ERR_UNSUPPORTED;
    if (G.yfaces != nullptr) return PP_ERR_UNSUPPORTED;
    // walls in y: the cosine transform runs as one complex FFT of even length
    if (G.bc[1] == PP_BC_WALL && (G.ny < 2 || (G.ny & 1) != 0)) return PP_ERR_UNSUPPORTED;
    if ((G.nx & 1) != 0 || G.nx > 2048 || G.ny > 2048) return PP_ERR_UNSUPPORTED;
    if ((long long)G.nx * G.ny * (G.nz + 1) > (1LL << 31)) return PP_ERR_UNSUPPORTED;  // 32-bit cell offsets
    FftDesc t;
    if (!factor(G.nx, &t) || !factor(G.ny, &t)) return PP_ERR_UNSUPPORTED;
    if (G.zfaces && !faces_ok(G.zfaces, G.nz)) return PP_ERR_INVALID_ARG;
  }
  pp_batch_s* B = new (std::nothrow) pp_batch_s();
  if (!B) return PP_ERR_OOM;
  B->n = ngrids;
  B->stream = (cudaStream_t)stream;
  B->grids.assign(grids, grids + ngrids);
  if (cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost((void**)&B->h_dev, ngrids * sizeof(GridDev)) != cudaSuccess ||
      cudaMallocHost((void**)&B->h_ctl, sizeof(BatchCtl)) != cudaSuccess ||
      cudaMallocHost((void**)&B->h_st, ngrids * sizeof(DevStatus)) != cudaSuccess ||
      cudaMalloc((void**)&B->d_dev, ngrids * sizeof(GridDev)) != cudaSuccess ||
      cudaMalloc((void**)&B->d_ctl, sizeof(BatchCtl)) != cudaSuccess) {
    free_batch(B);
    return PP_ERR_OOM;
  }
  std::memset(B->h_dev, 0, ngrids * sizeof(GridDev));

  // pool layout: per grid, every buffer and table
  struct Off {
    size_t spec, E, delta, sdelta, b, red, st, cx, cy, cz, diag, rhof, invd, mtab,
        twx, twy, dcty, idzf, idzc, dzf, za, zc, idzff, cwf, lamx, lamy, mtabf, invdf, zcf;
  };
  std::vector<Off> off(ngrids);
  Carve cv;
  B->cell_off.resize(ngrids);
  B->wface_off.resize(ngrids);
  for (int i = 0; i < ngrids; ++i) {
    const pp_grid& G = grids[i];
    const size_t nc = (size_t)G.nx * G.ny * G.nz, nw = (size_t)G.nx * G.ny * (G.nz + 1);
    const size_t nsp = (size_t)(G.nx / 2 + 1) * G.ny * G.nz;
    const size_t nchunk = (nc + kChunk - 1) / kChunk;
    const size_t nred = std::max(nchunk, (size_t)G.ny * G.nz + 2);
    B->cell_off[i] = B->ncell_tot;
    B->wface_off[i] = B->nwface_tot;
    B->ncell_tot += (long long)nc;
    B->nwface_tot += (long long)nw;
    Off& o = off[i];
    // E is FP32; it gets 8 bytes a cell to double as the stand-in p of the tuning runs
    o.spec = cv.take(nsp * sizeof(float2)); o.E = cv.take(nc * 8); o.delta = cv.take(nc * 4);
    o.sdelta = cv.take(nc * 4);
    o.b = cv.take(nc * 8); o.red = cv.take(nred * 8); o.st = cv.take(sizeof(DevStatus));
    o.cx = cv.take(nc * 8); o.cy = cv.take(nc * 8); o.cz = cv.take(nw * 8); o.diag = cv.take(nc * 8);
    o.rhof = cv.take(nc * 4);
    o.invd = cv.take(nsp * 8); o.mtab = cv.take(nsp * 8);
    o.twx = cv.take((size_t)G.nx * sizeof(float2)); o.twy = cv.take((size_t)G.ny * sizeof(float2));
    o.dcty = cv.take((size_t)G.ny * sizeof(float2));
    o.idzf = cv.take((size_t)G.nz * 8); o.idzc = cv.take((size_t)(G.nz + 1) * 8); o.dzf = cv.take((size_t)G.nz * 8);
    o.za = cv.take((size_t)G.nz * 8); o.zc = cv.take((size_t)G.nz * 8); o.idzff = cv.take((size_t)G.nz * 4);
    o.cwf = cv.take(3 * (size_t)(G.nz + 1) * 4);
    o.lamx = cv.take((size_t)(G.nx / 2 + 1) * 8); o.lamy = cv.take((size_t)G.ny * 8);
    o.mtabf = cv.take(nsp * 4); o.invdf = cv.take(nsp * 4); o.zcf = cv.take((size_t)G.nz * 4);
  }
  if (cudaMalloc((void**)&B->pool, cv.off) != cudaSuccess) { free_batch(B); return PP_ERR_OOM; }
  if (cudaMemset(B->pool, 0, cv.off) != cudaSuccess) { free_batch(B); return PP_ERR_CUDA; }

  std::vector<int2> wc, wz;
  std::vector<int> low_all;     // ill-conditioned z columns of every grid, concatenated
  std::vector<size_t> low_off;
  const double pi = 3.14159265358979323846264338327950288;
  const double two_pi = 2.0 * pi;
  for (int i = 0; i < ngrids; ++i) {
    const pp_grid& G = grids[i];
    const Off& o = off[i];
    unsigned char* P = B->pool;
    GridDev& d = B->h_dev[i];
    const int nx = G.nx, ny = G.ny, nz = G.nz, nxh = nx / 2 + 1;
    std::vector<double> zf(nz + 1);
    for (int k = 0; k <= nz; ++k) zf[k] = G.zfaces ? G.zfaces[k] : G.lz * (double)k / (double)nz;  // checked above
    std::vector<double> dzf(nz), idzf(nz), zcen(nz), idzc(nz + 1, 0.0), za(nz, 0.0), zc(nz, 0.0);
    std::vector<float> idzff(nz), zcf(nz);
    for (int k = 0; k < nz; ++k) {
      dzf[k] = zf[k + 1] - zf[k];
      idzf[k] = 1.0 / dzf[k];
      idzff[k] = (float)idzf[k];
      zcen[k] = 0.5 * (zf[k] + zf[k + 1]);
    }
    for (int k = 1; k < nz; ++k) idzc[k] = 1.0 / (zcen[k] - zcen[k - 1]);
    for (int k = 1; k < nz; ++k) za[k] = idzc[k] * idzf[k];
    for (int k = 0; k < nz - 1; ++k) zc[k] = idzc[k + 1] * idzf[k];
    double dmax = 0.0;
    for (int k = 0; k < nz; ++k) { zcf[k] = (float)zc[k]; dmax = std::max(dmax, za[k] + zc[k]); }
    const double dx = G.lx / nx, dy = G.ly / ny;
    std::vector<double> lamx(nxh), lamy(ny);
    for (int k = 0; k < nxh; ++k) { const double sn = std::sin(pi * k / nx); lamx[k] = -4.0 / (dx * dx) * sn * sn; }
    // walls in y: the eigenvalues of the Neumann second difference on the
    // cosine modes cos(pi k (j + 1/2) / ny)
    const bool ywall = G.bc[1] == PP_BC_WALL;
    for (int k = 0; k < ny; ++k) {
      const double sn = std::sin(pi * k / (ywall ? 2.0 * ny : (double)ny));
      lamy[k] = -4.0 / (dy * dy) * sn * sn;
    }
    std::vector<float2> dcty(ny);
    for (int m = 0; m < ny; ++m)
      dcty[m] = make_float2((float)std::cos(pi * m / (2.0 * ny)), (float)(-std::sin(pi * m / (2.0 * ny))));
    const std::vector<float> cwf = layer_factors_f32(nz, dzf, idzc, 1.0 / (dx * dx), 1.0 / (dy * dy));
    std::vector<float2> twx(nx), twy(ny);
    for (int m = 0; m < nx; ++m) twx[m] = make_float2((float)std::cos(two_pi * m / nx), (float)std::sin(two_pi * m / nx));
    for (int m = 0; m < ny; ++m) twy[m] = make_float2((float)std::cos(two_pi * m / ny), (float)std::sin(two_pi * m / ny));
    struct Up { size_t off; const void* src; size_t bytes; } ups[] = {
        {o.twx, twx.data(), twx.size() * sizeof(float2)}, {o.twy, twy.data(), twy.size() * sizeof(float2)},
        {o.dzf, dzf.data(), dzf.size() * 8}, {o.idzf, idzf.data(), idzf.size() * 8},
        {o.idzc, idzc.data(), idzc.size() * 8}, {o.za, za.data(), za.size() * 8}, {o.zc, zc.data(), zc.size() * 8},
        {o.idzff, idzff.data(), idzff.size() * 4}, {o.lamx, lamx.data(), lamx.size() * 8},
        {o.lamy, lamy.data(), lamy.size() * 8}, {o.zcf, zcf.data(), zcf.size() * 4},
        {o.cwf, cwf.data(), cwf.size() * 4}, {o.dcty, dcty.data(), dcty.size() * sizeof(float2)}};
    for (const Up& u : ups)
      if (cudaMemcpy(P + u.off, u.src, u.bytes, cudaMemcpyHostToDevice) != cudaSuccess) { free_batch(B); return PP_ERR_CUDA; }
    Geo& g = d.g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.nxh = nxh; g.dx = dx; g.dy = dy;
    g.inv_dx2 = 1.0 / (dx * dx); g.inv_dy2 = 1.0 / (dy * dy);
    g.inv_dzf = (const double*)(P + o.idzf); g.inv_dzc = (const double*)(P + o.idzc);
    g.dzf = (const double*)(P + o.dzf); g.za = (const double*)(P + o.za); g.zc = (const double*)(P + o.zc);
    g.inv_dzf_f = (const float*)(P + o.idzff); g.cw_f = (const float*)(P + o.cwf); g.lz = zf[nz] - zf[0];
    g.ywall = ywall ? 1 : 0;
    g.ym = nullptr;
    g.ym_f = nullptr;
    d.fc.cx = (double*)(P + o.cx); d.fc.cy = (double*)(P + o.cy); d.fc.cz = (double*)(P + o.cz);
    d.fc.diag = (double*)(P + o.diag); d.fc.rhof = (float*)(P + o.rhof);
    factor(nx, &d.fx);
    factor(ny, &d.fy);
    d.twx = (const float2*)(P + o.twx); d.twy = (const float2*)(P + o.twy);
    d.dcty = ywall ? (const float2*)(P + o.dcty) : nullptr;
    d.invd = (const double*)(P + o.invd); d.mtab = (const double*)(P + o.mtab);
    d.spec = (float2*)(P + o.spec); d.E = (float*)(P + o.E); d.delta = (float*)(P + o.delta);
    d.sdelta = (float*)(P + o.sdelta);
    d.b = (double*)(P + o.b); d.red = (double*)(P + o.red); d.st = (DevStatus*)(P + o.st);
    d.ncell = (long long)nx * ny * nz;
    d.nchunk = (int)((d.ncell + kChunk - 1) / kChunk);
    d.scale = 1.0 / ((double)nx * ny);
    for (int c = 0; c < d.nchunk; ++c) wc.push_back(make_int2(i, c));
    const size_t ncol = (size_t)nxh * ny;
    const std::vector<int> lowi = tri_low_columns(lamx, lamy, 2.0 * dmax / 512.0);
    low_off.push_back(low_all.size());
    low_all.insert(low_all.end(), lowi.begin(), lowi.end());
    d.tri.nlow = (int)lowi.size();
    for (int b = 0; b < tri_mixed_blocks(ncol, d.tri.nlow); ++b) wz.push_back(make_int2(i, b));
    const size_t nsp = (size_t)nxh * ny * nz;
    if (launch_setup_pivots(g, (const double*)(P + o.lamx), (const double*)(P + o.lamy), (double*)(P + o.invd),
                            B->cap, (double*)(P + o.mtab)) != cudaSuccess ||
        launch_narrow((const double*)(P + o.mtab), (float*)(P + o.mtabf), nsp, B->cap) != cudaSuccess ||
        launch_narrow((const double*)(P + o.invd), (float*)(P + o.invdf), nsp, B->cap) != cudaSuccess) {
      free_batch(B);
      return PP_ERR_CUDA;
    }
    d.tri.mtab = (const float*)(P + o.mtabf);
    d.tri.invd = (const float*)(P + o.invdf);
    d.tri.zc = (const float*)(P + o.zcf);
    d.tri.lamx = (const double*)(P + o.lamx);
    d.tri.lamy = (const double*)(P + o.lamy);
    d.tri.thr = 2.0 * dmax / 512.0;
    // stand-ins for the per-call pointers while tuning: plan-owned, zeroed
    d.p = (double*)(P + o.E); d.rho = d.b; d.us = d.vs = d.b; d.ws = d.fc.cz; d.S = nullptr; d.u = d.v = d.w = nullptr;
    d.dt = 1.0; d.inv_dt = 1.0;
  }
  if (cudaMalloc((void**)&B->d_low, low_all.size() * sizeof(int)) != cudaSuccess) { free_batch(B); return PP_ERR_OOM; }
  if (cudaMemcpy(B->d_low, low_all.data(), low_all.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    free_batch(B);
    return PP_ERR_CUDA;
  }
  for (int i = 0; i < ngrids; ++i) B->h_dev[i].tri.low = B->d_low + low_off[i];
  pp_status s;
  if ((s = upload_list(wc, &B->w_cells, &B->n_cells)) != PP_OK || (s = upload_list(wz, &B->w_z, &B->n_z)) != PP_OK) {
    free_batch(B);
    return s;
  }
  // largest tuning candidate + the largest twiddle table
  const int smem_max = (int)((16 * kThreads + fft_pad_elems(16 * kThreads) + 2048) * sizeof(float2));
  if (cudaFuncSetAttribute(kb_resid, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) != cudaSuccess ||
      cudaFuncSetAttribute(kb_fftx_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) != cudaSuccess ||
      cudaFuncSetAttribute(kb_ffty<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) != cudaSuccess ||
      cudaFuncSetAttribute(kb_ffty<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) != cudaSuccess ||
      cudaStreamSynchronize(B->cap) != cudaSuccess) {
    free_batch(B);
    return PP_ERR_CUDA;
  }
  if ((s = autotune(B)) != PP_OK || (s = build_graph(B)) != PP_OK) { free_batch(B); return s; }
  if (cudaStreamSynchronize(B->cap) != cudaSuccess) { free_batch(B); return PP_ERR_CUDA; }
  *out = B;
  return PP_OK;
}

pp_status pressure_batch_destroy(pp_batch B) {
  if (!B) return PP_ERR_INVALID_ARG;
  cudaStreamSynchronize(B->stream);
  cudaStreamSynchronize(B->cap);
  free_batch(B);
  return PP_OK;
}

pp_status pressure_batch_layout(pp_batch B, long long* cell_offset, long long* wface_offset,
                                long long* totals, int* tiles) {
  if (!B) return PP_ERR_INVALID_ARG;
  for (int i = 0; i < B->n; ++i) {
    if (cell_offset) cell_offset[i] = B->cell_off[i];
    if (wface_offset) wface_offset[i] = B->wface_off[i];
  }
  if (totals) { totals[0] = B->ncell_tot; totals[1] = B->nwface_tot; }
  if (tiles) { tiles[0] = B->ept_x; tiles[1] = B->ept_y; }
  return PP_OK;
}

pp_status pressure_batch_mixture_density(pp_batch B, const double* phi, double rho_g, double rho_l,
                                         double* rho) {
  if (!B || !phi || !rho || !is_device(phi) || !is_device(rho)) return PP_ERR_INVALID_ARG;
  PP_CK(launch_mixture(phi, rho_g, rho_l, rho, (size_t)B->ncell_tot, B->stream));
  return PP_OK;
}

pp_status pressure_batch_correct(pp_batch B, const double* us, const double* vs, const double* ws,
                                 const double* rho, const double* S, double dt, double* p, double* u,
                                 double* v, double* w, double rtol, int maxit, pp_info* infos) {
  if (!B || !us || !vs || !ws || !rho || !p || !u || !v || !w) return PP_ERR_INVALID_ARG;
  if (!(dt > 0.0) || !(rtol >= 0.0) || maxit < 0) return PP_ERR_INVALID_ARG;
  const void* ptrs[] = {us, vs, ws, rho, p, u, v, w};
  for (const void* q : ptrs)
    if (!is_device(q)) return PP_ERR_INVALID_ARG;
  if (S && !is_device(S)) return PP_ERR_INVALID_ARG;
  for (int i = 0; i < B->n; ++i) {
    GridDev& d = B->h_dev[i];
    const long long co = B->cell_off[i], wo = B->wface_off[i];
    d.us = us + co; d.vs = vs + co; d.ws = ws + wo; d.rho = rho + co; d.S = S ? S + co : nullptr;
    d.p = p + co; d.u = u + co; d.v = v + co; d.w = w + wo;
    d.dt = dt; d.inv_dt = 1.0 / dt;
  }
  B->h_ctl->rtol = rtol;
  B->h_ctl->maxit = maxit;
  B->h_ctl->passes = 0;
  B->h_ctl->active = 1;
  PP_CK(cudaMemcpyAsync(B->d_dev, B->h_dev, B->n * sizeof(GridDev), cudaMemcpyHostToDevice, B->stream));
  PP_CK(cudaMemcpyAsync(B->d_ctl, B->h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, B->stream));
  PP_CK(cudaGraphLaunch(B->exec, B->stream));
  for (int i = 0; i < B->n; ++i)
    PP_CK(cudaMemcpyAsync(&B->h_st[i], B->h_dev[i].st, sizeof(DevStatus), cudaMemcpyDeviceToHost, B->stream));
  PP_CK(cudaStreamSynchronize(B->stream));
  pp_status worst = PP_OK;
  for (int i = 0; i < B->n; ++i) {
    const DevStatus& s = B->h_st[i];
    if (infos) {
      infos[i].iters = s.iters;
      infos[i].res0 = std::sqrt(s.e2_0) * dt;
      infos[i].res_final = s.rel;
      infos[i].res_l1_sum = s.e1 * dt;
      infos[i].mean_S_removed = s.mean_S;
      infos[i].status = s.code;
    }
    if (s.code != PP_OK && worst == PP_OK) worst = (pp_status)s.code;
  }
  return worst;
}

}  // extern "C"
