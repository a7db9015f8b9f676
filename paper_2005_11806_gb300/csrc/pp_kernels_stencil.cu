// Stencil, reduction and set-up kernels of the projection: mixture density
// (Eq. 22), face coefficients, the loop-invariant right-hand side of
// Algorithm 1, its loop control, the correction step (Eq. corr), the gauge
// removal, the adjoint stencils and the Thomas pivots of the z solve.
#include "pp_cells.cuh"

namespace pp {

namespace {
constexpr int kRedBlocks = 1024;  // partial sums written by the reduction kernels
constexpr int kThreads = 256;

inline int grid_for(size_t n) {
  size_t b = (n + kThreads - 1) / kThreads;
  if (b > (size_t)152 * 64) b = (size_t)152 * 64;
  return (int)(b == 0 ? 1 : b);
}
}  // namespace

int reduce_blocks() { return kRedBlocks; }

__global__ void k_mixture(const double* __restrict__ phi, double rho_g, double rho_l,
                          double* __restrict__ rho, size_t n) {
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const double f = phi[c];
    rho[c] = rho_g * f + rho_l * (1.0 - f);
  }
}

// beta on every face: arithmetic face density, beta = 2 / (rho_a + rho_b);
// x/y coefficients carry the width dzf_k of their layer (row scaling).
__global__ void k_prep_faces(Geo g, const double* __restrict__ rho, Faces fc) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    cell_prep_faces(g, rho, fc, c);
}

// diag = sum of the six (row-scaled) coefficients of each cell.
__global__ void k_prep_diag(Geo g, Faces fc) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    cell_prep_diag(g, fc, c);
}

// Fixed-order partial sums of dzf_k * f (dzf_k s_j * f on a stretched y:
// the cell volume over dx dy) (grid of kRedBlocks blocks).
__global__ void k_weighted_partial(Geo g, const double* __restrict__ f, double* __restrict__ red) {
  __shared__ double sh[32];
  const size_t plane = (size_t)g.nx * g.ny, n = plane * g.nz;
  double s = 0.0;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const double wy = g.ym ? g.ym[(c / g.nx) % g.ny] : 1.0;
    s += g.dzf[c / plane] * wy * f[c];
  }
  s = block_sum<double>(s, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = s;
}

// out = scale * sum_b red[b * stride + off]
__global__ void k_finalize(const double* __restrict__ red, int nblk, int stride, int off, double scale,
                           double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += red[(size_t)b * stride + off];
  s = block_sum<double>(s, sh);
  if (threadIdx.x == 0) *out = scale * s;
}

// b_s = dzf_k (D u* - (S - <S>_V)) / dt (row-scaled); wall values of w* are
// taken as zero; block partial sums of (D u* - S_c)^2.
__global__ void k_rhs_b(Geo g, const double* __restrict__ us, const double* __restrict__ vs,
                        const double* __restrict__ ws, const double* __restrict__ S,
                        const DevStatus* __restrict__ st, double* __restrict__ b,
                        double* __restrict__ red, double inv_dt) {
  __shared__ double sh[32];
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  const double meanS = st->mean_S;
  double s2 = 0.0;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const double d = cell_rhs_b(g, us, vs, ws, S, meanS, b, inv_dt, c);
    s2 += d * d;
  }
  s2 = block_sum<double>(s2, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = s2;
}

__global__ void k_init_status(DevStatus* st) { status_init(st); }

// Loop control of Algorithm 1: reduce the residual partial sums, decide.
__global__ void k_check(DevStatus* st, const double* __restrict__ red, int nblk, double rtol, int maxit,
                        int kexact) {
  __shared__ double sh[32];
  if (st->done) return;
  double s2 = 0.0, s1 = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    s2 += red[2 * (size_t)b];
    s1 += red[2 * (size_t)b + 1];
  }
  s2 = block_sum<double>(s2, sh);
  s1 = block_sum<double>(s1, sh);
  if (threadIdx.x != 0) return;
  status_update(st, s2, s1, rtol, maxit, kexact);
}

// u = u* - dt beta G p  (Eq. corr); w wall planes are written as zero.
__global__ void k_correct(Geo g, Faces fc, const double* __restrict__ us, const double* __restrict__ vs,
                          const double* __restrict__ ws, const double* __restrict__ p, double dt,
                          double* __restrict__ u, double* __restrict__ v, double* __restrict__ w) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    cell_correct(g, fc, us, vs, ws, p, dt, u, v, w, c);
}

__global__ void k_sub_mean(double* __restrict__ p, size_t n, const DevStatus* __restrict__ st) {
  const double m = st->pmean;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    p[c] -= m;
}

// Inverse Thomas pivots of (L_z + lambda_x(kx) + lambda_y(ky)) per column.
__global__ void k_setup_pivots(Geo g, const double* __restrict__ lamx, const double* __restrict__ lamy,
                               double* __restrict__ invd, double* __restrict__ mtab) {
  const size_t ncol = (size_t)g.ny * g.nxh;
  const size_t col = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  const int j = (int)(col / g.nxh), kx = (int)(col % g.nxh);
  const double lam = lamx[kx] + lamy[j];
  double d = -(g.za[0] + g.zc[0]) + lam;
  if (mtab != nullptr) mtab[col] = 0.0;
  if (col == 0 && g.nz == 1) { invd[0] = 0.0; return; }
  invd[col] = 1.0 / d;
  for (int k = 1; k < g.nz; ++k) {
    const double dinv_prev = invd[(size_t)(k - 1) * ncol + col];
    if (mtab != nullptr) mtab[(size_t)k * ncol + col] = g.za[k] * dinv_prev;
    d = (-(g.za[k] + g.zc[k]) + lam) - g.za[k] * g.zc[k - 1] / d;
    const bool pin = (col == 0 && k == g.nz - 1);  // singular (0, 0) column: pin the last unknown
    invd[(size_t)k * ncol + col] = pin ? 0.0 : 1.0 / d;
  }
}

// Tables of the PP_MIXED_Z64 z solve (TriZ64), one thread per table column
// tc = ky' nxh + kx with lambda = lambda_x(kx) + lambda_y(ky'): the same
// pivot recurrence as k_setup_pivots, stored as m_k = a_k / d_{k-1},
// e_k = c_k / d_k (FP64) and 1 / d_k (FP32).  Column 0 is the singular
// (0, 0) system: its last inverse pivot is 0.
__global__ void k_setup_z64(Geo g, const double* __restrict__ lamx, const double* __restrict__ lamy, int nyt,
                            double* __restrict__ m, double* __restrict__ e, float* __restrict__ dinv) {
  const size_t ntc = (size_t)nyt * g.nxh;
  const size_t tc = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tc >= ntc) return;
  const int j = (int)(tc / g.nxh), kx = (int)(tc % g.nxh);
  const double lam = lamx[kx] + lamy[j];
  double d = -(g.za[0] + g.zc[0]) + lam;
  double inv_prev = 0.0;
  for (int k = 0; k < g.nz; ++k) {
    if (k > 0) d = (-(g.za[k] + g.zc[k]) + lam) - g.za[k] * g.zc[k - 1] / d;
    const bool pin = (tc == 0 && k == g.nz - 1);  // singular (0, 0) column: pin the last unknown
    const double inv = pin ? 0.0 : 1.0 / d;
    const size_t o = (size_t)k * ntc + tc;
    m[o] = (k == 0) ? 0.0 : g.za[k] * inv_prev;
    e[o] = (k + 1 < g.nz) ? g.zc[k] * inv : 0.0;
    dinv[o] = (float)inv;
    inv_prev = inv;
  }
}

// ---- Methods I and II (Sec. 3.3.1) -------------------------------------------
constexpr int kExtBlocks = kRedBlocks / 2;  // (min, max) pairs fit the partial-sum buffer

// Block partial minimum and maximum of rho into red[2 b], red[2 b + 1].
__global__ void k_rho_extrema(size_t n, const double* __restrict__ rho, double* __restrict__ red) {
  __shared__ double smin[kThreads / 32], smax[kThreads / 32];
  double lo = INFINITY, hi = -INFINITY;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const double r = rho[c];
    lo = fmin(lo, r);
    hi = fmax(hi, r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { smin[wid] = lo; smax[wid] = hi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { lo = fmin(lo, smin[k]); hi = fmax(hi, smax[k]); }
    red[2 * (size_t)blockIdx.x] = lo;
    red[2 * (size_t)blockIdx.x + 1] = hi;
  }
}

// rho0 = min rho (Method I, Eq. poisson_me1); the harmonic mean
// 2 rho_min rho_max / (rho_min + rho_max) of the two phase densities
// (Method II, Eq. poisson_laizet).  One thread.
__global__ void k_rho_tilde(const double* __restrict__ red, int nblk, int method, double* __restrict__ out) {
  double lo = INFINITY, hi = -INFINITY;
  for (int b = 0; b < nblk; ++b) {
    lo = fmin(lo, red[2 * (size_t)b]);
    hi = fmax(hi, red[2 * (size_t)b + 1]);
  }
  *out = (method == 1) ? lo : 2.0 * lo * hi / (lo + hi);
}

// Eq. poisson_me2 with p^q = p - delta:
//   u = u* - dt beta G p + dt (beta - 1/rho0) G delta  on every face.
// beta is recovered from the row-scaled coefficients: cx = dzf_k beta / dx^2,
// cy = dzf_k beta / dy^2, cz = beta / dzc.
template <typename T>
__global__ void k_correct_method1(Geo g, Faces fc, const double* __restrict__ us,
                                  const double* __restrict__ vs, const double* __restrict__ ws,
                                  const double* __restrict__ p, const T* __restrict__ delta, double dt,
                                  double* __restrict__ u, double* __restrict__ v, double* __restrict__ w) {
  const size_t plane = (size_t)g.nx * g.ny, n = plane * g.nz;
  const double ir0 = 1.0 / *fc.rho_tilde;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    cell_correct(g, fc, us, vs, ws, p, dt, u, v, w, c);
    const CellIdx x = cell_index(g, c);
    const double idzf = g.inv_dzf[x.k];
    const double dc = (double)delta[c];
    // stretched y: cx, cz carry s_j and cy carries t_j = dy / dyc_j (t_0 = 0
    // on the walls, where v is not corrected)
    const double is = g.ym ? g.ym[2 * g.ny + x.j] : 1.0;
    const double tj = g.ym ? g.ym[g.ny + x.j] : 1.0;
    const double bx = fc.cx[c] * idzf * is / g.inv_dx2;
    u[c] += dt * (bx - ir0) * (dc - (double)delta[x.cim]) / g.dx;
    if (!(g.ywall && x.j == 0)) {
      const double by = fc.cy[c] * idzf / (g.inv_dy2 * tj);
      v[c] += dt * (by - ir0) * (dc - (double)delta[x.cjm]) * tj / g.dy;
    }
    if (x.k > 0) w[c] += dt * (fc.cz[c] * is - ir0 * g.inv_dzc[x.k]) * (dc - (double)delta[c - plane]);
  }
}

// ---- divergence source from the thermodynamics (Eqs. 30, 34, v_gas) ----------

// Block partial sums of Phi div(k grad T) dV, Phi div(u) dV and Phi dV into
// red[3 b + {0, 1, 2}] (wall values of w taken as zero).
__global__ void k_thermo_partial(Geo g, const double* __restrict__ phi, const double* __restrict__ kc,
                                 const double* __restrict__ T, const double* __restrict__ u,
                                 const double* __restrict__ v, const double* __restrict__ w,
                                 double* __restrict__ red) {
  __shared__ double sh[32];
  const size_t plane = (size_t)g.nx * g.ny, n = plane * g.nz;
  const double dxdy = g.dx * g.dy;
  double a = 0.0, b = 0.0, vg = 0.0;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const CellIdx x = cell_index(g, c);
    const double f = phi[c];
    const double sj = g.ym ? g.ym[x.j] : 1.0;  // stretched y: dyf_j = s_j dy
    const double dv = dxdy * g.dzf[x.k] * sj;
    const double wlo = (x.k == 0) ? 0.0 : w[c];
    const double whi = (x.k == g.nz - 1) ? 0.0 : w[c + plane];
    // the wall row of v (walls in y) carries no flux, like the wall planes of w
    const double vlo = (g.ywall && x.j == 0) ? 0.0 : v[c];
    const double vhi = (g.ywall && x.j == g.ny - 1) ? 0.0 : v[x.cjp];
    const double div = (u[x.cip] - u[c]) / g.dx + (vhi - vlo) / (g.dy * sj) + (whi - wlo) * g.inv_dzf[x.k];
    a += f * cell_conduction(g, kc, T, c) * dv;
    b += f * div * dv;
    vg += f * dv;
  }
  a = block_sum<double>(a, sh);
  __syncthreads();
  b = block_sum<double>(b, sh);
  __syncthreads();
  vg = block_sum<double>(vg, sh);
  if (threadIdx.x == 0) {
    red[3 * (size_t)blockIdx.x] = a;
    red[3 * (size_t)blockIdx.x + 1] = b;
    red[3 * (size_t)blockIdx.x + 2] = vg;
  }
}

// out = {sum a, sum b, V_g, RP} with RP of Eq. 30 (RP = NaN when V_g = 0).
__global__ void k_thermo_rate(const double* __restrict__ red, int nblk, double p0, double gamma,
                              double* __restrict__ out) {
  __shared__ double sh[32];
  double s[3];
  for (int q = 0; q < 3; ++q) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) t += red[3 * (size_t)b + q];
    s[q] = block_sum<double>(t, sh);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s[0];
    out[1] = s[1];
    out[2] = s[2];
    out[3] = (s[2] > 0.0) ? gamma / s[2] * ((gamma - 1.0) / gamma * s[0] - p0 * s[1]) : NAN;
  }
}

// S = (1/p0) [ (gamma - 1)/gamma div(k grad T) - dp0dt / gamma ] Phi  (Eq. 34).
__global__ void k_divergence_source(Geo g, const double* __restrict__ phi, const double* __restrict__ kc,
                                    const double* __restrict__ T, double p0, double gamma, double dp0dt,
                                    double* __restrict__ S) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  const double a = (gamma - 1.0) / gamma, b = dp0dt / gamma, ip0 = 1.0 / p0;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    S[c] = (a * cell_conduction(g, kc, T, c) - b) * phi[c] * ip0;
}

// ---- momentum predictor (Eqs. 29, 32) ---------------------------------------

__global__ void k_cell_divergence(Geo g, const double* __restrict__ u, const double* __restrict__ v,
                                  const double* __restrict__ w, double* __restrict__ D) {
  const size_t plane = (size_t)g.nx * g.ny, n = plane * g.nz;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const CellIdx x = cell_index(g, c);
    // walls in y: the wall row of v carries no flux
    const double vlo = (g.ywall && x.j == 0) ? 0.0 : v[c];
    const double vhi = (g.ywall && x.j == g.ny - 1) ? 0.0 : v[x.cjp];
    D[c] = (u[x.cip] - u[c]) / g.dx + (vhi - vlo) / g.dy + (w[c + plane] - w[c]) * g.inv_dzf[x.k];
  }
}

// Predicted velocity at the three low faces of cell (i, j, k): the u-face
// i-1/2, the v-face j-1/2 and (k >= 1) the w-face k-1/2.  RU = -C(u) +
// (1/rho_f)[div tau + f] + g with C(u) = div(u u) - u div(u) (central
// divergence form: normal products at cell centres, cross products at edges,
// a velocity carried to an edge by the mean of its two values) and the
// Newton-Stokes stress (normal parts at cell centres with the cell's mu,
// shear parts at edges with the mean mu of the cells around the edge;
// no-slip z walls: wall velocity zero, half-cell distance to the wall).
// With walls in y the y walls are no-slip too: the wall row of v is zero
// (read as zero, written as zero), the edges on y = 0 (edge row 0) and
// y = ly (edge row ny) carry the wall shear of u and w over half a cell and
// no convective flux, and the edges where a y wall meets a z wall carry
// nothing.  Edge rows are passed unwrapped (0 .. ny); periodic y wraps ny
// to 0.  u* = u + dt (a RU - b RU_prev).  D: cell divergence.
__global__ void k_predictor(Geo g, const double* __restrict__ u, const double* __restrict__ v,
                            const double* __restrict__ w, const double* __restrict__ rho,
                            const double* __restrict__ mu, const double* __restrict__ D,
                            const double* __restrict__ fx, const double* __restrict__ fy,
                            const double* __restrict__ fz, const double* __restrict__ pu,
                            const double* __restrict__ pv, const double* __restrict__ pw, double gx, double gy,
                            double gz, double dt, double a, double b, double* __restrict__ us,
                            double* __restrict__ vs, double* __restrict__ ws, double* __restrict__ ru,
                            double* __restrict__ rv, double* __restrict__ rw) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const bool ywall = g.ywall != 0;
  const size_t plane = (size_t)nx * ny, n = plane * nz;
  const double idx = 1.0 / g.dx, idy = 1.0 / g.dy;
  const double two3 = 2.0 / 3.0;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / plane);
    const int im = i == 0 ? nx - 1 : i - 1, ip = i + 1 == nx ? 0 : i + 1;
    const int jm = j == 0 ? ny - 1 : j - 1, jp = j + 1 == ny ? 0 : j + 1;
    auto at = [&](int ii, int jj, int kk) { return ((size_t)kk * ny + jj) * nx + ii; };
    // v at the face row jj (0 .. ny - 1); the wall row reads as zero
    auto vv = [&](int ii, int jj, int kk) { return (ywall && jj == 0) ? 0.0 : v[at(ii, jj, kk)]; };
    const double idzf = g.inv_dzf[k];
    // is the edge row jj (0 .. ny) a y wall?
    auto ywall_edge = [&](int jj) { return ywall && (jj == 0 || jj == ny); };
    // mean mu over the four cells around an x-y edge (i'-1/2, j'-1/2) of layer kk (interior edge row)
    auto mxy = [&](int ii, int jj, int kk) {
      const int iim = ii == 0 ? nx - 1 : ii - 1, jjm = jj == 0 ? ny - 1 : jj - 1;
      return 0.25 * (mu[at(ii, jj, kk)] + mu[at(iim, jj, kk)] + mu[at(ii, jjm, kk)] + mu[at(iim, jjm, kk)]);
    };
    // shear stress tau_xy at the edge (i'-1/2, jj-1/2) of layer kk, jj in [0, ny]
    auto txy = [&](int ii, int jj, int kk) {
      const int iim = ii == 0 ? nx - 1 : ii - 1;
      if (ywall_edge(jj)) {  // no-slip y wall: u = 0 half a cell away, v = 0 along it
        const int jr = jj == 0 ? 0 : ny - 1;
        const double m = 0.5 * (mu[at(ii, jr, kk)] + mu[at(iim, jr, kk)]);
        return (jj == 0 ? 2.0 : -2.0) * m * u[at(ii, jr, kk)] * idy;
      }
      const int jw = jj == ny ? 0 : jj, jjm = jw == 0 ? ny - 1 : jw - 1;
      return mxy(ii, jw, kk) * ((u[at(ii, jw, kk)] - u[at(ii, jjm, kk)]) * idy +
                                (vv(ii, jw, kk) - vv(iim, jw, kk)) * idx);
    };
    // tau_xz at the edge (i'-1/2, kk-1/2), kk in [0, nz]; tau_yz likewise
    auto txz = [&](int ii, int jj, int kk) {
      const int iim = ii == 0 ? nx - 1 : ii - 1;
      if (kk == 0) return 0.5 * (mu[at(ii, jj, 0)] + mu[at(iim, jj, 0)]) * u[at(ii, jj, 0)] * 2.0 * g.inv_dzf[0];
      if (kk == nz)
        return -0.5 * (mu[at(ii, jj, nz - 1)] + mu[at(iim, jj, nz - 1)]) * u[at(ii, jj, nz - 1)] * 2.0 *
               g.inv_dzf[nz - 1];
      const double m = 0.25 * (mu[at(ii, jj, kk)] + mu[at(iim, jj, kk)] + mu[at(ii, jj, kk - 1)] +
                               mu[at(iim, jj, kk - 1)]);
      return m * ((u[at(ii, jj, kk)] - u[at(ii, jj, kk - 1)]) * g.inv_dzc[kk] +
                  (w[at(ii, jj, kk)] - w[at(iim, jj, kk)]) * idx);
    };
    // tau_yz at the edge (jj-1/2, kk-1/2), jj in [0, ny], kk in [0, nz]
    auto tyz = [&](int ii, int jj, int kk) {
      if (ywall_edge(jj)) {  // no-slip y wall: w = 0 half a cell away, v = 0 along it
        if (kk == 0 || kk == nz) return 0.0;  // a y wall meets a z wall
        const int jr = jj == 0 ? 0 : ny - 1;
        const double m = 0.5 * (mu[at(ii, jr, kk)] + mu[at(ii, jr, kk - 1)]);
        return (jj == 0 ? 2.0 : -2.0) * m * w[at(ii, jr, kk)] * idy;
      }
      const int jw = jj == ny ? 0 : jj, jjm = jw == 0 ? ny - 1 : jw - 1;
      if (kk == 0) return 0.5 * (mu[at(ii, jw, 0)] + mu[at(ii, jjm, 0)]) * vv(ii, jw, 0) * 2.0 * g.inv_dzf[0];
      if (kk == nz)
        return -0.5 * (mu[at(ii, jw, nz - 1)] + mu[at(ii, jjm, nz - 1)]) * vv(ii, jw, nz - 1) * 2.0 *
               g.inv_dzf[nz - 1];
      const double m = 0.25 * (mu[at(ii, jw, kk)] + mu[at(ii, jjm, kk)] + mu[at(ii, jw, kk - 1)] +
                               mu[at(ii, jjm, kk - 1)]);
      return m * ((vv(ii, jw, kk) - vv(ii, jw, kk - 1)) * g.inv_dzc[kk] +
                  (w[at(ii, jw, kk)] - w[at(ii, jjm, kk)]) * idy);
    };
    // convective cross products at edges (zero on the walls, where the
    // wall-normal velocity vanishes)
    auto fxy = [&](int ii, int jj, int kk) {  // u v at (i'-1/2, jj-1/2), jj in [0, ny]
      if (ywall_edge(jj)) return 0.0;
      const int jw = jj == ny ? 0 : jj;
      const int iim = ii == 0 ? nx - 1 : ii - 1, jjm = jw == 0 ? ny - 1 : jw - 1;
      return 0.25 * (u[at(ii, jw, kk)] + u[at(ii, jjm, kk)]) * (vv(ii, jw, kk) + vv(iim, jw, kk));
    };
    auto fxz = [&](int ii, int jj, int kk) {  // u w at (i'-1/2, kk-1/2); zero at the walls
      if (kk == 0 || kk == nz) return 0.0;
      const int iim = ii == 0 ? nx - 1 : ii - 1;
      return 0.25 * (u[at(ii, jj, kk)] + u[at(ii, jj, kk - 1)]) * (w[at(ii, jj, kk)] + w[at(iim, jj, kk)]);
    };
    auto fyz = [&](int ii, int jj, int kk) {  // v w at (jj-1/2, kk-1/2), jj in [0, ny]
      if (kk == 0 || kk == nz || ywall_edge(jj)) return 0.0;
      const int jw = jj == ny ? 0 : jj, jjm = jw == 0 ? ny - 1 : jw - 1;
      return 0.25 * (vv(ii, jw, kk) + vv(ii, jw, kk - 1)) * (w[at(ii, jw, kk)] + w[at(ii, jjm, kk)]);
    };
    const double Dc = D[c];
    // ---- x momentum at the u-face (i-1/2, j, k)
    {
      const size_t cm = at(im, j, k);
      const double uc0 = 0.5 * (u[c] + u[at(ip, j, k)]), ucm = 0.5 * (u[cm] + u[c]);
      const double conv = (uc0 * uc0 - ucm * ucm) * idx + (fxy(i, j + 1, k) - fxy(i, j, k)) * idy +
                          (fxz(i, j, k + 1) - fxz(i, j, k)) * idzf - u[c] * 0.5 * (Dc + D[cm]);
      const double t0 = mu[c] * (2.0 * (u[at(ip, j, k)] - u[c]) * idx - two3 * Dc);
      const double tm = mu[cm] * (2.0 * (u[c] - u[cm]) * idx - two3 * D[cm]);
      double visc = (t0 - tm) * idx + (txy(i, j + 1, k) - txy(i, j, k)) * idy +
                    (txz(i, j, k + 1) - txz(i, j, k)) * idzf;
      if (fx != nullptr) visc += fx[c];
      const double r = -conv + visc / (0.5 * (rho[c] + rho[cm])) + gx;
      us[c] = u[c] + dt * (a * r - (pu != nullptr ? b * pu[c] : 0.0));
      if (ru != nullptr) ru[c] = r;
    }
    // ---- y momentum at the v-face (i, j-1/2, k); with walls in y the wall row stays zero
    if (ywall && j == 0) {
      vs[c] = 0.0;
      if (rv != nullptr) rv[c] = 0.0;
    } else {
      const size_t cm = at(i, jm, k);
      const double vvc = vv(i, j, k), vvp = vv(i, jp, k), vvm = vv(i, jm, k);
      const double vc0 = 0.5 * (vvc + vvp), vcm = 0.5 * (vvm + vvc);
      const double conv = (fxy(ip, j, k) - fxy(i, j, k)) * idx + (vc0 * vc0 - vcm * vcm) * idy +
                          (fyz(i, j, k + 1) - fyz(i, j, k)) * idzf - vvc * 0.5 * (Dc + D[cm]);
      const double t0 = mu[c] * (2.0 * (vvp - vvc) * idy - two3 * Dc);
      const double tm = mu[cm] * (2.0 * (vvc - vvm) * idy - two3 * D[cm]);
      double visc = (txy(ip, j, k) - txy(i, j, k)) * idx + (t0 - tm) * idy + (tyz(i, j, k + 1) - tyz(i, j, k)) * idzf;
      if (fy != nullptr) visc += fy[c];
      const double r = -conv + visc / (0.5 * (rho[c] + rho[cm])) + gy;
      vs[c] = vvc + dt * (a * r - (pv != nullptr ? b * pv[c] : 0.0));
      if (rv != nullptr) rv[c] = r;
    }
    // ---- z momentum at the w-face (i, j, k-1/2), interior faces only
    if (k == 0) {
      ws[c] = 0.0;
      if (rw != nullptr) rw[c] = 0.0;
    } else {
      const size_t cm = c - plane;
      const double wc0 = 0.5 * (w[c] + w[c + plane]), wcm = 0.5 * (w[cm] + w[c]);
      const double idzc = g.inv_dzc[k];
      const double conv = (fxz(ip, j, k) - fxz(i, j, k)) * idx + (fyz(i, j + 1, k) - fyz(i, j, k)) * idy +
                          (wc0 * wc0 - wcm * wcm) * idzc - w[c] * 0.5 * (Dc + D[cm]);
      const double t0 = mu[c] * (2.0 * (w[c + plane] - w[c]) * idzf - two3 * Dc);
      const double tm = mu[cm] * (2.0 * (w[c] - w[cm]) * g.inv_dzf[k - 1] - two3 * D[cm]);
      double visc = (txz(ip, j, k) - txz(i, j, k)) * idx + (tyz(i, j + 1, k) - tyz(i, j, k)) * idy + (t0 - tm) * idzc;
      if (fz != nullptr) visc += fz[c];
      const double r = -conv + visc / (0.5 * (rho[c] + rho[cm])) + gz;
      ws[c] = w[c] + dt * (a * r - (pw != nullptr ? b * pw[c] : 0.0));
      if (rw != nullptr) rw[c] = r;
    }
    if (k == nz - 1) {
      ws[c + plane] = 0.0;
      if (rw != nullptr) rw[c + plane] = 0.0;
    }
  }
}

// ---- adjoint ---------------------------------------------------------------
// y = -dt * beta * W_f^{-1} g  (W_f = dzf of the layer on x/y faces, dzc on
// interior z faces; wall z-faces zero).
__global__ void k_adj_rhs(Geo g, const double* __restrict__ rho, const double* __restrict__ gu,
                          const double* __restrict__ gv, const double* __restrict__ gw, double dt,
                          double* __restrict__ yu, double* __restrict__ yv, double* __restrict__ yw) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const size_t plane = (size_t)nx * ny, n = plane * nz;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx);
    const int j = (int)((c / nx) % ny);
    const int k = (int)(c / plane);
    const size_t cim = c - i + (i == 0 ? nx - 1 : i - 1);
    const size_t cjm = c - (size_t)j * nx + (size_t)(j == 0 ? ny - 1 : j - 1) * nx;
    const double r = rho[c];
    const double idzf = g.inv_dzf[k];
    // stretched y (face weights dzf s_j on x faces, dzf / t_j on y faces,
    // dzc s_j on z faces; s_j = dyf_j / dy, t_j = dy / dyc_j)
    const double is = g.ym ? g.ym[2 * ny + j] : 1.0, tj = g.ym ? g.ym[ny + j] : 1.0;
    yu[c] = -dt * (2.0 / (r + rho[cim])) * gu[c] * idzf * is;
    // with walls in y the wall row of v is not an unknown: no gradient enters there
    yv[c] = (g.ywall && j == 0) ? 0.0 : -dt * (2.0 / (r + rho[cjm])) * gv[c] * idzf * tj;
    yw[c] = (k == 0) ? 0.0 : -dt * (2.0 / (r + rho[c - plane])) * gw[c] * g.inv_dzc[k] * is;
    if (k == nz - 1) yw[c + plane] = 0.0;
  }
}

// gus = g + W_f G mu; t = d beta/d rho * g_beta with g_beta = -dt (G p) gus.
__global__ void k_adj_finish(Geo g, const double* __restrict__ rho, const double* __restrict__ p,
                             const double* __restrict__ mu, double dt, const double* __restrict__ gu,
                             const double* __restrict__ gv, const double* __restrict__ gw,
                             double* __restrict__ gus, double* __restrict__ gvs, double* __restrict__ gws,
                             double* __restrict__ tx, double* __restrict__ ty, double* __restrict__ tz) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const size_t plane = (size_t)nx * ny, n = plane * nz;
  const double idx = 1.0 / g.dx, idy = 1.0 / g.dy;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx);
    const int j = (int)((c / nx) % ny);
    const int k = (int)(c / plane);
    const size_t cim = c - i + (i == 0 ? nx - 1 : i - 1);
    const size_t cjm = c - (size_t)j * nx + (size_t)(j == 0 ? ny - 1 : j - 1) * nx;
    const double dzf = g.dzf[k];
    const double r = rho[c];
    // stretched y: x-face weight dzf s_j, y-face weight dzf / t_j against
    // G_y = t_j / dy (the two cancel), z-face weight dzc s_j
    const double sj = g.ym ? g.ym[j] : 1.0, tj = g.ym ? g.ym[ny + j] : 1.0;
    const double a = gu[c] + dzf * sj * (mu[c] - mu[cim]) * idx;
    const bool vwall = g.ywall && j == 0;  // wall row of v: zero gradient, no density dependence
    const double bb = vwall ? 0.0 : gv[c] + dzf * (mu[c] - mu[cjm]) * idy;
    gus[c] = a;
    gvs[c] = bb;
    const double bx = 2.0 / (r + rho[cim]), by = 2.0 / (r + rho[cjm]);
    tx[c] = -0.5 * bx * bx * (-dt * (p[c] - p[cim]) * idx * a);
    ty[c] = vwall ? 0.0 : -0.5 * by * by * (-dt * (p[c] - p[cjm]) * idy * tj * bb);
    if (k == 0) {
      gws[c] = 0.0;
      tz[c] = 0.0;
    } else {
      const double cc = gw[c] + sj * (mu[c] - mu[c - plane]);
      gws[c] = cc;
      const double bz = 2.0 / (r + rho[c - plane]);
      tz[c] = -0.5 * bz * bz * (-dt * (p[c] - p[c - plane]) * g.inv_dzc[k] * cc);
    }
    if (k == nz - 1) { gws[c + plane] = 0.0; tz[c + plane] = 0.0; }
  }
}

__global__ void k_adj_grho(Geo g, const double* __restrict__ tx, const double* __restrict__ ty,
                           const double* __restrict__ tz, double* __restrict__ grho) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const size_t plane = (size_t)nx * ny, n = plane * nz;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx);
    const int j = (int)((c / nx) % ny);
    const size_t cip = c - i + (i + 1 == nx ? 0 : i + 1);
    const size_t cjp = c - (size_t)j * nx + (size_t)(j + 1 == ny ? 0 : j + 1) * nx;
    grho[c] = tx[c] + tx[cip] + ty[c] + ty[cjp] + tz[c] + tz[c + plane];
  }
  (void)nz;
}

// ---------------------------------------------------------------------------
cudaError_t launch_mixture(const double* phi, double rho_g, double rho_l, double* rho, size_t n,
                           cudaStream_t s) {
  k_mixture<<<grid_for(n), kThreads, 0, s>>>(phi, rho_g, rho_l, rho, n);
  return cudaGetLastError();
}

cudaError_t launch_prep_faces(const Geo& g, const double* rho, Faces fc, cudaStream_t s) {
  k_prep_faces<<<grid_for((size_t)g.nx * g.ny * g.nz), kThreads, 0, s>>>(g, rho, fc);
  k_prep_diag<<<grid_for((size_t)g.nx * g.ny * g.nz), kThreads, 0, s>>>(g, fc);
  return cudaGetLastError();
}

cudaError_t launch_weighted_mean(const Geo& g, const double* f, double* red, double* out_mean,
                                 cudaStream_t s) {
  k_weighted_partial<<<kRedBlocks, kThreads, 0, s>>>(g, f, red);
  k_finalize<<<1, 1024, 0, s>>>(red, kRedBlocks, 1, 0, 1.0 / (g.lz * (double)g.nx * g.ny), out_mean);
  return cudaGetLastError();
}

cudaError_t launch_rhs_b(const Geo& g, const double* us, const double* vs, const double* ws,
                         const double* S, double* b, double* red, DevStatus* st, double inv_dt,
                         cudaStream_t s) {
  k_rhs_b<<<kRedBlocks, kThreads, 0, s>>>(g, us, vs, ws, S, st, b, red, inv_dt);
  k_finalize<<<1, 1024, 0, s>>>(red, kRedBlocks, 1, 0, inv_dt * inv_dt, &st->e2_0);
  return cudaGetLastError();
}

cudaError_t launch_check(DevStatus* st, const double* red, int nblk, double rtol, int maxit,
                         int kexact, cudaStream_t s) {
  k_check<<<1, 1024, 0, s>>>(st, red, nblk, rtol, maxit, kexact);
  return cudaGetLastError();
}

cudaError_t launch_init_status(DevStatus* st, cudaStream_t s) {
  k_init_status<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_correct(const Geo& g, const Faces& fc, const double* us, const double* vs,
                           const double* ws, const double* p, double dt, double* u, double* v,
                           double* w, cudaStream_t s) {
  k_correct<<<grid_for((size_t)g.nx * g.ny * g.nz), kThreads, 0, s>>>(g, fc, us, vs, ws, p, dt, u, v, w);
  return cudaGetLastError();
}

cudaError_t launch_rho_tilde(const Geo& g, const double* rho, int method, double* red, double* out,
                             cudaStream_t s) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  k_rho_extrema<<<kExtBlocks, kThreads, 0, s>>>(n, rho, red);
  k_rho_tilde<<<1, 1, 0, s>>>(red, kExtBlocks, method, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_correct_method1(const Geo& g, const Faces& fc, const double* us, const double* vs,
                                   const double* ws, const double* p, const T* delta, double dt,
                                   double* u, double* v, double* w, cudaStream_t s) {
  k_correct_method1<T><<<grid_for((size_t)g.nx * g.ny * g.nz), kThreads, 0, s>>>(g, fc, us, vs, ws, p, delta,
                                                                               dt, u, v, w);
  return cudaGetLastError();
}
template cudaError_t launch_correct_method1<double>(const Geo&, const Faces&, const double*, const double*,
                                                    const double*, const double*, const double*, double,
                                                    double*, double*, double*, cudaStream_t);
template cudaError_t launch_correct_method1<float>(const Geo&, const Faces&, const double*, const double*,
                                                   const double*, const double*, const float*, double,
                                                   double*, double*, double*, cudaStream_t);

cudaError_t launch_thermo_rate(const Geo& g, const double* phi, const double* kc, const double* T,
                               const double* u, const double* v, const double* w, double p0, double gamma,
                               double* red, double* out, cudaStream_t s) {
  constexpr int kThermoBlocks = kRedBlocks / 3;  // three partial sums per block fit the buffer
  k_thermo_partial<<<kThermoBlocks, kThreads, 0, s>>>(g, phi, kc, T, u, v, w, red);
  k_thermo_rate<<<1, 1024, 0, s>>>(red, kThermoBlocks, p0, gamma, out);
  return cudaGetLastError();
}

cudaError_t launch_divergence_source(const Geo& g, const double* phi, const double* kc, const double* T,
                                     double p0, double gamma, double dp0dt, double* S, cudaStream_t s) {
  k_divergence_source<<<grid_for((size_t)g.nx * g.ny * g.nz), kThreads, 0, s>>>(g, phi, kc, T, p0, gamma, dp0dt, S);
  return cudaGetLastError();
}

cudaError_t launch_predictor(const Geo& g, const double* u, const double* v, const double* w, const double* rho,
                             const double* mu, const double* const f[3], const double* const prev[3],
                             const double grav[3], double dt, double a, double b, double* D, double* const out[3],
                             double* const ru[3], cudaStream_t s) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  k_cell_divergence<<<grid_for(n), kThreads, 0, s>>>(g, u, v, w, D);
  k_predictor<<<grid_for(n), kThreads, 0, s>>>(g, u, v, w, rho, mu, D, f[0], f[1], f[2], prev[0], prev[1], prev[2],
                                               grav[0], grav[1], grav[2], dt, a, b, out[0], out[1], out[2], ru[0],
                                               ru[1], ru[2]);
  return cudaGetLastError();
}

cudaError_t launch_remove_mean(const Geo& g, double* p, double* red, DevStatus* st, cudaStream_t s) {
  cudaError_t e = launch_weighted_mean(g, p, red, &st->pmean, s);
  if (e != cudaSuccess) return e;
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  k_sub_mean<<<grid_for(n), kThreads, 0, s>>>(p, n, st);
  return cudaGetLastError();
}

cudaError_t launch_setup_pivots(const Geo& g, const double* lamx, const double* lamy, double* invd,
                                cudaStream_t s, double* mtab) {
  const size_t ncol = (size_t)g.ny * g.nxh;
  k_setup_pivots<<<(int)((ncol + 127) / 128), 128, 0, s>>>(g, lamx, lamy, invd, mtab);
  return cudaGetLastError();
}

cudaError_t launch_setup_z64(const Geo& g, const double* lamx, const double* lamy, int nyt, int ysym,
                             double* m, double* e, float* d, cudaStream_t s) {
  (void)ysym;  // the table rows are ky' = 0 .. nyt - 1 either way
  const size_t ntc = (size_t)nyt * g.nxh;
  k_setup_z64<<<(int)((ntc + 127) / 128), 128, 0, s>>>(g, lamx, lamy, nyt, m, e, d);
  return cudaGetLastError();
}

cudaError_t launch_adj_rhs(const Geo& g, const double* rho, const double* gu, const double* gv,
                           const double* gw, double dt, double* yu, double* yv, double* yw,
                           cudaStream_t s) {
  k_adj_rhs<<<grid_for((size_t)g.nx * g.ny * g.nz), kThreads, 0, s>>>(g, rho, gu, gv, gw, dt, yu, yv, yw);
  return cudaGetLastError();
}

cudaError_t launch_adj_finish(const Geo& g, const double* rho, const double* p, const double* mu,
                              double dt, const double* gu, const double* gv, const double* gw,
                              double* gus, double* gvs, double* gws, double* tx, double* ty,
                              double* tz, cudaStream_t s) {
  k_adj_finish<<<grid_for((size_t)g.nx * g.ny * g.nz), kThreads, 0, s>>>(g, rho, p, mu, dt, gu, gv, gw,
                                                                         gus, gvs, gws, tx, ty, tz);
  return cudaGetLastError();
}

cudaError_t launch_adj_grho(const Geo& g, const double* tx, const double* ty, const double* tz,
                            double* grho, cudaStream_t s) {
  k_adj_grho<<<grid_for((size_t)g.nx * g.ny * g.nz), kThreads, 0, s>>>(g, tx, ty, tz, grho);
  return cudaGetLastError();
}

cudaError_t launch_copy_resid_sums(DevStatus*, const double*, int, cudaStream_t) { return cudaSuccess; }

}  // namespace pp
