// Per-cell bodies of the stencil kernels, shared by the single-grid kernels
// (pp_kernels_stencil.cu) and the grouped multi-grid kernels (pp_batch.cu).
#pragma once
#include "pp_fft.cuh"

namespace pp {

struct CellIdx {
  int i, j, k;
  size_t cim, cip, cjm, cjp;
};

__device__ __forceinline__ CellIdx cell_index(const Geo& g, size_t c) {
  const int nx = g.nx, ny = g.ny;
  const size_t plane = (size_t)nx * ny;
  CellIdx x;
  x.i = (int)(c % nx);
  x.j = (int)((c / nx) % ny);
  x.k = (int)(c / plane);
  x.cim = c - x.i + (x.i == 0 ? nx - 1 : x.i - 1);
  x.cip = c - x.i + (x.i + 1 == nx ? 0 : x.i + 1);
  x.cjm = c - (size_t)x.j * nx + (size_t)(x.j == 0 ? ny - 1 : x.j - 1) * nx;
  x.cjp = c - (size_t)x.j * nx + (size_t)(x.j + 1 == ny ? 0 : x.j + 1) * nx;
  return x;
}

// Face coefficients of cell c (beta = 2/(rho_a + rho_b) on its x-, y- and
// z-face "below", x/y coefficients scaled by the layer width dzf_k).  Wall
// faces get 0: the z walls, and with walls in y the y-face below row 0,
// which the periodic indexing also reaches as the face above row ny - 1.
__device__ __forceinline__ void cell_prep_faces(const Geo& g, const double* __restrict__ rho,
                                                const Faces& fc, size_t c) {
  const CellIdx x = cell_index(g, c);
  const size_t plane = (size_t)g.nx * g.ny;
  const double r = rho[c];
  const double w = g.dzf[x.k];
  // stretched y: the row of cell j is scaled by dzf_k s_j; the y face below
  // it carries t_j = dy / dyc_j
  const double sj = g.ym ? g.ym[x.j] : 1.0, tj = g.ym ? g.ym[g.ny + x.j] : 1.0;
  fc.cx[c] = 2.0 / (r + rho[x.cim]) * g.inv_dx2 * w * sj;
  fc.cy[c] = (g.ywall && x.j == 0) ? 0.0 : 2.0 / (r + rho[x.cjm]) * g.inv_dy2 * w * tj;
  fc.cz[c] = (x.k == 0) ? 0.0 : 2.0 / (r + rho[c - plane]) * g.inv_dzc[x.k] * sj;
  if (x.k == g.nz - 1) fc.cz[c + plane] = 0.0;
  fc.rhof[c] = (float)r;
}

// diag = sum of the six (row-scaled) coefficients of cell c.
__device__ __forceinline__ void cell_prep_diag(const Geo& g, const Faces& fc, size_t c) {
  const CellIdx x = cell_index(g, c);
  const size_t plane = (size_t)g.nx * g.ny;
  fc.diag[c] = ((fc.cx[c] + fc.cx[x.cip]) + (fc.cy[c] + fc.cy[x.cjp])) + (fc.cz[c] + fc.cz[c + plane]);
  if (fc.diagf != nullptr) fc.diagf[c] = (float)fc.diag[c];
}

// d = D u* - (S - meanS) at cell c (wall values of w*, and of v* with walls
// in y, taken as zero); stores the row-scaled b_s = dzf_k d / dt (dzf_k s_j
// d / dt on a stretched y, where the row width is dyf_j = s_j dy) and
// returns d.
__device__ __forceinline__ double cell_rhs_b(const Geo& g, const double* __restrict__ us,
                                             const double* __restrict__ vs,
                                             const double* __restrict__ ws,
                                             const double* __restrict__ S, double meanS,
                                             double* __restrict__ b, double inv_dt, size_t c) {
  const CellIdx x = cell_index(g, c);
  const size_t plane = (size_t)g.nx * g.ny;
  const double wlo = (x.k == 0) ? 0.0 : ws[c];
  const double whi = (x.k == g.nz - 1) ? 0.0 : ws[c + plane];
  const double vlo = (g.ywall && x.j == 0) ? 0.0 : vs[c];
  const double vhi = (g.ywall && x.j == g.ny - 1) ? 0.0 : vs[x.cjp];
  const double sj = g.ym ? g.ym[x.j] : 1.0;
  double d = (us[x.cip] - us[c]) / g.dx + (vhi - vlo) / (g.dy * sj) + (whi - wlo) * g.inv_dzf[x.k];
  if (S != nullptr) d -= (S[c] - meanS);
  b[c] = d * g.dzf[x.k] * sj * inv_dt;
  return d;
}

// div(k grad T) at cell c: D(k_f G T) with k_f the arithmetic mean of the
// two cells of a face, no flux through the z walls, nor through the y walls
// when y is bounded (Eqs. 30 and 34).
__device__ __forceinline__ double cell_conduction(const Geo& g, const double* __restrict__ kc,
                                                  const double* __restrict__ T, size_t c) {
  const CellIdx x = cell_index(g, c);
  const size_t plane = (size_t)g.nx * g.ny;
  const double k0 = kc[c], t0 = T[c];
  double sx = 0.5 * (k0 + kc[x.cip]) * (T[x.cip] - t0) + 0.5 * (k0 + kc[x.cim]) * (T[x.cim] - t0);
  // with walls in y no heat crosses the faces below row 0 and above row ny - 1
  const bool yhi = !(g.ywall && x.j + 1 == g.ny), ylo = !(g.ywall && x.j == 0);
  // stretched y: the face below row j is dyc_j = dy / t_j from the centre
  // below, and the row is dyf_j = s_j dy wide
  const double thi = (g.ym && yhi) ? g.ym[g.ny + x.j + 1] : 1.0, tlo = g.ym ? g.ym[g.ny + x.j] : 1.0;
  const double isj = g.ym ? g.ym[2 * g.ny + x.j] : 1.0;
  double sy = (yhi ? 0.5 * (k0 + kc[x.cjp]) * (T[x.cjp] - t0) * thi : 0.0) +
              (ylo ? 0.5 * (k0 + kc[x.cjm]) * (T[x.cjm] - t0) * tlo : 0.0);
  sy *= isj;
  double sz = 0.0;
  if (x.k + 1 < g.nz) sz += 0.5 * (k0 + kc[c + plane]) * (T[c + plane] - t0) * g.inv_dzc[x.k + 1];
  if (x.k > 0) sz += 0.5 * (k0 + kc[c - plane]) * (T[c - plane] - t0) * g.inv_dzc[x.k];
  return sx * g.inv_dx2 + sy * g.inv_dy2 + sz * g.inv_dzf[x.k];
}

// u = u* - dt beta G p at the faces of cell c (Eq. corr); w walls = 0, and
// with walls in y the wall row 0 of v = 0.
__device__ __forceinline__ void cell_correct(const Geo& g, const Faces& fc,
                                             const double* __restrict__ us,
                                             const double* __restrict__ vs,
                                             const double* __restrict__ ws,
                                             const double* __restrict__ p, double dt,
                                             double* __restrict__ u, double* __restrict__ v,
                                             double* __restrict__ w, size_t c) {
  const CellIdx x = cell_index(g, c);
  const size_t plane = (size_t)g.nx * g.ny;
  const double pc = p[c];
  // dt beta_x / dx = dt dx cx / dzf_k (cx carries dzf_k); on a stretched y
  // cx and cz also carry s_j, and dt beta_y / dyc_j = dt dy cy / dzf_k
  // (cy carries dzf_k t_j = dzf_k dy / dyc_j)
  const double is = g.ym ? g.ym[2 * g.ny + x.j] : 1.0;
  const double ax = dt * g.dx * g.inv_dzf[x.k] * is, ay = dt * g.dy * g.inv_dzf[x.k];
  u[c] = us[c] - ax * fc.cx[c] * (pc - p[x.cim]);
  v[c] = (g.ywall && x.j == 0) ? 0.0 : vs[c] - ay * fc.cy[c] * (pc - p[x.cjm]);
  w[c] = (x.k == 0) ? 0.0 : ws[c] - dt * is * fc.cz[c] * (pc - p[c - plane]);
  if (x.k == g.nz - 1) w[c + plane] = 0.0;
}

// Loop control of Algorithm 1 for one grid, run by thread 0 with the
// reduced residual sums s2 (sum e^2) and s1 (sum |e|).  kexact: recompute
// the residual exactly every kexact passes (<= 1: every pass); convergence
// is only accepted on an exact residual.
__device__ __forceinline__ void status_update(DevStatus* st, double s2, double s1, double rtol,
                                              int maxit, int kexact) {
  st->e2 = s2;
  st->e1 = s1;
  const double e20 = st->e2_0;
  const double rel = (e20 > 0.0) ? sqrt(s2 / e20) : 0.0;
  st->rel = rel;
  const int exact = st->need_exact;
  st->last_exact = exact;
  if (!isfinite(s2) || !isfinite(e20)) { st->done = 1; st->code = PP_ERR_NUMERIC; }
  else if (e20 == 0.0 || (rel <= rtol && exact)) { st->done = 1; st->code = PP_OK; }
  else if (st->iters >= maxit) { st->done = 1; st->code = PP_ERR_NOT_CONVERGED; }
  else {
    st->iters += 1;
    if (kexact <= 1) {
      st->need_exact = 1;
    } else if (exact) {
      st->need_exact = 0;
      st->since_exact = 1;
    } else {
      st->since_exact += 1;
      // an updated residual below the tolerance is confirmed by an exact one
      st->need_exact = (rel <= rtol || st->since_exact >= kexact) ? 1 : 0;
    }
  }
}

__device__ __forceinline__ void status_init(DevStatus* st) {
  st->e2 = 0; st->e1 = 0; st->e2_0 = 0; st->rel = 0; st->mean_S = 0; st->pmean = 0;
  st->iters = 0; st->done = 0; st->code = PP_OK; st->pad = 0;
  st->need_exact = 1; st->since_exact = 0; st->last_exact = 1;
}

}  // namespace pp
