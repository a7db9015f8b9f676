// Host eigen decompositions of the symmetric tridiagonal second
// differences of a stretched direction (the eigenexpansion method of
// Sec. 3.3.1 with a numerical eigenbasis): L = W^{-1} T with W = diag(cell
// widths) and T symmetric, so its eigenvectors V = W^{-1/2} Q come from the
// symmetric S = W^{-1/2} T W^{-1/2} (S Q = Q Lambda) and are W-orthonormal.
// Used for the z expansion on the tensor cores (PP_MIXED_TC) and for a
// stretched y between walls.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "pp_internal.cuh"

namespace pp {

namespace {

// number of eigenvalues of the symmetric tridiagonal (d, e) below x
int sturm_count(const std::vector<double>& d, const std::vector<double>& e2, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    q = (d[i] - x) - (i > 0 ? e2[i - 1] / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// solve (S - s I) y = b in place (tridiagonal Gaussian elimination with
// partial pivoting; S has diagonal d and off-diagonal e)
void shifted_solve(const std::vector<double>& d, const std::vector<double>& e, double s, std::vector<double>& b) {
  const int n = (int)d.size();
  // band storage after pivoting: row i has entries at columns i, i+1, i+2
  std::vector<double> r0(n), r1(n, 0.0), r2(n, 0.0);
  std::vector<double> sub(n, 0.0);
  for (int i = 0; i < n; ++i) {
    r0[i] = d[i] - s;
    if (i + 1 < n) r1[i] = e[i];
    if (i > 0) sub[i] = e[i - 1];
  }
  const double tiny = 1e-300;
  for (int i = 0; i + 1 < n; ++i) {
    // rows i and i+1; sub[i+1] is row i+1's entry in column i
    if (std::fabs(sub[i + 1]) > std::fabs(r0[i])) {
      std::swap(r0[i], sub[i + 1]);
      std::swap(r1[i], r0[i + 1]);
      std::swap(r2[i], r1[i + 1]);
      std::swap(b[i], b[i + 1]);
    }
    const double piv = (r0[i] == 0.0) ? tiny : r0[i];
    const double f = sub[i + 1] / piv;
    r0[i + 1] -= f * r1[i];
    r1[i + 1] -= f * r2[i];
    b[i + 1] -= f * b[i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = b[i];
    if (i + 1 < n) v -= r1[i] * b[i + 1];
    if (i + 2 < n) v -= r2[i] * b[i + 2];
    b[i] = v / ((r0[i] == 0.0) ? tiny : r0[i]);
  }
}

}  // namespace

// Eigenpairs of the symmetric tridiagonal (d, e), ascending: Sturm-sequence
// bisection for the eigenvalues, inverse iteration with two Gram-Schmidt
// passes for the eigenvectors, and a residual check of every pair.
bool sym_tridiag_eigen(const std::vector<double>& d, const std::vector<double>& e, std::vector<double>& lam,
                       std::vector<double>& Q) {
  const int n = (int)d.size();
  std::vector<double> e2(n, 0.0);
  for (int k = 0; k + 1 < n; ++k) e2[k] = e[k] * e[k];
  double lo = 0.0, hi = 0.0;  // Gershgorin interval
  for (int k = 0; k < n; ++k) {
    const double r = (k > 0 ? std::fabs(e[k - 1]) : 0.0) + (k + 1 < n ? std::fabs(e[k]) : 0.0);
    lo = std::min(lo, d[k] - r);
    hi = std::max(hi, d[k] + r);
  }
  lam.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    double a = lo, b = hi;
    for (int it = 0; it < 200 && b - a > 1e-15 * std::max(1.0, std::max(std::fabs(a), std::fabs(b))); ++it) {
      const double m = 0.5 * (a + b);
      if (sturm_count(d, e2, m) > j) b = m; else a = m;
    }
    lam[j] = 0.5 * (a + b);
  }
  Q.assign((size_t)n * n, 0.0);
  unsigned long long seed = 0x9E3779B97F4A7C15ull;
  for (int j = 0; j < n; ++j) {
    std::vector<double> v(n);
    for (int k = 0; k < n; ++k) {
      seed = seed * 6364136223846793005ull + 1442695040888963407ull;
      v[k] = (double)(seed >> 11) / 9007199254740992.0 - 0.5;
    }
    const double shift = lam[j] + 1e-10 * std::max(1.0, std::fabs(lam[j]));
    for (int it = 0; it < 3; ++it) {
      shifted_solve(d, e, shift, v);
      for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < j; ++i) {
          double dot = 0.0;
          for (int k = 0; k < n; ++k) dot += Q[(size_t)k * n + i] * v[k];
          for (int k = 0; k < n; ++k) v[k] -= dot * Q[(size_t)k * n + i];
        }
      double nrm = 0.0;
      for (int k = 0; k < n; ++k) nrm += v[k] * v[k];
      nrm = std::sqrt(nrm);
      if (!(nrm > 0.0)) return false;
      for (int k = 0; k < n; ++k) v[k] /= nrm;
    }
    for (int k = 0; k < n; ++k) Q[(size_t)k * n + j] = v[k];
  }
  // self-check: residual of S q = lambda q for every pair
  for (int j = 0; j < n; ++j) {
    double res = 0.0;
    for (int k = 0; k < n; ++k) {
      double sq = d[k] * Q[(size_t)k * n + j];
      if (k > 0) sq += e[k - 1] * Q[(size_t)(k - 1) * n + j];
      if (k + 1 < n) sq += e[k] * Q[(size_t)(k + 1) * n + j];
      res = std::max(res, std::fabs(sq - lam[j] * Q[(size_t)k * n + j]));
    }
    if (res > 1e-8 * std::max(1.0, std::fabs(lo))) return false;
  }
  return true;
}

// The eigen decomposition of L_z = W^{-1} T (W = diag(dzf)) for the
// tensor-core z expansion: the eigenvalues mu (ascending, FP32 copy padded
// with zeros to `pad` entries), the index of the zero eigenvalue, and the
// row-major n x n matrices of its two products, V^T W (mode x level) and V
// (level x mode).  False when the decomposition failed its own checks.
bool build_zeigen_host(int nz, const double* dzf, const double* inv_dzc, int pad, std::vector<float>& mu_out,
                       int* zero_mode, std::vector<double>& m_fwd, std::vector<double>& m_inv) {
  // S = W^{-1/2} T W^{-1/2}, T_kk = -(1/dzc_k + 1/dzc_{k+1}), T_{k,k+1} = 1/dzc_{k+1}
  std::vector<double> d(nz), e(nz > 1 ? nz - 1 : 1, 0.0);
  for (int k = 0; k < nz; ++k) d[k] = -(inv_dzc[k] + inv_dzc[k + 1]) / dzf[k];
  for (int k = 0; k + 1 < nz; ++k) e[k] = inv_dzc[k + 1] / std::sqrt(dzf[k] * dzf[k + 1]);
  std::vector<double> lam, Q;
  if (!sym_tridiag_eigen(d, e, lam, Q)) return false;
  int zm = 0;
  for (int j = 1; j < nz; ++j)
    if (std::fabs(lam[j]) < std::fabs(lam[zm])) zm = j;
  *zero_mode = zm;
  mu_out.assign(std::max(pad, nz), 0.0f);
  for (int j = 0; j < nz; ++j) mu_out[j] = (float)lam[j];
  m_fwd.assign((size_t)nz * nz, 0.0);
  m_inv.assign((size_t)nz * nz, 0.0);
  for (int j = 0; j < nz; ++j)
    for (int k = 0; k < nz; ++k) {
      const double q = Q[(size_t)k * nz + j];
      m_fwd[(size_t)j * nz + k] = q * std::sqrt(dzf[k]);  // (V^T W)[mode j][level k]
      m_inv[(size_t)k * nz + j] = q / std::sqrt(dzf[k]);  // V[level k][mode j]
    }
  return true;
}

// The same decomposition for a stretched y between walls, in the order the
// spectrum's rows take (mode 0 = the constant, eigenvalue 0, first).  The
// constant mode is set exactly (q_0 = W^{1/2} 1 / sqrt(ly)) and the others
// are made orthogonal to it once more.
bool build_yeigen_host(int ny, const double* dyf, const double* inv_dyc, std::vector<double>& lam,
                       std::vector<double>& mt_fwd, std::vector<double>& mt_inv) {
  std::vector<double> d(ny), e(ny > 1 ? ny - 1 : 1, 0.0);
  for (int j = 0; j < ny; ++j) d[j] = -(inv_dyc[j] + inv_dyc[j + 1]) / dyf[j];
  for (int j = 0; j + 1 < ny; ++j) e[j] = inv_dyc[j + 1] / std::sqrt(dyf[j] * dyf[j + 1]);
  std::vector<double> asc, Q;
  if (!sym_tridiag_eigen(d, e, asc, Q)) return false;
  double ly = 0.0;
  for (int j = 0; j < ny; ++j) ly += dyf[j];
  // mode m of the spectrum = ascending pair ny - 1 - m
  std::vector<double> q((size_t)ny * ny);  // q[m * ny + j]
  for (int m = 0; m < ny; ++m)
    for (int j = 0; j < ny; ++j) q[(size_t)m * ny + j] = Q[(size_t)j * ny + (ny - 1 - m)];
  for (int j = 0; j < ny; ++j) q[j] = std::sqrt(dyf[j] / ly);
  for (int m = 1; m < ny; ++m) {
    double dot = 0.0, nrm = 0.0;
    for (int j = 0; j < ny; ++j) dot += q[j] * q[(size_t)m * ny + j];
    for (int j = 0; j < ny; ++j) {
      q[(size_t)m * ny + j] -= dot * q[j];
      nrm += q[(size_t)m * ny + j] * q[(size_t)m * ny + j];
    }
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0)) return false;
    for (int j = 0; j < ny; ++j) q[(size_t)m * ny + j] /= nrm;
  }
  lam.assign(ny, 0.0);
  for (int m = 1; m < ny; ++m) lam[m] = asc[ny - 1 - m];
  mt_fwd.assign((size_t)ny * ny, 0.0);
  mt_inv.assign((size_t)ny * ny, 0.0);
  for (int m = 0; m < ny; ++m)
    for (int j = 0; j < ny; ++j) {
      const double v = q[(size_t)m * ny + j];
      mt_fwd[(size_t)j * ny + m] = v * std::sqrt(dyf[j]);  // (V^T W)[m][j], stored [j][m]
      mt_inv[(size_t)m * ny + j] = v / std::sqrt(dyf[j]);  // V[j][m], stored [m][j]
    }
  return true;
}

}  // namespace pp
