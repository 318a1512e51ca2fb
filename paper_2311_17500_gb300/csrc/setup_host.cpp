// Host-side 1D set-up in FP64 (Sec. 2 and Sec. 3.1 of the paper):
// open knot vectors, Gauss-Legendre rules, local B-spline values and
// derivatives per knot span, the banded 1D matrices M_l, K_l, M_t, W_t, the
// SU functions tau_k of Eq. (tau), and Greville abscissae.
#include <cmath>
#include <algorithm>
#include <cstring>
#include "st_internal.h"

namespace {

// Legendre polynomials P_n(z) and P_{n-1}(z) by the three-term recurrence.
void legendre_pair(int n, double z, double &pn, double &pm) {
  pm = 1.0;
  pn = z;
  for (int k = 2; k <= n; ++k) {
    double pk = ((2.0 * k - 1.0) * z * pn - (k - 1.0) * pm) / k;
    pm = pn;
    pn = pk;
  }
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  if (n == 1) { w[0] = 2.0; return; }
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double pn, pm, dp;
    for (int it = 0; it < 100; ++it) {
      legendre_pair(n, z, pn, pm);
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre_pair(n, z, pn, pm);
    dp = n * (z * pn - pm) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Values of the degree-j functions nonzero on span s (knots[s] <= x < knots[s+1]),
// for j = 0..p: N[j][r] = b_{s-j+r, j}(x).  Triangular de Boor scheme.
void local_values(const std::vector<double> &kn, int s, int p, double x, double N[ST_MAXP + 1][ST_MAXP + 1]) {
  for (int j = 0; j <= p; ++j)
    for (int r = 0; r <= p; ++r) N[j][r] = 0.0;
  N[0][0] = 1.0;
  for (int j = 1; j <= p; ++j) {
    for (int r = 0; r <= j; ++r) {
      int i = s - j + r;
      double v = 0.0;
      if (r - 1 >= 0) {   // b_{i, j-1} = N[j-1][r-1]
        double den = kn[i + j] - kn[i];
        if (den > 0) v += (x - kn[i]) / den * N[j - 1][r - 1];
      }
      if (r <= j - 1) {   // b_{i+1, j-1} = N[j-1][r]
        double den = kn[i + j + 1] - kn[i + 1];
        if (den > 0) v += (kn[i + j + 1] - x) / den * N[j - 1][r];
      }
      N[j][r] = v;
    }
  }
}

// k-th parametric derivative of the p+1 degree-p functions on span s at x.
// The derivative of sum_m c_m b_{i+m,q} is expanded into degree q-1 functions
// with the knot-difference rule, k times, then evaluated with N[p-k].
void local_derivs(const std::vector<double> &kn, int s, int p, double x, int kmax,
                  double out[ST_MAXP + 1][ST_MAXP + 1]) {
  double N[ST_MAXP + 1][ST_MAXP + 1];
  local_values(kn, s, p, x, N);
  for (int r = 0; r <= p; ++r) {
    int i = s - p + r;            // global index of the r-th local function
    double c[ST_MAXP + 2];
    for (int m = 0; m < ST_MAXP + 2; ++m) c[m] = 0.0;
    c[0] = 1.0;
    for (int k = 0; k <= kmax; ++k) {
      if (k > 0) {
        int q = p - k + 1;        // degree before this differentiation
        double nc[ST_MAXP + 2];
        for (int m = 0; m < ST_MAXP + 2; ++m) nc[m] = 0.0;
        for (int m = 0; m < k; ++m) {   // k terms at degree q
          int ii = i + m;
          double d1 = kn[ii + q] - kn[ii];
          double d2 = kn[ii + q + 1] - kn[ii + 1];
          if (d1 > 0) nc[m] += c[m] * q / d1;
          if (d2 > 0) nc[m + 1] -= c[m] * q / d2;
        }
        for (int m = 0; m < ST_MAXP + 2; ++m) c[m] = nc[m];
      }
      // evaluate sum_m c[m] b_{i+m, p-k}
      int deg = p - k;
      double v = 0.0;
      for (int m = 0; m <= k; ++m) {
        int rr = r + m - k;       // index in the degree-deg table
        if (rr >= 0 && rr <= deg) v += c[m] * N[deg][rr];
      }
      out[k][r] = v;
    }
  }
}

// Open knot vector of maximal regularity on [0, 1] with the breakpoints
// `breaks` (n_el + 1 increasing values from 0 to 1; null: uniform), the Gauss
// rule of each span and the local basis derivatives 0..kmax there.
void build_dir(Dir1D &dr, int n_el, int p, double scale, int kmax, int nq = 0, const double *breaks = nullptr) {
  dr.n_el = n_el;
  dr.p = p;
  dr.n = n_el + p;
  dr.nq = nq > 0 ? nq : p + 1;
  dr.kmax = kmax;
  dr.scale = scale;
  dr.knots.assign(dr.n + p + 1, 0.0);
  for (int i = 0; i <= p; ++i) dr.knots[dr.n + i] = 1.0;
  for (int i = 1; i < n_el; ++i) dr.knots[p + i] = breaks ? breaks[i] : (double)i / n_el;
  std::vector<double> gx, gw;
  gauss_legendre(dr.nq, gx, gw);
  dr.xq.assign((size_t)n_el * dr.nq, 0.0);
  dr.wq.assign((size_t)n_el * dr.nq, 0.0);
  dr.tab.assign((size_t)(kmax + 1) * n_el * dr.nq * (p + 1), 0.0);
  for (int e = 0; e < n_el; ++e) {
    int s = e + p;
    double a = dr.knots[s], b = dr.knots[s + 1];
    for (int q = 0; q < dr.nq; ++q) {
      double x = 0.5 * (a + b) + 0.5 * (b - a) * gx[q];
      dr.xq[e * dr.nq + q] = scale * x;
      dr.wq[e * dr.nq + q] = scale * 0.5 * (b - a) * gw[q];
      double D[ST_MAXP + 1][ST_MAXP + 1];
      local_derivs(dr.knots, s, p, x, kmax, D);
      for (int k = 0; k <= kmax; ++k) {
        double f = std::pow(scale, -k);
        for (int r = 0; r <= p; ++r)
          dr.tab[(((size_t)k * n_el + e) * dr.nq + q) * (p + 1) + r] = f * D[k][r];
      }
    }
  }
  dr.greville.assign(dr.n, 0.0);
  for (int i = 0; i < dr.n && p > 0; ++i) {
    double s = 0.0;
    for (int j = 1; j <= p; ++j) s += dr.knots[i + j];
    dr.greville[i] = scale * s / p;
  }
}

}  // namespace

// Collocation of the basis at its own Greville abscissae, banded (n x (2p+1)):
// entry (i, j) = b_j(gamma_i), nonzero for |i - j| <= p since gamma_i lies in
// the support of b_i.  `shift` = 1 drops the first function from rows and
// columns (time: the functions of X_t at their Greville points).
std::vector<double> greville_band(const Dir1D &dr, int shift) {
  const int p = dr.p, B = 2 * p + 1, n = dr.n - shift;
  std::vector<double> out((size_t)n * B, 0.0);
  for (int i = 0; i < n; ++i) {
    const int f = i + shift;
    double x = 0.0;
    for (int j = 1; j <= p; ++j) x += dr.knots[f + j];
    x = p > 0 ? x / p : 0.5 * (dr.knots[f] + dr.knots[f + 1]);
    // span s with knots[s] <= x < knots[s+1] (the last span holds x = 1)
    int s = p;
    while (s + 1 < dr.n && dr.knots[s + 1] <= x) ++s;
    double N[ST_MAXP + 1][ST_MAXP + 1];
    local_values(dr.knots, s, p, x, N);
    for (int r = 0; r <= p; ++r) {
      const int j = s - p + r - shift;
      if (j < 0 || j >= n) continue;
      out[(size_t)i * B + (j - i + p)] = N[p][r];
    }
  }
  return out;
}

namespace {

// Banded Gram matrix sum_e sum_q w (d^ki b_i)(d^kj b_j) over the full basis;
// `shift` removes the first function (time: X_t) when 1.  Row = index of the
// function carrying derivative ki (test), column = kj (trial).
std::vector<double> band_matrix(const Dir1D &dr, int ki, int kj, int shift) {
  int p = dr.p, B = 2 * p + 1;
  int n = dr.n - shift;
  std::vector<double> out((size_t)n * B, 0.0);
  for (int e = 0; e < dr.n_el; ++e)
    for (int q = 0; q < dr.nq; ++q) {
      double w = dr.wq[e * dr.nq + q];
      for (int a = 0; a <= p; ++a) {
        int i = e + a - shift;
        if (i < 0) continue;
        for (int c = 0; c <= p; ++c) {
          int j = e + c - shift;
          if (j < 0) continue;
          out[(size_t)i * B + (j - i + p)] += w * dr.at(ki, e, q, a) * dr.at(kj, e, q, c);
        }
      }
    }
  return out;
}

// Symmetric positive definite banded Cholesky (dense storage, band bw), in place.
bool chol_band_factor(std::vector<double> &A, int n, int bw) {
  for (int j = 0; j < n; ++j) {
    double s = A[(size_t)j * n + j];
    for (int k = std::max(0, j - bw); k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(s > 0)) return false;
    double l = std::sqrt(s);
    A[(size_t)j * n + j] = l;
    for (int i = j + 1; i <= std::min(n - 1, j + bw); ++i) {
      double t = A[(size_t)i * n + j];
      for (int k = std::max(0, i - bw); k < j; ++k) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = t / l;
    }
  }
  return true;
}

// b <- (L L^T)^{-1} b with the factor of chol_band_factor.
void chol_band_apply(const std::vector<double> &A, int n, int bw, std::vector<double> &b) {
  for (int i = 0; i < n; ++i) {
    double t = b[i];
    for (int k = std::max(0, i - bw); k < i; ++k) t -= A[(size_t)i * n + k] * b[k];
    b[i] = t / A[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = b[i];
    for (int k = i + 1; k <= std::min(n - 1, i + bw); ++k) t -= A[(size_t)k * n + i] * b[k];
    b[i] = t / A[(size_t)i * n + i];
  }
}

// tau_k (k = 1..p) of Eq. (tau): splines of degree p-k on the time breakpoints,
// the minimum-norm solution in the scaled coefficients y = c / h_t^(2k-1) of
// the conditions "strict upper band of W_t + sum_k S_k vanishes", obtained
// from the normal equations (C C^T) z = rhs, y = C^T z.  Returns the tau_k at
// the time Gauss points, [k-1][e][q].
bool tau_setup(const Dir1D &td, std::vector<double> &tau_q) {
  int p = td.p, n_el = td.n_el, nq = td.nq;
  int Nt = td.n - 1;
  // unknowns scaled by h^(2k-1), h the largest element in the support of the
  // unknown's B-spline (the mesh size itself on a uniform mesh)
  std::vector<double> hel(n_el);
  for (int e = 0; e < n_el; ++e) hel[e] = (td.knots[e + p + 1] - td.knots[e + p]) * td.scale;
  auto hsc = [&](int k, int m) {   // m-th B-spline of degree p-k spans elements m-(p-k) .. m
    double h = 0.0;
    for (int e = std::max(0, m - (p - k)); e <= std::min(n_el - 1, m); ++e) h = std::max(h, hel[e]);
    return std::pow(h, 2 * k - 1);
  };
  // unknown spaces
  // unknown (k, m) of tau_k's m-th B-spline sits in column m*p + (k-1), so
  // that the columns a condition touches stay local and C C^T is banded
  std::vector<Dir1D> sp(p + 1);
  // on the breakpoints of the time mesh, evaluated at its Gauss points
  std::vector<double> br(n_el + 1);
  for (int e = 0; e <= n_el; ++e) br[e] = td.knots[e + p];
  for (int k = 1; k <= p; ++k) build_dir(sp[k], n_el, p - k, td.scale, 0, nq, br.data());
  int nu = p * (n_el + p - 1);
  auto col = [p](int k, int m) { return m * p + (k - 1); };
  // conditions
  struct Row { std::vector<double> v; int c0, c1; double rhs; };
  std::vector<Row> rows;
  for (int i = 0; i < Nt - 1; ++i)
    for (int l = 1; l <= std::min(p, Nt - 1 - i); ++l) {
      int j = i + l;
      Row r;
      r.v.assign(nu, 0.0);
      r.rhs = 0.0;
      // X_t index i <-> full index i+1; on span e, local a = full - e
      for (int e = 0; e < n_el; ++e) {
        int ai = i + 1 - e, aj = j + 1 - e;
        if (ai < 0 || ai > p || aj < 0 || aj > p) continue;
        for (int q = 0; q < nq; ++q) {
          double w = td.wq[e * nq + q];
          r.rhs -= w * td.at(1, e, q, aj) * td.at(0, e, q, ai);
          for (int k = 1; k <= p; ++k) {
            double prod = w * td.at(k, e, q, aj) * td.at(k, e, q, ai);
            const Dir1D &s = sp[k];
            for (int m = 0; m <= s.p; ++m) r.v[col(k, e + m)] += prod * hsc(k, e + m) * s.at(0, e, q, m);
          }
        }
      }
      r.c0 = nu; r.c1 = -1;
      for (int c = 0; c < nu; ++c)
        if (r.v[c] != 0.0) { r.c0 = std::min(r.c0, c); r.c1 = std::max(r.c1, c); }
      rows.push_back(std::move(r));
    }
  int nr = (int)rows.size();
  std::vector<double> y(nu, 0.0);
  if (nr > 0) {
    // bandwidth of C C^T: largest row distance with overlapping column ranges
    int bw = 0;
    for (int a = 0; a < nr; ++a)
      for (int b = a + 1; b < nr; ++b)
        if (rows[b].c0 <= rows[a].c1 && rows[b].c1 >= rows[a].c0) bw = std::max(bw, b - a);
    std::vector<double> G((size_t)nr * nr, 0.0);
    for (int a = 0; a < nr; ++a)
      for (int b = std::max(0, a - bw); b <= a; ++b) {
        int lo = std::max(rows[a].c0, rows[b].c0), hi = std::min(rows[a].c1, rows[b].c1);
        double s = 0.0;
        for (int c = lo; c <= hi; ++c) s += rows[a].v[c] * rows[b].v[c];
        G[(size_t)a * nr + b] = s;
        G[(size_t)b * nr + a] = s;
      }
    // Cholesky of C C^T once; y = C^T z, then refinement steps on the
    // residual rhs - C y (the normal equations square the condition number,
    // which graded time meshes raise further); every update stays in the
    // range of C^T, so y tends to the minimum-norm solution
    std::vector<double> z(nr), res(nr);
    for (int a = 0; a < nr; ++a) z[a] = rows[a].rhs;
    if (!chol_band_factor(G, nr, bw)) return false;
    for (int pass = 0; pass < 6; ++pass) {
      if (pass == 0) {
        for (int a = 0; a < nr; ++a) res[a] = rows[a].rhs;
      } else {
        for (int a = 0; a < nr; ++a) {
          double t = rows[a].rhs;
          for (int c = rows[a].c0; c <= rows[a].c1; ++c) t -= rows[a].v[c] * y[c];
          res[a] = t;
        }
      }
      chol_band_apply(G, nr, bw, res);
      for (int a = 0; a < nr; ++a)
        for (int c = rows[a].c0; c <= rows[a].c1; ++c) y[c] += rows[a].v[c] * res[a];
    }
    (void)z;
  }
  tau_q.assign((size_t)p * n_el * nq, 0.0);
  for (int k = 1; k <= p; ++k) {
    const Dir1D &s = sp[k];
    for (int e = 0; e < n_el; ++e)
      for (int q = 0; q < nq; ++q) {
        double v = 0.0;
        for (int m = 0; m <= s.p; ++m) v += y[col(k, e + m)] * hsc(k, e + m) * s.at(0, e, q, m);
        tau_q[((size_t)(k - 1) * n_el + e) * nq + q] = v;
      }
  }
  return true;
}

}  // namespace

int band_lu_inplace(double *a, int n, int p) {
  int B = 2 * p + 1;
  for (int k = 0; k < n; ++k) {
    double piv = a[(size_t)k * B + p];
    if (!(std::fabs(piv) > 0) || !std::isfinite(piv)) return -1;
    for (int i = k + 1; i <= std::min(n - 1, k + p); ++i) {
      double l = a[(size_t)i * B + (k - i + p)] / piv;
      a[(size_t)i * B + (k - i + p)] = l;
      for (int j = k + 1; j <= std::min(n - 1, k + p); ++j) a[(size_t)i * B + (j - i + p)] -= l * a[(size_t)k * B + (j - k + p)];
    }
  }
  for (int k = 0; k < n; ++k) a[(size_t)k * B + p] = 1.0 / a[(size_t)k * B + p];
  return 0;
}

namespace {
// M_t, W_t on X_t and the banded LU of W_t + b d_e M_t (the time matrix of the
// w-system, Eq. lin_sys_L) for the time direction `td`: the one definition
// shared by the handle set-up and the handle-free w-update.
st_status time_bands(const Dir1D &td, const st_problem_desc &d, std::vector<double> &Mt, std::vector<double> &Wt,
                     std::vector<double> &wlu) {
  const int p = d.p;
  Mt = band_matrix(td, 0, 0, 1);
  Wt = band_matrix(td, 0, 1, 1);   // row i tests b_i, column j carries b_j'
  const int Nt = td.n - 1;
  const int B = 2 * p + 1;
  wlu.assign((size_t)Nt * B, 0.0);
  for (size_t i = 0; i < wlu.size(); ++i) wlu[i] = Wt[i] + d.b * d.d_e * Mt[i];
  if (band_lu_inplace(wlu.data(), Nt, p) != 0) return ST_ERR_BREAKDOWN;
  return ST_OK;
}
}  // namespace

st_status host_setup(const st_problem_desc &d, HostSetup &hs) {
  int p = d.p;
  for (int l = 0; l < d.d; ++l) {
    build_dir(hs.sdir[l], d.n_el[l], p, 1.0, std::min(2, p), 0, d.breaks[l]);
    hs.M[l] = band_matrix(hs.sdir[l], 0, 0, 0);
    hs.K[l] = band_matrix(hs.sdir[l], 1, 1, 0);
  }
  build_dir(hs.tdir, d.n_el_t, p, d.T, p, 0, d.breaks_t);
  if (!tau_setup(hs.tdir, hs.tau_q)) return ST_ERR_BREAKDOWN;
  return time_bands(hs.tdir, d, hs.Mt, hs.Wt, hs.wlu);
}

// Time bands only (M_t and the banded LU of W_t + b d_e M_t); used by the
// handle-free w-update.
st_status host_time_bands(const st_problem_desc &d, std::vector<double> &Mt, std::vector<double> &wlu) {
  Dir1D td;
  build_dir(td, d.n_el_t, d.p, d.T, d.p, 0, d.breaks_t);
  std::vector<double> Wt;
  return time_bands(td, d, Mt, Wt, wlu);
}
