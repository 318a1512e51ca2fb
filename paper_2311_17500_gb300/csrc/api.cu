// C ABI of libst.so: set-up, operator, preconditioner, Krylov solver and the
// nonlinear loop of the space-time IgA monodomain solver (include/st.h).
#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>
#include "st_internal.h"

void launch_gemm64(cudaStream_t s, double *C, const double *A, const double *X, int M, int N, int K,
                   long long sam, long long sak, long long sbk, long long sbc, long long scm, long long scc,
                   double alpha, double beta, double *work = nullptr, long long work_elems = 0);

namespace {

struct Sizes {
  int d, p, nq, B;
  int n[3], nel[3], Q[3];
  int Nt, nel_t, Qt;
  long long Ns, Ndof, Qs, Nel_s, NtQs;
  int m, nmax, cap;
  bool lean;
  long long rows_x, wcap;
  long long gpart;   // values of a separate Gram partial-sum buffer (0: the first work buffer holds them)
  size_t bytes;
};

// The lean operator form applies to d >= 2 with an x row in one block.
bool lean_applies(const st_problem_desc &D) { return D.d >= 2 && xlean_feasible(D.n_el[0], D.p); }

// Device bytes above which ST_FORM_AUTO takes the lean form.
constexpr size_t kBandFormLimit = (size_t)160 << 30;

Sizes plan(const st_problem_desc &D);

st_status validate(const st_problem_desc *d) {
  if (!d) return ST_ERR_ARG;
  if (d->d < 1 || d->d > 3 || d->p < 1 || d->p > ST_MAXP) return ST_ERR_ARG;
  for (int l = 0; l < d->d; ++l)
    if (d->n_el[l] < 1 || d->n_el[l] > 1024 || !(d->D[l] > 0)) return ST_ERR_ARG;
  if (d->n_el_t < 1 || d->n_el_t > 60000) return ST_ERR_ARG;
  if (!(d->T > 0) || !(d->C_m > 0)) return ST_ERR_ARG;
  if (d->source_kind < ST_SRC_ZERO || d->source_kind > ST_SRC_E1_MMS) return ST_ERR_ARG;
  if (d->source_kind == ST_SRC_E1_MMS && d->d != 1) return ST_ERR_ARG;
  if (d->n_stim < 0 || d->n_stim > ST_MAX_STIM) return ST_ERR_ARG;
  if (d->stabilization != ST_GALERKIN && d->stabilization != ST_SU) return ST_ERR_ARG;
  if (d->suppext != ST_SUPPEXT_LITERAL && d->suppext != ST_SUPPEXT_SYMMETRIC) return ST_ERR_ARG;
  if (d->nonlinear != ST_PICARD && d->nonlinear != ST_NEWTON) return ST_ERR_ARG;
  if (d->precision != ST_FP64 && d->precision != ST_MIXED) return ST_ERR_ARG;
  if (d->gmres_m < 1 || d->gmres_m > 500 || !(d->rtol > 0) || d->max_it < 1) return ST_ERR_ARG;
  if (!(d->eps_theta >= 0) || !(d->alpha > 0) || d->alpha > 1 || !(d->delta >= 0) || d->max_fp < 1)
    return ST_ERR_ARG;
  if (d->operator_form < ST_FORM_AUTO || d->operator_form > ST_FORM_LEAN) return ST_ERR_ARG;
  if (d->inner_op < ST_INNER_AUTO || d->inner_op > ST_INNER_DF) return ST_ERR_ARG;
  if (!(d->eps_reaction == d->eps_reaction)) return ST_ERR_ARG;   // NaN
  if (d->precond_arith < ST_PRECOND_AUTO || d->precond_arith > ST_PRECOND_FP64) return ST_ERR_ARG;
  auto breaks_ok = [](const double *b, int n_el) {
    if (!b) return true;
    if (!(b[0] == 0.0) || !(b[n_el] == 1.0)) return false;
    for (int e = 0; e < n_el; ++e)
      if (!(b[e + 1] > b[e])) return false;
    return true;
  };
  for (int l = 0; l < d->d; ++l)
    if (!breaks_ok(d->breaks[l], d->n_el[l])) return ST_ERR_ARG;
  if (!breaks_ok(d->breaks_t, d->n_el_t)) return ST_ERR_ARG;
  if (d->operator_form == ST_FORM_LEAN && !lean_applies(*d)) return ST_ERR_ARG;
  return ST_OK;
}

Sizes plan(const st_problem_desc &D) {
  Sizes z;
  z.d = D.d; z.p = D.p; z.nq = D.p + 1; z.B = 2 * D.p + 1;
  z.Ns = 1; z.Qs = 1; z.Nel_s = 1;
  for (int l = 0; l < 3; ++l) {
    if (l < D.d) { z.nel[l] = D.n_el[l]; z.n[l] = D.n_el[l] + D.p; z.Q[l] = D.n_el[l] * z.nq; }
    else { z.nel[l] = 1; z.n[l] = 1; z.Q[l] = 1; }
    z.Ns *= z.n[l]; z.Qs *= z.Q[l]; z.Nel_s *= z.nel[l];
  }
  z.nel_t = D.n_el_t;
  z.Nt = D.n_el_t + D.p - 1;
  z.Qt = D.n_el_t * z.nq;
  z.Ndof = z.Ns * z.Nt;
  z.NtQs = (long long)z.Nt * z.Qs;
  z.m = D.gmres_m;
  z.nmax = z.Nt;
  for (int l = 0; l < D.d; ++l) z.nmax = std::max(z.nmax, z.n[l]);
  z.cap = (int)std::min<long long>(z.Nt, z.Ns);
  // automatic form: the band form, faster per apply wherever it fits (FP32
  // apply on GB300: 0.30 against 1.23 ms on the 2D p = 3, 128^2 x 256 mesh,
  // 5.1 against 16 ms on the 3D p = 2, 64^3 x 128 one), unless its footprint
  // exceeds kBandFormLimit and the lean form applies
  z.lean = D.operator_form == ST_FORM_LEAN;
  if (D.operator_form == ST_FORM_AUTO && lean_applies(D)) {
    st_problem_desc b = D;
    b.operator_form = ST_FORM_BANDS;
    z.lean = plan(b).bytes > kBandFormLimit;
  }
  z.rows_x = 1;
  for (int l = 1; l < D.d; ++l) z.rows_x *= z.Q[l];
  // values per Gauss-point work buffer: every spatial Gauss point of every time
  // row in the band form; in the lean form the Gauss rows of the other axes
  // with x in coefficients (the largest array of the apply), at least N_dof
  z.wcap = z.lean ? std::max<long long>((long long)z.Nt * z.rows_x * z.n[0], z.Ndof) : z.NtQs;
  // the Gram matrix of the low-rank steps sums 64 x 64 tiles of partial sums,
  // at least one per upper-triangle tile pair: small problems need more room
  // than their work buffer
  {
    const long long nt = (z.Nt + kGramTile - 1) / kGramTile;
    const long long need = nt * (nt + 1) / 2 * kGramTile * kGramTile;
    z.gpart = need > z.wcap ? need : 0;
  }
  size_t b = 0;
  size_t d8 = sizeof(double), f4 = sizeof(float);
  // 1D data (generous)
  b += (size_t)(6 * z.nmax * z.B + 4 * z.nmax * z.nmax) * (d8 + f4) + (size_t)z.Qt * (z.p + 2) * z.nq * d8 * 4;
  b += (size_t)(3 * z.nmax * z.nq * z.nq * 4) * d8;
  // rows padded to a multiple of 4 (FP32 LU and the tensor-core transforms)
  const size_t nxp = (size_t)(z.n[0] + 3) / 4 * 4;
  const size_t Ns_pad = (size_t)z.Ns / z.n[0] * nxp;
  size_t np = (size_t)z.Nt;
  for (int l = 0; l < z.d; ++l) np *= (size_t)(z.n[l] + 3) / 4 * 4;
  b += (size_t)z.Ns * d8;                                          // mu
  b += (size_t)z.Nt * z.B * (z.Ns * d8 + Ns_pad * f4);             // LU per eigen-index (FP64, padded FP32)
  if (z.lean) {
    b += (size_t)z.wcap * d8 * 2;                                  // two work buffers (FP32 ones alias them)
    b += (size_t)z.Nt * z.rows_x * z.n[0] * d8 * 2;                // u^k, w^k rows (pairs)
    b += (size_t)z.cap * d8 + (size_t)z.Qt * d8;                   // rank scales, time weight pairs
  } else {
    b += (size_t)(z.p + 1) * z.NtQs * (f4 + f4);                   // bands (high + low parts)
    b += (size_t)z.NtQs * d8 * 5;                                  // two work buffers + ionic fields
    b += (size_t)z.NtQs * f4 * 2;
  }
  b += (size_t)z.Ndof * d8 * 9;                                    // f, theta, FP64 vectors
  b += (size_t)z.Ndof * f4 * 4;                                    // FP32 vectors
  b += (size_t)z.nel_t * z.Nel_s * 8;                              // element maxima
  b += (size_t)z.Nt * z.Nt * d8 * 2 + (size_t)z.nmax * z.nmax * (12 * d8 + 2 * f4);
  b += (size_t)z.cap * (z.Nt + z.Ns + 1 + z.Qt + 2 * (z.p + 1) * z.Nt) * d8;
  b += (size_t)z.Ndof * (d8 + f4) * 7;                             // Kronecker temporaries
  b += 2 * (std::max<size_t>(np, 2 * (size_t)z.Ndof) + 64) * f4;   // padded transform buffers
  if (D.precision == ST_FP64) b += (size_t)(2 * z.m + 1) * (z.Ndof + 64) * d8;
  else b += (size_t)(2 * z.m + 1) * (z.Ndof + 64) * f4;
  if (D.eps_reaction >= 0.0) {                                     // low-rank reaction factors and bands
    b += (size_t)z.cap * (z.Nt + z.Ns + 2 + z.Qt + (z.p + 1) * z.Nt) * d8 + (size_t)z.cap * (z.p + 1) * z.Nt * 8;
    b += (size_t)(2 * z.nmax + z.Nt) * z.B * d8;
  }
  b += (size_t)z.gpart * d8;                                       // Gram partial sums (small problems)
  b += (size_t)(608 * (2 * z.m + 56) + 4096) * d8;                 // reduction scratch
  b += 2 * (size_t)(2 * (z.m + 2) + 8) * d8 + 256;                 // Hessenberg column, DCGS2 coefficients, flags
  b += 64 * 1024;   // small tables: 1D data of tiny meshes (one element at least each), Gauss-point hats
  z.bytes = b;
  return z;
}

template <typename T>
T *dalloc(st_handle *h, size_t count, st_status *err) {
  return (T *)st_alloc(h, count * sizeof(T), err);
}

template <typename T>
st_status upload(st_handle *h, T **dst, const std::vector<double> &src) {
  st_status e = ST_OK;
  *dst = dalloc<T>(h, std::max<size_t>(src.size(), 1), &e);
  if (e != ST_OK) return e;
  std::vector<T> tmp(src.begin(), src.end());
  if (!tmp.empty()) ST_CUDA(cudaMemcpyAsync(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  ST_CUDA(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

template <typename T>
st_status upload_vec(st_handle *h, T **dst, const std::vector<T> &src) {
  st_status e = ST_OK;
  *dst = dalloc<T>(h, std::max<size_t>(src.size(), 1), &e);
  if (e != ST_OK) return e;
  if (!src.empty()) ST_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  ST_CUDA(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

st_status upload_i(st_handle *h, int **dst, const std::vector<int> &src) {
  st_status e = ST_OK;
  *dst = dalloc<int>(h, std::max<size_t>(src.size(), 1), &e);
  if (e != ST_OK) return e;
  if (!src.empty()) ST_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  ST_CUDA(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

// left node and weight of the linear interpolation on `grid` at each point
void hat_data(const std::vector<double> &grid, const std::vector<double> &pts, std::vector<int> &idx,
              std::vector<double> &lam) {
  int n = (int)grid.size();
  idx.assign(pts.size(), 0);
  lam.assign(pts.size(), 0.0);
  if (n < 2) return;
  for (size_t k = 0; k < pts.size(); ++k) {
    double x = pts[k];
    int i = (int)(std::upper_bound(grid.begin(), grid.end(), x) - grid.begin()) - 1;
    i = std::max(0, std::min(n - 2, i));
    double l = (x - grid[i]) / (grid[i + 1] - grid[i]);
    idx[k] = i;
    lam[k] = std::max(0.0, std::min(1.0, l));
  }
}

double host_scalar(st_handle *h, const double *dptr) {
  double v = 0.0;
  cudaMemcpyAsync(&v, dptr, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  return v;
}

double norm2_64(st_handle *h, const double *x) {
  launch_norm2_64(h->stream, h->red + 4000, x, h->Ndof, h->red + 4096);
  return std::sqrt(host_scalar(h, h->red + 4000));
}

double absmax_diff(st_handle *h, const double *x, const double *y) {
  launch_absmax64(h->stream, h->red + 4000, x, y, h->Ndof, h->red + 4096);
  return host_scalar(h, h->red + 4000);
}

// Krylov basis accessors
template <typename T> T *basis(st_handle *h);
template <> double *basis<double>(st_handle *h) { return h->V64; }
template <> float *basis<float>(st_handle *h) { return h->V32; }

// Flexible right-preconditioned GMRES(m) on A_T d = b from d = 0, one cycle of
// at most `maxit` (<= m) iterations; stops when the Arnoldi residual estimate
// drops to tol * ||b||.  The preconditioned vectors z_j = M^{-1} v_j are kept
// (Z basis) and d = Z y, so the update matches the Arnoldi relation even when
// the preconditioner is applied with rounded (TF32) transform inputs.
// Gram-Schmidt: classical with one reorthogonalization, inner products
// accumulated in FP64 in a fixed order; Hessenberg and Givens in FP64.
template <typename T> T *zbasis(st_handle *h);
template <> double *zbasis<double>(st_handle *h) { return h->Z64; }
template <> float *zbasis<float>(st_handle *h) { return h->Z32; }

// The operator inside a Krylov cycle: the FP64 cycle applies it in FP64; the
// FP32 cycle in FP32, or in double-float on its FP32 vectors (converted to
// FP64 around the FP64 operator) when the handle's inner solve needs the
// accuracy.
template <typename T> st_status inner_apply(st_handle *h, const T *z, T *w);
template <> st_status inner_apply<double>(st_handle *h, const double *z, double *w) { return apply_T<double>(h, z, w); }
template <> st_status inner_apply<float>(st_handle *h, const float *z, float *w) {
  if (!h->inner_df) return apply_T<float>(h, z, w);
  launch_f2d(h->stream, h->z64, z, h->Ndof);
  ST_TRY(apply_T<double>(h, h->z64, h->t64a));
  launch_d2f(h->stream, w, h->t64a, 1.0, h->Ndof);
  return ST_OK;
}

// The preconditioner inside a Krylov cycle: FP64 in the FP64 cycle; in the
// FP32 cycle the FP32 (TF32) one, or the FP64 one on the FP32 vectors
// (converted around it) when the handle's inner solve needs the accuracy.
template <typename T> st_status inner_precond(st_handle *h, const T *v, T *z);
template <> st_status inner_precond<double>(st_handle *h, const double *v, double *z) { return precond_T<double>(h, v, z); }
template <> st_status inner_precond<float>(st_handle *h, const float *v, float *z) {
  if (!h->pre64) return precond_T<float>(h, v, z);
  launch_f2d(h->stream, h->r64, v, h->Ndof);
  ST_TRY(precond_T<double>(h, h->r64, h->t64b));
  launch_d2f(h->stream, z, h->t64b, 1.0, h->Ndof);
  return ST_OK;
}

template <typename T>
st_status gmres_cycle(st_handle *h, const T *b, T *d, double tol, int maxit, int *its, double *est) {
  cudaStream_t s = h->stream;
  long long N = h->Ndof, ld = h->ldv;
  T *V = basis<T>(h);
  T *Z = zbasis<T>(h);
  int m = std::min(maxit, h->m);
  double *hd = h->hcol;           // device: dots D[0 .. 2(m+2)), then (nu, gam, sw)
  double *sc = hd + 2 * (m + 2);
  double *scratch = h->red + 4096;
  launch_multi_dot<T>(s, hd, b, N, 1, b, N, scratch);
  double beta = std::sqrt(host_scalar(h, hd));
  *its = 0;
  if (!(beta > 0.0) || !std::isfinite(beta)) {
    ST_CUDA(cudaMemsetAsync(d, 0, N * sizeof(T), s));
    *est = std::isfinite(beta) ? 0.0 : INFINITY;
    return std::isfinite(beta) ? ST_OK : ST_ERR_NAN;
  }
  launch_scale_copy<T>(s, V, b, 1.0 / beta, N);   // u_0
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), g(m + 1, 0.0);
  std::vector<double> hh(2 * (m + 2) + 3);
  // first-projection coefficients of the previous column: <V_i, w> (i < j-1),
  // <v_{j-1}, w> and the scale of the vector it left behind
  std::vector<double> bprev(m + 1, 0.0);
  double gprev = 0.0, sprev = 1.0;
  double res = beta;
  int k = 0;
  bool done = false;
  // Givens rotations of the finished column c, residual estimate |g[c+1]|
  auto close_column = [&](int c) {
    for (int i = 0; i < c; ++i) {
      double a = H[(size_t)i * m + c], e = H[(size_t)(i + 1) * m + c];
      H[(size_t)i * m + c] = cs[i] * a + sn[i] * e;
      H[(size_t)(i + 1) * m + c] = -sn[i] * a + cs[i] * e;
    }
    double a = H[(size_t)c * m + c], e = H[(size_t)(c + 1) * m + c];
    double r = std::hypot(a, e);
    cs[c] = r > 0 ? a / r : 1.0;
    sn[c] = r > 0 ? e / r : 0.0;
    H[(size_t)c * m + c] = r;
    H[(size_t)(c + 1) * m + c] = 0.0;
    g[c + 1] = -sn[c] * g[c];
    g[c] = cs[c] * g[c];
    res = std::fabs(g[c + 1]);
  };
  // column c = j-1 from its first projection and the reorthogonalization of
  // u_j (a_i = <V_i, u_j>, nu = |u_j - V a|):  A z_c = V (b + a/s) + (nu/s) v_j
  auto finish_column = [&](int j, const double *a, double nu) {
    const int c = j - 1;
    for (int i = 0; i < c; ++i) H[(size_t)i * m + c] = bprev[i] + a[i] / sprev;
    H[(size_t)c * m + c] = gprev + a[c] / sprev;
    H[(size_t)j * m + c] = nu / sprev;
    close_column(c);
  };
  std::vector<double> acol(m + 1);
  // Iterations are enqueued one ahead of the host: iteration j+1 goes to the
  // stream before the coefficients of iteration j are read back (into one of
  // two pinned slots), unless the residual estimate extrapolated from the
  // last two columns says iteration j may end the cycle.  An iteration
  // launched past the end of the cycle only writes basis columns that are
  // not used.
  const int nhh = (int)hh.size();
  const size_t slot = (size_t)nhh + 1;   // coefficients, then the tensor-core error flag
  auto launch_iter = [&](int jj) -> st_status {
    T *uj = V + (long long)jj * ld, *w = V + (long long)(jj + 1) * ld, *zj = Z + (long long)jj * ld;
    ST_TRY(inner_precond<T>(h, uj, zj));
    ST_TRY(inner_apply<T>(h, zj, w));
    {
      // delayed CGS2: one dot pass of [V_0..V_{j-1}, u_j, w] against (u_j, w),
      // one update pass writing v_j and u_{j+1}
      double vb = (double)N * sizeof(T);
      ProfScope ps(h, PROF_ARNOLDI, vb * (2.0 * (jj + 2) + 2.0), 8.0 * (jj + 2) * (double)N);
      launch_multi_dot2<T>(s, hd, V, ld, jj + 2, uj, w, N, scratch);
      launch_dcgs2_update<T>(s, V, ld, jj, hd, N, sc, reinterpret_cast<T *>(h->gs_coef));
    }
    double *hs = h->red_host + (size_t)(jj & 1) * slot;
    ST_CUDA(cudaMemcpyAsync(hs, hd, nhh * sizeof(double), cudaMemcpyDeviceToHost, s));
    ST_CUDA(cudaMemcpyAsync(hs + nhh, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    ST_CUDA(cudaEventRecord(h->arn_ev[jj & 1], s));
    return ST_OK;
  };
  std::vector<double> resv(1, beta);   // residual estimate after c finished columns
  // Upper triangle of the rotated H against g over the first kk columns.
  auto solve_y = [&](int kk, std::vector<double> &y) {
    y.assign(kk, 0.0);
    for (int i = kk - 1; i >= 0; --i) {
      double t = g[i];
      for (int l = i + 1; l < kk; ++l) t -= H[(size_t)i * m + l] * y[l];
      const double piv = H[(size_t)i * m + i];
      y[i] = piv != 0.0 ? t / piv : 0.0;
    }
  };
  // The FP32 cycle's Arnoldi estimate keeps falling after the true residual of
  // its iterate has stopped at the level set by the FP32 vectors (about
  // u_32 ||A|| ||d|| / ||b||, which depends on the problem).  Past that level
  // the cycle only adds iterations: the outer FP64 residual takes it from
  // there.  So when the estimate first drops below each decade from 1e-3, and
  // every 10 columns after the first check, the cycle forms its iterate
  // (Z y, one operator application) and ends once the true residual exceeds
  // twice the estimate.  (Above that level the two agree to rounding, also
  // through the plateaus of a slowly converging cycle.)
  const bool check_floor = sizeof(T) == 4;
  double next_decade = 1e-3;
  int last_check = -1;
  std::vector<double> ychk;
  auto true_residual = [&](int kk, double *rt) -> st_status {
    solve_y(kk, ychk);
    for (int i = 0; i < kk; ++i) ychk[i] = -ychk[i];
    ychk.push_back(1.0);
    T *xc = reinterpret_cast<T *>(h->t32a), *ax = reinterpret_cast<T *>(h->t32b);
    ST_CUDA(cudaMemcpyAsync(hd, ychk.data(), (kk + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
    ST_CUDA(cudaMemsetAsync(xc, 0, N * sizeof(T), s));
    launch_multi_axpy<T>(s, xc, Z, ld, kk, hd, N);          // xc = Z y
    ST_TRY(inner_apply<T>(h, xc, ax));
    launch_scale_copy<T>(s, d, b, 1.0, N);
    launch_multi_axpy<T>(s, d, ax, ld, 1, hd + kk, N);      // d = b - A xc
    launch_multi_dot<T>(s, hd, d, N, 1, d, N, scratch);
    *rt = std::sqrt(host_scalar(h, hd)) / beta;
    return std::isfinite(*rt) ? ST_OK : ST_ERR_NAN;
  };
  ST_TRY(launch_iter(0));
  int launched = 1;
  int j = 0;
  for (; j < m; ++j) {
    if (launched == j + 1 && j + 1 < m) {
      bool ahead = true;
      if (j >= 2 && resv.size() >= (size_t)j) {
        const double r1 = resv[j - 1], r2 = resv[j - 2];
        ahead = r2 > 0.0 && r1 * (r1 / r2) > 2.0 * tol * beta;
      }
      if (ahead) {
        ST_TRY(launch_iter(j + 1));
        ++launched;
      }
    }
    ST_CUDA(cudaEventSynchronize(h->arn_ev[j & 1]));
    const double *hs = h->red_host + (size_t)(j & 1) * slot;
    int tc_flag = 0;
    std::memcpy(&tc_flag, hs + nhh, sizeof(int));
    if (tc_flag) return ST_ERR_TIMEOUT;
    std::copy(hs, hs + nhh, hh.begin());
    const double nu = hh[2 * (m + 2)], gam = hh[2 * (m + 2) + 1], sw = hh[2 * (m + 2) + 2];
    if (!std::isfinite(nu) || !std::isfinite(gam) || !std::isfinite(sw)) return ST_ERR_NAN;
    if (j == 0) {
      g[0] = beta * nu;   // b = beta u_0 = beta nu v_0
    } else {
      for (int i = 0; i < j; ++i) acol[i] = hh[2 * i];
      finish_column(j, acol.data(), nu);
      resv.push_back(res);
      if (res <= tol * beta || nu == 0.0) { k = j; done = true; break; }
      const double e = res / beta;
      if (check_floor && (e < next_decade || (last_check >= 0 && j - last_check >= 10))) {
        while (next_decade > e) next_decade *= 0.1;
        double rt = 0.0;
        ST_TRY(true_residual(j, &rt));
        const bool stop = rt <= tol || rt > 2.0 * e;
        last_check = j;
        if (stop) { k = j; done = true; break; }
      }
    }
    for (int i = 0; i < j; ++i) bprev[i] = hh[2 * i + 1];
    gprev = gam;
    sprev = sw;
    if (launched == j + 1 && j + 1 < m) {
      ST_TRY(launch_iter(j + 1));
      ++launched;
    }
  }
  if (!done) {
    // the last column: reorthogonalization dots of u_m alone
    launch_multi_dot<T>(s, hd, V, ld, m + 1, V + (long long)m * ld, N, scratch);
    ST_CUDA(cudaMemcpyAsync(hh.data(), hd, (m + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    ST_CUDA(cudaStreamSynchronize(s));
    double q = hh[m];
    for (int i = 0; i < m; ++i) q -= hh[i] * hh[i];
    const double nu = q > 0.0 ? std::sqrt(q) : 0.0;
    if (!std::isfinite(nu)) return ST_ERR_NAN;
    finish_column(m, hh.data(), nu);
    k = m;
  }
  // back substitution H(0:k,0:k) y = g(0:k)
  std::vector<double> y;
  solve_y(k, y);
  // d = Z y, accumulated with the multi-axpy (d -= sum (-y_i) Z_i)
  for (int i = 0; i < k; ++i) y[i] = -y[i];
  ST_CUDA(cudaMemcpyAsync(hd, y.data(), std::max(k, 1) * sizeof(double), cudaMemcpyHostToDevice, s));
  ST_CUDA(cudaMemsetAsync(d, 0, N * sizeof(T), s));
  if (k > 0) launch_multi_axpy<T>(s, d, Z, ld, k, hd, N);
  *its = done ? k + 1 : k;   // operator applications (a converged cycle has one past its last column)
  *est = res / beta;
  ST_CUDA(cudaStreamSynchronize(s));
  return ST_OK;
}

}  // namespace

// ---------------------------------------------------------------- internals
namespace {
// A handle's entry points run on the handle's device, whatever device the
// calling thread has current; the thread's device is restored on return.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    int cur = 0;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess) prev = cur;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};
}  // namespace

static std::atomic<long long> g_launches{0};

namespace {
// Source positions of this thread's launches: the last one, and the one after
// which a CUDA error was first found pending (cleared once the error is gone).
struct LaunchNote {
  const char *file = nullptr;
  int line = 0;
  cudaError_t err = cudaSuccess;
  const char *efile = nullptr;
  int eline = 0;
};
thread_local LaunchNote g_launch_note;

const char *base_name(const char *file) {
  const char *base = file;
  for (const char *c = file; *c; ++c)
    if (*c == '/') base = c + 1;
  return base;
}
}  // namespace

void st_count_launch_at(const char *file, int line) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  LaunchNote &n = g_launch_note;
  const cudaError_t e = cudaPeekAtLastError();
  if (e == cudaSuccess) {
    n.err = cudaSuccess;
  } else if (n.err == cudaSuccess && n.file) {
    n.err = e;
    n.efile = n.file;
    n.eline = n.line;
  }
  n.file = file;
  n.line = line;
}

// the CUDA error behind the last ST_ERR_CUDA / ST_ERR_OOM, per thread
static thread_local char g_cuda_detail[320] = "";
void st_note_cuda_error(cudaError_t e, const char *file, int line) {
  LaunchNote &n = g_launch_note;
  if (n.err == e && n.efile) {
    std::snprintf(g_cuda_detail, sizeof(g_cuda_detail), "%s (%d) at %s:%d, pending since the launch at %s:%d",
                  cudaGetErrorName(e), (int)e, base_name(file), line, base_name(n.efile), n.eline);
  } else if (n.file) {
    std::snprintf(g_cuda_detail, sizeof(g_cuda_detail), "%s (%d) at %s:%d, last launch at %s:%d",
                  cudaGetErrorName(e), (int)e, base_name(file), line, base_name(n.file), n.line);
  } else {
    std::snprintf(g_cuda_detail, sizeof(g_cuda_detail), "%s (%d) at %s:%d", cudaGetErrorName(e), (int)e,
                  base_name(file), line);
  }
  n.err = cudaSuccess;
  n.efile = nullptr;
}
const char *st_cuda_detail() { return g_cuda_detail; }
static cudaEvent_t prof_event(st_handle *h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

ProfScope::ProfScope(st_handle *hh, int cat, double bytes, double flops) : h(hh), idx((size_t)-1) {
  if (!h->prof_on) return;
  st_handle::ProfRec r;
  r.cat = cat;
  r.a = prof_event(h);
  r.b = prof_event(h);
  r.bytes = bytes;
  r.flops = flops;
  cudaEventRecord(r.a, h->stream);
  idx = h->prof.size();
  h->prof.push_back(r);
}

ProfScope::~ProfScope() {
  if (idx != (size_t)-1) cudaEventRecord(h->prof[idx].b, h->stream);
}

void *st_alloc(st_handle *h, size_t bytes, st_status *err) {
  void *p = nullptr;
  const size_t n = std::max<size_t>(bytes, 16);
  const cudaError_t e = h->pooled ? cudaMallocAsync(&p, n, h->stream) : cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *err = ST_ERR_OOM;
    return nullptr;
  }
  h->allocs.push_back(p);
  return p;
}

namespace {
// Page-locked host slots of the Arnoldi coefficients, reused across handles:
// allocating and freeing page-locked memory per handle would synchronize the
// device each time.  One slot holds 2 (2 (m + 2) + 4) doubles for m <= 500.
constexpr size_t kPinnedSlot = 16384;
static_assert(2 * (2 * (500 + 2) + 4) * sizeof(double) <= kPinnedSlot, "pinned slot too small for m = 500");
std::mutex g_pinned_mutex;
std::vector<void *> g_pinned_free;

double *pinned_acquire() {
  {
    std::lock_guard<std::mutex> lk(g_pinned_mutex);
    if (!g_pinned_free.empty()) {
      void *p = g_pinned_free.back();
      g_pinned_free.pop_back();
      return static_cast<double *>(p);
    }
  }
  void *p = nullptr;
  if (cudaHostAlloc(&p, kPinnedSlot, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return static_cast<double *>(p);
}

void pinned_release(void *p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pinned_mutex);
  g_pinned_free.push_back(p);
}

// Whether the device has stream-ordered memory pools (checked once per device).
bool pools_supported(int dev) {
  static std::atomic<unsigned long long> known{0}, yes{0};
  const unsigned long long bit = 1ull << (dev & 63);
  if (known.load(std::memory_order_acquire) & bit) return (yes.load(std::memory_order_acquire) & bit) != 0;
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMemoryPoolsSupported, dev) != cudaSuccess) {
    cudaGetLastError();
    v = 0;
  }
  if (v) yes.fetch_or(bit, std::memory_order_release);
  known.fetch_or(bit, std::memory_order_release);
  return v != 0;
}
}  // namespace

template <typename T> struct Prec;
template <> struct Prec<double> {
  static const double *Mb(st_handle *h, int l) { return h->Mb[l]; }
  static const double *Kb(st_handle *h, int l) { return h->Kb[l]; }
  static const double *Mt(st_handle *h) { return h->Mtb; }
  static const double *Wt(st_handle *h) { return h->Wtb; }
  static const double *Bq(st_handle *h, int l) { return h->Bq[l]; }
  static double *W(st_handle *h, int i) { return h->W64[i]; }
  static double *K(st_handle *h, int i) { return h->K64[i]; }
  static const float *band_lo(st_handle *h) { return h->band_lo; }
  static const double *UT(st_handle *h, int l) { return h->UT64[l]; }
  static const double *U(st_handle *h, int l) { return h->U64[l]; }
  static const double *lu(st_handle *h) { return h->lu64; }
};
template <> struct Prec<float> {
  static const float *Mb(st_handle *h, int l) { return h->Mb32[l]; }
  static const float *Kb(st_handle *h, int l) { return h->Kb32[l]; }
  static const float *Mt(st_handle *h) { return h->Mtb32; }
  static const float *Wt(st_handle *h) { return h->Wtb32; }
  static const float *Bq(st_handle *h, int l) { return h->Bq32[l]; }
  static float *W(st_handle *h, int i) { return h->W32[i]; }
  static float *K(st_handle *h, int i) { return h->K32[i]; }
  static const float *band_lo(st_handle *) { return nullptr; }
  static const float *UT(st_handle *h, int l) { return h->UT32[l]; }
  static const float *U(st_handle *h, int l) { return h->U32[l]; }
  static const float *lu(st_handle *h) { return h->lu32; }
};

LeanTerms lean_terms(st_handle *h) {
  LeanTerms L;
  const st_problem_desc &D = h->desc;
  L.exact = 1;
  L.U1 = h->U1;
  L.W1 = h->W1;
  L.bt = h->bt2;   // k = 0 block of [k][e][gt][a]
  L.wt = h->wt2;
  for (int l = 0; l < 3; ++l) {
    L.ws[l] = h->wqs[l];
    L.hi[l] = h->hat_i_s[l];
    L.hl[l] = h->hat_l_s[l];
    L.n[l] = h->n[l];
    L.Q[l] = h->Q[l];
  }
  L.Rt = D.stabilization == ST_SU ? h->rank : 0;
  L.V = h->Vr;
  L.cf = h->cfr;
  L.Tb = h->Tr2;
  L.newton = h->lin_kind == ST_NEWTON;
  if (D.eps_reaction >= 0.0) {
    // the reaction term as rank terms of its own (no Gauss-point evaluation)
    L.exact = 0;
    L.V2 = h->VrC; L.cf2 = h->cfc; L.Tb2 = h->Tc2; L.R2 = h->rankC;
  }
  L.c1 = D.c1; L.c2 = D.c2; L.a = D.a;
  L.d = h->d; L.p = h->p; L.nel = h->nel[0]; L.Nt = h->Nt; L.nel_t = h->nel_t;
  return L;
}

// Arithmetic of one lean-kernel launch (flops, for the per-stage record): per
// element-thread and step, the x interpolation of three new rows, the band
// of the rank terms, the time integration of one element and the projection.
static double lean_flops(st_handle *h) {
  const double P = h->p, nq = h->nq;
  const bool exact = h->desc.eps_reaction < 0.0;
  const double R = (h->desc.stabilization == ST_SU ? h->rank : 0) + (exact ? 0 : h->rankC);
  const double per = (exact ? 3 : 1) * nq * (P + 1) + R * (P + 1) * nq + (2 * P + 1) * nq +
                     (exact ? nq * nq * (4 * (P + 1) + 6) : 0) + nq * (P + 1);
  return 2.0 * per * (double)h->nel[0] * (double)h->rows_x * (double)h->Nt;
}

// y = A x (Eq. lin_sys_A): Kronecker part C_m W_t (x) M_s + M_t (x) K_s by
// banded passes, then the reaction + SU part (I (x) B_s^T) band (I (x) B_s)
// by sum factorization in space and one banded product along time per
// spatial Gauss point.
template <typename T>
st_status apply_T(st_handle *h, const T *x, T *y) {
  typedef Prec<T> P;
  cudaStream_t s = h->stream;
  const st_problem_desc &D = h->desc;
  int p = h->p;
  long long nx = h->n[0], ny = h->n[1], nz = h->n[2], Nt = h->Nt, Ns = h->Ns;
  const double sz = sizeof(T);
  const double vec = (double)h->Ndof * sz;
  // FP64 with d >= 2: x as double-float pairs (in the second Gauss-point work
  // buffer, which the reaction part below only overwrites after its first
  // pass), read by the 2D Kronecker kernel and the first interpolation pass
  const bool fused = h->d >= 2 && (h->nel[0] + p + 31) / 32 * 32 <= xband_fused_limit(sizeof(T), p);
  float2 *xs = nullptr;
  if (sizeof(T) == 8 && (h->d == 2 || fused)) {
    xs = reinterpret_cast<float2 *>(h->W64[1]);
    ProfScope ps(h, PROF_APPLY64, 3.0 * (double)h->Ndof * sizeof(double));
    launch_split_df(s, xs, reinterpret_cast<const double *>(x), h->Ndof);
  }
  // --- Kronecker part
  const bool plane2 = h->d == 2;
  ProfScope *pk = new ProfScope(h, sizeof(T) == 8 ? PROF_APPLY64 : PROF_KRON, vec * (h->d == 1 ? 7 : plane2 ? 2 : 19));
  if (plane2 && launch_kron2d<T>(s, y, x, xs, P::Wt(h), P::Mt(h), P::Mb(h, 0), P::Kb(h, 0),
                                 P::Mb(h, 1), P::Kb(h, 1), (int)nx, (int)ny, (int)Nt, p, D.C_m, D.D[0], D.D[1])) {
    delete pk;
    pk = nullptr;
  }
  const T *bands[3];
  const T *ins[3];
  double cf[3];
  if (pk) {
    T *m = nullptr, *sK = nullptr;
    if (h->d == 1) {
      m = P::K(h, 0); sK = P::K(h, 1);
      bands[0] = P::Mb(h, 0); ins[0] = x; cf[0] = 1.0;
      launch_band_pass<T>(s, m, 1, bands, ins, cf, (int)nx, 1, Nt, p, false);
      bands[0] = P::Kb(h, 0); cf[0] = D.D[0];
      launch_band_pass<T>(s, sK, 1, bands, ins, cf, (int)nx, 1, Nt, p, false);
    } else if (h->d == 2) {
      T *a = P::K(h, 0), *b = P::K(h, 1);
      m = P::K(h, 2); sK = P::K(h, 3);
      bands[0] = P::Mb(h, 0); ins[0] = x; cf[0] = 1.0;
      launch_band_pass<T>(s, a, 1, bands, ins, cf, (int)nx, 1, Nt * ny, p, false);
      bands[0] = P::Kb(h, 0);
      launch_band_pass<T>(s, b, 1, bands, ins, cf, (int)nx, 1, Nt * ny, p, false);
      bands[0] = P::Mb(h, 1); ins[0] = a;
      launch_band_pass<T>(s, m, 1, bands, ins, cf, (int)ny, nx, Nt, p, false);
      bands[0] = P::Mb(h, 1); ins[0] = b; cf[0] = D.D[0];
      bands[1] = P::Kb(h, 1); ins[1] = a; cf[1] = D.D[1];
      launch_band_pass<T>(s, sK, 2, bands, ins, cf, (int)ny, nx, Nt, p, false);
    } else {
      T *a = P::K(h, 0), *b = P::K(h, 1), *c = P::K(h, 2), *e = P::K(h, 3), *g = P::K(h, 4);
      m = P::K(h, 5); sK = P::K(h, 6);
      cf[0] = 1.0;
      bands[0] = P::Mb(h, 0); ins[0] = x;
      launch_band_pass<T>(s, a, 1, bands, ins, cf, (int)nx, 1, Nt * ny * nz, p, false);
      bands[0] = P::Kb(h, 0);
      launch_band_pass<T>(s, b, 1, bands, ins, cf, (int)nx, 1, Nt * ny * nz, p, false);
      bands[0] = P::Mb(h, 1); ins[0] = a;
      launch_band_pass<T>(s, c, 1, bands, ins, cf, (int)ny, nx, Nt * nz, p, false);
      ins[0] = b;
      launch_band_pass<T>(s, e, 1, bands, ins, cf, (int)ny, nx, Nt * nz, p, false);
      bands[0] = P::Kb(h, 1); ins[0] = a;
      launch_band_pass<T>(s, g, 1, bands, ins, cf, (int)ny, nx, Nt * nz, p, false);
      bands[0] = P::Mb(h, 2); ins[0] = c;
      launch_band_pass<T>(s, m, 1, bands, ins, cf, (int)nz, nx * ny, Nt, p, false);
      bands[0] = P::Mb(h, 2); ins[0] = e; cf[0] = D.D[0];
      bands[1] = P::Mb(h, 2); ins[1] = g; cf[1] = D.D[1];
      bands[2] = P::Kb(h, 2); ins[2] = c; cf[2] = D.D[2];
      launch_band_pass<T>(s, sK, 3, bands, ins, cf, (int)nz, nx * ny, Nt, p, false);
    }
    bands[0] = P::Wt(h); ins[0] = m; cf[0] = D.C_m;
    bands[1] = P::Mt(h); ins[1] = sK; cf[1] = 1.0;
    launch_band_pass<T>(s, y, 2, bands, ins, cf, (int)Nt, Ns, 1, p, false);
    delete pk;
  }
  // --- reaction + SU part
  long long qd[3] = {h->Q[0], h->Q[1], h->Q[2]};
  long long nd[3] = {h->n[0], h->n[1], h->n[2]};
  const T *cur = x;
  int ping = 0;
  if (fused && sizeof(T) == 8) {
    // the FP64 operator on double-float pairs from the split x to the last
    // backward pass (no FP64 instruction per value); passes as below
    const float2 *cur2 = xs;
    for (int l = h->d - 1; l >= 1; --l) {
      long long inner = 1, outer = Nt;
      for (int k = 0; k < l; ++k) inner *= nd[k];
      for (int k = l + 1; k < h->d; ++k) outer *= qd[k];
      float2 *out2 = reinterpret_cast<float2 *>(P::W(h, ping));
      ProfScope ps(h, PROF_APPLY64, sz * (double)outer * inner * (h->n[l] + (double)h->Q[l]));
      launch_interp_fwd_pairs(s, out2, cur2, h->Bq2[l], h->nel[l], p, inner, outer);
      cur2 = out2;
      ping ^= 1;
    }
    long long rows = 1;
    for (int k = 1; k < h->d; ++k) rows *= qd[k];
    float2 *Y2 = reinterpret_cast<float2 *>(P::W(h, ping));
    if (h->lean) {
      ProfScope ps(h, PROF_APPLY64, (2.0 * sz + 16.0) * (double)Nt * rows * nx, lean_flops(h));
      ST_TRY(launch_xlean<float2>(s, lean_terms(h), Y2, cur2, h->Bq2[0], rows));
    } else {
      ProfScope ps(h, PROF_APPLY64, sz * ((double)(p + 1) * h->NtQs + 2.0 * (double)Nt * rows * nx));
      launch_xband_fused<float2>(s, Y2, cur2, h->band32, h->band_lo, h->Bq2[0], h->nel[0], (int)Nt, rows, p,
                                 h->tc_err);
    }
    cur2 = Y2;
    ping ^= 1;
    for (int l = 1; l < h->d; ++l) {
      long long inner = 1, outer = Nt;
      for (int k = 0; k < l; ++k) inner *= nd[k];
      for (int k = l + 1; k < h->d; ++k) outer *= qd[k];
      const bool last = l == h->d - 1;
      ProfScope ps(h, PROF_APPLY64, sz * (double)outer * inner * (h->n[l] * (last ? 2.0 : 1.0) + (double)h->Q[l]));
      if (last) {
        launch_interp_bwd_pairs<double>(s, reinterpret_cast<double *>(y), cur2, h->Bq2[l], h->nel[l], p, inner,
                                        outer, true);
      } else {
        float2 *out2 = reinterpret_cast<float2 *>(P::W(h, ping));
        launch_interp_bwd_pairs<float2>(s, out2, cur2, h->Bq2[l], h->nel[l], p, inner, outer, false);
        cur2 = out2;
        ping ^= 1;
      }
    }
    ST_CUDA(cudaGetLastError());
    return ST_OK;
  }
  if (fused) {
    // the other axes to their Gauss points (last axis first), x kept in
    // coefficients; then the fused x pass; then the other axes back, the
    // last one accumulated onto the Kronecker part
    for (int l = h->d - 1; l >= 1; --l) {
      long long inner = 1, outer = Nt;
      for (int k = 0; k < l; ++k) inner *= nd[k];
      for (int k = l + 1; k < h->d; ++k) outer *= qd[k];
      T *out = P::W(h, ping);
      ProfScope ps(h, sizeof(T) == 8 ? PROF_APPLY64 : PROF_INTERP, sz * (double)outer * inner * (h->n[l] + (double)h->Q[l]));
      launch_interp_fwd<T>(s, out, cur, P::Bq(h, l), h->nel[l], p, h->nq, inner, outer);
      cur = out;
      ping ^= 1;
    }
    long long rows = 1;
    for (int k = 1; k < h->d; ++k) rows *= qd[k];
    T *Y1 = P::W(h, ping);
    if (h->lean) {
      // the FP32 operator (the FP64 one takes the pair branch above)
      ProfScope ps(h, PROF_QBAND, (2.0 * sz + 16.0) * (double)Nt * rows * nx, lean_flops(h));
      ST_TRY(launch_xlean<float>(s, lean_terms(h), reinterpret_cast<float *>(Y1), reinterpret_cast<const float *>(cur),
                                 h->Bq32[0], rows));
    } else {
      ProfScope ps(h, sizeof(T) == 8 ? PROF_APPLY64 : PROF_QBAND, sz * ((double)(p + 1) * h->NtQs + 2.0 * (double)Nt * rows * nx));
      launch_xband_fused<T>(s, Y1, cur, h->band32, P::band_lo(h), P::Bq(h, 0), h->nel[0], (int)Nt, rows, p, h->tc_err);
    }
    cur = Y1;
    ping ^= 1;
    for (int l = 1; l < h->d; ++l) {
      long long inner = 1, outer = Nt;
      for (int k = 0; k < l; ++k) inner *= nd[k];
      for (int k = l + 1; k < h->d; ++k) outer *= qd[k];
      const bool last = l == h->d - 1;
      T *out = last ? y : P::W(h, ping);
      ProfScope ps(h, sizeof(T) == 8 ? PROF_APPLY64 : PROF_INTERP, sz * (double)outer * inner * (h->n[l] * (last ? 2.0 : 1.0) + (double)h->Q[l]));
      launch_interp_bwd<T>(s, out, cur, P::Bq(h, l), h->nel[l], p, h->nq, inner, outer, last);
      cur = out;
      ping ^= 1;
    }
    ST_CUDA(cudaGetLastError());
    return ST_OK;
  }
  for (int l = 0; l < h->d; ++l) {
    long long inner = 1, outer = Nt;
    for (int k = 0; k < l; ++k) inner *= qd[k];
    for (int k = l + 1; k < h->d; ++k) outer *= nd[k];
    T *out = P::W(h, ping);
    ProfScope ps(h, sizeof(T) == 8 ? PROF_APPLY64 : PROF_INTERP, sz * (double)outer * inner * (h->n[l] + (double)h->Q[l]));
    launch_interp_fwd<T>(s, out, cur, P::Bq(h, l), h->nel[l], p, h->nq, inner, outer);
    cur = out;
    ping ^= 1;
  }
  T *zq = P::W(h, ping);
  {
    ProfScope ps(h, sizeof(T) == 8 ? PROF_APPLY64 : PROF_QBAND, sz * (double)h->NtQs * (p + 3));
    launch_qband_apply<T>(s, zq, cur, h->band32, P::band_lo(h), h->Nt, h->Qs, p);
  }
  cur = zq;
  ping ^= 1;
  for (int l = h->d - 1; l >= 0; --l) {
    long long inner = 1, outer = Nt;
    for (int k = 0; k < l; ++k) inner *= qd[k];
    for (int k = l + 1; k < h->d; ++k) outer *= nd[k];
    T *out = (l == 0) ? y : P::W(h, ping);
    ProfScope ps(h, sizeof(T) == 8 ? PROF_APPLY64 : PROF_INTERP, sz * (double)outer * inner * (h->n[l] * (l == 0 ? 2.0 : 1.0) + (double)h->Q[l]));
    launch_interp_bwd<T>(s, out, cur, P::Bq(h, l), h->nel[l], p, h->nq, inner, outer, l == 0);
    cur = out;
    ping ^= 1;
  }
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

// z = A-hat^{-1} r by fast diagonalization (Eq. factorized).  Each spatial
// transform contracts the contiguous axis and writes the result rotated
// ([T][a][b] -> [T][j][a]), so after the d forward transforms (with U_l^T)
// the eigen-indices are back in the natural order for the banded LU solves
// along time, and the d backward transforms (with U_l) restore [T][z][y][x].
// FP32 transforms run on the tensor cores (TF32) when the self-test passed.
// One transform of the sequence: contract the innermost axis (length n_l,
// row stride in_stride) and write [T][j][remaining axes], the new innermost
// axis of length A_inner stored with row stride A_stride.
struct RotStep {
  int l;
  long long Aa, A_inner, A_stride;
};

// Steps of the forward (and, identically, the backward) sequence: axis order
// outer -> inner starts as (z, y, x); each step contracts the innermost axis
// and moves the new index to the front.
static void rot_plan(const st_handle *h, RotStep *steps, bool pad_last) {
  int order[3], no = 0;
  for (int l = h->d - 1; l >= 0; --l) order[no++] = l;   // outer .. inner
  for (int s = 0; s < h->d; ++s) {
    int c = order[no - 1];
    long long Aa = 1;
    for (int i = 0; i < no - 1; ++i) Aa *= h->n[order[i]];
    long long A_inner = no >= 2 ? h->n[order[no - 2]] : 1;
    bool last = (s == h->d - 1);
    long long A_stride = (!last || pad_last) ? (A_inner + 3) / 4 * 4 : A_inner;
    if (no == 1) A_stride = 1;
    steps[s] = RotStep{c, Aa, A_inner, A_stride};
    // new order: [j_c, order[0 .. no-2]]
    for (int i = no - 1; i > 0; --i) order[i] = order[i - 1];
    order[0] = c;
  }
}

template <typename T>
static void rot_simt(st_handle *h, T *out, const T *in, int l, bool fwd);
template <>
void rot_simt<double>(st_handle *h, double *out, const double *in, int l, bool fwd) {
  launch_rot_gemm<double>(h->stream, out, in, fwd ? h->UT64[l] : h->U64[l], h->n[l], h->n[l], h->Ns / h->n[l], h->Nt);
}
template <>
void rot_simt<float>(st_handle *h, float *out, const float *in, int l, bool fwd) {
  launch_rot_gemm<float>(h->stream, out, in, fwd ? h->UT32[l] : h->U32[l], h->n[l], h->n[l], h->Ns / h->n[l], h->Nt);
}

// Tensor-core sequence of d transforms (FP32).  Intermediate results use
// rows padded to a multiple of 4 floats (16-byte aligned for TMA).  The input
// is either the natural layout (copied into a padded buffer first) or already
// padded; the result is written to `out` in the natural layout, or, when out
// is null, padded into one of the two ping-pong buffers, returned in *res.
static st_status tc_sequence(st_handle *h, const float *in, bool in_padded, float *out, bool fwd, float **res) {
  cudaStream_t s = h->stream;
  RotStep st[3];
  rot_plan(h, st, out == nullptr);
  const float *cur = in;
  long long cur_stride = h->n[st[0].l];
  float *P[2] = {h->P32[0], h->P32[1]};
  int ping = (in == P[0]) ? 1 : 0;   // never write the buffer being read
  if (in_padded) {
    cur_stride = (cur_stride + 3) / 4 * 4;
  } else if (cur_stride % 4 != 0) {
    long long rows = h->Ndof / cur_stride;
    long long sp = (cur_stride + 3) / 4 * 4;
    ProfScope ps(h, PROF_FD_GEMM, 2.0 * h->Ndof * sizeof(float));
    launch_pad_rows(s, P[ping], cur, rows, cur_stride, sp);
    cur = P[ping];
    cur_stride = sp;
    ping ^= 1;
  }
  for (int k = 0; k < h->d; ++k) {
    const RotStep &r = st[k];
    int l = r.l;
    float *dst = (k == h->d - 1 && out) ? out : P[ping];
    ProfScope ps(h, PROF_FD_GEMM, 2.0 * h->Ndof * sizeof(float), 2.0 * h->n[l] * (double)h->Ndof);
    ST_TRY(launch_tc_xform(s, dst, cur, (long long)h->Nt * r.Aa, h->n[l], cur_stride, fwd ? h->UTp[l] : h->Up[l],
                           h->n[l], h->Npad[l], h->Kpad[l], r.Aa, r.A_inner, r.A_stride, h->tc_err));
    cur = dst;
    cur_stride = r.A_stride;
    ping ^= 1;
  }
  if (res) *res = const_cast<float *>(cur);
  return ST_OK;
}

// z = A-hat^{-1} r by fast diagonalization (Eq. factorized).  Each spatial
// transform contracts the contiguous axis and writes the result rotated
// ([T][a][b] -> [T][j][a]), so after the d forward transforms (with U_l^T)
// the eigen-indices are back in the natural order for the banded LU solves
// along time, and the d backward transforms (with U_l) restore [T][z][y][x].
// FP32 transforms run on the tensor cores (TF32) when the self-test passed.
template <typename T>
st_status precond_T(st_handle *h, const T *r, T *z) {
  typedef Prec<T> P;
  cudaStream_t s = h->stream;
  T *bufs[2] = {P::K(h, 0), P::K(h, 1)};
  const double vec = (double)h->Ndof * sizeof(T);
  const bool tc = (sizeof(T) == 4) && h->use_tc;
  if (tc && h->d == 1) {
    ST_TRY(tc_sequence(h, (const float *)r, false, (float *)bufs[0], true, nullptr));
    {
      ProfScope ps(h, PROF_FD_LU, vec * (2 + h->B));
      launch_tline_lu_solve<float>(s, (float *)bufs[1], (const float *)bufs[0], h->lu32, h->Nt, h->Ns, h->p, h->tc_err);
    }
    ST_TRY(tc_sequence(h, (const float *)bufs[1], false, (float *)z, false, nullptr));
    ST_CUDA(cudaGetLastError());
    return ST_OK;
  }
  if (tc) {
    // padded layout from the forward transforms through the LU to the
    // backward transforms
    float *fw = nullptr;
    ST_TRY(tc_sequence(h, (const float *)r, false, nullptr, true, &fw));
    float *lu_out = (fw == h->P32[0]) ? h->P32[1] : h->P32[0];
    {
      ProfScope ps(h, PROF_FD_LU, vec * (2 + h->B));
      launch_tline_lu_solve<float>(s, lu_out, fw, h->lu32, h->Nt, h->Ns_pad, h->p, h->tc_err);
    }
    ST_TRY(tc_sequence(h, lu_out, true, (float *)z, false, nullptr));
    ST_CUDA(cudaGetLastError());
    return ST_OK;
  } else {
    // r -> ... -> bufs[0], alternating so that no step writes its input
    const T *cur = r;
    for (int l = 0; l < h->d; ++l) {
      T *dst = bufs[(h->d - 1 - l) % 2];
      ProfScope ps(h, PROF_FD_GEMM, 2 * vec, 2.0 * h->n[l] * (double)h->Ndof);
      rot_simt<T>(h, dst, cur, l, true);
      cur = dst;
    }
  }
  {
    ProfScope ps(h, PROF_FD_LU, vec * (2 + h->B));
    launch_tline_lu_solve<T>(s, bufs[1], bufs[0], P::lu(h), h->Nt, h->Ns, h->p, h->tc_err);
  }
  {
    const T *cur = bufs[1];
    for (int l = 0; l < h->d; ++l) {
      T *dst = (l == h->d - 1) ? z : bufs[l % 2];
      ProfScope ps(h, PROF_FD_GEMM, 2 * vec, 2.0 * h->n[l] * (double)h->Ndof);
      rot_simt<T>(h, dst, cur, l, false);
      cur = dst;
    }
  }
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

template st_status apply_T<double>(st_handle *, const double *, double *);
template st_status apply_T<float>(st_handle *, const float *, float *);
template st_status precond_T<double>(st_handle *, const double *, double *);
template st_status precond_T<float>(st_handle *, const float *, float *);

// ---------------------------------------------------------------- C ABI
extern "C" {

const char *st_last_cuda_error(void) { return st_cuda_detail(); }

const char *st_error_string(st_status s) {
  switch (s) {
    case ST_OK: return "ok";
    case ST_ERR_ARG: return "invalid argument";
    case ST_ERR_OOM: return "device out of memory";
    case ST_ERR_CUDA: return "CUDA error";
    case ST_ERR_NOT_CONVERGED: return "not converged";
    case ST_ERR_BREAKDOWN: return "breakdown (zero pivot)";
    case ST_ERR_NAN: return "NaN or Inf detected";
    case ST_ERR_TIMEOUT: return "device wait timed out";
    case ST_ERR_STATE: return "invalid call order";
    case ST_ERR_CAPACITY: return "problem exceeds the fixed scratch of st_wupdate_static (2 N_t (2p+1) > ST_WUPDATE_STATIC_CAPACITY doubles)";
  }
  return "unknown status";
}

st_status st_footprint(const st_problem_desc *desc, size_t *bytes) {
  ST_TRY(validate(desc));
  if (!bytes) return ST_ERR_ARG;
  *bytes = plan(*desc).bytes;
  return ST_OK;
}

st_status st_destroy(st_handle *h) {
  if (!h) return ST_OK;
  {
    DeviceScope ds(h->dev);
    cudaStreamSynchronize(h->stream);
    if (h->pooled) {
      // freed in stream order, then waited for on this stream alone, so the
      // memory is back in the pool when the call returns
      for (void *p : h->allocs) cudaFreeAsync(p, h->stream);
      cudaStreamSynchronize(h->stream);
    } else {
      for (void *p : h->allocs) cudaFree(p);
    }
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : h->arn_ev)
      if (e) cudaEventDestroy(e);
    pinned_release(h->red_host);
  }
  delete h;
  return ST_OK;
}

st_status st_get_dims(const st_handle *h, st_dims *out) {
  if (!h || !out) return ST_ERR_ARG;
  out->N_s = h->Ns; out->N_t = h->Nt; out->N_dof = h->Ndof; out->Q_s = h->Qs;
  for (int l = 0; l < 3; ++l) out->n[l] = h->n[l];
  out->operator_form = h->lean ? ST_FORM_LEAN : ST_FORM_BANDS;
  out->precond_tc = h->use_tc ? 1 : 0;
  return ST_OK;
}

static st_status setup_impl(st_handle *h) {
  const st_problem_desc &D = h->desc;
  Sizes z = plan(D);
  h->d = z.d; h->p = z.p; h->nq = z.nq; h->B = z.B;
  for (int l = 0; l < 3; ++l) { h->n[l] = z.n[l]; h->nel[l] = z.nel[l]; h->Q[l] = z.Q[l]; }
  h->Nt = z.Nt; h->nel_t = z.nel_t; h->Qt = z.Qt;
  h->Ns = z.Ns; h->Ndof = z.Ndof; h->Qs = z.Qs; h->Nel_s = z.Nel_s; h->NtQs = z.NtQs;
  h->m = z.m;
  h->lean = z.lean;
  h->rows_x = z.rows_x;
  h->wcap = z.wcap;
  h->gpart_cap = z.gpart;
  h->ldv = (z.Ndof + 63) / 64 * 64;
  h->rank_cap = z.cap;
  ST_TRY(host_setup(D, h->hs));
  HostSetup &hs = h->hs;
  st_status e = ST_OK;
  // ---- 1D data
  for (int l = 0; l < h->d; ++l) {
    const Dir1D &dr = hs.sdir[l];
    ST_TRY(upload<double>(h, &h->Mb[l], hs.M[l]));
    ST_TRY(upload<double>(h, &h->Kb[l], hs.K[l]));
    ST_TRY(upload<float>(h, &h->Mb32[l], hs.M[l]));
    ST_TRY(upload<float>(h, &h->Kb32[l], hs.K[l]));
    size_t per = (size_t)dr.n_el * dr.nq * (dr.p + 1);
    std::vector<double> b0(dr.tab.begin(), dr.tab.begin() + per);
    std::vector<double> b2(per, 0.0);
    if (dr.kmax >= 2) b2.assign(dr.tab.begin() + 2 * per, dr.tab.begin() + 3 * per);
    ST_TRY(upload<double>(h, &h->Bq[l], b0));
    ST_TRY(upload<double>(h, &h->B2q[l], b2));
    {
      auto split = [](const std::vector<double> &v) {
        std::vector<float2> out(v.size());
        for (size_t i = 0; i < v.size(); ++i) {
          float hi = (float)v[i];
          out[i] = make_float2(hi, (float)(v[i] - (double)hi));
        }
        return out;
      };
      ST_TRY(upload_vec<float2>(h, &h->Bq2[l], split(b0)));
      ST_TRY(upload_vec<float2>(h, &h->B2q2[l], split(b2)));
    }
    ST_TRY(upload<float>(h, &h->Bq32[l], b0));
    ST_TRY(upload<double>(h, &h->wqs[l], dr.wq));
    ST_TRY(upload<double>(h, &h->xs[l], dr.xq));
  }
  ST_TRY(upload<double>(h, &h->Mtb, hs.Mt));
  ST_TRY(upload<double>(h, &h->Wtb, hs.Wt));
  ST_TRY(upload<float>(h, &h->Mtb32, hs.Mt));
  ST_TRY(upload<float>(h, &h->Wtb32, hs.Wt));
  ST_TRY(upload<double>(h, &h->bt, hs.tdir.tab));
  {
    // products w_t b_i b_{i+k} at the time Gauss points for the reaction bands
    const Dir1D &td = hs.tdir;
    int np = (h->p + 1) * (h->p + 2) / 2;
    std::vector<double> bp((size_t)td.n_el * td.nq * np);
    for (int e = 0; e < td.n_el; ++e)
      for (int q = 0; q < td.nq; ++q) {
        int pr = 0;
        for (int i = 0; i <= h->p; ++i)
          for (int k = 0; k <= h->p - i; ++k)
            bp[((size_t)e * td.nq + q) * np + pr++] = td.wq[e * td.nq + q] * td.at(0, e, q, i) * td.at(0, e, q, i + k);
      }
    ST_TRY(upload<double>(h, &h->bprod, bp));
    // the same tables split into double-float pairs for the ionic kernel
    auto split = [](const double *v, size_t n) {
      std::vector<float2> out(n);
      for (size_t i = 0; i < n; ++i) {
        float hi = (float)v[i];
        out[i] = make_float2(hi, (float)(v[i] - (double)hi));
      }
      return out;
    };
    const size_t nbt = (size_t)2 * td.n_el * td.nq * (h->p + 1);   // k = 0, 1 of [k][e][q][a]
    ST_TRY(upload_vec<float2>(h, &h->bt2, split(hs.tdir.tab.data(), nbt)));
    ST_TRY(upload_vec<float2>(h, &h->bprod2, split(bp.data(), bp.size())));
  }
  ST_TRY(upload<double>(h, &h->wt, hs.tdir.wq));
  {
    std::vector<float2> w2(hs.tdir.wq.size());
    for (size_t i = 0; i < w2.size(); ++i) {
      const float hi = (float)hs.tdir.wq[i];
      w2[i] = make_float2(hi, (float)(hs.tdir.wq[i] - (double)hi));
    }
    ST_TRY(upload_vec<float2>(h, &h->wt2, w2));
  }
  ST_TRY(upload<double>(h, &h->xt, hs.tdir.xq));
  {
    // stimulus windows of each time quadrature point ([t0, t1), as in the
    // source assembly)
    std::vector<int> tm(hs.tdir.xq.size(), 0);
    if (D.source_kind == ST_SRC_STIM)
      for (size_t i = 0; i < tm.size(); ++i)
        for (int b = 0; b < D.n_stim; ++b)
          if (hs.tdir.xq[i] >= D.stim[b].t0 && hs.tdir.xq[i] < D.stim[b].t1) tm[i] |= 1 << b;
    ST_TRY(upload_i(h, &h->tmask, tm));
  }
  ST_TRY(upload<double>(h, &h->tauq, hs.tau_q));
  ST_TRY(upload<double>(h, &h->wlu, hs.wlu));
  {
    std::vector<double> gt(hs.tdir.greville.begin() + 1, hs.tdir.greville.end());
    std::vector<int> ii;
    std::vector<double> ll;
    hat_data(gt, hs.tdir.xq, ii, ll);
    ST_TRY(upload_i(h, &h->hat_i_t, ii));
    ST_TRY(upload<double>(h, &h->hat_l_t, ll));
    for (int l = 0; l < h->d; ++l) {
      hat_data(hs.sdir[l].greville, hs.sdir[l].xq, ii, ll);
      ST_TRY(upload_i(h, &h->hat_i_s[l], ii));
      ST_TRY(upload<double>(h, &h->hat_l_s[l], ll));
    }
  }
  // ---- buffers
  int nmax = z.nmax;
  for (int l = 0; l < h->d; ++l) {
    size_t nn = (size_t)h->n[l] * h->n[l];
    h->U64[l] = dalloc<double>(h, nn, &e); h->UT64[l] = dalloc<double>(h, nn, &e);
    h->U32[l] = dalloc<float>(h, nn, &e); h->UT32[l] = dalloc<float>(h, nn, &e);
    h->lam[l] = dalloc<double>(h, h->n[l], &e);
  }
  h->mu = dalloc<double>(h, h->Ns, &e);
  h->lu64 = dalloc<double>(h, (size_t)h->Nt * h->B * h->Ns, &e);
  h->nxp = (h->n[0] + 3) / 4 * 4;
  h->Ns_pad = h->Ns / h->n[0] * h->nxp;
  h->lu32 = dalloc<float>(h, (size_t)h->Nt * h->B * h->Ns_pad, &e);
  if (!h->lean) {
    h->band32 = dalloc<float>(h, (size_t)(h->p + 1) * h->NtQs, &e);
    h->band_lo = dalloc<float>(h, (size_t)(h->p + 1) * h->NtQs, &e);
  } else {
    const size_t rn = (size_t)h->Nt * h->rows_x * h->n[0];
    h->U1 = dalloc<float2>(h, rn, &e);
    h->W1 = dalloc<float2>(h, rn, &e);
    h->cfr = dalloc<double>(h, h->rank_cap, &e);
  }
  h->f64 = dalloc<double>(h, h->Ndof, &e);
  h->emax = dalloc<unsigned long long>(h, (size_t)h->nel_t * h->Nel_s, &e);
  h->stats = dalloc<double>(h, 8, &e);
  h->theta = dalloc<double>(h, h->Ndof, &e);
  h->gram = dalloc<double>(h, (size_t)h->Nt * h->Nt, &e);
  h->evec = dalloc<double>(h, (size_t)h->Nt * h->Nt, &e);
  h->eval = dalloc<double>(h, h->Nt, &e);
  h->eig_work = dalloc<double>(h, (size_t)12 * nmax * nmax + 16 * (size_t)nmax + 64, &e);
  h->eig32 = dalloc<float>(h, (size_t)2 * nmax * nmax, &e);
  int cap = h->rank_cap;
  h->Ur = dalloc<double>(h, (size_t)h->Nt * cap, &e);
  h->sr = dalloc<double>(h, cap, &e);
  h->Vr = dalloc<double>(h, (size_t)h->Ns * cap, &e);
  h->th_t = dalloc<double>(h, (size_t)cap * h->Qt, &e);
  h->Tr = dalloc<double>(h, (size_t)cap * (h->p + 1) * h->Nt, &e);
  h->Tr2 = dalloc<float2>(h, (size_t)cap * (h->p + 1) * h->Nt, &e);
  if (D.eps_reaction >= 0.0) {
    for (int l = 0; l < h->d; ++l) ST_TRY(upload<double>(h, &h->Gsb[l], greville_band(hs.sdir[l], 0)));
    ST_TRY(upload<double>(h, &h->Gtb, greville_band(hs.tdir, 1)));
    h->UrC = dalloc<double>(h, (size_t)h->Nt * cap, &e);
    h->srC = dalloc<double>(h, cap, &e);
    h->cfc = dalloc<double>(h, cap, &e);
    h->VrC = dalloc<double>(h, (size_t)h->Ns * cap, &e);
    h->thC = dalloc<double>(h, (size_t)cap * h->Qt, &e);
    h->Tc = dalloc<double>(h, (size_t)cap * (h->p + 1) * h->Nt, &e);
    h->Tc2 = dalloc<float2>(h, (size_t)cap * (h->p + 1) * h->Nt, &e);
  }
  if (h->gpart_cap > 0) h->gpart = dalloc<double>(h, h->gpart_cap, &e);
  for (int i = 0; i < 2; ++i) {
    h->W64[i] = dalloc<double>(h, h->wcap, &e);
    // the lean form's FP32 work buffers share the FP64 ones: the two operators
    // run one after the other on the handle's stream and keep nothing there
    h->W32[i] = h->lean ? reinterpret_cast<float *>(h->W64[i]) : dalloc<float>(h, h->wcap, &e);
  }
  for (int i = 0; i < 7; ++i) {
    h->K64[i] = dalloc<double>(h, h->Ndof, &e);
    h->K32[i] = dalloc<float>(h, h->Ndof, &e);
  }
  if (!h->lean) {
    h->U0 = dalloc<double>(h, h->NtQs, &e);
    h->L0 = dalloc<double>(h, h->NtQs, &e);
    h->Wq0 = dalloc<double>(h, h->NtQs, &e);
  }
  h->red = dalloc<double>(h, 4096 + 608 * (size_t)(2 * h->m + 56), &e);
  if (D.precision == ST_FP64) {
    h->V64 = dalloc<double>(h, (size_t)(h->m + 1) * h->ldv, &e);
    h->Z64 = dalloc<double>(h, (size_t)h->m * h->ldv, &e);
  } else {
    h->V32 = dalloc<float>(h, (size_t)(h->m + 1) * h->ldv, &e);
    h->Z32 = dalloc<float>(h, (size_t)h->m * h->ldv, &e);
  }
  h->r64 = dalloc<double>(h, h->Ndof, &e);
  h->x64 = dalloc<double>(h, h->Ndof, &e);
  h->t64a = dalloc<double>(h, h->Ndof, &e);
  h->t64b = dalloc<double>(h, h->Ndof, &e);
  h->z64 = dalloc<double>(h, h->Ndof, &e);
  h->b64 = dalloc<double>(h, h->Ndof, &e);
  h->r32 = dalloc<float>(h, h->Ndof, &e);
  h->t32a = dalloc<float>(h, h->Ndof, &e);
  h->t32b = dalloc<float>(h, h->Ndof, &e);
  h->d32 = dalloc<float>(h, h->Ndof, &e);
  h->hcol = dalloc<double>(h, (size_t)2 * (h->m + 2) + 8, &e);
  // pinned host slots for the Arnoldi coefficients (two iterations in flight)
  // and the events that mark their arrival
  h->red_host = pinned_acquire();
  if (!h->red_host) return ST_ERR_OOM;
  for (int i = 0; i < 2; ++i) ST_CUDA(cudaEventCreateWithFlags(&h->arn_ev[i], cudaEventDisableTiming));
  h->gs_coef = dalloc<double>(h, (size_t)2 * (h->m + 2) + 8, &e);
  if (e != ST_OK) return e;
  {
    // padded layouts of the tensor-core preconditioner: every axis rounded up to 4
    size_t np = (size_t)h->Nt;
    for (int l = 0; l < h->d; ++l) np *= (size_t)((h->n[l] + 3) / 4 * 4);
    h->P32[0] = dalloc<float>(h, std::max<size_t>(np, 2 * h->Ndof) + 64, &e);
    h->P32[1] = dalloc<float>(h, std::max<size_t>(np, 2 * h->Ndof) + 64, &e);
  }
  h->tc_err = dalloc<int>(h, 4, &e);
  if (e != ST_OK) return e;
  ST_CUDA(cudaMemsetAsync(h->tc_err, 0, 4 * sizeof(int), h->stream));
  // ---- device set-up: fast diagonalization, right-hand side
  ST_TRY(fd_setup(h));
  {
    // zero-padded FP32 copies of U_l^T and U_l for the tensor-core transforms
    bool fits = true;
    for (int l = 0; l < h->d; ++l) fits = fits && h->n[l] <= 256;
    const bool want_tc = D.precond_arith == ST_PRECOND_TF32 || (D.precond_arith == ST_PRECOND_AUTO && h->d <= 2);
    if (fits && want_tc && tc_state(h->stream, nullptr) == 1) {
      for (int l = 0; l < h->d; ++l) {
        int n = h->n[l];
        h->Npad[l] = (n + 15) / 16 * 16;
        h->Kpad[l] = (n + 31) / 32 * 32;
        std::vector<double> U((size_t)n * n);
        ST_CUDA(cudaMemcpyAsync(U.data(), h->U64[l], U.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        ST_CUDA(cudaStreamSynchronize(h->stream));
        std::vector<double> ut((size_t)h->Npad[l] * h->Kpad[l], 0.0), uu((size_t)h->Npad[l] * h->Kpad[l], 0.0);
        for (int j = 0; j < n; ++j)
          for (int k = 0; k < n; ++k) {
            ut[(size_t)j * h->Kpad[l] + k] = U[(size_t)k * n + j];   // (U^T)[j][k]
            uu[(size_t)j * h->Kpad[l] + k] = U[(size_t)j * n + k];   // U[j][k]
          }
        ST_TRY(upload<float>(h, &h->UTp[l], ut));
        ST_TRY(upload<float>(h, &h->Up[l], uu));
      }
      h->use_tc = true;
      // FP32 LU factors in the padded layout of the tensor-core sequence (d >= 2)
      if (h->d >= 2)
        launch_pad_d2f(h->stream, h->lu32, h->lu64, (long long)h->Nt * h->B * (h->Ns / h->n[0]), h->n[0], h->nxp);
    }
  }
  ST_TRY(source_assemble(h));
  ST_CUDA(cudaStreamSynchronize(h->stream));
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

st_status st_setup(const st_problem_desc *desc, void *cuda_stream, st_handle **out) {
  if (!out) return ST_ERR_ARG;
  *out = nullptr;
  ST_TRY(validate(desc));
  st_handle *h = new st_handle();
  h->desc = *desc;
  h->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&h->dev);
  h->pooled = pools_supported(h->dev);
  st_status s = setup_impl(h);
  // the breakpoint arrays belong to the caller: the handle keeps only the
  // tables built from them
  for (int l = 0; l < 3; ++l) h->desc.breaks[l] = nullptr;
  h->desc.breaks_t = nullptr;
  if (s != ST_OK) {
    st_destroy(h);
    return s;
  }
  *out = h;
  return ST_OK;
}

st_status st_linearize(st_handle *h, const double *u, const double *w, int kind, int keep_theta,
                       st_ionic_info *info) {
  if (!h || !u || !w) return ST_ERR_ARG;
  if (kind != ST_PICARD && kind != ST_NEWTON) return ST_ERR_ARG;
  DeviceScope ds(h->dev);
  bool su = h->desc.stabilization == ST_SU;
  bool stats = !keep_theta;
  {
    ProfScope ps(h, PROF_IONIC, 8.0 * (double)h->NtQs * (3 + h->p + 1));
    ST_TRY(ionic_run(h, u, w, kind, stats));
  }
  ProfScope plr(h, PROF_LOWRANK, 0.0);
  if (stats) {
    if (su) {
      ST_TRY(theta_and_lowrank(h, info));
    } else {
      double st[4];
      ST_CUDA(cudaMemcpyAsync(st, h->stats, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      ST_CUDA(cudaStreamSynchronize(h->stream));
      h->rank = 0;
      if (info) {
        info->u_max = st[0]; info->ut_max = st[1]; info->r_max = st[2];
        info->den = h->desc.C_m * (st[0] / h->desc.T + st[1]);
        info->rank = 0; info->theta_fro = 0.0;
      }
      if (!std::isfinite(st[0]) || !std::isfinite(st[1])) return ST_ERR_NAN;
    }
  } else if (info) {
    info->rank = h->rank;
    info->theta_fro = h->theta_fro;
  }
  if (h->desc.eps_reaction >= 0.0) ST_TRY(reaction_lowrank(h, u, w, kind));
  if (info) info->rank_reaction = h->desc.eps_reaction >= 0.0 ? h->rankC : 0;
  ST_TRY(su_band_add(h));   // also writes the FP32 copy of the bands
  ST_CUDA(cudaStreamSynchronize(h->stream));
  ST_CUDA(cudaGetLastError());
  h->have_lin = true;
  return ST_OK;
}

st_status st_ionic(st_handle *h, const double *u, const double *w, st_ionic_info *info) {
  if (!h) return ST_ERR_ARG;
  return st_linearize(h, u, w, h->desc.nonlinear, 0, info);
}

st_status st_apply(st_handle *h, int prec, const void *x, void *y) {
  if (!h || !x || !y || x == y) return ST_ERR_ARG;
  if (!h->have_lin) return ST_ERR_STATE;
  DeviceScope ds(h->dev);
  if (prec == ST_FP64) return apply_T<double>(h, (const double *)x, (double *)y);
  if (prec == ST_MIXED) return apply_T<float>(h, (const float *)x, (float *)y);
  return ST_ERR_ARG;
}

st_status st_precond(st_handle *h, int prec, const void *r, void *z) {
  if (!h || !r || !z) return ST_ERR_ARG;
  DeviceScope ds(h->dev);
  if (prec == ST_FP64) return precond_T<double>(h, (const double *)r, (double *)z);
  if (prec == ST_MIXED) return precond_T<float>(h, (const float *)r, (float *)z);
  return ST_ERR_ARG;
}

st_status st_rhs(st_handle *h, double *f) {
  if (!h || !f) return ST_ERR_ARG;
  DeviceScope ds(h->dev);
  ST_CUDA(cudaMemcpyAsync(f, h->f64, h->Ndof * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  return ST_OK;
}

st_status st_wupdate(st_handle *h, const double *u, double *w) {
  if (!h || !u || !w || u == w) return ST_ERR_ARG;
  DeviceScope ds(h->dev);
  return wupdate_run(h, u, w);
}

// Handle-free w-update for callers that cannot allocate device memory: the
// time bands are built on the host and staged in a fixed device array.
st_status st_wupdate_static(const st_problem_desc *desc, const double *u, double *w, void *stream) {
  ST_TRY(validate(desc));
  if (!u || !w || u == w) return ST_ERR_ARG;
  const Sizes z = plan(*desc);
  if (2 * (long long)z.Nt * z.B > ST_WUPDATE_STATIC_CAPACITY) return ST_ERR_CAPACITY;
  std::vector<double> Mt, lu;
  ST_TRY(host_time_bands(*desc, Mt, lu));
  return wupdate_static_run((cudaStream_t)stream, u, w, Mt.data(), lu.data(), desc->b, (int)z.Nt, z.Ns, desc->p);
}

st_status st_linsolve(st_handle *h, const double *b, double *x, st_stats *stats) {
  if (!h || !b || !x) return ST_ERR_ARG;
  if (!h->have_lin) return ST_ERR_STATE;
  DeviceScope ds(h->dev);
  cudaStream_t s = h->stream;
  const st_problem_desc &D = h->desc;
  long long N = h->Ndof;
  double bn = norm2_64(h, b);
  if (!std::isfinite(bn)) return ST_ERR_NAN;
  if (stats) { stats->gmres_iters = 0; stats->outer_iters = 0; stats->rel_res = 0.0; stats->rank = h->rank; }
  if (bn == 0.0) {
    ST_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), s));
    ST_CUDA(cudaStreamSynchronize(s));
    return ST_OK;
  }
  int total = 0, outer = 0;
  double rel = INFINITY, rel_prev = INFINITY;
  st_status status = ST_ERR_NOT_CONVERGED;
  if (D.precision == ST_MIXED && D.inner_op == ST_INNER_DF) h->inner_df = true;
  if (D.precision == ST_MIXED && D.inner_op == ST_INNER_FP32) h->inner_df = false;
  if (D.precision == ST_MIXED && D.precond_arith == ST_PRECOND_FP64) h->pre64 = true;
  while (true) {
    ST_TRY(apply_T<double>(h, x, h->t64a));
    launch_sub64(s, h->r64, b, h->t64a, N);
    double rn = norm2_64(h, h->r64);
    if (!std::isfinite(rn)) return ST_ERR_NAN;
    rel = rn / bn;
    if (rel <= D.rtol) { status = ST_OK; break; }
    // a refinement step that failed (the true residual fell by less than a
    // factor 2): first the FP64 preconditioner, then the double-float
    // operator (both kept for the handle's later solves)
    if (D.precision == ST_MIXED && rel > rel_prev / 2.0) {
      if (D.precond_arith == ST_PRECOND_AUTO && !h->pre64) h->pre64 = true;
      else if (D.inner_op == ST_INNER_AUTO && !h->inner_df) h->inner_df = true;
    }
    rel_prev = rel;
    if (total >= D.max_it) break;
    int its = 0;
    double est = 0.0;
    double tol_in = D.rtol * bn / rn;
    int maxit = std::min(h->m, D.max_it - total);
    if (D.precision == ST_FP64) {
      ST_TRY(gmres_cycle<double>(h, h->r64, h->t64a, 0.5 * tol_in, maxit, &its, &est));
      launch_axpby64(s, x, h->t64a, 1.0, 1.0, N);
    } else {
      // FP32 inner solve on the scaled residual, FP64 update
      launch_d2f(s, h->r32, h->r64, 1.0 / rn, N);
      double tin = std::max(0.5 * tol_in, 1e-6);
      ST_TRY(gmres_cycle<float>(h, h->r32, h->d32, tin, maxit, &its, &est));
      launch_f2d_axpy(s, x, h->d32, rn, N);
    }
    total += its;
    ++outer;
    if (its == 0) break;
  }
  ST_CUDA(cudaStreamSynchronize(s));
  if (stats) { stats->gmres_iters = total; stats->outer_iters = outer; stats->rel_res = rel; stats->rank = h->rank; }
  return status;
}

st_status st_solve(st_handle *h, double *u, double *w, st_stats *stats) {
  if (!h || !u || !w) return ST_ERR_ARG;
  DeviceScope ds(h->dev);
  cudaStream_t s = h->stream;
  const st_problem_desc &D = h->desc;
  long long N = h->Ndof;
  double *unew = h->x64, *wnew = h->t64b;
  st_stats ls;
  int total = 0;
  double diff = INFINITY;
  int k = 0;
  st_status status = ST_ERR_NOT_CONVERGED;
  for (; k < D.max_fp; ++k) {
    st_ionic_info info;
    if (D.nonlinear == ST_NEWTON) {
      // rhs = f - A_P(u^k) u^k, then J du = rhs with theta frozen
      ST_TRY(st_linearize(h, u, w, ST_PICARD, 0, &info));
      ST_TRY(apply_T<double>(h, u, h->t64a));
      launch_sub64(s, h->b64, h->f64, h->t64a, N);
      ST_TRY(st_linearize(h, u, w, ST_NEWTON, 1, &info));
      ST_CUDA(cudaMemsetAsync(unew, 0, N * sizeof(double), s));
      st_status ls_s = st_linsolve(h, h->b64, unew, &ls);
      if (ls_s != ST_OK && ls_s != ST_ERR_NOT_CONVERGED) return ls_s;
      total += ls.gmres_iters;
      diff = absmax_diff(h, unew, nullptr);
      launch_axpby64(s, unew, u, 1.0, 1.0, N);   // u + du
      if (D.fix_w_zero) ST_CUDA(cudaMemsetAsync(wnew, 0, N * sizeof(double), s));
      else ST_TRY(wupdate_run(h, u, wnew));
    } else {
      ST_TRY(st_linearize(h, u, w, ST_PICARD, 0, &info));
      ST_CUDA(cudaMemcpyAsync(unew, u, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      st_status ls_s = st_linsolve(h, h->f64, unew, &ls);
      if (ls_s != ST_OK && ls_s != ST_ERR_NOT_CONVERGED) return ls_s;
      total += ls.gmres_iters;
      if (D.fix_w_zero) ST_CUDA(cudaMemsetAsync(wnew, 0, N * sizeof(double), s));
      else ST_TRY(wupdate_run(h, u, wnew));
      // relaxation
      launch_axpby64(s, unew, u, 1.0 - D.alpha, D.alpha, N);   // unew = alpha unew + (1-alpha) u
      launch_axpby64(s, wnew, w, 1.0 - D.alpha, D.alpha, N);
      diff = absmax_diff(h, unew, u);
    }
    ST_CUDA(cudaMemcpyAsync(u, unew, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    ST_CUDA(cudaMemcpyAsync(w, wnew, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (!std::isfinite(diff)) { status = ST_ERR_NAN; ++k; break; }
    if (diff <= D.delta) { status = ST_OK; ++k; break; }
  }
  ST_CUDA(cudaStreamSynchronize(s));
  if (stats) {
    *stats = ls;
    stats->fp_iters = k;
    stats->total_gmres = total;
    stats->last_diff = diff;
    stats->rank = h->rank;
  }
  return status;
}

long long st_launch_count(void) { return g_launches.load(); }

st_status st_tc_selftest(int *usable, double *max_rel_err) {
  if (!usable || !max_rel_err) return ST_ERR_ARG;
  double err = 0.0;
  int st = tc_state(nullptr, &err);
  *usable = st == 1 ? 1 : 0;
  *max_rel_err = err;
  return ST_OK;
}

st_status st_profile(st_handle *h, int enable) {
  if (!h) return ST_ERR_ARG;
  DeviceScope ds(h->dev);
  ST_CUDA(cudaStreamSynchronize(h->stream));
  h->prof.clear();
  h->ev_used = 0;
  h->prof_on = enable != 0;
  return ST_OK;
}

st_status st_profile_read(st_handle *h, int cat, double *ms, double *bytes, double *flops, long long *launches) {
  if (!h || cat < 0 || cat >= PROF_NCAT || !ms || !bytes || !flops || !launches) return ST_ERR_ARG;
  DeviceScope ds(h->dev);
  ST_CUDA(cudaStreamSynchronize(h->stream));
  double t = 0.0, b = 0.0, f = 0.0;
  long long n = 0;
  for (const auto &r : h->prof) {
    if (r.cat != cat) continue;
    float e = 0.0f;
    if (cudaEventElapsedTime(&e, r.a, r.b) != cudaSuccess) { cudaGetLastError(); continue; }
    t += e; b += r.bytes; f += r.flops; ++n;
  }
  *ms = t; *bytes = b; *flops = f; *launches = n;
  return ST_OK;
}

st_status st_get(st_handle *h, int what, void *dst, size_t bytes) {
  if (!h || !dst) return ST_ERR_ARG;
  DeviceScope ds(h->dev);
  cudaStream_t s = h->stream;
  size_t need = 0;
  const void *src = nullptr;
  std::vector<double> tmp;
  switch (what) {
    case ST_GET_THETA_HAT: need = h->Ndof * sizeof(double); src = h->theta; break;
    case ST_GET_LOWRANK_S: need = h->rank * sizeof(double); src = h->sr; break;
    case ST_GET_LOWRANK_U: need = (size_t)h->Nt * h->rank * sizeof(double); src = h->Ur; break;
    case ST_GET_LOWRANK_V: need = (size_t)h->Ns * h->rank * sizeof(double); src = h->Vr; break;
    case ST_GET_REACTION_S: need = (size_t)h->rankC * sizeof(double); src = h->srC; if (!src) return ST_ERR_STATE; break;
    case ST_GET_REACTION_U: need = (size_t)h->Nt * h->rankC * sizeof(double); src = h->UrC; if (!src) return ST_ERR_STATE; break;
    case ST_GET_REACTION_V: need = (size_t)h->Ns * h->rankC * sizeof(double); src = h->VrC; if (!src) return ST_ERR_STATE; break;
    case ST_GET_REACTION_TB:
      need = (size_t)h->rankC * (h->p + 1) * h->Nt * sizeof(double); src = h->Tc; if (!src) return ST_ERR_STATE; break;
    case ST_GET_TAU_Q: tmp = h->hs.tau_q; break;
    case ST_GET_FD_EIG: {
      size_t tot = 0;
      for (int l = 0; l < h->d; ++l) tot += h->n[l];
      need = tot * sizeof(double);
      if (bytes != need) return ST_ERR_ARG;
      size_t off = 0;
      for (int l = 0; l < h->d; ++l) {
        ST_CUDA(cudaMemcpyAsync((double *)dst + off, h->lam[l], h->n[l] * sizeof(double), cudaMemcpyDeviceToHost, s));
        off += h->n[l];
      }
      ST_CUDA(cudaStreamSynchronize(s));
      return ST_OK;
    }
    case ST_GET_BANDS_1D:
      for (int l = 0; l < h->d; ++l) {
        tmp.insert(tmp.end(), h->hs.M[l].begin(), h->hs.M[l].end());
        tmp.insert(tmp.end(), h->hs.K[l].begin(), h->hs.K[l].end());
      }
      tmp.insert(tmp.end(), h->hs.Mt.begin(), h->hs.Mt.end());
      tmp.insert(tmp.end(), h->hs.Wt.begin(), h->hs.Wt.end());
      break;
    default: return ST_ERR_ARG;
  }
  if (!src) {
    need = tmp.size() * sizeof(double);
    if (bytes != need) return ST_ERR_ARG;
    std::memcpy(dst, tmp.data(), need);
    return ST_OK;
  }
  if (bytes != need) return ST_ERR_ARG;
  if (need) ST_CUDA(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToHost, s));
  ST_CUDA(cudaStreamSynchronize(s));
  return ST_OK;
}

}  // extern "C"
