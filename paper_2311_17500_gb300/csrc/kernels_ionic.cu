// Ionic quadrature, Theta-hat, the low-rank theta, the SU and reaction time
// bands, the right-hand side and the w-update (Sec. 3 and Sec. 3.1).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include "st_internal.h"
#include "df.cuh"

void launch_gemm64(cudaStream_t s, double *C, const double *A, const double *X, int M, int N, int K,
                   long long sam, long long sak, long long sbk, long long sbc, long long scm, long long scc,
                   double alpha, double beta, double *work = nullptr, long long work_elems = 0);

namespace {

constexpr double kPi = 3.14159265358979323846;

// f of eq. 3.1 at one point (stimulus boxes, or the manufactured sources).
__device__ double source_at(const st_problem_desc &D, const double *x, double t) {
  if (D.source_kind == ST_SRC_STIM) {
    double f = 0.0;
    for (int b = 0; b < D.n_stim; ++b) {
      const st_stim &s = D.stim[b];
      bool in = (t >= s.t0) && (t < s.t1);
      for (int l = 0; l < D.d; ++l) in = in && (x[l] >= s.lo[l]) && (x[l] <= s.hi[l]);
      if (in) f += s.amp;
    }
    return f;
  }
  if (D.source_kind == ST_SRC_HEAT_MMS) {
    // u = prod cos(pi x_l) sin t, w = 0
    double c = 1.0, lapc = 0.0;
    for (int l = 0; l < D.d; ++l) { c *= cos(kPi * x[l]); lapc += D.D[l]; }
    double u = c * sin(t);
    return D.C_m * c * cos(t) + kPi * kPi * lapc * u + D.c1 * u * (u - D.a) * (u - 1.0);
  }
  if (D.source_kind == ST_SRC_E1_MMS) {
    // u = 10 g(x) h(t), g = sin(pi x)(1-e^-x)(1-e^(x-1)), h = sin(pi t)(1-e^(t-1)), w = 0
    double xx = x[0];
    double s0 = sin(kPi * xx), s1 = kPi * cos(kPi * xx), s2 = -kPi * kPi * sin(kPi * xx);
    double em = exp(-xx), ep = exp(xx - 1.0);
    double A0 = 1.0 - em, A1 = em, A2 = -em;
    double B0 = 1.0 - ep, B1 = -ep, B2 = -ep;
    double g = s0 * A0 * B0;
    double g2 = s2 * A0 * B0 + s0 * A2 * B0 + s0 * A0 * B2 + 2.0 * (s1 * A1 * B0 + s1 * A0 * B1 + s0 * A1 * B1);
    double et = exp(t - 1.0);
    double h = sin(kPi * t) * (1.0 - et);
    double h1 = kPi * cos(kPi * t) * (1.0 - et) - sin(kPi * t) * et;
    double u = 10.0 * g * h;
    return D.C_m * 10.0 * g * h1 - D.D[0] * 10.0 * g2 * h + D.c1 * u * (u - D.a) * (u - 1.0);
  }
  return 0.0;
}

struct SpatialPoint {
  double ws;        // product of the 1D weights
  double x[3];      // coordinates
  long long es;     // spatial element (colexicographic)
};

struct GeomArgs {
  int d, nq;
  int Q[3], nel[3];
  const double *wqs[3];
  const double *xs[3];
};

__device__ SpatialPoint spatial_point(const GeomArgs &g, long long q) {
  SpatialPoint sp;
  sp.ws = 1.0;
  sp.es = 0;
  long long stride = 1, rem = q;
  for (int l = 0; l < 3; ++l) sp.x[l] = 0.0;
  for (int l = 0; l < g.d; ++l) {
    int ql = (int)(rem % g.Q[l]);
    rem /= g.Q[l];
    sp.ws *= g.wqs[l][ql];
    sp.x[l] = g.xs[l][ql];
    sp.es += (long long)(ql / g.nq) * stride;
    stride *= g.nel[l];
  }
  return sp;
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long *addr, double v) {
  // non-negative doubles order like their bit patterns; NaN maps to +inf
  if (v != v) v = INFINITY;
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

struct IonicArgs {
  st_problem_desc D;
  GeomArgs g;
  const float2 *U0, *L0, *W0;   // [Nt][Qs]: u, sum D_l d_ll u, w at spatial Gauss points (double-float)
  const double *bt, *xt;        // time tables: values/derivatives, points
  const double *bprod;          // [e][qt][pair]: w_t b_i b_{i+k} for the band pairs (i, k), k <= P - i
  const float2 *bt2, *bprod2;   // the same tables as double-float pairs (bt for k = 0, 1)
  const int *tmask;             // [e*nq+qt]: bit b set if time point (e, qt) lies in stimulus window b
  float2 amp2[ST_MAX_STIM];     // stimulus amplitudes as double-float pairs
  int Nt, nel_t;
  long long Qs, Nel_s;
  int kind;                     // ST_PICARD: C_r, ST_NEWTON: C_J
  int want_stats;
  float *band_hi, *band_lo;     // [k][it][q] as double-float pairs; null: no bands (lean form)
  unsigned long long *emax;     // [et][es]
  unsigned long long *stats;    // max|u|, max|d_t u|, max|R| (bit patterns)
  // rows mode (lean form): the fields are interpolated along x here from
  // their coefficients at the Gauss rows of the other axes, [N_t][rows][n_x]:
  // U1 = u, W1 = w, L1 = the other axes' part of sum_l D_ll d_ll u (null in 1D)
  int no_reaction_band;         // bands without the reaction term (it comes in low rank)
  int rows_mode;
  const float2 *U1, *L1, *W1;
  const float2 *tbx, *tb2x;     // x basis values and second derivatives [ex][g][a], pairs
  double Dx;
  int nx, Qx;
  long long rows;
};

// |v| as the bit pattern of a non-negative double: the unsigned order of these
// patterns is the order of the values (NaN above +inf), so maxima are
// integer operations.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// One thread per spatial Gauss point sweeps the time elements: evaluates u,
// d_t u, the Laplacian and w at the time Gauss points from the time
// coefficients, forms the residual R = C_m d_t u - lap + C_r u - f (Eq.
// theta_ce_u numerator, with the ionic current written as C_r u) and the
// linearization coefficient (C_r of Eq. reaction, or its u-derivative for
// Newton), keeps max |R| per space-time element, and assembles the time band
// sum_qt w_t C b_i b_j of the reaction mass term at this spatial point
// (times its spatial weight).  Rows are written once complete.
// The arithmetic is double-float (about 48 bits): the fields arrive as
// double-float pairs and the band rows are stored as their (high, low) float
// parts; FP64 is used only for the element maxima.
template <int P>
__global__ void __launch_bounds__(128, P <= 3 ? 4 : 2) ionic_tline_kernel(IonicArgs a) {
  constexpr int nq = P + 1, NPAIR = (P + 1) * (P + 2) / 2;
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  __shared__ unsigned long long red[3][4];
  unsigned long long mu = 0, mut = 0, mr = 0;
  if (q < a.Qs) {
    SpatialPoint sp = spatial_point(a.g, q);
    // stimulus boxes containing this point (the spatial factor of f)
    unsigned inbox = 0;
    const bool stim = a.D.source_kind == ST_SRC_STIM;
    if (stim)
      for (int b = 0; b < a.D.n_stim; ++b) {
        bool in = true;
        for (int l = 0; l < a.D.d; ++l) in = in && (sp.x[l] >= a.D.stim[b].lo[l]) && (sp.x[l] <= a.D.stim[b].hi[l]);
        if (in) inbox |= 1u << b;
      }
    const df c1 = df_from(a.D.c1), c2 = df_from(a.D.c2), aa = df_from(a.D.a), Cm = df_from(a.D.C_m);
    const df apl = df_from(1.0 + a.D.a), apl2 = df_from(2.0 * (1.0 + a.D.a)), three = {3.f, 0.f};
    const df ws = df_from(sp.ws);
    const df zero = {0.f, 0.f};
    const bool newton = a.kind == ST_NEWTON;
    const bool bands = a.band_hi != nullptr;
    const long long plane = (long long)a.Nt * a.Qs;
    // rows mode: this point's x element and its basis values
    const long long o = a.rows_mode ? q / a.Qx : 0;
    const int gx = a.rows_mode ? (int)(q % a.Qx) : 0;
    const int ex = gx / nq;
    df bx[P + 1], b2x[P + 1];
    if (a.rows_mode) {
#pragma unroll
      for (int j = 0; j <= P; ++j) {
        bx[j] = df_from2(a.tbx[(size_t)gx * (P + 1) + j]);
        b2x[j] = df_from2(a.tb2x[(size_t)gx * (P + 1) + j]);
      }
    }
    const df Dx = df_from(a.Dx);
    // u, the Laplacian term and w of coefficient row `row` at this point
    auto fetch = [&](int row, df &fu, df &fl, df &fw) {
      if (!a.rows_mode) {
        const long long off = (long long)row * a.Qs + q;
        fu = df_from2(a.U0[off]); fl = df_from2(a.L0[off]); fw = df_from2(a.W0[off]);
        return;
      }
      const long long base = ((long long)row * a.rows + o) * a.nx + ex;
      df su = zero, s2 = zero, sl = zero, sw = zero;
#pragma unroll
      for (int j = 0; j <= P; ++j) {
        const df cu_j = df_from2(a.U1[base + j]);
        su = df_fma(bx[j], cu_j, su);
        s2 = df_fma(b2x[j], cu_j, s2);
        if (a.L1) sl = df_fma(bx[j], df_from2(a.L1[base + j]), sl);
        sw = df_fma(bx[j], df_from2(a.W1[base + j]), sw);
      }
      fu = su; fl = df_fma(Dx, s2, sl); fw = sw;
    };
    df acc[P + 1][P + 1];
#pragma unroll
    for (int r = 0; r <= P; ++r)
#pragma unroll
      for (int k = 0; k <= P; ++k) acc[r][k] = zero;
    // window of coefficient rows e-1 .. e+P-1 (row -1 is zero)
    df cu[P + 1], cl[P + 1], cw[P + 1];
    cu[0] = cl[0] = cw[0] = zero;
#pragma unroll
    for (int j = 1; j <= P; ++j) fetch(j - 1, cu[j], cl[j], cw[j]);
    df mu_d = zero, mut_d = zero;
    for (int e = 0; e < a.nel_t; ++e) {
      // next row (e + P), requested before this element's work
      df nu = zero, nl = zero, nw = zero;
      if (e + 1 < a.nel_t) fetch(e + P, nu, nl, nw);
      df rloc = zero;
#pragma unroll
      for (int qt = 0; qt < nq; ++qt) {
        const float2 *b0 = a.bt2 + ((size_t)(0 * a.nel_t + e) * nq + qt) * (P + 1);
        const float2 *b1 = a.bt2 + ((size_t)(1 * a.nel_t + e) * nq + qt) * (P + 1);
        df u = zero, ut = zero, lap = zero, w = zero;
#pragma unroll
        for (int j = 0; j <= P; ++j) {
          const df v0 = df_from2(__ldg(b0 + j)), v1 = df_from2(__ldg(b1 + j));
          u = df_fma(v0, cu[j], u);
          ut = df_fma(v1, cu[j], ut);
          lap = df_fma(v0, cl[j], lap);
          w = df_fma(v0, cw[j], w);
        }
        df fd = zero;
        if (stim) {
          // boxes containing this point whose time window holds this time
          // point, their amplitudes summed in box order
          unsigned act = inbox & (unsigned)__ldg(a.tmask + e * nq + qt);
          while (act) {
            const int b = __ffs(act) - 1;
            act &= act - 1;
            fd = df_add(fd, df_from2(a.amp2[b]));
          }
        } else if (a.D.source_kind != ST_SRC_ZERO) {
          const double f = source_at(a.D, sp.x, a.xt[e * nq + qt]);
          if (f != 0.0) fd = df_from(f);
        }
        // C_r = c1 (u - a)(u - 1) + c2 w = c1 ((u - (1 + a)) u + a) + c2 w
        const df c2w = df_mul(c2, w);
        const df Cr = df_fma(c1, df_fma(df_sub(u, apl), u, aa), c2w);
        const df R = df_fma(Cr, u, df_sub(df_sub(df_mul(Cm, ut), lap), fd));
        df C = Cr;
        if (newton) C = df_fma(c1, df_fma(df_sub(df_mul(three, u), apl2), u, aa), c2w);
        rloc = df_max_nonneg(rloc, df_abs(R));
        mu_d = df_max_nonneg(mu_d, df_abs(u));
        mut_d = df_max_nonneg(mut_d, df_abs(ut));
        if (bands) {
          const df wc = a.no_reaction_band ? zero : df_mul(ws, C);
          const float2 *bp = a.bprod2 + ((size_t)e * nq + qt) * NPAIR;
          int pr = 0;
#pragma unroll
          for (int i = 0; i <= P; ++i)
#pragma unroll
            for (int k = 0; k <= P - i; ++k) { acc[i][k] = df_fma(wc, df_from2(__ldg(bp + pr)), acc[i][k]); ++pr; }
        }
      }
      const unsigned long long rb = abs_bits(df_to(rloc));
      mr = mr > rb ? mr : rb;
      if (a.want_stats) atomicMax(&a.emax[(long long)e * a.Nel_s + sp.es], rb);
      // row e-1 is complete
      int row = e - 1;
      if (bands && row >= 0)
#pragma unroll
        for (int k = 0; k <= P; ++k) {
          const long long bi = k * plane + (long long)row * a.Qs + q;
          a.band_hi[bi] = acc[0][k].hi;
          a.band_lo[bi] = acc[0][k].lo;
        }
#pragma unroll
      for (int r = 0; r < P; ++r)
#pragma unroll
        for (int k = 0; k <= P; ++k) acc[r][k] = acc[r + 1][k];
#pragma unroll
      for (int k = 0; k <= P; ++k) acc[P][k] = zero;
#pragma unroll
      for (int j = 0; j < P; ++j) { cu[j] = cu[j + 1]; cl[j] = cl[j + 1]; cw[j] = cw[j + 1]; }
      cu[P] = nu; cl[P] = nl; cw[P] = nw;
    }
    for (int r = 0; bands && r < P; ++r) {
      int row = a.nel_t - 1 + r;
      if (row < a.Nt)
        for (int k = 0; k <= P; ++k) {
          const long long bi = k * plane + (long long)row * a.Qs + q;
          a.band_hi[bi] = acc[r][k].hi;
          a.band_lo[bi] = acc[r][k].lo;
        }
    }
    mu = abs_bits(df_to(mu_d));
    mut = abs_bits(df_to(mut_d));
  }
  if (a.want_stats) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      unsigned long long o0 = __shfl_down_sync(0xffffffffu, mu, off);
      unsigned long long o1 = __shfl_down_sync(0xffffffffu, mut, off);
      unsigned long long o2 = __shfl_down_sync(0xffffffffu, mr, off);
      mu = mu > o0 ? mu : o0;
      mut = mut > o1 ? mut : o1;
      mr = mr > o2 ? mr : o2;
    }
    if (lane == 0) { red[0][warp] = mu; red[1][warp] = mut; red[2][warp] = mr; }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m0 = 0, m1 = 0, m2 = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
        m0 = m0 > red[0][i] ? m0 : red[0][i];
        m1 = m1 > red[1][i] ? m1 : red[1][i];
        m2 = m2 > red[2][i] ? m2 : red[2][i];
      }
      atomicMax(&a.stats[0], m0);
      atomicMax(&a.stats[1], m1);
      atomicMax(&a.stats[2], m2);
    }
  }
}

// Right-hand side of Eq. (rhsfun), first stage: for each spatial Gauss point,
// Fq[it][q] = ws(q) sum over time Gauss points of wt f(x_q, t) b_it(t).
template <int P>
__global__ void source_tline_kernel(st_problem_desc D, GeomArgs g, const double *bt, const double *wt,
                                    const double *xt, int Nt, int nel_t, long long Qs, int r0, int nr, double *Fq) {
  // rows r0 .. r0 + nr - 1 of Fq (row i at Fq[(i - r0) Qs + q]); row i takes
  // the time elements i + 1 - P .. i + 1
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= Qs) return;
  const int nq = P + 1;
  SpatialPoint sp = spatial_point(g, q);
  double acc[P + 1];
#pragma unroll
  for (int r = 0; r <= P; ++r) acc[r] = 0.0;
  const int e_lo = max(0, r0 + 1 - P), e_hi = min(nel_t - 1, r0 + nr);
  const int r1 = min(Nt, r0 + nr);
  for (int e = e_lo; e <= e_hi; ++e) {
    for (int qt = 0; qt < nq; ++qt) {
      const double *b0 = bt + ((size_t)e * nq + qt) * (P + 1);
      double v = wt[e * nq + qt] * sp.ws * source_at(D, sp.x, xt[e * nq + qt]);
#pragma unroll
      for (int j = 0; j <= P; ++j) acc[j] += v * b0[j];
    }
    const int row = e - 1;
    if (row >= r0 && row < r1) Fq[(long long)(row - r0) * Qs + q] = acc[0];
#pragma unroll
    for (int r = 0; r < P; ++r) acc[r] = acc[r + 1];
    acc[P] = 0.0;
  }
  if (e_hi == nel_t - 1)
    for (int r = 0; r < P; ++r) {
      const int row = e_hi + r;
      if (row >= r0 && row < r1) Fq[(long long)(row - r0) * Qs + q] = acc[r];
    }
}

// Support-extension maximum along one axis (Eq. suppext), separable over the
// axes of the box: out[o][i][c] = max_{e in window(i)} in[o][e][c] with
// window(i) = [i+shift-2p, i+shift] (literal) or [i+shift-2p, i+shift+p]
// (symmetric), clamped to the spans; shift = 1 for the time axis (X_t index
// i is the (i+1)-th B-spline).
__global__ void window_max_kernel(double *__restrict__ out, const double *__restrict__ in, int nel, int nout,
                                  int p, int shift, int symmetric, long long inner, long long outer) {
  long long total = outer * nout * inner;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long c = idx % inner;
    long long r = idx / inner;
    int i = (int)(r % nout);
    long long o = r / nout;
    int lo = max(0, i + shift - 2 * p);
    int hi = min(nel - 1, i + shift + (symmetric ? p : 0));
    double m = 0.0;
    for (int e = lo; e <= hi; ++e) m = fmax(m, in[(o * nel + e) * inner + c]);
    out[idx] = m;
  }
}

// Theta-hat = min(num / den, 1), with 1 for num > 0 = den and 0 for num = 0 = den.
__global__ void theta_kernel(double *__restrict__ th, const double *__restrict__ num, double den, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double v = num[e];
    th[e] = den > 0.0 ? fmin(v / den, 1.0) : (v > 0.0 ? 1.0 : 0.0);
  }
}

// theta_{t,r} at the time Gauss points: linear interpolation of U[:, r] on
// the time Greville grid, constant before the first node.  thq[r][qt].
__global__ void theta_t_kernel(double *__restrict__ thq, const double *__restrict__ U, int R, int Qt,
                               const int *hi, const double *hl) {
  int total = Qt * R;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int qt = idx % Qt, r = idx / Qt;
    int i = hi[qt];
    double l = hl[qt];
    double v = (1.0 - l) * U[(long long)i * R + r];
    if (l != 0.0) v += l * U[(long long)(i + 1) * R + r];
    thq[idx] = v;
  }
}

// SU time bands per rank (Eq. tildeS, matrices S^t_{r,l} summed over l):
// Tr[r][k][it] = sum_l int tau_l theta_{t,r} d^l b_it d^l b_{it+k} dt.
__global__ void su_time_band_kernel(double *__restrict__ Tr, const double *__restrict__ tht,
                                    const double *__restrict__ tauq, const double *__restrict__ bt,
                                    const double *__restrict__ wt, int R, int Nt, int nel_t, int p) {
  int nq = p + 1;
  int total = R * (p + 1) * Nt;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int it = idx % Nt;
    int k = (idx / Nt) % (p + 1);
    int r = idx / (Nt * (p + 1));
    double s = 0.0;
    if (it + k < Nt) {
      int e0 = max(0, it + k + 1 - p), e1 = min(nel_t - 1, it + 1);
      for (int e = e0; e <= e1; ++e) {
        int ai = it + 1 - e, ci = it + k + 1 - e;
        for (int qt = 0; qt < nq; ++qt) {
          double w = wt[e * nq + qt] * tht[(long long)r * nel_t * nq + e * nq + qt];
          double acc = 0.0;
          for (int l = 1; l <= p; ++l) {
            const double *bl = bt + (((size_t)l * nel_t + e) * nq + qt) * (p + 1);
            acc += tauq[((size_t)(l - 1) * nel_t + e) * nq + qt] * bl[ai] * bl[ci];
          }
          s += w * acc;
        }
      }
    }
    Tr[idx] = s;
  }
}

// Time mass bands of the low-rank reaction ranks (the time factor of M_R in
// low rank): Tc[r][k][it] = int rho_{t,r} b_it b_{it+k} dt, with rho_{t,r}
// the linear interpolant of U[:, r] at the time Gauss points (rho[r][qt]).
__global__ void mass_time_band_kernel(double *__restrict__ Tc, const double *__restrict__ rho,
                                      const double *__restrict__ bt, const double *__restrict__ wt, int R, int Nt,
                                      int nel_t, int p) {
  int nq = p + 1;
  int total = R * (p + 1) * Nt;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int it = idx % Nt;
    int k = (idx / Nt) % (p + 1);
    int r = idx / (Nt * (p + 1));
    double s = 0.0;
    if (it + k < Nt) {
      int e0 = max(0, it + k + 1 - p), e1 = min(nel_t - 1, it + 1);
      for (int e = e0; e <= e1; ++e) {
        int ai = it + 1 - e, ci = it + k + 1 - e;
        for (int qt = 0; qt < nq; ++qt) {
          const double *b0 = bt + ((size_t)e * nq + qt) * (p + 1);
          s += wt[e * nq + qt] * rho[(long long)r * nel_t * nq + e * nq + qt] * b0[ai] * b0[ci];
        }
      }
    }
    Tc[idx] = s;
  }
}

// The reaction coefficient (C_r of Eq. reaction, or C_J for Newton) of the
// values u, w (FP64, elementwise).
__global__ void reaction_coef_kernel(double *__restrict__ C, const double *__restrict__ u,
                                     const double *__restrict__ w, double c1, double c2, double a, int newton,
                                     long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double uu = u[i];
    C[i] = newton ? c1 * ((3.0 * uu - 2.0 * (1.0 + a)) * uu + a) + c2 * w[i]
                  : c1 * ((uu - (1.0 + a)) * uu + a) + c2 * w[i];
  }
}

struct HatArgs {
  const int *idx[3];
  const double *lam[3];
  int n[3];
};

// Cq[r][q] = C_m sigma_r ws(q) theta_{s,r}(x_q): the spatial factors of the SU
// ranks, with theta_{s,r} the d-linear interpolation of V[:, r] on the
// spatial Greville grid (Sec. 3.1) evaluated at the spatial Gauss point x_q.
__global__ void su_space_coef_kernel(double *__restrict__ Cq, const double *__restrict__ V,
                                     const double *__restrict__ sig, GeomArgs g, HatArgs hat, double Cm, int R,
                                     long long Qs) {
  long long total = Qs * R;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long q = idx % Qs;
    int r = (int)(idx / Qs);
    SpatialPoint sp = spatial_point(g, q);
    int il[3] = {0, 0, 0};
    double ll[3] = {0.0, 0.0, 0.0};
    long long rem = q;
    for (int l = 0; l < g.d; ++l) {
      int ql = (int)(rem % g.Q[l]);
      rem /= g.Q[l];
      il[l] = hat.idx[l][ql];
      ll[l] = hat.lam[l][ql];
    }
    double s = 0.0;
    int nc = 1 << g.d;
    for (int c = 0; c < nc; ++c) {
      double w = 1.0;
      long long j = 0, stride = 1;
      for (int l = 0; l < g.d; ++l) {
        int cl = (c >> l) & 1;
        w *= cl ? ll[l] : 1.0 - ll[l];
        j += (long long)(il[l] + cl) * stride;
        stride *= hat.n[l];
      }
      if (w != 0.0) s += w * V[j * R + r];
    }
    Cq[idx] = Cm * sig[r] * sp.ws * s;
  }
}

// w-update (Sec. 3.2): w[:, j] = b (W_t + b d_e M_t)^{-1} M_t u[:, j] for every
// spatial index j; the LU factors of the time matrix are shared by all columns.
template <int P>
__global__ void wupdate_kernel(double *__restrict__ w, const double *__restrict__ u, const double *__restrict__ Mt,
                               const double *__restrict__ lu, double bcoef, int Nt, long long Ns) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= Ns) return;
  constexpr int B = 2 * P + 1;
  double uw[2 * P + 1];
#pragma unroll
  for (int i = 0; i < 2 * P + 1; ++i) uw[i] = 0.0;
#pragma unroll
  for (int k = 0; k < P; ++k) uw[P + 1 + k] = (k < Nt) ? u[(long long)k * Ns + j] : 0.0;
  double yw[P];
#pragma unroll
  for (int k = 0; k < P; ++k) yw[k] = 0.0;
  for (int it = 0; it < Nt; ++it) {
#pragma unroll
    for (int i = 0; i < 2 * P; ++i) uw[i] = uw[i + 1];
    uw[2 * P] = (it + P < Nt) ? u[(long long)(it + P) * Ns + j] : 0.0;
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < B; ++k) {
      int c = it - P + k;
      if (c >= 0 && c < Nt) v += Mt[(size_t)it * B + k] * uw[k];
    }
    double s = bcoef * v;
#pragma unroll
    for (int k = 1; k <= P; ++k)
      if (it - k >= 0) s -= lu[(size_t)it * B + (P - k)] * yw[P - k];
#pragma unroll
    for (int k = 0; k < P - 1; ++k) yw[k] = yw[k + 1];
    yw[P - 1] = s;
    w[(long long)it * Ns + j] = s;
  }
  double zw[P];
#pragma unroll
  for (int k = 0; k < P; ++k) zw[k] = 0.0;
  for (int it = Nt - 1; it >= 0; --it) {
    double s = w[(long long)it * Ns + j];
#pragma unroll
    for (int k = 1; k <= P; ++k)
      if (it + k < Nt) s -= lu[(size_t)it * B + (P + k)] * zw[k - 1];
    s *= lu[(size_t)it * B + P];
#pragma unroll
    for (int k = P - 1; k > 0; --k) zw[k] = zw[k - 1];
    zw[0] = s;
    w[(long long)it * Ns + j] = s;
  }
}

// FP64 values split into double-float pairs.
__global__ void d2df_kernel(float2 *__restrict__ out, const double *__restrict__ in, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const df v = df_from(in[e]);
    out[e] = make_float2(v.hi, v.lo);
  }
}

// band[m][q] += sum_{r0 <= r < r0 + RMAX, r < R} Tr[r][m] Cq[r][q] (SU ranks of
// Eq. tildeS added to the reaction band) in double-float arithmetic on the
// (high, low) pairs; Tr and Cq come split into pairs.
template <int RMAX>
__global__ void __launch_bounds__(256) su_band_update_kernel(float *__restrict__ bhi, float *__restrict__ blo,
                                                             const float2 *__restrict__ Tr,
                                                             const float2 *__restrict__ Cq, int r0, int R,
                                                             long long Mrows, long long Qs) {
  // thread = 4 consecutive spatial points q (their rank coefficients stay in
  // registers), blockIdx.y strides over the band rows m, two rows at a time
  const long long q0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * 4;
  if (q0 >= Qs) return;
  const int nr = min(RMAX, R - r0);
  const bool vec = (Qs % 4) == 0;   // rows start on 16-byte boundaries
  const int nu = (int)min(4LL, Qs - q0);
  df c[RMAX][4];
#pragma unroll
  for (int rr = 0; rr < RMAX; ++rr)
#pragma unroll
    for (int u = 0; u < 4; ++u)
      c[rr][u] = (rr < nr && u < nu) ? df_from2(Cq[(long long)(r0 + rr) * Qs + q0 + u]) : df{0.f, 0.f};
  auto update = [&](long long m, float (&h)[4], float (&l)[4]) {
    df t[RMAX];
#pragma unroll
    for (int rr = 0; rr < RMAX; ++rr)
      t[rr] = rr < nr ? df_from2(__ldg(Tr + (long long)(r0 + rr) * Mrows + m)) : df{0.f, 0.f};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      df v = {h[u], l[u]};
#pragma unroll
      for (int rr = 0; rr < RMAX; ++rr)
        if (rr < nr) v = df_fma(t[rr], c[rr][u], v);
      h[u] = v.hi;
      l[u] = v.lo;
    }
  };
  auto load = [&](long long idx, float (&h)[4], float (&l)[4]) {
    if (vec) {
      const float4 a = *reinterpret_cast<const float4 *>(bhi + idx), b = *reinterpret_cast<const float4 *>(blo + idx);
      h[0] = a.x; h[1] = a.y; h[2] = a.z; h[3] = a.w;
      l[0] = b.x; l[1] = b.y; l[2] = b.z; l[3] = b.w;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        h[u] = u < nu ? bhi[idx + u] : 0.f;
        l[u] = u < nu ? blo[idx + u] : 0.f;
      }
    }
  };
  auto store = [&](long long idx, const float (&h)[4], const float (&l)[4]) {
    if (vec) {
      *reinterpret_cast<float4 *>(bhi + idx) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4 *>(blo + idx) = make_float4(l[0], l[1], l[2], l[3]);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (u < nu) { bhi[idx + u] = h[u]; blo[idx + u] = l[u]; }
    }
  };
  const long long step = gridDim.y;
  for (long long m = blockIdx.y; m < Mrows; m += 2 * step) {
    const long long m2 = m + step;
    float h0[4], l0[4], h1[4], l1[4];
    load(m * Qs + q0, h0, l0);
    if (m2 < Mrows) load(m2 * Qs + q0, h1, l1);
    update(m, h0, l0);
    store(m * Qs + q0, h0, l0);
    if (m2 < Mrows) {
      update(m2, h1, l1);
      store(m2 * Qs + q0, h1, l1);
    }
  }
}

// Gram matrix G = Theta Theta^T (n x n, Theta n x K row-major, FP64) in
// double-float arithmetic: upper-triangle 64 x 64 tiles, K split into chunks;
// each block stages 64 x 32 slices of the two row panels as double-float pairs
// and accumulates 4 x 4 outputs per thread; part[split][tile][64][64] holds
// the chunk sums as FP64.
constexpr int kGT = kGramTile, kGK = 32;

__global__ void __launch_bounds__(256) gram_df_kernel(double *__restrict__ part, const double *__restrict__ Th, int n,
                                                      long long K, int ntile, int kchunk) {
  __shared__ float2 sa[kGK][kGT + 1], sb[kGK][kGT + 1];
  // tile pair (ti <= tj) from the linear index
  int tp = blockIdx.x, ti = 0;
  while (tp >= ntile - ti) { tp -= ntile - ti; ++ti; }
  const int tj = ti + tp;
  const long long k0 = (long long)blockIdx.y * kchunk, k1 = min(K, k0 + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, 4 x 4 outputs each
  df acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = {0.f, 0.f};
  for (long long kb = k0; kb < k1; kb += kGK) {
    for (int e = threadIdx.x; e < kGK * kGT; e += blockDim.x) {
      const int rr = e / kGK, kk = e - rr * kGK;
      const long long kx = kb + kk;
      const int ra = ti * kGT + rr, rb = tj * kGT + rr;
      const df va = (ra < n && kx < k1) ? df_from(Th[(long long)ra * K + kx]) : df{0.f, 0.f};
      const df vb = (rb < n && kx < k1) ? df_from(Th[(long long)rb * K + kx]) : df{0.f, 0.f};
      sa[kk][rr] = make_float2(va.hi, va.lo);
      sb[kk][rr] = make_float2(vb.hi, vb.lo);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kGK; ++kk) {
      df av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = df_from2(sa[kk][ty * 4 + a]);
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = df_from2(sb[kk][tx * 4 + b]);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = df_fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
  double *dst = part + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * kGT * kGT;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) dst[(ty * 4 + a) * kGT + tx * 4 + b] = df_to(acc[a][b]);
}

// G[i][j] = G[j][i] = sum over the K chunks (fixed order, FP64).
__global__ void gram_reduce_kernel(double *__restrict__ G, const double *__restrict__ part, int n, int ntile,
                                   int npair, int nsplit) {
  const long long total = (long long)npair * kGT * kGT;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int pr = (int)(e / (kGT * kGT)), w = (int)(e - (long long)pr * kGT * kGT);
    int tp = pr, ti = 0;
    while (tp >= ntile - ti) { tp -= ntile - ti; ++ti; }
    const int tj = ti + tp;
    const int i = ti * kGT + w / kGT, j = tj * kGT + w % kGT;
    if (i >= n || j >= n || (ti == tj && j < i)) continue;
    double v = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) v += part[((long long)sp * npair + pr) * kGT * kGT + w];
    G[(long long)i * n + j] = v;
    G[(long long)j * n + i] = v;
  }
}

__global__ void zero_ull_kernel(unsigned long long *p, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    p[e] = 0ull;
}

__global__ void scale_cols_kernel(double *V, const double *sig, int R, long long n) {
  long long total = n * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e % R);
    V[e] = sig[r] > 0.0 ? V[e] / sig[r] : 0.0;
  }
}

inline int grid_for(long long total, int threads = 256) {
  long long g = (total + threads - 1) / threads;
  if (g > 152LL * 64) g = 152LL * 64;
  if (g < 1) g = 1;
  return (int)g;
}

GeomArgs geom(st_handle *h) {
  GeomArgs g;
  g.d = h->d;
  g.nq = h->nq;
  for (int l = 0; l < 3; ++l) {
    g.Q[l] = h->Q[l];
    g.nel[l] = h->nel[l];
    g.wqs[l] = h->wqs[l];
    g.xs[l] = h->xs[l];
  }
  return g;
}

// One spatial axis from coefficients to Gauss points in double-float:
// out[o][e*nq+g][c] (= or += coef *) sum_a tab[e][g][a] in[o][e+a][c].
// Grid y runs over o, grid x over the (e*nq+g, c) outputs of one o slice, so
// consecutive threads write consecutive addresses whatever the inner extent.
template <int P>
__global__ void interp_df_kernel(float2 *__restrict__ out, const float2 *__restrict__ in,
                                 const float2 *__restrict__ tab, int nel, unsigned inner, long long outer,
                                 int accumulate, double coef) {
  constexpr int nq = P + 1;
  const int nin = nel + P;
  const unsigned slice = (unsigned)(nel * nq) * inner;
  const df cf = df_from(coef);
  for (long long o = blockIdx.y; o < outer; o += gridDim.y) {
    const float2 *src0 = in + (size_t)o * nin * inner;
    float2 *dst0 = out + (size_t)o * slice;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < slice; i += gridDim.x * blockDim.x) {
      const unsigned eq = i / inner, c = i - eq * inner, e = eq / nq;
      const float2 *tb = tab + (size_t)eq * (P + 1);
      const float2 *src = src0 + (size_t)e * inner + c;
      df v = {0.f, 0.f};
#pragma unroll
      for (int a = 0; a <= P; ++a) v = df_fma(df_from2(__ldg(tb + a)), df_from2(src[(size_t)a * inner]), v);
      if (accumulate) v = df_fma(cf, v, df_from2(dst0[i]));
      else if (coef != 1.0) v = df_mul(cf, v);
      dst0[i] = make_float2(v.hi, v.lo);
    }
  }
}

void launch_interp_df(cudaStream_t s, float2 *out, const float2 *in, const float2 *tab, int nel, int p,
                      long long inner, long long outer, int accumulate, double coef) {
  const long long slice = (long long)nel * (p + 1) * inner;
  const int threads = 256;
  dim3 g((unsigned)std::min<long long>((slice + threads - 1) / threads, 1024),
         (unsigned)std::min<long long>(outer, 65535));
  const unsigned in32 = (unsigned)inner;
  switch (p) {
    case 1: st_count_launch(); interp_df_kernel<1><<<g, threads, 0, s>>>(out, in, tab, nel, in32, outer, accumulate, coef); break;
    case 2: st_count_launch(); interp_df_kernel<2><<<g, threads, 0, s>>>(out, in, tab, nel, in32, outer, accumulate, coef); break;
    case 3: st_count_launch(); interp_df_kernel<3><<<g, threads, 0, s>>>(out, in, tab, nel, in32, outer, accumulate, coef); break;
    default: st_count_launch(); interp_df_kernel<4><<<g, threads, 0, s>>>(out, in, tab, nel, in32, outer, accumulate, coef); break;
  }
}

// The three fields of the ionic model in two dimensions by sum factorization,
// every input read once per pass, double-float.  One axis, inner extent
// `inner` (1 for x), tables B (values) and B2 (second derivatives):
//  first pass (x):  o0 = B i0,  o1 = B2 i0,  o2 = B i1      (i0 = u, i1 = w)
//  last pass (y):   o0 = B i0,  o1 = c1 B i1 + c2 B2 i0,  o2 = B i2
// so that with i0 = B_x u, i1 = B2_x u, i2 = B_x w the outputs are u,
// D_x d_xx u + D_y d_yy u and w at the spatial Gauss points.
// Grid y runs over the outer index, grid x over one outer slice.
template <int P, bool LAST>
__global__ void fields_interp_kernel(float2 *__restrict__ o0, float2 *__restrict__ o1, float2 *__restrict__ o2,
                                     const float2 *__restrict__ i0, const float2 *__restrict__ i1,
                                     const float2 *__restrict__ i2, const float2 *__restrict__ tb,
                                     const float2 *__restrict__ tb2, int nel, unsigned inner, long long outer,
                                     double c1, double c2) {
  constexpr int nq = P + 1;
  const int nin = nel + P;
  const unsigned slice = (unsigned)(nel * nq) * inner;
  const df d1 = df_from(c1), d2 = df_from(c2);
  for (long long o = blockIdx.y; o < outer; o += gridDim.y) {
    const size_t ibase = (size_t)o * nin * inner, obase = (size_t)o * slice;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < slice; i += gridDim.x * blockDim.x) {
      const unsigned eq = i / inner, c = i - eq * inner, e = eq / nq;
      const size_t src = ibase + (size_t)e * inner + c;
      df s0 = {0.f, 0.f}, s1 = s0, s2 = s0, s3 = s0;
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        const df b = df_from2(__ldg(tb + (size_t)eq * nq + a)), b2 = df_from2(__ldg(tb2 + (size_t)eq * nq + a));
        const size_t k = src + (size_t)a * inner;
        const df x0 = df_from2(i0[k]), x1 = df_from2(i1[k]);
        s0 = df_fma(b, x0, s0);
        s1 = df_fma(b2, x0, s1);
        s2 = df_fma(b, x1, s2);
        if (LAST) s3 = df_fma(b, df_from2(i2[k]), s3);
      }
      const size_t d = obase + i;
      o0[d] = make_float2(s0.hi, s0.lo);
      if (LAST) {
        const df l = df_fma(d1, s2, df_mul(d2, s1));
        o1[d] = make_float2(l.hi, l.lo);
        o2[d] = make_float2(s3.hi, s3.lo);
      } else {
        o1[d] = make_float2(s1.hi, s1.lo);
        o2[d] = make_float2(s2.hi, s2.lo);
      }
    }
  }
}

template <bool LAST>
void launch_fields_interp(cudaStream_t s, int p, float2 *o0, float2 *o1, float2 *o2, const float2 *i0,
                          const float2 *i1, const float2 *i2, const float2 *tb, const float2 *tb2, int nel,
                          long long inner, long long outer, double c1, double c2) {
  const long long slice = (long long)nel * (p + 1) * inner;
  const int threads = 256;
  dim3 g((unsigned)std::min<long long>((slice + threads - 1) / threads, 1024),
         (unsigned)std::min<long long>(outer, 65535));
  const unsigned in32 = (unsigned)inner;
  switch (p) {
    case 1: st_count_launch(); fields_interp_kernel<1, LAST><<<g, threads, 0, s>>>(o0, o1, o2, i0, i1, i2, tb, tb2, nel, in32, outer, c1, c2); break;
    case 2: st_count_launch(); fields_interp_kernel<2, LAST><<<g, threads, 0, s>>>(o0, o1, o2, i0, i1, i2, tb, tb2, nel, in32, outer, c1, c2); break;
    case 3: st_count_launch(); fields_interp_kernel<3, LAST><<<g, threads, 0, s>>>(o0, o1, o2, i0, i1, i2, tb, tb2, nel, in32, outer, c1, c2); break;
    default: st_count_launch(); fields_interp_kernel<4, LAST><<<g, threads, 0, s>>>(o0, o1, o2, i0, i1, i2, tb, tb2, nel, in32, outer, c1, c2); break;
  }
}

// The 2D fields through the two passes above when the three x-pass results
// fit in the two Gauss-point work buffers; false (nothing launched) if not.
bool fields_to_qpts_2d(st_handle *h, const float2 *u2, const float2 *w2, float2 *U0, float2 *L0, float2 *W0) {
  if (h->d != 2) return false;
  const long long sz = h->Nt * h->n[1] * h->Q[0];   // one x-pass result [N_t][n_y][Q_x]
  const long long cap = h->NtQs;                      // pairs per work buffer
  float2 *B0 = reinterpret_cast<float2 *>(h->W64[0]), *B1 = reinterpret_cast<float2 *>(h->W64[1]);
  float2 *X[3];
  if (3 * sz <= cap) {
    X[0] = B0; X[1] = B0 + sz; X[2] = B0 + 2 * sz;
  } else if (2 * sz <= cap) {
    X[0] = B0; X[1] = B0 + sz; X[2] = B1;
  } else {
    return false;
  }
  cudaStream_t s = h->stream;
  launch_fields_interp<false>(s, h->p, X[0], X[1], X[2], u2, w2, nullptr, h->Bq2[0], h->B2q2[0], h->nel[0], 1,
                              h->Nt * h->n[1], 1.0, 1.0);
  launch_fields_interp<true>(s, h->p, U0, L0, W0, X[0], X[1], X[2], h->Bq2[1], h->B2q2[1], h->nel[1], h->Q[0],
                             h->Nt, h->desc.D[0], h->desc.D[1]);
  return true;
}

// A field at the spatial Gauss points (all time rows), double-float: the
// coefficient tensor [N_t][n_z][n_y][n_x] as pairs to [N_t][Q_z][Q_y][Q_x];
// deriv_dir selects the axis taking the second derivative (-1: none); the
// result is written to dst, or added to it times coef.  Intermediate axes use
// both Gauss-point work buffers.
void spatial_to_qpts(st_handle *h, const float2 *x, int deriv_dir, float2 *dst, int accumulate, double coef) {
  cudaStream_t s = h->stream;
  const float2 *cur = x;
  long long dims[3] = {h->n[0], h->n[1], h->n[2]};
  int ping = 0;
  for (int l = 0; l < h->d; ++l) {
    long long inner = 1, outer = h->Nt;
    for (int m = 0; m < l; ++m) inner *= h->Q[m];
    for (int m = l + 1; m < h->d; ++m) outer *= dims[m];
    const bool last = l == h->d - 1;
    float2 *out = last ? dst : reinterpret_cast<float2 *>(h->W64[ping]);
    const float2 *tab = (l == deriv_dir) ? h->B2q2[l] : h->Bq2[l];
    launch_interp_df(s, out, cur, tab, h->nel[l], h->p, inner, outer, last ? accumulate : 0, last ? coef : 1.0);
    cur = out;
    ping ^= 1;
  }
}

// A field at the Gauss rows of the axes other than x, with x kept in
// coefficients (the layout of the lean operator's rows, [N_t][rows][n_x]),
// double-float: the axes d-1 .. 1 in turn (the order of the operator's own
// forward passes); deriv_dir selects the axis taking the second derivative
// (-1: none); the result is written to dst or added to it times coef.  The
// intermediate of three dimensions uses the second work buffer.
void rows_forward(st_handle *h, const float2 *x, int deriv_dir, float2 *dst, int accumulate, double coef) {
  cudaStream_t s = h->stream;
  const float2 *cur = x;
  for (int l = h->d - 1; l >= 1; --l) {
    long long inner = 1, outer = h->Nt;
    for (int m = 0; m < l; ++m) inner *= h->n[m];
    for (int m = l + 1; m < h->d; ++m) outer *= h->Q[m];
    const bool last = l == 1;
    float2 *out = last ? dst : reinterpret_cast<float2 *>(h->W64[1]);
    const float2 *tab = (l == deriv_dir) ? h->B2q2[l] : h->Bq2[l];
    launch_interp_df(s, out, cur, tab, h->nel[l], h->p, inner, outer, last ? accumulate : 0, last ? coef : 1.0);
    cur = out;
  }
}

// The arguments of the ionic kernel shared by both operator forms (no field
// source, no bands, not in rows mode).
IonicArgs ionic_args(st_handle *h, int kind, bool want_stats) {
  IonicArgs a;
  std::memset(&a, 0, sizeof(a));
  a.D = h->desc;
  a.g = geom(h);
  a.bt = h->bt; a.xt = h->xt; a.bprod = h->bprod;
  a.bt2 = h->bt2; a.bprod2 = h->bprod2;
  a.tmask = h->tmask;
  for (int b = 0; b < ST_MAX_STIM; ++b) {
    const double v = b < h->desc.n_stim ? h->desc.stim[b].amp : 0.0;
    const float hi = (float)v;
    a.amp2[b] = make_float2(hi, (float)(v - (double)hi));
  }
  a.Nt = h->Nt; a.nel_t = h->nel_t;
  a.Qs = h->Qs; a.Nel_s = h->Nel_s;
  a.kind = kind;
  a.want_stats = want_stats ? 1 : 0;
  a.emax = h->emax;
  a.stats = (unsigned long long *)h->stats;
  return a;
}

st_status ionic_launch(st_handle *h, const IonicArgs &a) {
  cudaStream_t s = h->stream;
  if (a.want_stats) {
    st_count_launch(); zero_ull_kernel<<<grid_for((long long)h->nel_t * h->Nel_s), 256, 0, s>>>(h->emax, (long long)h->nel_t * h->Nel_s);
    st_count_launch(); zero_ull_kernel<<<1, 32, 0, s>>>((unsigned long long *)h->stats, 4);
  }
  unsigned blocks = (unsigned)((h->Qs + 127) / 128);
  switch (h->p) {
    case 1: st_count_launch(); ionic_tline_kernel<1><<<blocks, 128, 0, s>>>(a); break;
    case 2: st_count_launch(); ionic_tline_kernel<2><<<blocks, 128, 0, s>>>(a); break;
    case 3: st_count_launch(); ionic_tline_kernel<3><<<blocks, 128, 0, s>>>(a); break;
    default: st_count_launch(); ionic_tline_kernel<4><<<blocks, 128, 0, s>>>(a); break;
  }
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

// The lean form's linearization: u^k and w^k at the Gauss rows of the other
// axes (the rows the operator reads), and, when the statistics are wanted,
// the residual maxima of Eq. (theta_ce_u) from the same rows (the other axes'
// Laplacian part in the first work buffer); no time bands.
st_status ionic_rows(st_handle *h, const float2 *u2, const float2 *w2, int kind, bool want_stats) {
  rows_forward(h, u2, -1, h->U1, 0, 1.0);
  rows_forward(h, w2, -1, h->W1, 0, 1.0);
  if (!want_stats) {
    ST_CUDA(cudaGetLastError());
    return ST_OK;
  }
  float2 *L1 = reinterpret_cast<float2 *>(h->W64[0]);
  for (int l = 1; l < h->d; ++l) rows_forward(h, u2, l, L1, l > 1 ? 1 : 0, h->desc.D[l]);
  IonicArgs a = ionic_args(h, kind, want_stats);
  a.rows_mode = 1;
  a.U1 = h->U1; a.W1 = h->W1; a.L1 = h->d >= 2 ? L1 : nullptr;
  a.tbx = h->Bq2[0]; a.tb2x = h->B2q2[0];
  a.Dx = h->desc.D[0];
  a.nx = h->n[0]; a.Qx = h->Q[0];
  a.rows = h->rows_x;
  return ionic_launch(h, a);
}

}  // namespace

st_status ionic_run(st_handle *h, const double *u, const double *w, int kind, bool want_stats) {
  cudaStream_t s = h->stream;
  // fields at spatial Gauss points as double-float pairs: u, sum_l D_ll d_ll u, w
  // (u and w split into pairs first; the FP64 field buffers hold the pairs)
  float2 *u2 = reinterpret_cast<float2 *>(h->t64a), *w2 = reinterpret_cast<float2 *>(h->t64b);
  st_count_launch(); d2df_kernel<<<grid_for(h->Ndof), 256, 0, s>>>(u2, u, h->Ndof);
  st_count_launch(); d2df_kernel<<<grid_for(h->Ndof), 256, 0, s>>>(w2, w, h->Ndof);
  h->lin_kind = kind;
  if (h->lean) return ionic_rows(h, u2, w2, kind, want_stats);
  float2 *U0 = reinterpret_cast<float2 *>(h->U0), *L0 = reinterpret_cast<float2 *>(h->L0);
  float2 *W0 = reinterpret_cast<float2 *>(h->Wq0);
  if (!fields_to_qpts_2d(h, u2, w2, U0, L0, W0)) {
    spatial_to_qpts(h, u2, -1, U0, 0, 1.0);
    for (int l = 0; l < h->d; ++l) spatial_to_qpts(h, u2, l, L0, l > 0 ? 1 : 0, h->desc.D[l]);
    spatial_to_qpts(h, w2, -1, W0, 0, 1.0);
  }
  IonicArgs a = ionic_args(h, kind, want_stats);
  a.no_reaction_band = h->desc.eps_reaction >= 0.0 ? 1 : 0;
  a.U0 = U0; a.L0 = L0; a.W0 = W0;
  a.band_hi = h->band32;
  a.band_lo = h->band_lo;
  return ionic_launch(h, a);
}

// C[m][c] = sum_k A[k][m] X[k][c] for the columns c0 <= c < min(c0 + 8, nc)
// (A: K x M row-major, X: K x nc, C: M x nc): one thread per m, the few
// columns in registers, X read by every thread of a warp at once.  For the
// tall, narrow products of the low-rank step a tiled GEMM would compute
// mostly padding.
__global__ void skinny_atx_kernel(double *__restrict__ C, const double *__restrict__ A, const double *__restrict__ X,
                                  long long M, int nc, int c0, int K) {
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int n = min(8, nc - c0);
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < K; ++k) {
    const double a = A[(long long)k * M + m];
    const double *xr = X + (long long)k * nc + c0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c < n) acc[c] = fma(a, __ldg(xr + c), acc[c]);
  }
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (c < n) C[m * nc + c0 + c] = acc[c];
}

// Truncated SVD of the N_t x N_s matrix M (row-major, FP64) through its Gram
// matrix (Eq. tol): the smallest rank R <= cap with
// ||M - U diag(sigma) V^T||_F <= eps ||M||_F; U (N_t x R), sigma (R, device
// and host), V = M^T U diag(1/sigma) (N_s x R).  R = 0 for M = 0.
static st_status truncated_svd(st_handle *h, const double *M, double eps, int cap, double *Uo, double *so,
                               double *Vo, int *R_out, double *fro_out, std::vector<double> &sig) {
  cudaStream_t s = h->stream;
  const int Nt = h->Nt;
  {
    // G = M M^T in double-float, upper-triangle tiles, K split so that the
    // grid holds several blocks per SM; the partials go to the first work
    // buffer, or to the handle's own buffer where that one is too small for a
    // single split (set-up sizes it for exactly that)
    const int ntile = (Nt + kGT - 1) / kGT, npair = ntile * (ntile + 1) / 2;
    double *part = h->gpart ? h->gpart : h->W64[0];
    const long long cap = h->gpart ? h->gpart_cap : h->wcap;
    if ((long long)npair * kGT * kGT > cap) return ST_ERR_STATE;  // set-up sizes the buffer: not reached
    int nsplit = (int)std::max<long long>(1, std::min<long long>((152LL * 6 + npair - 1) / npair, (h->Ns + 255) / 256));
    while ((long long)nsplit * npair * kGT * kGT > cap && nsplit > 1) --nsplit;
    const int kchunk = (int)((h->Ns + nsplit - 1) / nsplit);
    st_count_launch(); gram_df_kernel<<<dim3(npair, nsplit), 256, 0, s>>>(part, M, Nt, h->Ns, ntile, kchunk);
    st_count_launch(); gram_reduce_kernel<<<grid_for((long long)npair * kGT * kGT), 256, 0, s>>>(h->gram, part, Nt, ntile, npair, nsplit);
  }
  std::vector<double> G((size_t)Nt * Nt);
  // trace = ||M||_F^2
  ST_CUDA(cudaMemcpyAsync(G.data(), h->gram, G.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  ST_CUDA(cudaStreamSynchronize(s));
  double tr = 0.0;
  for (int i = 0; i < Nt; ++i) tr += G[(size_t)i * Nt + i];
  *fro_out = std::sqrt(tr);
  *R_out = 0;
  sig.clear();
  if (!(tr > 0.0)) return std::isfinite(tr) ? ST_OK : ST_ERR_NAN;
  // leading eigenpairs of G and the rank R: smallest R with
  // ||M - U S V^T||_F^2 = tr - sum_{i<=R} lam_i <= eps^2 tr (Eq. tol)
  std::vector<double> lam;
  int R = 0;
  st_status lz = gram_top_eigs(h, h->gram, Nt, tr, eps, cap, Uo, &R, lam);
  if (lz == ST_ERR_NAN) return lz;
  if (lz != ST_OK) {
    // full decomposition (eigenvalues descending) when Lanczos did not settle
    ST_TRY(sym_eig_desc(h, h->gram, Nt, h->evec, h->eval));
    lam.assign(Nt, 0.0);
    ST_CUDA(cudaMemcpyAsync(lam.data(), h->eval, Nt * sizeof(double), cudaMemcpyDeviceToHost, s));
    ST_CUDA(cudaStreamSynchronize(s));
    double kept = 0.0;
    R = Nt;
    for (int r = 1; r <= Nt; ++r) {
      kept += std::max(lam[r - 1], 0.0);
      if (tr - kept <= eps * eps * tr) { R = r; break; }
    }
    if (R > cap) R = cap;
    // U_R (N_t x R) = first R columns of evec (evec[i][c], c sorted descending)
    ST_CUDA(cudaMemcpy2DAsync(Uo, R * sizeof(double), h->evec, Nt * sizeof(double), R * sizeof(double), Nt,
                              cudaMemcpyDeviceToDevice, s));
  }
  sig.assign(R, 0.0);
  for (int r = 0; r < R; ++r) sig[r] = std::sqrt(std::max(lam[r], 0.0));
  ST_CUDA(cudaMemcpyAsync(so, sig.data(), R * sizeof(double), cudaMemcpyHostToDevice, s));
  // V = M^T U_R diag(1/sigma): (N_s x R)
  for (int c0 = 0; c0 < R; c0 += 8) {
    st_count_launch();
    skinny_atx_kernel<<<(unsigned)((h->Ns + 127) / 128), 128, 0, s>>>(Vo, M, Uo, h->Ns, R, c0, Nt);
  }
  st_count_launch(); scale_cols_kernel<<<grid_for(h->Ns * R), 256, 0, s>>>(Vo, so, R, h->Ns);
  *R_out = R;
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

st_status theta_and_lowrank(st_handle *h, st_ionic_info *info) {
  cudaStream_t s = h->stream;
  const st_problem_desc &D = h->desc;
  double st[4];
  ST_CUDA(cudaMemcpyAsync(st, h->stats, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  ST_CUDA(cudaStreamSynchronize(s));
  double umax = st[0], utmax = st[1], rmax = st[2];
  double den = D.C_m * (umax / D.T + utmax);
  if (info) {
    info->u_max = umax; info->ut_max = utmax; info->den = den; info->r_max = rmax;
  }
  if (!std::isfinite(umax) || !std::isfinite(utmax) || !std::isfinite(rmax)) return ST_ERR_NAN;
  // numerators: window maxima of the element maxima, axis by axis
  const double *cur = (const double *)h->emax;
  long long dimsE[4] = {h->nel[0], h->nel[1], h->nel[2], h->nel_t};
  long long dimsB[4] = {h->n[0], h->n[1], h->n[2], h->Nt};
  long long cdims[4];
  for (int l = 0; l < 3; ++l) cdims[l] = l < h->d ? dimsE[l] : 1;
  cdims[3] = h->nel_t;
  int ping = 0;
  int axes[4];
  int na = 0;
  for (int l = 0; l < h->d; ++l) axes[na++] = l;
  axes[na++] = 3;
  for (int ai = 0; ai < na; ++ai) {
    int l = axes[ai];
    long long inner = 1, outer = 1;
    for (int m = 0; m < l; ++m) inner *= cdims[m];
    for (int m = l + 1; m < 4; ++m) outer *= cdims[m];
    int nel = (int)dimsE[l], nout = (int)dimsB[l];
    double *out = h->W64[ping];
    long long total = outer * nout * inner;
    st_count_launch(); window_max_kernel<<<grid_for(total), 256, 0, s>>>(out, cur, nel, nout, h->p, l == 3 ? 1 : 0,
                                                       D.suppext == ST_SUPPEXT_SYMMETRIC, inner, outer);
    cdims[l] = nout;
    cur = out;
    ping ^= 1;
  }
  long long NtNs = h->Ndof;
  st_count_launch(); theta_kernel<<<grid_for(NtNs), 256, 0, s>>>(h->theta, cur, den, NtNs);
  std::vector<double> sig;
  int R = 0;
  double fro = 0.0;
  ST_TRY(truncated_svd(h, h->theta, D.eps_theta, h->rank_cap, h->Ur, h->sr, h->Vr, &R, &fro, sig));
  h->theta_fro = fro;
  h->rank = R;
  if (info) { info->theta_fro = fro; info->rank = R; }
  if (h->lean && R > 0) {
    // scale of each SU rank term in the lean operator: C_m sigma_r
    std::vector<double> cf(R);
    for (int r = 0; r < R; ++r) cf[r] = D.C_m * sig[r];
    ST_CUDA(cudaMemcpyAsync(h->cfr, cf.data(), R * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

// Band form: band[(k,it)][q] += sum_r T[r][(k,it)] Cq[r][q], with the spatial
// factors Cq[r][q] = scale sigma_r ws(q) phi_r(x_q) (phi_r the d-linear
// interpolant of V[:, r] on the spatial Greville grid), 8 ranks per pass;
// both factors split into double-float pairs first (Cq in the work buffers,
// R Q_s <= N_t Q_s values).
static st_status bands_add_ranks(st_handle *h, const double *V, const double *sig, double scale, const double *T,
                                 float2 *T2, int R) {
  cudaStream_t s = h->stream;
  const int p = h->p;
  double *Cq = h->W64[0];
  HatArgs hat;
  for (int l = 0; l < 3; ++l) {
    hat.idx[l] = h->hat_i_s[l];
    hat.lam[l] = h->hat_l_s[l];
    hat.n[l] = h->n[l];
  }
  st_count_launch(); su_space_coef_kernel<<<grid_for(h->Qs * R), 256, 0, s>>>(Cq, V, sig, geom(h), hat, scale, R, h->Qs);
  const int Mrows = (p + 1) * h->Nt;
  float2 *Cq2 = reinterpret_cast<float2 *>(h->W64[1]);
  st_count_launch(); d2df_kernel<<<grid_for((long long)R * h->Qs), 256, 0, s>>>(Cq2, Cq, (long long)R * h->Qs);
  st_count_launch(); d2df_kernel<<<grid_for((long long)R * Mrows), 256, 0, s>>>(T2, T, (long long)R * Mrows);
  // thread = 4 spatial points; about 8 blocks per SM in all
  const long long gx = (h->Qs + 1023) / 1024;
  const dim3 g2((unsigned)gx, (unsigned)std::max<long long>(1, std::min<long long>(Mrows, (152LL * 8 + gx - 1) / gx)));
  for (int r0 = 0; r0 < R; r0 += 8) {
    const int left = R - r0;
    if (left <= 2) {
      st_count_launch(); su_band_update_kernel<2><<<g2, 256, 0, s>>>(h->band32, h->band_lo, T2, Cq2, r0, R, Mrows, h->Qs);
    } else if (left <= 4) {
      st_count_launch(); su_band_update_kernel<4><<<g2, 256, 0, s>>>(h->band32, h->band_lo, T2, Cq2, r0, R, Mrows, h->Qs);
    } else {
      st_count_launch(); su_band_update_kernel<8><<<g2, 256, 0, s>>>(h->band32, h->band_lo, T2, Cq2, r0, R, Mrows, h->Qs);
    }
  }
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

st_status su_band_add(st_handle *h) {
  cudaStream_t s = h->stream;
  const int p = h->p;
  const bool su = h->desc.stabilization == ST_SU && h->rank > 0;
  if (su) {
    const int R = h->rank;
    st_count_launch(); theta_t_kernel<<<grid_for((long long)h->Qt * R), 256, 0, s>>>(h->th_t, h->Ur, R, h->Qt, h->hat_i_t, h->hat_l_t);
    st_count_launch(); su_time_band_kernel<<<grid_for((long long)R * (p + 1) * h->Nt), 256, 0, s>>>(h->Tr, h->th_t, h->tauq, h->bt,
                                                                                h->wt, R, h->Nt, h->nel_t, p);
    if (h->lean) {
      // the lean operator reads the rank factors themselves: only the time
      // bands, as double-float pairs
      st_count_launch(); d2df_kernel<<<grid_for((long long)R * (p + 1) * h->Nt), 256, 0, s>>>(h->Tr2, h->Tr, (long long)R * (p + 1) * h->Nt);
    } else {
      ST_TRY(bands_add_ranks(h, h->Vr, h->sr, h->desc.C_m, h->Tr, h->Tr2, R));
    }
  }
  // the low-rank reaction (its time bands are ready): into the bands of the band form
  if (!h->lean && h->desc.eps_reaction >= 0.0 && h->rankC > 0)
    ST_TRY(bands_add_ranks(h, h->VrC, h->srC, 1.0, h->Tc, h->Tc2, h->rankC));
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

st_status reaction_lowrank(st_handle *h, const double *u, const double *w, int kind) {
  cudaStream_t s = h->stream;
  const st_problem_desc &D = h->desc;
  // values at the Greville grid: one banded collocation pass per axis (x
  // first, time last) into the Kronecker temporaries
  auto greville = [&](const double *in, double *out) {
    const double *cur = in;
    const int naxes = h->d + 1;
    int ping = 0;
    for (int ax = 0; ax < naxes; ++ax) {
      const bool time = ax == h->d;
      const int n = time ? h->Nt : h->n[ax];
      long long inner = 1, outer = 1;
      if (time) {
        inner = h->Ns;
      } else {
        for (int m = 0; m < ax; ++m) inner *= h->n[m];
        outer = h->Nt;
        for (int m = ax + 1; m < h->d; ++m) outer *= h->n[m];
      }
      double *dst = ax == naxes - 1 ? out : h->K64[ping];
      const double *band = time ? h->Gtb : h->Gsb[ax];
      const double *bands[1] = {band};
      const double *ins[1] = {cur};
      const double cf[1] = {1.0};
      launch_band_pass<double>(s, dst, 1, bands, ins, cf, n, inner, outer, h->p, false);
      cur = dst;
      ping ^= 1;
    }
  };
  double *Ug = h->K64[2], *Wg = h->K64[3], *Cg = h->K64[4];
  greville(u, Ug);
  greville(w, Wg);
  st_count_launch(); reaction_coef_kernel<<<grid_for(h->Ndof), 256, 0, s>>>(Cg, Ug, Wg, D.c1, D.c2, D.a, kind == ST_NEWTON, h->Ndof);
  std::vector<double> sig;
  int R = 0;
  double fro = 0.0;
  ST_TRY(truncated_svd(h, Cg, D.eps_reaction, h->rank_cap, h->UrC, h->srC, h->VrC, &R, &fro, sig));
  h->rankC = R;
  if (R > 0) {
    const int p = h->p;
    st_count_launch(); theta_t_kernel<<<grid_for((long long)h->Qt * R), 256, 0, s>>>(h->thC, h->UrC, R, h->Qt, h->hat_i_t, h->hat_l_t);
    st_count_launch(); mass_time_band_kernel<<<grid_for((long long)R * (p + 1) * h->Nt), 256, 0, s>>>(h->Tc, h->thC, h->bt, h->wt,
                                                                                  R, h->Nt, h->nel_t, p);
    st_count_launch(); d2df_kernel<<<grid_for((long long)R * (p + 1) * h->Nt), 256, 0, s>>>(h->Tc2, h->Tc, (long long)R * (p + 1) * h->Nt);
    ST_CUDA(cudaMemcpyAsync(h->cfc, sig.data(), R * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

st_status source_assemble(st_handle *h) {
  cudaStream_t s = h->stream;
  // f at the spatial Gauss points of a block of time rows (all rows at once
  // in the band form, whose field buffer holds them; blocks of rows that fit
  // one work buffer in the lean form), then the spatial test functions
  double *Fq = h->lean ? h->W64[0] : h->U0;
  const long long cap = h->lean ? h->wcap : h->NtQs;
  const int nr = (int)std::max<long long>(1, std::min<long long>(h->Nt, cap / h->Qs));
  unsigned blocks = (unsigned)((h->Qs + 127) / 128);
  GeomArgs g = geom(h);
  long long qd[3] = {h->Q[0], h->Q[1], h->Q[2]};
  long long nd[3] = {h->n[0], h->n[1], h->n[2]};
  for (int r0 = 0; r0 < h->Nt; r0 += nr) {
    const int rows = std::min(nr, h->Nt - r0);
    switch (h->p) {
      case 1: st_count_launch(); source_tline_kernel<1><<<blocks, 128, 0, s>>>(h->desc, g, h->bt, h->wt, h->xt, h->Nt, h->nel_t, h->Qs, r0, rows, Fq); break;
      case 2: st_count_launch(); source_tline_kernel<2><<<blocks, 128, 0, s>>>(h->desc, g, h->bt, h->wt, h->xt, h->Nt, h->nel_t, h->Qs, r0, rows, Fq); break;
      case 3: st_count_launch(); source_tline_kernel<3><<<blocks, 128, 0, s>>>(h->desc, g, h->bt, h->wt, h->xt, h->Nt, h->nel_t, h->Qs, r0, rows, Fq); break;
      default: st_count_launch(); source_tline_kernel<4><<<blocks, 128, 0, s>>>(h->desc, g, h->bt, h->wt, h->xt, h->Nt, h->nel_t, h->Qs, r0, rows, Fq); break;
    }
    // spatial test functions: Gauss points -> coefficients, last axis first
    const double *cur = Fq;
    int ping = h->lean ? 1 : 0;   // the lean form's rows sit in the first work buffer
    for (int l = h->d - 1; l >= 0; --l) {
      long long inner = 1, outer = rows;
      for (int m = 0; m < l; ++m) inner *= qd[m];
      for (int m = l + 1; m < h->d; ++m) outer *= nd[m];
      double *out = (l == 0) ? h->f64 + (long long)r0 * h->Ns : h->W64[ping];
      launch_interp_bwd<double>(s, out, cur, h->Bq[l], h->nel[l], h->p, h->nq, inner, outer, false);
      cur = out;
      ping ^= 1;
    }
  }
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

// Fixed scratch of the handle-free w-update: M_t at [0, Nt B) and the LU of
// W_t + b d_e M_t at [Nt B, 2 Nt B), B = 2p+1.  It lives in the module's
// static device storage, so that call allocates no device memory; every call
// on a device shares it, and each call rewrites both bands before reading.
static __device__ __align__(256) double g_wupdate_scratch[ST_WUPDATE_STATIC_CAPACITY];

namespace {
constexpr int kScratchDevices = 64;
std::atomic<double *> g_wupdate_scratch_addr[kScratchDevices];

// Device address of the scratch on the current device.  The first call on a
// device asks the runtime (cudaGetSymbolAddress) and caches the answer.
st_status wupdate_scratch_addr(double **out) {
  int dev = 0;
  ST_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < kScratchDevices) {
    double *p = g_wupdate_scratch_addr[dev].load(std::memory_order_acquire);
    if (p) { *out = p; return ST_OK; }
  }
  void *p = nullptr;
  ST_CUDA(cudaGetSymbolAddress(&p, g_wupdate_scratch));
  if (!p) return ST_ERR_CUDA;
  if (dev >= 0 && dev < kScratchDevices) g_wupdate_scratch_addr[dev].store((double *)p, std::memory_order_release);
  *out = (double *)p;
  return ST_OK;
}
}  // namespace

st_status wupdate_static_run(cudaStream_t s, const double *u, double *w, const double *Mt_host,
                             const double *lu_host, double bcoef, int Nt, long long Ns, int p) {
  const long long band = (long long)Nt * (2 * p + 1);
  if (Nt < 1 || p < 1 || p > 4 || Ns < 1) return ST_ERR_ARG;
  if (2 * band > ST_WUPDATE_STATIC_CAPACITY) return ST_ERR_CAPACITY;
  double *scratch = nullptr;
  ST_TRY(wupdate_scratch_addr(&scratch));
  double *Mt = scratch, *lu = scratch + band;
  // Pageable-host sources: each copy returns once its source has been staged,
  // and stays ordered on s before the kernel that reads it.
  ST_CUDA(cudaMemcpyAsync(Mt, Mt_host, band * sizeof(double), cudaMemcpyHostToDevice, s));
  ST_CUDA(cudaMemcpyAsync(lu, lu_host, band * sizeof(double), cudaMemcpyHostToDevice, s));
  unsigned blocks = (unsigned)((Ns + 127) / 128);
  switch (p) {
    case 1: st_count_launch(); wupdate_kernel<1><<<blocks, 128, 0, s>>>(w, u, Mt, lu, bcoef, Nt, Ns); break;
    case 2: st_count_launch(); wupdate_kernel<2><<<blocks, 128, 0, s>>>(w, u, Mt, lu, bcoef, Nt, Ns); break;
    case 3: st_count_launch(); wupdate_kernel<3><<<blocks, 128, 0, s>>>(w, u, Mt, lu, bcoef, Nt, Ns); break;
    default: st_count_launch(); wupdate_kernel<4><<<blocks, 128, 0, s>>>(w, u, Mt, lu, bcoef, Nt, Ns); break;
  }
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

st_status wupdate_run(st_handle *h, const double *u, double *w) {
  cudaStream_t s = h->stream;
  double bcoef = h->desc.b;
  unsigned blocks = (unsigned)((h->Ns + 127) / 128);
  switch (h->p) {
    case 1: st_count_launch(); wupdate_kernel<1><<<blocks, 128, 0, s>>>(w, u, h->Mtb, h->wlu, bcoef, h->Nt, h->Ns); break;
    case 2: st_count_launch(); wupdate_kernel<2><<<blocks, 128, 0, s>>>(w, u, h->Mtb, h->wlu, bcoef, h->Nt, h->Ns); break;
    case 3: st_count_launch(); wupdate_kernel<3><<<blocks, 128, 0, s>>>(w, u, h->Mtb, h->wlu, bcoef, h->Nt, h->Ns); break;
    default: st_count_launch(); wupdate_kernel<4><<<blocks, 128, 0, s>>>(w, u, h->Mtb, h->wlu, bcoef, h->Nt, h->Ns); break;
  }
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}
