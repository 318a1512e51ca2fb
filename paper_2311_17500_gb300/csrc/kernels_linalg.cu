// Tensor kernels of the operator, the preconditioner and the Krylov solver.
//
// Every vector of unknowns is a tensor [N_t][n_z][n_y][n_x] (x fastest, time
// slowest).  A one-axis operation sees it as [outer][n][inner]: `n` entries
// along the axis, `inner` contiguous entries after it, `outer` blocks before.
#include <algorithm>
#include "st_internal.h"

namespace {

constexpr int kThreads = 256;

inline int grid_for(long long total, int threads = kThreads) {
  long long g = (total + threads - 1) / threads;
  if (g > 152LL * 64) g = 152LL * 64;   // grid-stride loops beyond 64 waves of 152 SMs
  if (g < 1) g = 1;
  return (int)g;
}

// Division by a fixed d of 32-bit unsigned x < 2^31 as a multiply and a shift:
// with s = ceil(log2 d) and m = floor(2^(32+s) / d) + 1, floor(x m / 2^(32+s))
// equals floor(x / d) because m d - 2^(32+s) lies in (0, d].
struct FastDiv {
  unsigned d;
  int s;
  unsigned long long m;
  FastDiv() : d(1), s(0), m((1ull << 32) + 1) {}
  explicit FastDiv(long long dd) {
    d = (unsigned)dd;
    s = 0;
    while ((1ull << s) < d) ++s;
    m = ((1ull << (32 + s)) / d) + 1;
  }
  __device__ __forceinline__ unsigned div(unsigned x) const {
    return (unsigned)(((unsigned long long)x * m) >> (32 + s));
  }
};

// idx = (o * n + i) * inner + c  ->  (o, i, c)
struct Split3 {
  FastDiv inner, n;
  Split3(long long ninner, long long nn) : inner(ninner), n(nn) {}
  __device__ __forceinline__ void operator()(long long idx, long long &o, int &i, long long &c, bool small) const {
    if (small) {
      unsigned x = (unsigned)idx;
      unsigned r = inner.div(x);
      c = x - r * inner.d;
      unsigned oo = n.div(r);
      i = (int)(r - oo * n.d);
      o = oo;
    } else {
      c = idx % (long long)inner.d;
      long long r = idx / (long long)inner.d;
      i = (int)(r % (long long)n.d);
      o = r / (long long)n.d;
    }
  }
};

template <typename T>
struct BandTerms {
  const T *band[3];
  const T *in[3];
  T coef[3];
  int nterms;
};

// out[o][i][c] (+)= sum_t coef_t sum_k band_t[i][k] in_t[o][i-p+k][c]
// (banded 1D matrix n x (2p+1) applied along one axis: the Kronecker factors
// of W_t (x) M_s + M_t (x) K_s, Sec. 3.1).
template <typename T, int P>
__global__ void band_pass_kernel(T *__restrict__ out, BandTerms<T> bt, int n, long long inner,
                                 long long outer, int accumulate, Split3 sp) {
  constexpr int p = P, B = 2 * P + 1;
  long long total = outer * n * inner;
  const bool small = total < (1ll << 31);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long c, o;
    int i;
    sp(idx, o, i, c, small);
    T acc = accumulate ? out[idx] : T(0);
    int k0 = max(0, p - i), k1 = min(B - 1, n - 1 - i + p);
    for (int t = 0; t < bt.nterms; ++t) {
      const T *bd = bt.band[t] + (size_t)i * B;
      const T *src = bt.in[t] + (o * n + (i - p)) * inner + c;
      T s = T(0);
      if (k0 == 0 && k1 == B - 1) {
#pragma unroll
        for (int k = 0; k < B; ++k) s += __ldg(bd + k) * src[(long long)k * inner];
      } else {
        for (int k = k0; k <= k1; ++k) s += __ldg(bd + k) * src[(long long)k * inner];
      }
      acc += bt.coef[t] * s;
    }
    out[idx] = acc;
  }
}

// Coefficients -> Gauss points along one axis (sum factorization, Sec. 3.1):
// out[o][e*nq+q][c] = sum_a tab[e][q][a] in[o][e+a][c].
template <typename T, int P>
__global__ void interp_fwd_kernel(T *__restrict__ out, const T *__restrict__ in, const T *__restrict__ tab,
                                  int nel, long long inner, long long outer, Split3 sp) {
  constexpr int p = P, nq = P + 1;
  int nout = nel * nq, nin = nel + p;
  long long total = outer * nout * inner;
  const bool small = total < (1ll << 31);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long c, o;
    int eq;
    sp(idx, o, eq, c, small);
    int e = eq / nq;
    const T *tb = tab + (size_t)eq * (p + 1);
    const T *src = in + (o * nin + e) * inner + c;
    T s = T(0);
#pragma unroll
    for (int a = 0; a <= p; ++a) s += __ldg(tb + a) * src[(long long)a * inner];
    out[idx] = s;
  }
}

// Gauss points -> coefficients (transpose of interp_fwd):
// out[o][i][c] (+)= sum_{e=i-p..i} sum_q tab[e][q][i-e] in[o][e*nq+q][c].
template <typename T, int P>
__global__ void interp_bwd_kernel(T *__restrict__ out, const T *__restrict__ in, const T *__restrict__ tab,
                                  int nel, long long inner, long long outer, int accumulate, Split3 sp) {
  constexpr int p = P, nq = P + 1;
  int nin = nel * nq, nout = nel + p;
  long long total = outer * nout * inner;
  const bool small = total < (1ll << 31);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long c, o;
    int i;
    sp(idx, o, i, c, small);
    T s = T(0);
#pragma unroll
    for (int a = 0; a <= p; ++a) {
      int e = i - a;
      if (e < 0 || e >= nel) continue;
      const T *src = in + (o * nin + (long long)e * nq) * inner + c;
      const T *tb = tab + (size_t)e * nq * (p + 1) + a;
#pragma unroll
      for (int q = 0; q < nq; ++q) s += __ldg(tb + q * (p + 1)) * src[(long long)q * inner];
    }
    out[idx] = accumulate ? out[idx] + s : s;
  }
}

// Per spatial Gauss point q, the symmetric time band of the reaction and SU
// terms: z[it][q] = sum_{k=-P..P} band(it, it+k; q) x[it+k][q], band stored as
// the upper half [k][it][q] (entry (it, it+k)), k = 0..P.  One thread sweeps
// the whole time line of a column; the window of x and band rows lives in
// registers, so every band entry and x value is read once.
template <typename T, int P>
__global__ void qband_kernel(T *__restrict__ z, const T *__restrict__ x, const T *__restrict__ band,
                             int Nt, long long Qs) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= Qs) return;
  const long long plane = (long long)Nt * Qs;
  T xw[2 * P + 1];           // x[it-P .. it+P]
  T bl[P][P + 1];            // band rows it-P .. it-1 (upper parts)
#pragma unroll
  for (int i = 0; i < 2 * P + 1; ++i) xw[i] = T(0);
#pragma unroll
  for (int r = 0; r < P; ++r)
#pragma unroll
    for (int k = 0; k <= P; ++k) bl[r][k] = T(0);
#pragma unroll
  for (int k = 0; k < P; ++k) xw[P + 1 + k] = (k < Nt) ? x[(long long)k * Qs + q] : T(0);
  for (int it = 0; it < Nt; ++it) {
    // shift the window: xw[j] = x[it - P + j]
#pragma unroll
    for (int j = 0; j < 2 * P; ++j) xw[j] = xw[j + 1];
    xw[2 * P] = (it + P < Nt) ? x[(long long)(it + P) * Qs + q] : T(0);
    T b[P + 1];
#pragma unroll
    for (int k = 0; k <= P; ++k) b[k] = band[k * plane + (long long)it * Qs + q];
    T s = b[0] * xw[P];
#pragma unroll
    for (int k = 1; k <= P; ++k) s += b[k] * xw[P + k] + bl[P - k][k] * xw[P - k];
    z[(long long)it * Qs + q] = s;
#pragma unroll
    for (int r = 0; r < P - 1; ++r)
#pragma unroll
      for (int k = 0; k <= P; ++k) bl[r][k] = bl[r + 1][k];
#pragma unroll
    for (int k = 0; k <= P; ++k) bl[P - 1][k] = b[k];
  }
}

// Dense strided GEMM C[b](m, c) = sum_k A(m, k) X[b](k, c) with 64x64 tiles,
// 256 threads, 4x4 outputs per thread: the spatial transforms U_l, U_l^T of
// the fast-diagonalization preconditioner (Eq. factorized), the Gram matrix
// of Theta-hat and the products of the eigen-refinement.
struct GemmDesc {
  int M, N, K, batch;
  long long sam, sak;            // A(m,k) = A[m*sam + k*sak]
  long long sbb, sbk, sbc;       // X(b,k,c)
  long long scb, scm, scc;       // C(b,m,c)
};

template <typename T>
__global__ void __launch_bounds__(256) gemm_kernel(T *__restrict__ C, const T *__restrict__ A,
                                                   const T *__restrict__ X, GemmDesc g, T alpha, T beta) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Xs[BK][BN + 1];
  int b = blockIdx.z;
  int m0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  int tid = threadIdx.x;
  int tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  const T *Xb = X + (long long)b * g.sbb;
  bool a_k_fast = (g.sak == 1);
  bool x_c_fast = (g.sbc == 1);
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int l = tid; l < BM * BK; l += 256) {
      int mm, kk;
      if (a_k_fast) { kk = l % BK; mm = l / BK; } else { mm = l % BM; kk = l / BM; }
      int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < g.M && k < g.K) ? A[m * g.sam + k * g.sak] : T(0);
    }
    for (int l = tid; l < BN * BK; l += 256) {
      int cc, kk;
      if (x_c_fast) { cc = l % BN; kk = l / BN; } else { kk = l % BK; cc = l / BK; }
      int c = c0 + cc, k = k0 + kk;
      Xs[kk][cc] = (c < g.N && k < g.K) ? Xb[k * g.sbk + c * g.sbc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[4], xv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) xv[j] = Xs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * xv[j];
    }
    __syncthreads();
  }
  T *Cb = C + (long long)b * g.scb;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int m = m0 + ty * 4 + i, c = c0 + tx + 16 * j;
      if (m < g.M && c < g.N) {
        long long off = m * g.scm + c * g.scc;
        Cb[off] = beta == T(0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * Cb[off];
      }
    }
}

// One banded LU solve along time per spatial eigen-index j (the block-diagonal
// middle factor of the fast-diagonalization preconditioner): lu[it][k][j] holds
// L below the diagonal (unit diagonal), 1/u_ii on it and U above.
template <typename T, int P>
__global__ void tline_lu_kernel(T *__restrict__ z, const T *__restrict__ r, const T *__restrict__ lu, int Nt,
                                long long Ns) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= Ns) return;
  constexpr int B = 2 * P + 1;
  constexpr int U = 8;     // time steps whose operands are loaded ahead of the recurrence
  T yw[P];
#pragma unroll
  for (int k = 0; k < P; ++k) yw[k] = T(0);
  // forward substitution with the unit lower factor
  for (int it0 = 0; it0 < Nt; it0 += U) {
    T rv[U], lv[U][P];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int it = it0 + u;
      bool ok = it < Nt;
      rv[u] = ok ? r[(long long)it * Ns + j] : T(0);
#pragma unroll
      for (int k = 1; k <= P; ++k) lv[u][k - 1] = (ok && it - k >= 0) ? lu[((long long)it * B + (P - k)) * Ns + j] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int it = it0 + u;
      if (it >= Nt) break;
      T s = rv[u];
#pragma unroll
      for (int k = 1; k <= P; ++k) s -= lv[u][k - 1] * yw[P - k];
#pragma unroll
      for (int k = 0; k < P - 1; ++k) yw[k] = yw[k + 1];
      yw[P - 1] = s;
      z[(long long)it * Ns + j] = s;
    }
  }
  // backward substitution with the upper factor (1/u_ii stored on the diagonal)
  T zw[P];
#pragma unroll
  for (int k = 0; k < P; ++k) zw[k] = T(0);
  for (int it0 = Nt - 1; it0 >= 0; it0 -= U) {
    T yv[U], uv[U][P + 1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int it = it0 - u;
      bool ok = it >= 0;
      yv[u] = ok ? z[(long long)it * Ns + j] : T(0);
#pragma unroll
      for (int k = 0; k <= P; ++k) uv[u][k] = (ok && it + k < Nt) ? lu[((long long)it * B + (P + k)) * Ns + j] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int it = it0 - u;
      if (it < 0) break;
      T s = yv[u];
#pragma unroll
      for (int k = 1; k <= P; ++k) s -= uv[u][k] * zw[k - 1];
      s *= uv[u][0];
#pragma unroll
      for (int k = P - 1; k > 0; --k) zw[k] = zw[k - 1];
      zw[0] = s;
      z[(long long)it * Ns + j] = s;
    }
  }
}

template <typename T> struct Acc;
template <> struct Acc<float> { typedef float type; };
template <> struct Acc<double> { typedef double type; };

// 16-byte vector type of the Krylov kernels
template <typename T> struct V16;
template <> struct V16<float> {
  typedef float4 type;
  static constexpr int W = 4;
  __device__ static float dot(const float4 &a, const float4 &b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
  __device__ static float4 fma(float h, const float4 &v, float4 acc) {
    acc.x += h * v.x; acc.y += h * v.y; acc.z += h * v.z; acc.w += h * v.w; return acc;
  }
  __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static float4 upd(const float4 &w, const float4 &a, float s) {
    return make_float4((w.x - a.x) * s, (w.y - a.y) * s, (w.z - a.z) * s, (w.w - a.w) * s);
  }
};
template <> struct V16<double> {
  typedef double2 type;
  static constexpr int W = 2;
  __device__ static double dot(const double2 &a, const double2 &b) { return a.x * b.x + a.y * b.y; }
  __device__ static double2 fma(double h, const double2 &v, double2 acc) {
    acc.x += h * v.x; acc.y += h * v.y; return acc;
  }
  __device__ static double2 zero() { return make_double2(0.0, 0.0); }
  __device__ static double2 upd(const double2 &w, const double2 &a, double s) {
    return make_double2((w.x - a.x) * s, (w.y - a.y) * s);
  }
};

// Partial inner products <V_i, w>, i in [G*blockIdx.y, G*blockIdx.y + G) ∩ [0, nv),
// over the block's contiguous chunk of elements: 16-byte loads of G basis
// vectors per step, accumulation in the storage precision over short chains
// (8 steps), widened to FP64 and reduced in a fixed order by warp shuffles and
// shared memory; partial[i][block].  V rows (stride ldv) and w are 16-byte aligned.
// Compensated (Kahan) accumulation in the storage precision: FP32 vectors
// get close to FP64-accurate sums without FP64 instructions in the loop.
template <typename T>
struct KahanAcc {
  T s, c;
  __device__ __forceinline__ void zero() { s = T(0); c = T(0); }
  __device__ __forceinline__ void add(T x) {
    T y = x - c;
    T t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Partial inner products <V_i, w>, i in [G*blockIdx.y, G*blockIdx.y + G) ∩ [0, nv),
// over the block's contiguous chunk of elements: 16-byte loads of G basis
// vectors per step, compensated accumulation per thread, FP64 block reduction
// in a fixed order (warp shuffles, shared memory); partial[i][block].
// V rows (stride ldv) and w are 16-byte aligned.
template <typename T, int G>
__global__ void __launch_bounds__(256) mdot_kernel(double *__restrict__ partial, const T *__restrict__ V,
                                                   long long ldv, int nv, const T *__restrict__ w, long long n) {
  typedef V16<T> X;
  typedef typename X::type VT;
  constexpr int W = X::W;
  __shared__ double red[G][8];
  const int i0 = blockIdx.y * G;
  const int cnt = min(G, nv - i0);
  const long long nvec = n / W;
  const long long chunk = (nvec + gridDim.x - 1) / gridDim.x;
  const long long beg = (long long)blockIdx.x * chunk, end = min(nvec, beg + chunk);
  KahanAcc<T> acc[G];
#pragma unroll
  for (int g = 0; g < G; ++g) acc[g].zero();
  const VT *wv = reinterpret_cast<const VT *>(w);
  for (long long e = beg + threadIdx.x; e < end; e += blockDim.x) {
    VT x = wv[e];
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < cnt) acc[g].add(X::dot(reinterpret_cast<const VT *>(V + (long long)(i0 + g) * ldv)[e], x));
  }
  if (blockIdx.x == gridDim.x - 1)
    for (long long e = nvec * W + threadIdx.x; e < n; e += blockDim.x)
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (g < cnt) acc[g].add(V[(long long)(i0 + g) * ldv + e] * w[e]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    if (g >= cnt) break;
    double t = acc[g].value();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if (lane == 0) red[g][warp] = t;
  }
  __syncthreads();
  if ((int)threadIdx.x < cnt) {
    double t = 0.0;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) t += red[threadIdx.x][wi];
    partial[(long long)(i0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void reduce_blocks_kernel(double *__restrict__ out, const double *__restrict__ partial, int nblocks,
                                     int nv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  double t = 0.0;
  const double *p = partial + (long long)i * nblocks;
  for (int b = 0; b < nblocks; ++b) t += p[b];
  out[i] = t;
}

// w <- (w - sum_{i<nv} h_i V_i) * s, with s = 1 or, when nrm is given,
// s = 1 / sqrt(nrm[0] - sum h_i^2): the norm of the updated vector by
// Pythagoras from <w, w> and the projection coefficients (classical
// Gram-Schmidt update fused with the normalization).  16-byte aligned rows.
template <typename T>
__global__ void __launch_bounds__(256) maxpy_kernel(T *__restrict__ w, const T *__restrict__ V, long long ldv,
                                                    int nv, const double *__restrict__ h, long long n,
                                                    const double *__restrict__ nrm) {
  typedef V16<T> X;
  typedef typename X::type VT;
  constexpr int W = X::W;
  __shared__ T hs[512];
  __shared__ double sc;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = (T)h[i];
  if (threadIdx.x == 0) {
    double s = 1.0;
    if (nrm) {
      double q = nrm[0];
      for (int i = 0; i < nv; ++i) q -= h[i] * h[i];
      q = q > 0.0 ? sqrt(q) : 0.0;
      s = q > 0.0 ? 1.0 / q : 0.0;
    }
    sc = s;
  }
  __syncthreads();
  const T s = (T)sc;
  const long long nvec = n / W;
  VT *wv = reinterpret_cast<VT *>(w);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nvec;
       e += (long long)gridDim.x * blockDim.x) {
    VT a = X::zero();
#pragma unroll 8
    for (int i = 0; i < nv; ++i) a = X::fma(hs[i], reinterpret_cast<const VT *>(V + (long long)i * ldv)[e], a);
    wv[e] = X::upd(wv[e], a, s);
  }
  if (blockIdx.x == 0)
    for (long long e = nvec * W + threadIdx.x; e < n; e += blockDim.x) {
      T a = T(0);
      for (int i = 0; i < nv; ++i) a += hs[i] * V[(long long)i * ldv + e];
      w[e] = (w[e] - a) * s;
    }
}

template <typename T>
__global__ void scale_copy_kernel(T *__restrict__ y, const T *__restrict__ x, double alpha, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = (T)(alpha * (double)x[e]);
}

__global__ void axpby64_kernel(double *__restrict__ y, const double *__restrict__ x, double a, double b,
                               long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = b == 0.0 ? a * x[e] : a * x[e] + b * y[e];
}

__global__ void sub64_kernel(double *__restrict__ r, const double *__restrict__ b, const double *__restrict__ ax,
                             long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    r[e] = b[e] - ax[e];
}

__global__ void d2f_kernel(float *__restrict__ y, const double *__restrict__ x, double scale, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = (float)(scale * x[e]);
}

__global__ void f2d_axpy_kernel(double *__restrict__ y, const float *__restrict__ x, double scale, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    y[e] += scale * (double)x[e];
}

// max |x - y| (y may be null: max |x|), per block to scratch; NaN counts as +inf.
__device__ __forceinline__ double nan_as_inf(double v) { return v != v ? INFINITY : v; }

__global__ void absmax_kernel(double *__restrict__ scratch, const double *__restrict__ x,
                              const double *__restrict__ y, long long n) {
  __shared__ double red[32];
  double m = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double v = y ? x[e] - y[e] : x[e];
    m = fmax(m, nan_as_inf(fabs(v)));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, red[i]);
    scratch[blockIdx.x] = t;
  }
}

__global__ void max_blocks_kernel(double *__restrict__ out, const double *__restrict__ scratch, int nb) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t = fmax(t, scratch[b]);
    out[0] = t;
  }
}

__global__ void to_f32_kernel(float *__restrict__ y, const double *__restrict__ x, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = (float)x[e];
}

constexpr int kDotBlocks = 608;

}  // namespace

// ---------------------------------------------------------------- launchers
template <typename T>
void launch_band_pass(cudaStream_t s, T *out, int nterms, const T *const *bands, const T *const *ins,
                      const double *coefs, int n, long long inner, long long outer, int p, bool accumulate) {
  BandTerms<T> bt;
  bt.nterms = nterms;
  for (int t = 0; t < 3; ++t) {
    bt.band[t] = t < nterms ? bands[t] : nullptr;
    bt.in[t] = t < nterms ? ins[t] : nullptr;
    bt.coef[t] = t < nterms ? (T)coefs[t] : T(0);
  }
  long long total = outer * n * inner;
  int acc = accumulate ? 1 : 0;
  Split3 sp(inner, n);
  int g = grid_for(total);
  st_count_launch();
  switch (p) {
    case 1: band_pass_kernel<T, 1><<<g, kThreads, 0, s>>>(out, bt, n, inner, outer, acc, sp); break;
    case 2: band_pass_kernel<T, 2><<<g, kThreads, 0, s>>>(out, bt, n, inner, outer, acc, sp); break;
    case 3: band_pass_kernel<T, 3><<<g, kThreads, 0, s>>>(out, bt, n, inner, outer, acc, sp); break;
    default: band_pass_kernel<T, 4><<<g, kThreads, 0, s>>>(out, bt, n, inner, outer, acc, sp); break;
  }
}

template <typename T>
void launch_interp_fwd(cudaStream_t s, T *out, const T *in, const T *tab, int nel, int p, int nq,
                       long long inner, long long outer) {
  long long total = outer * (long long)nel * nq * inner;
  Split3 sp(inner, (long long)nel * nq);
  int g = grid_for(total);
  st_count_launch();
  switch (p) {
    case 1: interp_fwd_kernel<T, 1><<<g, kThreads, 0, s>>>(out, in, tab, nel, inner, outer, sp); break;
    case 2: interp_fwd_kernel<T, 2><<<g, kThreads, 0, s>>>(out, in, tab, nel, inner, outer, sp); break;
    case 3: interp_fwd_kernel<T, 3><<<g, kThreads, 0, s>>>(out, in, tab, nel, inner, outer, sp); break;
    default: interp_fwd_kernel<T, 4><<<g, kThreads, 0, s>>>(out, in, tab, nel, inner, outer, sp); break;
  }
}

template <typename T>
void launch_interp_bwd(cudaStream_t s, T *out, const T *in, const T *tab, int nel, int p, int nq,
                       long long inner, long long outer, bool accumulate) {
  long long total = outer * (long long)(nel + p) * inner;
  Split3 sp(inner, nel + p);
  int acc = accumulate ? 1 : 0;
  int g = grid_for(total);
  st_count_launch();
  switch (p) {
    case 1: interp_bwd_kernel<T, 1><<<g, kThreads, 0, s>>>(out, in, tab, nel, inner, outer, acc, sp); break;
    case 2: interp_bwd_kernel<T, 2><<<g, kThreads, 0, s>>>(out, in, tab, nel, inner, outer, acc, sp); break;
    case 3: interp_bwd_kernel<T, 3><<<g, kThreads, 0, s>>>(out, in, tab, nel, inner, outer, acc, sp); break;
    default: interp_bwd_kernel<T, 4><<<g, kThreads, 0, s>>>(out, in, tab, nel, inner, outer, acc, sp); break;
  }
}

template <typename T>
void launch_qband_apply(cudaStream_t s, T *z, const T *x, const T *band, int Nt, long long Qs, int p) {
  int threads = 128;
  long long blocks = (Qs + threads - 1) / threads;
  switch (p) {
    case 1: st_count_launch(); qband_kernel<T, 1><<<(unsigned)blocks, threads, 0, s>>>(z, x, band, Nt, Qs); break;
    case 2: st_count_launch(); qband_kernel<T, 2><<<(unsigned)blocks, threads, 0, s>>>(z, x, band, Nt, Qs); break;
    case 3: st_count_launch(); qband_kernel<T, 3><<<(unsigned)blocks, threads, 0, s>>>(z, x, band, Nt, Qs); break;
    default: st_count_launch(); qband_kernel<T, 4><<<(unsigned)blocks, threads, 0, s>>>(z, x, band, Nt, Qs); break;
  }
}

template <typename T>
void launch_gemm(cudaStream_t s, T *C, const T *A, const T *X, const GemmDesc &g, double alpha, double beta) {
  dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, g.batch);
  st_count_launch(); gemm_kernel<T><<<grid, 256, 0, s>>>(C, A, X, g, (T)alpha, (T)beta);
}

// out[o][j][c] = sum_k A[j*n + k] in[o][k][c]
template <typename T>
void launch_mode_gemm(cudaStream_t s, T *out, const T *in, const T *A, int n, long long inner, long long outer) {
  GemmDesc g;
  if (inner == 1) {
    g.M = n; g.N = (int)outer; g.K = n; g.batch = 1;
    g.sam = n; g.sak = 1;
    g.sbb = 0; g.sbk = 1; g.sbc = n;
    g.scb = 0; g.scm = 1; g.scc = n;
    launch_gemm<T>(s, out, A, in, g, 1.0, 0.0);
  } else {
    g.M = n; g.N = (int)inner; g.K = n; g.batch = (int)outer;
    g.sam = n; g.sak = 1;
    g.sbb = (long long)n * inner; g.sbk = inner; g.sbc = 1;
    g.scb = (long long)n * inner; g.scm = inner; g.scc = 1;
    // gridDim.z is limited to 65535: split very large batches
    const int maxb = 65535;
    for (int b0 = 0; b0 < (int)outer; b0 += maxb) {
      GemmDesc gb = g;
      gb.batch = (int)std::min<long long>(maxb, outer - b0);
      launch_gemm<T>(s, out + (long long)b0 * g.scb, A, in + (long long)b0 * g.sbb, gb, 1.0, 0.0);
    }
  }
}

template <typename T>
void launch_tline_lu_solve(cudaStream_t s, T *z, const T *r, const T *lu, int Nt, long long Ns, int p) {
  int threads = 128;
  unsigned blocks = (unsigned)((Ns + threads - 1) / threads);
  switch (p) {
    case 1: st_count_launch(); tline_lu_kernel<T, 1><<<blocks, threads, 0, s>>>(z, r, lu, Nt, Ns); break;
    case 2: st_count_launch(); tline_lu_kernel<T, 2><<<blocks, threads, 0, s>>>(z, r, lu, Nt, Ns); break;
    case 3: st_count_launch(); tline_lu_kernel<T, 3><<<blocks, threads, 0, s>>>(z, r, lu, Nt, Ns); break;
    default: st_count_launch(); tline_lu_kernel<T, 4><<<blocks, threads, 0, s>>>(z, r, lu, Nt, Ns); break;
  }
}

template <typename T>
void launch_multi_dot(cudaStream_t s, double *out, const T *V, long long ldv, int nv, const T *w, long long n,
                      double *scratch) {
  constexpr int G = 8;
  int bx = (int)std::min<long long>(kDotBlocks, std::max<long long>(1, (n + 2047) / 2048));
  dim3 grid(bx, (nv + G - 1) / G);
  st_count_launch(); mdot_kernel<T, G><<<grid, 256, 0, s>>>(scratch, V, ldv, nv, w, n);
  st_count_launch(); reduce_blocks_kernel<<<(nv + 127) / 128, 128, 0, s>>>(out, scratch, bx, nv);
}

template <typename T>
void launch_multi_axpy(cudaStream_t s, T *w, const T *V, long long ldv, int nv, const double *h, long long n,
                       const double *nrm) {
  long long nvec = n / V16<T>::W;
  st_count_launch(); maxpy_kernel<T><<<grid_for(std::max<long long>(nvec, 1)), kThreads, 0, s>>>(w, V, ldv, nv, h, n, nrm);
}

template <typename T>
void launch_scale_copy(cudaStream_t s, T *y, const T *x, double alpha, long long n) {
  st_count_launch(); scale_copy_kernel<T><<<grid_for(n), kThreads, 0, s>>>(y, x, alpha, n);
}

void launch_axpby64(cudaStream_t s, double *y, const double *x, double a, double b, long long n) {
  st_count_launch(); axpby64_kernel<<<grid_for(n), kThreads, 0, s>>>(y, x, a, b, n);
}
void launch_sub64(cudaStream_t s, double *r, const double *b, const double *ax, long long n) {
  st_count_launch(); sub64_kernel<<<grid_for(n), kThreads, 0, s>>>(r, b, ax, n);
}
void launch_d2f(cudaStream_t s, float *y, const double *x, double scale, long long n) {
  st_count_launch(); d2f_kernel<<<grid_for(n), kThreads, 0, s>>>(y, x, scale, n);
}
void launch_f2d_axpy(cudaStream_t s, double *y, const float *x, double scale, long long n) {
  st_count_launch(); f2d_axpy_kernel<<<grid_for(n), kThreads, 0, s>>>(y, x, scale, n);
}
void launch_absmax64(cudaStream_t s, double *out, const double *x, const double *y, long long n, double *scratch) {
  int blocks = (int)std::min<long long>(kDotBlocks, std::max<long long>(1, (n + 1023) / 1024));
  st_count_launch(); absmax_kernel<<<blocks, 256, 0, s>>>(scratch, x, y, n);
  st_count_launch(); max_blocks_kernel<<<1, 32, 0, s>>>(out, scratch, blocks);
}
void launch_norm2_64(cudaStream_t s, double *out, const double *x, long long n, double *scratch) {
  launch_multi_dot<double>(s, out, x, n, 1, x, n, scratch);
}
void launch_band_to_f32(cudaStream_t s, float *out, const double *in, long long n) {
  st_count_launch(); to_f32_kernel<<<grid_for(n), kThreads, 0, s>>>(out, in, n);
}

void launch_gemm64(cudaStream_t s, double *C, const double *A, const double *X, int M, int N, int K,
                   long long sam, long long sak, long long sbk, long long sbc, long long scm, long long scc,
                   double alpha, double beta) {
  GemmDesc g;
  g.M = M; g.N = N; g.K = K; g.batch = 1;
  g.sam = sam; g.sak = sak; g.sbb = 0; g.sbk = sbk; g.sbc = sbc; g.scb = 0; g.scm = scm; g.scc = scc;
  launch_gemm<double>(s, C, A, X, g, alpha, beta);
}

#define INST(T)                                                                                        \
  template void launch_band_pass<T>(cudaStream_t, T *, int, const T *const *, const T *const *,       \
                                    const double *, int, long long, long long, int, bool);            \
  template void launch_interp_fwd<T>(cudaStream_t, T *, const T *, const T *, int, int, int, long long, \
                                     long long);                                                      \
  template void launch_interp_bwd<T>(cudaStream_t, T *, const T *, const T *, int, int, int, long long, \
                                     long long, bool);                                                \
  template void launch_qband_apply<T>(cudaStream_t, T *, const T *, const T *, int, long long, int);   \
  template void launch_mode_gemm<T>(cudaStream_t, T *, const T *, const T *, int, long long, long long); \
  template void launch_tline_lu_solve<T>(cudaStream_t, T *, const T *, const T *, int, long long, int); \
  template void launch_multi_dot<T>(cudaStream_t, double *, const T *, long long, int, const T *,      \
                                    long long, double *);                                             \
  template void launch_multi_axpy<T>(cudaStream_t, T *, const T *, long long, int, const double *,     \
                                     long long, const double *);                                      \
  template void launch_scale_copy<T>(cudaStream_t, T *, const T *, double, long long);
INST(float)
INST(double)
#undef INST
