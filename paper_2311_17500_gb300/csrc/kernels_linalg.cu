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
template <typename T>
__global__ void band_pass_kernel(T *__restrict__ out, BandTerms<T> bt, int n, long long inner,
                                 long long outer, int p, int accumulate) {
  const int B = 2 * p + 1;
  long long total = outer * n * inner;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long c = idx % inner;
    long long r = idx / inner;
    int i = (int)(r % n);
    long long o = r / n;
    T acc = accumulate ? out[idx] : T(0);
    int k0 = max(0, p - i), k1 = min(B - 1, n - 1 - i + p);
    for (int t = 0; t < bt.nterms; ++t) {
      const T *bd = bt.band[t] + (size_t)i * B;
      const T *src = bt.in[t] + (o * n + (i - p)) * inner + c;
      T s = T(0);
      for (int k = k0; k <= k1; ++k) s += __ldg(bd + k) * src[(long long)k * inner];
      acc += bt.coef[t] * s;
    }
    out[idx] = acc;
  }
}

// Coefficients -> Gauss points along one axis (sum factorization, Sec. 3.1):
// out[o][e*nq+q][c] = sum_a tab[e][q][a] in[o][e+a][c].
template <typename T>
__global__ void interp_fwd_kernel(T *__restrict__ out, const T *__restrict__ in, const T *__restrict__ tab,
                                  int nel, int p, int nq, long long inner, long long outer) {
  int nout = nel * nq, nin = nel + p;
  long long total = outer * nout * inner;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long c = idx % inner;
    long long r = idx / inner;
    int eq = (int)(r % nout);
    long long o = r / nout;
    int e = eq / nq;
    const T *tb = tab + (size_t)eq * (p + 1);
    const T *src = in + (o * nin + e) * inner + c;
    T s = T(0);
    for (int a = 0; a <= p; ++a) s += __ldg(tb + a) * src[(long long)a * inner];
    out[idx] = s;
  }
}

// Gauss points -> coefficients (transpose of interp_fwd):
// out[o][i][c] (+)= sum_{e=i-p..i} sum_q tab[e][q][i-e] in[o][e*nq+q][c].
template <typename T>
__global__ void interp_bwd_kernel(T *__restrict__ out, const T *__restrict__ in, const T *__restrict__ tab,
                                  int nel, int p, int nq, long long inner, long long outer, int accumulate) {
  int nin = nel * nq, nout = nel + p;
  long long total = outer * nout * inner;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long c = idx % inner;
    long long r = idx / inner;
    int i = (int)(r % nout);
    long long o = r / nout;
    T s = T(0);
    int e0 = max(0, i - p), e1 = min(nel - 1, i);
    for (int e = e0; e <= e1; ++e) {
      const T *src = in + (o * nin + (long long)e * nq) * inner + c;
      const T *tb = tab + (size_t)e * nq * (p + 1) + (i - e);
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
  T yw[P];
#pragma unroll
  for (int k = 0; k < P; ++k) yw[k] = T(0);
  for (int it = 0; it < Nt; ++it) {
    T s = r[(long long)it * Ns + j];
#pragma unroll
    for (int k = 1; k <= P; ++k)
      if (it - k >= 0) s -= lu[((long long)it * B + (P - k)) * Ns + j] * yw[P - k];
#pragma unroll
    for (int k = 0; k < P - 1; ++k) yw[k] = yw[k + 1];
    yw[P - 1] = s;
    z[(long long)it * Ns + j] = s;
  }
  T zw[P];
#pragma unroll
  for (int k = 0; k < P; ++k) zw[k] = T(0);
  for (int it = Nt - 1; it >= 0; --it) {
    T s = z[(long long)it * Ns + j];
#pragma unroll
    for (int k = 1; k <= P; ++k)
      if (it + k < Nt) s -= lu[((long long)it * B + (P + k)) * Ns + j] * zw[k - 1];
    s *= lu[((long long)it * B + P) * Ns + j];
#pragma unroll
    for (int k = P - 1; k > 0; --k) zw[k] = zw[k - 1];
    zw[0] = s;
    z[(long long)it * Ns + j] = s;
  }
}

template <typename T> struct Acc;
template <> struct Acc<float> { typedef float type; };
template <> struct Acc<double> { typedef double type; };

// Partial inner products <V_i, w> for i < nv: each thread accumulates its
// elements in the storage precision (FP32 for FP32 vectors: short chains of at
// most `per_thread` products), then the partial is widened to FP64 and reduced
// by warp shuffles and shared memory in a fixed order; scratch[block][i].
template <typename T>
__global__ void multi_dot_kernel(double *__restrict__ scratch, const T *__restrict__ V, long long ldv, int nv,
                                 const T *__restrict__ w, long long n) {
  __shared__ double red[32][8];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long chunk = (n + gridDim.x - 1) / gridDim.x;
  long long beg = (long long)blockIdx.x * chunk, end = min(n, beg + chunk);
  for (int i0 = 0; i0 < nv; i0 += 32) {
    int cnt = min(32, nv - i0);
    for (int ii = 0; ii < cnt; ++ii) {
      const T *v = V + (long long)(i0 + ii) * ldv;
      double tot = 0.0;
      typename Acc<T>::type s = 0;
      int c = 0;
      for (long long e = beg + threadIdx.x; e < end; e += blockDim.x) {
        s += v[e] * w[e];
        if (++c == 16) { tot += (double)s; s = 0; c = 0; }
      }
      tot += (double)s;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, off);
      if (lane == 0) red[ii][warp] = tot;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double t = 0.0;
      for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) t += red[threadIdx.x][wi];
      scratch[(long long)blockIdx.x * nv + i0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

__global__ void reduce_blocks_kernel(double *__restrict__ out, const double *__restrict__ scratch, int nblocks,
                                     int nv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  double t = 0.0;
  for (int b = 0; b < nblocks; ++b) t += scratch[(long long)b * nv + i];
  out[i] = t;
}

// w -= sum_i h_i V_i (classical Gram-Schmidt update).
template <typename T>
__global__ void multi_axpy_kernel(T *__restrict__ w, const T *__restrict__ V, long long ldv, int nv,
                                  const double *__restrict__ h, long long n) {
  __shared__ T hs[512];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = (T)h[i];
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    T s = T(0);
    for (int i = 0; i < nv; ++i) s += hs[i] * V[(long long)i * ldv + e];
    w[e] -= s;
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

constexpr int kDotBlocks = 304;

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
  st_count_launch(); band_pass_kernel<T><<<grid_for(total), kThreads, 0, s>>>(out, bt, n, inner, outer, p, accumulate ? 1 : 0);
}

template <typename T>
void launch_interp_fwd(cudaStream_t s, T *out, const T *in, const T *tab, int nel, int p, int nq,
                       long long inner, long long outer) {
  long long total = outer * (long long)nel * nq * inner;
  st_count_launch(); interp_fwd_kernel<T><<<grid_for(total), kThreads, 0, s>>>(out, in, tab, nel, p, nq, inner, outer);
}

template <typename T>
void launch_interp_bwd(cudaStream_t s, T *out, const T *in, const T *tab, int nel, int p, int nq,
                       long long inner, long long outer, bool accumulate) {
  long long total = outer * (long long)(nel + p) * inner;
  st_count_launch(); interp_bwd_kernel<T><<<grid_for(total), kThreads, 0, s>>>(out, in, tab, nel, p, nq, inner, outer,
                                                            accumulate ? 1 : 0);
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
  int blocks = (int)std::min<long long>(kDotBlocks, std::max<long long>(1, (n + 1023) / 1024));
  st_count_launch(); multi_dot_kernel<T><<<blocks, 256, 0, s>>>(scratch, V, ldv, nv, w, n);
  st_count_launch(); reduce_blocks_kernel<<<(nv + 127) / 128, 128, 0, s>>>(out, scratch, blocks, nv);
}

template <typename T>
void launch_multi_axpy(cudaStream_t s, T *w, const T *V, long long ldv, int nv, const double *h, long long n) {
  st_count_launch(); multi_axpy_kernel<T><<<grid_for(n), kThreads, 0, s>>>(w, V, ldv, nv, h, n);
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
                                     long long);                                                      \
  template void launch_scale_copy<T>(cudaStream_t, T *, const T *, double, long long);
INST(float)
INST(double)
#undef INST
