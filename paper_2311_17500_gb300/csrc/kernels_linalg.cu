// Tensor kernels of the operator, the preconditioner and the Krylov solver.
//
// Every vector of unknowns is a tensor [N_t][n_z][n_y][n_x] (x fastest, time
// slowest).  A one-axis operation sees it as [outer][n][inner]: `n` entries
// along the axis, `inner` contiguous entries after it, `outer` blocks before.
#include <algorithm>
#include "st_internal.h"
#include "dev_sync.cuh"
#include "df.cuh"
#include "pdl.cuh"

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

// Division-free variants of the three axis passes.  "rows" kernels serve the
// fastest axis (inner == 1): a thread per position along the axis, blockIdx.y
// over the outer index.  "cols" kernels serve the other axes: a thread per
// inner index c, blockIdx.y over the axis position, blockIdx.z over the outer
// index.  Outer indices beyond the grid limit are covered by a stride loop.
template <typename T, int P>
__global__ void band_rows_kernel(T *__restrict__ out, BandTerms<T> bt, int n, long long outer, int accumulate) {
  constexpr int B = 2 * P + 1;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k0 = max(0, P - i), k1 = min(B - 1, n - 1 - i + P);
  for (long long o = blockIdx.y; o < outer; o += gridDim.y) {
    long long idx = o * n + i;
    T acc = accumulate ? out[idx] : T(0);
    for (int t = 0; t < bt.nterms; ++t) {
      const T *bd = bt.band[t] + (size_t)i * B;
      const T *src = bt.in[t] + o * n + (i - P);
      T s = T(0);
      for (int k = k0; k <= k1; ++k) s += __ldg(bd + k) * src[k];
      acc += bt.coef[t] * s;
    }
    out[idx] = acc;
  }
}

template <typename T, int P>
__global__ void band_cols_kernel(T *__restrict__ out, BandTerms<T> bt, int n, long long inner, long long outer,
                                 int accumulate) {
  constexpr int B = 2 * P + 1;
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= inner) return;
  const int i = blockIdx.y;
  const int k0 = max(0, P - i), k1 = min(B - 1, n - 1 - i + P);
  for (long long o = blockIdx.z; o < outer; o += gridDim.z) {
    long long idx = (o * n + i) * inner + c;
    T acc = accumulate ? out[idx] : T(0);
    for (int t = 0; t < bt.nterms; ++t) {
      const T *bd = bt.band[t] + (size_t)i * B;
      const T *src = bt.in[t] + (o * n + (i - P)) * inner + c;
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

template <typename T, int P>
__global__ void ifwd_rows_kernel(T *__restrict__ out, const T *__restrict__ in, const T *__restrict__ tab, int nel,
                                 long long outer) {
  constexpr int nq = P + 1;
  const int nout = nel * nq, nin = nel + P;
  int eq = blockIdx.x * blockDim.x + threadIdx.x;
  if (eq >= nout) return;
  const int e = eq / nq;
  T tb[P + 1];
#pragma unroll
  for (int a = 0; a <= P; ++a) tb[a] = __ldg(tab + (size_t)eq * (P + 1) + a);
  for (long long o = blockIdx.y; o < outer; o += gridDim.y) {
    const T *src = in + o * nin + e;
    T s = T(0);
#pragma unroll
    for (int a = 0; a <= P; ++a) s += tb[a] * src[a];
    out[o * nout + eq] = s;
  }
}

template <typename T, int P>
__global__ void ifwd_cols_kernel(T *__restrict__ out, const T *__restrict__ in, const T *__restrict__ tab, int nel,
                                 long long inner, long long outer) {
  constexpr int nq = P + 1;
  const int nout = nel * nq, nin = nel + P;
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= inner) return;
  const int eq = blockIdx.y, e = eq / nq;
  T tb[P + 1];
#pragma unroll
  for (int a = 0; a <= P; ++a) tb[a] = __ldg(tab + (size_t)eq * (P + 1) + a);
  for (long long o = blockIdx.z; o < outer; o += gridDim.z) {
    const T *src = in + (o * nin + e) * inner + c;
    T s = T(0);
#pragma unroll
    for (int a = 0; a <= P; ++a) s += tb[a] * src[(long long)a * inner];
    out[(o * nout + eq) * inner + c] = s;
  }
}

template <typename T, int P>
__global__ void ibwd_rows_kernel(T *__restrict__ out, const T *__restrict__ in, const T *__restrict__ tab, int nel,
                                 long long outer, int accumulate) {
  constexpr int nq = P + 1;
  const int nin = nel * nq, nout = nel + P;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nout) return;
  for (long long o = blockIdx.y; o < outer; o += gridDim.y) {
    T s = T(0);
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      int e = i - a;
      if (e < 0 || e >= nel) continue;
      const T *src = in + o * nin + (long long)e * nq;
      const T *tb = tab + (size_t)e * nq * (P + 1) + a;
#pragma unroll
      for (int q = 0; q < nq; ++q) s += __ldg(tb + q * (P + 1)) * src[q];
    }
    long long idx = o * nout + i;
    out[idx] = accumulate ? out[idx] + s : s;
  }
}

template <typename T, int P>
__global__ void ibwd_cols_kernel(T *__restrict__ out, const T *__restrict__ in, const T *__restrict__ tab, int nel,
                                 long long inner, long long outer, int accumulate) {
  constexpr int nq = P + 1;
  const int nin = nel * nq, nout = nel + P;
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= inner) return;
  const int i = blockIdx.y;
  T tb[P + 1][P + 1];
#pragma unroll
  for (int a = 0; a <= P; ++a)
#pragma unroll
    for (int q = 0; q < nq; ++q) {
      int e = i - a;
      tb[a][q] = (e >= 0 && e < nel) ? __ldg(tab + ((size_t)e * nq + q) * (P + 1) + a) : T(0);
    }
  for (long long o = blockIdx.z; o < outer; o += gridDim.z) {
    T s = T(0);
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      int e = i - a;
      if (e < 0 || e >= nel) continue;
      const T *src = in + (o * nin + (long long)e * nq) * inner + c;
#pragma unroll
      for (int q = 0; q < nq; ++q) s += tb[a][q] * src[(long long)q * inner];
    }
    long long idx = (o * nout + i) * inner + c;
    out[idx] = accumulate ? out[idx] + s : s;
  }
}

// ---------------------------------------------------------------------------
// Shared-memory tiled axis passes.  All three one-axis operations have the
// form out[o][i][c] = sum_{j in window(i)} W(i, j) in[o][j][c] with a
// contiguous window: OP_BAND (banded 1D matrix, j in [i-P, i+P]), OP_FWD
// (coefficients -> Gauss points, i = e*nq+q, j in [e, e+P]) and OP_BWD (Gauss
// points -> coefficients, j over the Gauss points of spans i-P..i).  A block
// stages the input rows of its output tile in shared memory once (coalesced
// along c, or along the axis for the fastest axis), then every output reads
// its window from shared memory.
enum { OP_BAND = 0, OP_FWD = 1, OP_BWD = 2 };

template <int P, int OP>
struct AxisWin {
  static constexpr int nq = P + 1;
  // first input row needed by output row i (clamped later), and window length bound
  __device__ __forceinline__ static int lo(int i) {
    return OP == OP_BAND ? i - P : OP == OP_FWD ? i / nq : (i - P) * nq;
  }
  __device__ __forceinline__ static int hi(int i) {
    return OP == OP_BAND ? i + P : OP == OP_FWD ? i / nq + P : i * nq + nq - 1;
  }
  // weight of input row j for output row i (j inside the window)
  template <typename T>
  __device__ __forceinline__ static T w(const T *tab, int i, int j) {
    if (OP == OP_BAND) return __ldg(tab + (size_t)i * (2 * P + 1) + (j - i + P));
    if (OP == OP_FWD) return __ldg(tab + (size_t)i * (P + 1) + (j - i / nq));
    const int e = j / nq, q = j - e * nq;
    return __ldg(tab + ((size_t)e * nq + q) * (P + 1) + (i - e));
  }
};

template <typename T>
struct TiledTerms {
  const T *in[3];
  const T *tab[3];
  T coef[3];
  int nterms;
};

constexpr int kTileC = 32, kTileI = 32;

template <typename T, int P, int OP>
__global__ void __launch_bounds__(256) tiled_cols_kernel(T *__restrict__ out, TiledTerms<T> tt, int nin, int nout,
                                                         long long inner, long long outer, int accumulate) {
  extern __shared__ unsigned char smem_raw[];
  T *tile = reinterpret_cast<T *>(smem_raw);
  typedef AxisWin<P, OP> Win;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const long long c = (long long)blockIdx.x * kTileC + tx;
  const int i0 = blockIdx.y * kTileI;
  const int i1 = min(nout, i0 + kTileI);
  const int jlo = max(0, Win::lo(i0)), jhi = min(nin - 1, Win::hi(i1 - 1));
  const int rows = jhi - jlo + 1;
  for (long long o = blockIdx.z; o < outer; o += gridDim.z) {
    for (int t = 0; t < tt.nterms; ++t) {
      const T *src = tt.in[t] + (o * nin + jlo) * inner;
      T *dst = tile + (size_t)t * rows * kTileC;
      for (int r = ty; r < rows; r += 8) dst[r * kTileC + tx] = (c < inner) ? src[(long long)r * inner + c] : T(0);
    }
    __syncthreads();
    for (int i = i0 + ty; i < i1; i += 8) {
      const int a = max(jlo, Win::lo(i)), b = min(jhi, Win::hi(i));
      T acc = T(0);
      for (int t = 0; t < tt.nterms; ++t) {
        const T *tl = tile + (size_t)t * rows * kTileC;
        T s = T(0);
        for (int j = a; j <= b; ++j) s += Win::w(tt.tab[t], i, j) * tl[(j - jlo) * kTileC + tx];
        acc += tt.coef[t] * s;
      }
      if (c < inner) {
        long long idx = (o * nout + i) * inner + c;
        out[idx] = accumulate ? out[idx] + acc : acc;
      }
    }
    __syncthreads();
  }
}

template <typename T, int P, int OP>
__global__ void __launch_bounds__(256) tiled_rows_kernel(T *__restrict__ out, TiledTerms<T> tt, int nin, int nout,
                                                         long long outer, int rb, int accumulate) {
  extern __shared__ unsigned char smem_raw[];
  T *tile = reinterpret_cast<T *>(smem_raw);   // [term][rb][nin]
  typedef AxisWin<P, OP> Win;
  for (long long o0 = (long long)blockIdx.x * rb; o0 < outer; o0 += (long long)gridDim.x * rb) {
    const int nr = (int)min((long long)rb, outer - o0);
    for (int t = 0; t < tt.nterms; ++t) {
      const T *src = tt.in[t] + o0 * nin;
      T *dst = tile + (size_t)t * rb * nin;
      for (int k = threadIdx.x; k < nr * nin; k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nr * nout; k += blockDim.x) {
      const int r = k / nout, i = k - r * nout;
      const int a = max(0, Win::lo(i)), b = min(nin - 1, Win::hi(i));
      T acc = T(0);
      for (int t = 0; t < tt.nterms; ++t) {
        const T *tl = tile + ((size_t)t * rb + r) * nin;
        T s = T(0);
        for (int j = a; j <= b; ++j) s += Win::w(tt.tab[t], i, j) * tl[j];
        acc += tt.coef[t] * s;
      }
      long long idx = (o0 + r) * nout + i;
      out[idx] = accumulate ? out[idx] + acc : acc;
    }
    __syncthreads();
  }
}

// Streaming variants for the non-fastest axes (inner > 1): a thread owns one
// inner index c, one outer index o and a run of output rows along the axis,
// and slides a register window over the input rows it needs, so every input
// row of the run is loaded once (coalesced across c) and no barrier is used.
constexpr int kRun = 32;

template <typename T, int P>
__global__ void band_stream_kernel(T *__restrict__ out, TiledTerms<T> tt, int n, long long inner, long long outer,
                                   int nruns, int accumulate) {
  constexpr int B = 2 * P + 1, U = 8;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= inner) return;
  for (long long yr = blockIdx.y; yr < outer * nruns; yr += gridDim.y) {
    const long long o = yr / nruns;
    const int i0 = (int)(yr - o * nruns) * kRun, i1 = min(n, i0 + kRun);
    T w[3][B];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      if (t >= tt.nterms) break;
      const T *src = tt.in[t] + o * n * inner + c;
#pragma unroll
      for (int k = 0; k < B - 1; ++k) {
        int j = i0 - P + k;   // w[k+1] holds row i0-P+k before the first shift
        w[t][k + 1] = (j >= 0 && j < n) ? src[(long long)j * inner] : T(0);
      }
    }
    for (int ib = i0; ib < i1; ib += U) {
      // request the U next rows of every term before using them
      T nx[3][U];
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        if (t >= tt.nterms) break;
        const T *src = tt.in[t] + o * n * inner + c;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          int j = ib + u + P;
          nx[t][u] = (ib + u < i1 && j < n) ? src[(long long)j * inner] : T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = ib + u;
        if (i >= i1) break;
        T acc = accumulate ? out[(o * n + i) * inner + c] : T(0);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          if (t >= tt.nterms) break;
#pragma unroll
          for (int k = 0; k < B - 1; ++k) w[t][k] = w[t][k + 1];
          w[t][B - 1] = nx[t][u];
          const T *bd = tt.tab[t] + (size_t)i * B;
          T sacc = T(0);
#pragma unroll
          for (int k = 0; k < B; ++k) sacc += __ldg(bd + k) * w[t][k];
          acc += tt.coef[t] * sacc;
        }
        out[(o * n + i) * inner + c] = acc;
      }
    }
  }
}

// One row of an interpolation table (P+1 values) in shared memory, aligned so
// that rows of 2 or 4 values are read with one vector access.
template <typename T, int N>
struct __align__((N == 4 ? 4 : N == 2 ? 2 : 1) * sizeof(T)) TabRow {
  T v[N];
};

// Runs of elements per block of the strided interpolation passes (shorter
// runs give more independent blocks; every run rereads P neighbours).
constexpr int kRunFwd = 8, kRunBwd = 16;

// Coefficients -> Gauss points along a strided axis: thread = column c of
// one outer slice o, block = a run of elements.  The run's table rows are
// staged in shared memory; the coefficients of the next U elements are
// loaded before their outputs are formed.
template <typename T, int P>
__global__ void __launch_bounds__(256) ifwd_stream_kernel(T *__restrict__ out, const T *__restrict__ in,
                                                          const T *__restrict__ tab, int nel, long long inner,
                                                          long long outer, int nruns) {
  pdl_trigger();
  pdl_wait();   // inputs and outputs are shared with the previous kernel
  constexpr int nq = P + 1, U = 8, RUN = kRunFwd;
  __shared__ TabRow<T, P + 1> st[RUN * nq];
  const int nin = nel + P, nout = nel * nq;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long yr = blockIdx.y; yr < outer * nruns; yr += gridDim.y) {
    const long long o = yr / nruns;
    const int e0 = (int)(yr - o * nruns) * RUN, e1 = min(nel, e0 + RUN);
    __syncthreads();   // the previous run's rows are no longer read
    for (int i = threadIdx.x; i < (e1 - e0) * nq * (P + 1); i += blockDim.x)
      st[i / (P + 1)].v[i % (P + 1)] = __ldg(tab + (size_t)e0 * nq * (P + 1) + i);
    __syncthreads();
    if (c >= inner) continue;
    const T *src = in + o * nin * inner + c;
    T *dst = out + o * nout * inner + c;
    T w[P + 1];
#pragma unroll
    for (int a = 0; a < P; ++a) w[a + 1] = src[(long long)(e0 + a) * inner];
    for (int eb = e0; eb < e1; eb += U) {
      T nx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) nx[u] = (eb + u < e1) ? src[(long long)(eb + u + P) * inner] : T(0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = eb + u;
        if (e >= e1) break;
#pragma unroll
        for (int a = 0; a < P; ++a) w[a] = w[a + 1];
        w[P] = nx[u];
#pragma unroll
        for (int q = 0; q < nq; ++q) {
          const TabRow<T, P + 1> tb = st[(e - e0) * nq + q];
          T sacc = T(0);
#pragma unroll
          for (int a = 0; a <= P; ++a) sacc += tb.v[a] * w[a];
          dst[((long long)e * nq + q) * inner] = sacc;
        }
      }
    }
  }
}

// Gauss points -> coefficients along a strided axis (transpose of the pass
// above): thread = column c, block = a run of output coefficients; the
// elements touching the run are swept in batches of UE whose Gauss values
// (and, when accumulating, the old outputs) are loaded together.
template <typename T, int P>
__global__ void __launch_bounds__(256) ibwd_stream_kernel(T *__restrict__ out, const T *__restrict__ in,
                                                          const T *__restrict__ tab, int nel, long long inner,
                                                          long long outer, int nruns, int accumulate) {
  pdl_trigger();
  pdl_wait();   // inputs and outputs are shared with the previous kernel
  constexpr int nq = P + 1, UE = 4, RUN = kRunBwd;
  __shared__ TabRow<T, P + 1> st[(RUN + P) * nq];
  const int nin = nel * nq, nout = nel + P;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long yr = blockIdx.y; yr < outer * nruns; yr += gridDim.y) {
    const long long o = yr / nruns;
    const int i0 = (int)(yr - o * nruns) * RUN, i1 = min(nout, i0 + RUN);
    const int ea = max(0, i0 - P), eb = min(nel - 1, i1 - 1);
    __syncthreads();
    for (int i = threadIdx.x; i < (eb - ea + 1) * nq * (P + 1); i += blockDim.x)
      st[i / (P + 1)].v[i % (P + 1)] = __ldg(tab + (size_t)ea * nq * (P + 1) + i);
    __syncthreads();
    if (c >= inner) continue;
    const T *src = in + o * nin * inner + c;
    T *dst = out + o * nout * inner + c;
    T acc[P + 1];   // acc[a]: coefficient e + a while element e is processed
#pragma unroll
    for (int a = 0; a <= P; ++a) acc[a] = T(0);
    for (int e0 = ea; e0 <= eb; e0 += UE) {
      T z[UE][nq], yo[UE];
#pragma unroll
      for (int u = 0; u < UE; ++u) {
        const bool ok = e0 + u <= eb;
#pragma unroll
        for (int q = 0; q < nq; ++q) z[u][q] = ok ? src[((long long)(e0 + u) * nq + q) * inner] : T(0);
        yo[u] = (accumulate && ok && e0 + u >= i0) ? dst[(long long)(e0 + u) * inner] : T(0);
      }
#pragma unroll
      for (int u = 0; u < UE; ++u) {
        const int e = e0 + u;
        if (e > eb) break;
        TabRow<T, P + 1> r[nq];
#pragma unroll
        for (int q = 0; q < nq; ++q) r[q] = st[(e - ea) * nq + q];
#pragma unroll
        for (int a = 0; a <= P; ++a) {
          T sacc = T(0);
#pragma unroll
          for (int q = 0; q < nq; ++q) sacc += r[q].v[a] * z[u][q];
          acc[a] += sacc;
        }
        // coefficient e receives nothing from later elements
        if (e >= i0) dst[(long long)e * inner] = accumulate ? yo[u] + acc[0] : acc[0];
#pragma unroll
        for (int a = 0; a < P; ++a) acc[a] = acc[a + 1];
        acc[P] = T(0);
      }
    }
    // coefficients eb+1 .. i1-1 (only past the last element); acc[0] is eb+1
    for (int i = eb + 1; i < i1; ++i) {
      if (i >= i0) {
        long long idx = (long long)i * inner;
        T v = acc[0];
        dst[idx] = accumulate ? dst[idx] + v : v;
      }
#pragma unroll
      for (int a = 0; a < P; ++a) acc[a] = acc[a + 1];
      acc[P] = T(0);
    }
  }
}

// The two passes above for the FP64 operator on double-float pairs: input
// and (forward) output as (high, low) float pairs, arithmetic in double-float,
// so no FP64 instruction is spent per value.  The backward pass writes pairs,
// or FP64 (optionally accumulated) for the last axis.
__device__ __forceinline__ df ld_df(const float2 *p) { const float2 v = *p; return {v.x, v.y}; }
__device__ __forceinline__ df ld_df(const double *p) { return df_from(*p); }

template <int P>
__global__ void __launch_bounds__(256) ifwd_pairs_kernel(float2 *__restrict__ out, const float2 *__restrict__ in,
                                                         const float2 *__restrict__ tab, int nel, long long inner,
                                                         long long outer, int nruns) {
  pdl_trigger();
  pdl_wait();   // inputs and outputs are shared with the previous kernel
  constexpr int nq = P + 1, U = 8, RUN = kRunFwd;
  __shared__ TabRow<float2, P + 1> st[RUN * nq];
  const int nin = nel + P, nout = nel * nq;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long yr = blockIdx.y; yr < outer * nruns; yr += gridDim.y) {
    const long long o = yr / nruns;
    const int e0 = (int)(yr - o * nruns) * RUN, e1 = min(nel, e0 + RUN);
    __syncthreads();
    for (int i = threadIdx.x; i < (e1 - e0) * nq * (P + 1); i += blockDim.x)
      st[i / (P + 1)].v[i % (P + 1)] = __ldg(tab + (size_t)e0 * nq * (P + 1) + i);
    __syncthreads();
    if (c >= inner) continue;
    const float2 *src = in + o * nin * inner + c;
    float2 *dst = out + o * nout * inner + c;
    df w[P + 1];
#pragma unroll
    for (int a = 0; a < P; ++a) w[a + 1] = ld_df(src + (long long)(e0 + a) * inner);
    for (int eb = e0; eb < e1; eb += U) {
      df nx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) nx[u] = (eb + u < e1) ? ld_df(src + (long long)(eb + u + P) * inner) : df{0.f, 0.f};
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = eb + u;
        if (e >= e1) break;
#pragma unroll
        for (int a = 0; a < P; ++a) w[a] = w[a + 1];
        w[P] = nx[u];
#pragma unroll
        for (int q = 0; q < nq; ++q) {
          const TabRow<float2, P + 1> tb = st[(e - e0) * nq + q];
          df sacc = {0.f, 0.f};
#pragma unroll
          for (int a = 0; a <= P; ++a) sacc = df_fma(df{tb.v[a].x, tb.v[a].y}, w[a], sacc);
          dst[((long long)e * nq + q) * inner] = make_float2(sacc.hi, sacc.lo);
        }
      }
    }
  }
}

template <int P, typename TO>
__global__ void __launch_bounds__(256) ibwd_pairs_kernel(TO *__restrict__ out, const float2 *__restrict__ in,
                                                         const float2 *__restrict__ tab, int nel, long long inner,
                                                         long long outer, int nruns, int accumulate) {
  pdl_trigger();
  pdl_wait();   // inputs and outputs are shared with the previous kernel
  constexpr int nq = P + 1, UE = 4, RUN = kRunBwd;
  __shared__ TabRow<float2, P + 1> st[(RUN + P) * nq];
  const int nin = nel * nq, nout = nel + P;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const df zero = {0.f, 0.f};
  for (long long yr = blockIdx.y; yr < outer * nruns; yr += gridDim.y) {
    const long long o = yr / nruns;
    const int i0 = (int)(yr - o * nruns) * RUN, i1 = min(nout, i0 + RUN);
    const int ea = max(0, i0 - P), eb = min(nel - 1, i1 - 1);
    __syncthreads();
    for (int i = threadIdx.x; i < (eb - ea + 1) * nq * (P + 1); i += blockDim.x)
      st[i / (P + 1)].v[i % (P + 1)] = __ldg(tab + (size_t)ea * nq * (P + 1) + i);
    __syncthreads();
    if (c >= inner) continue;
    const float2 *src = in + o * nin * inner + c;
    TO *dst = out + o * nout * inner + c;
    df acc[P + 1];   // acc[a]: coefficient e + a while element e is processed
#pragma unroll
    for (int a = 0; a <= P; ++a) acc[a] = zero;
    for (int e0 = ea; e0 <= eb; e0 += UE) {
      df z[UE][nq], yo[UE];
#pragma unroll
      for (int u = 0; u < UE; ++u) {
        const bool ok = e0 + u <= eb;
#pragma unroll
        for (int q = 0; q < nq; ++q) z[u][q] = ok ? ld_df(src + ((long long)(e0 + u) * nq + q) * inner) : zero;
        yo[u] = (accumulate && ok && e0 + u >= i0) ? ld_df(dst + (long long)(e0 + u) * inner) : zero;
      }
#pragma unroll
      for (int u = 0; u < UE; ++u) {
        const int e = e0 + u;
        if (e > eb) break;
        TabRow<float2, P + 1> r[nq];
#pragma unroll
        for (int q = 0; q < nq; ++q) r[q] = st[(e - ea) * nq + q];
#pragma unroll
        for (int a = 0; a <= P; ++a) {
          df sacc = zero;
#pragma unroll
          for (int q = 0; q < nq; ++q) sacc = df_fma(df{r[q].v[a].x, r[q].v[a].y}, z[u][q], sacc);
          acc[a] = df_add(acc[a], sacc);
        }
        // coefficient e receives nothing from later elements
        if (e >= i0) ct_store(dst + (long long)e * inner, accumulate ? df_add(yo[u], acc[0]) : acc[0]);
#pragma unroll
        for (int a = 0; a < P; ++a) acc[a] = acc[a + 1];
        acc[P] = zero;
      }
    }
    // coefficients eb+1 .. i1-1 (only past the last element); acc[0] is eb+1
    for (int i = eb + 1; i < i1; ++i) {
      if (i >= i0) {
        TO *p = dst + (long long)i * inner;
        ct_store(p, accumulate ? df_add(ld_df(p), acc[0]) : acc[0]);
      }
#pragma unroll
      for (int a = 0; a < P; ++a) acc[a] = acc[a + 1];
      acc[P] = zero;
    }
  }
}

// Fastest-axis passes: a block stages rb whole rows in shared memory
// (coalesced), and each thread keeps the weights of its output positions in
// registers across the rows of the block.
template <typename T, int P>
__global__ void __launch_bounds__(256) band_rows2_kernel(T *__restrict__ out, const T *__restrict__ in,
                                                         const T *__restrict__ band, T coef, int n, long long outer,
                                                         int rb, int accumulate) {
  extern __shared__ unsigned char smem_raw[];
  T *tile = reinterpret_cast<T *>(smem_raw);
  constexpr int B = 2 * P + 1;
  for (long long o0 = (long long)blockIdx.x * rb; o0 < outer; o0 += (long long)gridDim.x * rb) {
    const int nr = (int)min((long long)rb, outer - o0);
    for (int k = threadIdx.x; k < nr * n; k += blockDim.x) tile[k] = in[o0 * n + k];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      T wv[B];
#pragma unroll
      for (int k = 0; k < B; ++k) {
        int j = i - P + k;
        wv[k] = (j >= 0 && j < n) ? coef * __ldg(band + (size_t)i * B + k) : T(0);
      }
      for (int r = 0; r < nr; ++r) {
        const T *tl = tile + r * n;
        T sacc = T(0);
#pragma unroll
        for (int k = 0; k < B; ++k) {
          int j = i - P + k;
          if (j >= 0 && j < n) sacc += wv[k] * tl[j];
        }
        long long idx = (o0 + r) * n + i;
        out[idx] = accumulate ? out[idx] + sacc : sacc;
      }
    }
    __syncthreads();
  }
}

template <typename T, int P>
__global__ void __launch_bounds__(256) ifwd_rows2_kernel(T *__restrict__ out, const T *__restrict__ in,
                                                         const T *__restrict__ tab, int nel, long long outer, int rb) {
  extern __shared__ unsigned char smem_raw[];
  T *tile = reinterpret_cast<T *>(smem_raw);
  constexpr int nq = P + 1;
  const int nin = nel + P, nout = nel * nq;
  for (long long o0 = (long long)blockIdx.x * rb; o0 < outer; o0 += (long long)gridDim.x * rb) {
    const int nr = (int)min((long long)rb, outer - o0);
    for (int k = threadIdx.x; k < nr * nin; k += blockDim.x) tile[k] = in[o0 * nin + k];
    __syncthreads();
    for (int eq = threadIdx.x; eq < nout; eq += blockDim.x) {
      const int e = eq / nq;
      T wv[P + 1];
#pragma unroll
      for (int a = 0; a <= P; ++a) wv[a] = __ldg(tab + (size_t)eq * (P + 1) + a);
      for (int r = 0; r < nr; ++r) {
        const T *tl = tile + r * nin + e;
        T sacc = T(0);
#pragma unroll
        for (int a = 0; a <= P; ++a) sacc += wv[a] * tl[a];
        out[(o0 + r) * nout + eq] = sacc;
      }
    }
    __syncthreads();
  }
}

template <typename T, int P>
__global__ void __launch_bounds__(256) ibwd_rows2_kernel(T *__restrict__ out, const T *__restrict__ in,
                                                         const T *__restrict__ tab, int nel, long long outer, int rb,
                                                         int accumulate) {
  extern __shared__ unsigned char smem_raw[];
  T *tile = reinterpret_cast<T *>(smem_raw);
  constexpr int nq = P + 1;
  const int nin = nel * nq, nout = nel + P;
  for (long long o0 = (long long)blockIdx.x * rb; o0 < outer; o0 += (long long)gridDim.x * rb) {
    const int nr = (int)min((long long)rb, outer - o0);
    for (int k = threadIdx.x; k < nr * nin; k += blockDim.x) tile[k] = in[o0 * nin + k];
    __syncthreads();
    for (int i = threadIdx.x; i < nout; i += blockDim.x) {
      T wv[P + 1][nq];
#pragma unroll
      for (int a = 0; a <= P; ++a)
#pragma unroll
        for (int q = 0; q < nq; ++q) {
          int e = i - a;
          wv[a][q] = (e >= 0 && e < nel) ? __ldg(tab + ((size_t)e * nq + q) * (P + 1) + a) : T(0);
        }
      for (int r = 0; r < nr; ++r) {
        const T *tl = tile + r * nin;
        T sacc = T(0);
#pragma unroll
        for (int a = 0; a <= P; ++a) {
          int e = i - a;
          if (e < 0 || e >= nel) continue;
#pragma unroll
          for (int q = 0; q < nq; ++q) sacc += wv[a][q] * tl[e * nq + q];
        }
        long long idx = (o0 + r) * nout + i;
        out[idx] = accumulate ? out[idx] + sacc : sacc;
      }
    }
    __syncthreads();
  }
}

template <typename T, int P, int OP>
void launch_tiled(cudaStream_t s, T *out, const TiledTerms<T> &tt, int nin, int nout, long long inner,
                  long long outer, bool accumulate) {
  int acc = accumulate ? 1 : 0;
  st_count_launch();
  if (inner == 1) {
    // whole rows in shared memory, at most 40 KB per block
    int rb = (int)std::max<long long>(1, std::min<long long>(32, 40960 / ((long long)tt.nterms * sizeof(T) * std::max(nin, 1))));
    size_t sh = (size_t)tt.nterms * rb * nin * sizeof(T);
    long long blocks = std::min<long long>((outer + rb - 1) / rb, 152LL * 16);
    if (tt.nterms == 1 && OP == OP_BAND) {
      band_rows2_kernel<T, P><<<(unsigned)blocks, 256, sh, s>>>(out, tt.in[0], tt.tab[0], tt.coef[0], nin, outer, rb, acc);
    } else if (OP == OP_FWD) {
      ifwd_rows2_kernel<T, P><<<(unsigned)blocks, 256, sh, s>>>(out, tt.in[0], tt.tab[0], nin - P, outer, rb);
    } else if (OP == OP_BWD) {
      ibwd_rows2_kernel<T, P><<<(unsigned)blocks, 256, sh, s>>>(out, tt.in[0], tt.tab[0], nout - P, outer, rb, acc);
    } else {
      tiled_rows_kernel<T, P, OP><<<(unsigned)blocks, 256, sh, s>>>(out, tt, nin, nout, outer, rb, acc);
    }
  } else {
    int bx = (int)std::min<long long>(256, (inner + 31) / 32 * 32);
    long long gx = (inner + bx - 1) / bx;
    int nruns = OP == OP_FWD ? (nin - P + kRunFwd - 1) / kRunFwd
                : OP == OP_BWD ? (nout + kRunBwd - 1) / kRunBwd : (nout + kRun - 1) / kRun;
    long long gy = std::min<long long>(outer * nruns, 65535);
    dim3 grid((unsigned)gx, (unsigned)gy);
    if (OP == OP_BAND)
      band_stream_kernel<T, P><<<grid, bx, 0, s>>>(out, tt, nout, inner, outer, nruns, acc);
    else if (OP == OP_FWD)
      pdl_launch(ifwd_stream_kernel<T, P>, grid, dim3(bx), 0, s, out, tt.in[0], tt.tab[0], nin - P, inner, outer, nruns);
    else
      pdl_launch(ibwd_stream_kernel<T, P>, grid, dim3(bx), 0, s, out, tt.in[0], tt.tab[0], nout - P, inner, outer, nruns, acc);
  }
}

template <typename T, int OP>
void launch_tiled_p(cudaStream_t s, int p, T *out, const TiledTerms<T> &tt, int nin, int nout, long long inner,
                    long long outer, bool accumulate) {
  switch (p) {
    case 1: launch_tiled<T, 1, OP>(s, out, tt, nin, nout, inner, outer, accumulate); break;
    case 2: launch_tiled<T, 2, OP>(s, out, tt, nin, nout, inner, outer, accumulate); break;
    case 3: launch_tiled<T, 3, OP>(s, out, tt, nin, nout, inner, outer, accumulate); break;
    default: launch_tiled<T, 4, OP>(s, out, tt, nin, nout, inner, outer, accumulate); break;
  }
}

// Per spatial Gauss point q, the symmetric time band of the reaction and SU
// terms: z[it][q] = sum_{k=-P..P} band(it, it+k; q) x[it+k][q], band stored as
// the upper half [k][it][q] (entry (it, it+k)), k = 0..P.  One thread sweeps
// the whole time line of a column; the window of x and band rows lives in
// registers, so every band entry and x value is read once.
template <typename T, int P>
__global__ void qband_kernel(T *__restrict__ z, const T *__restrict__ x, const float *__restrict__ bhi,
                             const float *__restrict__ blo, int Nt, long long Qs) {
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
    for (int k = 0; k <= P; ++k) {
      const long long bi = k * plane + (long long)it * Qs + q;
      b[k] = sizeof(T) == 8 ? (T)((double)bhi[bi] + (double)blo[bi]) : (T)bhi[bi];
    }
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

// Per-thread asynchronous copies (cp.async, 4 or 8 bytes) into shared memory.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// nq consecutive values into shared memory with 16-byte copies where the
// size allows (addresses aligned as for load_nq), else element by element.
template <typename T, int NQ>
__device__ __forceinline__ void cp_async_nq(T *smem, const T *gmem) {
  constexpr int bytes = NQ * (int)sizeof(T);
  if constexpr (bytes % 16 == 0) {
#pragma unroll
    for (int c = 0; c < bytes / 16; ++c) {
      unsigned sa = (unsigned)__cvta_generic_to_shared(reinterpret_cast<char *>(smem) + 16 * c);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(reinterpret_cast<const char *>(gmem) + 16 * c)
                   : "memory");
    }
  } else if constexpr (bytes == 8) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
  } else {
#pragma unroll
    for (int g = 0; g < NQ; ++g) cp_async_elem(smem + g, gmem + g);
  }
}

// nq consecutive band values of one element (vector loads where aligned:
// nq = 4 floats or doubles start on a 16-byte boundary, nq = 2 on 8 bytes).
template <typename T, int NQ>
__device__ __forceinline__ void load_nq(T (&v)[NQ], const T *p) {
  if constexpr (NQ == 4 && sizeof(T) == 4) {
    float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else if constexpr (NQ == 4 && sizeof(T) == 8) {
    double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  } else if constexpr (NQ == 2 && sizeof(T) == 4) {
    float2 a = __ldg(reinterpret_cast<const float2 *>(p));
    v[0] = a.x; v[1] = a.y;
  } else {
#pragma unroll
    for (int g = 0; g < NQ; ++g) v[g] = __ldg(p + g);
  }
}

// nq consecutive values from shared memory (16-byte aligned slots).
template <typename T, int NQ>
__device__ __forceinline__ void load_nq_shared(T (&v)[NQ], const T *p) {
  if constexpr (NQ == 4 && sizeof(T) == 4) {
    float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else {
#pragma unroll
    for (int g = 0; g < NQ; ++g) v[g] = p[g];
  }
}

// Reaction + SU part of the operator (the M_R and S-tilde terms of Sec. 3.1.1,
// both folded into one symmetric time band per spatial Gauss point), fused
// along the fastest spatial axis:  Y1 = Bx^T (band) Bx X1  for every row o of
// the other axes (already at their Gauss points) and every time step.
//   X1, Y1 : [Nt][rows][nx]        x-coefficients of each Gauss row
//   band   : [k][Nt][rows][Qx]     band[k][it] = T(it, it+k), k = 0..P, as
//                                   double-float pairs (bhi, blo)
//   tab    : [ex][g][a]            local basis a at Gauss point g of element ex
// The FP32 instance reads bhi and computes in float; the FP64 instance reads
// both parts and computes in double-float (FP64 accuracy on the FP32 pipe).
// One block per (row, time segment), one thread per x element (its nq Gauss
// points) plus P threads for the trailing coefficients (at most 512 threads,
// 256 for FP64 or p = 4 so that the window stays in registers).  The block
// sweeps its segment with a register window x(it..it+P) per Gauss point and
// scatters the lower-triangle terms band[k][it] x(it) into accumulators of
// the steps it+k; a segment first replays the P steps before it (band and x,
// no output) to rebuild those accumulators, so every output is complete and
// each band entry is read once plus a halo of P(P+1)/2 rows per segment.
// Operands stream through an S-step ring in shared memory filled by cp.async
// S-1 steps ahead: each thread copies its element's band values and its own
// x coefficient of row it+P.  One barrier per step publishes the coefficient
// row and the cross-warp partial sums of the previous step: the projection
// onto coefficient ex+a collects the contributions of elements ex-a..ex by
// warp shuffles, and across warps through shared memory, in a fixed order.
template <typename T, int P>
constexpr int xband_max_threads() { return (sizeof(T) == 8 || P >= 4) ? 256 : 512; }

constexpr long long kXbWaitLimit = 1ll << 22;

template <typename T> struct XbandCT { typedef float type; };
template <> struct XbandCT<double> { typedef df type; };
template <> struct XbandCT<float2> { typedef df type; };   // double-float pairs in and out

template <typename T, int P>
constexpr int xband_min_blocks() { return (sizeof(T) == 8 && P <= 3) ? 2 : 1; }

template <typename T, int P, int S, bool BULK>
__global__ void __launch_bounds__(xband_max_threads<T, P>(), xband_min_blocks<T, P>()) xband_fused_kernel(
    T *__restrict__ Y1, const T *__restrict__ X1, const float *__restrict__ bhi, const float *__restrict__ blo,
    const T *__restrict__ tab, int nel, int Nt, long long rows, int seglen, int *err) {
  typedef typename XbandCT<T>::type CT;
  constexpr bool DF = sizeof(T) == 8;
  constexpr int nq = P + 1, NB = DF ? 2 : 1;   // band parts per value
  static_assert(S >= 2, "ring depth");
  __shared__ CT xch[2][16][P][P];   // [step parity][warp][a-1][lane-(32-P)]
  // BULK: the band slice of a step (Qx contiguous values per diagonal and
  // part) arrives by bulk copies issued by thread 0 on bfull[slot]
  __shared__ __align__(8) uint64_t bfull[S];
  __shared__ int bfail;
  extern __shared__ __align__(16) unsigned char xb_raw[];
  const int nth = blockDim.x;
  float *bring = reinterpret_cast<float *>(xb_raw);                  // [S][NB][P+1][thread][nq]
  T *xring = reinterpret_cast<T *>(bring + (size_t)S * NB * (P + 1) * nth * nq);   // [S][thread]
  const int nx = nel + P, Qx = nel * nq;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool owns = t < nel;
  const CT zero = ct_zero<CT>();
  CT wv[nq][P + 1];
#pragma unroll
  for (int g = 0; g < nq; ++g)
#pragma unroll
    for (int a = 0; a <= P; ++a) wv[g][a] = owns ? ct_from<CT>(__ldg(tab + ((size_t)t * nq + g) * (P + 1) + a)) : zero;
  const long long planeX = rows * nx, planeQ = rows * Qx, bandK = (long long)Nt * planeQ;
  const int nseg = (Nt + seglen - 1) / seglen;
  if (BULK) {
    if (t == 0) {
      for (int i = 0; i < S; ++i) mbar_init(&bfull[i], 1);
      mbar_fence_init();
      bfail = 0;
    }
    __syncthreads();
  }
  pdl_trigger();
  pdl_wait();   // the table and barriers above are set up before the previous kernel ends
  long long gbase = 0;   // steps issued by this block before the current segment
  for (long long blk = blockIdx.x; blk < rows * nseg; blk += gridDim.x) {
    const long long o = blk % rows;
    const int t0 = (int)(blk / rows) * seglen, t1 = min(Nt, t0 + seglen);
    const T *xrow = X1 + o * nx + t;
    const long long boff = o * Qx + (long long)t * nq;
    T *yrow = Y1 + o * nx;
    auto gauss = [&](const CT (&c)[P + 1], CT (&xq)[nq]) {
#pragma unroll
      for (int g = 0; g < nq; ++g) {
        CT v = zero;
#pragma unroll
        for (int a = 0; a <= P; ++a) v = ct_fma(wv[g][a], c[a], v);
        xq[g] = v;
      }
    };
    auto interp_global = [&](int it, CT (&xq)[nq]) {
      CT c[P + 1];
#pragma unroll
      for (int a = 0; a <= P; ++a)
        c[a] = (owns && it >= 0 && it < Nt) ? ct_from<CT>(xrow[(long long)it * planeX + a]) : zero;
      gauss(c, xq);
    };
    auto band_global = [&](long long idx, CT (&v)[nq]) {
      float h[nq];
      load_nq<float, nq>(h, bhi + idx);
      if constexpr (DF) {
        float l[nq];
        load_nq<float, nq>(l, blo + idx);
#pragma unroll
        for (int g = 0; g < nq; ++g) v[g] = CT{h[g], l[g]};
      } else {
#pragma unroll
        for (int g = 0; g < nq; ++g) v[g] = ct_from<CT>(h[g]);
      }
    };
    CT acc[P][nq];      // lower-triangle terms owed to steps it .. it+P-1
#pragma unroll
    for (int k = 0; k < P; ++k)
#pragma unroll
      for (int g = 0; g < nq; ++g) acc[k][g] = zero;
    // replay steps t0-P .. t0-1: band[k][it'] x(it') owed to t0 + m, m = it'+k-t0
#pragma unroll
    for (int r = P; r >= 1; --r) {
      const int itp = t0 - r;
      if (itp < 0 || !owns) continue;
      CT xp[nq];
      interp_global(itp, xp);
#pragma unroll
      for (int k = 1; k <= P; ++k) {
        const int m = k - r;
        if (m < 0) continue;
        CT bv[nq];
        band_global(boff + k * bandK + (long long)itp * planeQ, bv);
#pragma unroll
        for (int g = 0; g < nq; ++g) acc[m][g] = ct_fma(bv[g], xp[g], acc[m][g]);
      }
    }
    CT xw[P + 1][nq];   // x(it + k) at the element's Gauss points
#pragma unroll
    for (int k = 0; k < P; ++k) interp_global(t0 + k, xw[k + 1]);
    // step u needs band row u and coefficient row u + P
    auto bslot = [&](int u, int part, int k) -> float * {
      return bring + ((size_t)(((u % S) * NB + part) * (P + 1) + k) * nth + t) * nq;
    };
    auto xslot = [&](int u) -> T * { return xring + (size_t)(u % S) * nth; };
    auto issue = [&](int u) {
      if (u < t1) {
        if constexpr (BULK) {
          if (t == 0) {
            const long long g = gbase + (u - t0);
            uint64_t *bar = &bfull[g % S];
            const uint32_t bytes = (uint32_t)Qx * sizeof(float);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                         "r"(bytes * NB * (P + 1))
                         : "memory");
#pragma unroll
            for (int part = 0; part < NB; ++part)
#pragma unroll
              for (int k = 0; k <= P; ++k) {
                const float *src = (part ? blo : bhi) + o * Qx + k * bandK + (long long)u * planeQ;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(bring + (size_t)((((u % S) * NB + part) * (P + 1) + k) * nth) * nq)),
                    "l"(src), "r"(bytes), "r"(smem_u32(bar))
                    : "memory");
              }
          }
        } else if (owns) {
#pragma unroll
          for (int k = 0; k <= P; ++k) {
            const long long idx = boff + k * bandK + (long long)u * planeQ;
            cp_async_nq<float, nq>(bslot(u, 0, k), bhi + idx);
            if constexpr (DF) cp_async_nq<float, nq>(bslot(u, 1, k), blo + idx);
          }
        }
        if (t < nx && u + P < Nt) cp_async_elem(xslot(u) + t, X1 + (long long)(u + P) * planeX + o * nx + t);
      }
      cp_async_commit();
    };
#pragma unroll
    for (int u = 0; u < S - 1; ++u) issue(t0 + u);
    CT pend = zero;   // this thread's output of the previous step, before its cross-warp part
    for (int it = t0; it < t1; ++it) {
      cp_async_wait<S - 2>();
      if constexpr (BULK) {
        const long long g = gbase + (it - t0);
        if (!mbar_wait(smem_u32(&bfull[g % S]), (uint32_t)((g / S) & 1), kXbWaitLimit)) {
          bfail = 1;
          atomicExch(err, 1);
        }
      }
      __syncthreads();
      if (BULK && bfail) break;
      if (it > t0) {
        const int pp = (it - 1) & 1;
        if (lane < P && warp > 0) {
#pragma unroll
          for (int a = 1; a <= P; ++a)
            if (a > lane) pend = ct_add(pend, xch[pp][warp - 1][a - 1][lane + P - a]);
        }
        if (t < nx) ct_store(yrow + (long long)(it - 1) * planeX + t, pend);
      }
      issue(it + S - 1);
      CT b[P + 1][nq];
#pragma unroll
      for (int k = 0; k <= P; ++k) {
        if (owns) {
          float h[nq];
          load_nq_shared<float, nq>(h, bslot(it, 0, k));
          if constexpr (DF) {
            float l[nq];
            load_nq_shared<float, nq>(l, bslot(it, 1, k));
#pragma unroll
            for (int g = 0; g < nq; ++g) b[k][g] = CT{h[g], l[g]};
          } else {
#pragma unroll
            for (int g = 0; g < nq; ++g) b[k][g] = ct_from<CT>(h[g]);
          }
        } else {
#pragma unroll
          for (int g = 0; g < nq; ++g) b[k][g] = zero;
        }
      }
#pragma unroll
      for (int k = 0; k < P; ++k)
#pragma unroll
        for (int g = 0; g < nq; ++g) xw[k][g] = xw[k + 1][g];
      {
        CT c[P + 1];
        const T *xs = xslot(it);
        const bool ok = it + P < Nt;
        if constexpr (DF) {
          // each coefficient converted once: by its own thread, then shuffled
          // down to the elements that use it (across the warp edge, read again)
          const CT mine = (ok && t < nx) ? ct_from<CT>(xs[t]) : zero;
          c[0] = owns ? mine : zero;
#pragma unroll
          for (int a = 1; a <= P; ++a) {
            CT v = ct_shfl_down(mine, a);
            if (lane + a >= 32) v = (ok && t + a < nx) ? ct_from<CT>(xs[t + a]) : zero;
            c[a] = owns ? v : zero;
          }
        } else {
#pragma unroll
          for (int a = 0; a <= P; ++a) c[a] = (owns && ok) ? ct_from<CT>(xs[t + a]) : zero;
        }
        gauss(c, xw[P]);
      }
      CT yq[nq];
#pragma unroll
      for (int g = 0; g < nq; ++g) {
        CT v = ct_fma(b[0][g], xw[0][g], acc[0][g]);
#pragma unroll
        for (int k = 1; k <= P; ++k) v = ct_fma(b[k][g], xw[k][g], v);
        yq[g] = v;
      }
#pragma unroll
      for (int k = 0; k < P - 1; ++k)
#pragma unroll
        for (int g = 0; g < nq; ++g) acc[k][g] = ct_fma(b[k + 1][g], xw[0][g], acc[k + 1][g]);
#pragma unroll
      for (int g = 0; g < nq; ++g) acc[P - 1][g] = ct_fma(b[P][g], xw[0][g], zero);
      // contributions c[a] of this element to coefficient t + a
      CT c[P + 1];
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        CT v = zero;
#pragma unroll
        for (int g = 0; g < nq; ++g) v = ct_fma(wv[g][a], yq[g], v);
        c[a] = v;
      }
      CT out = c[0];
#pragma unroll
      for (int a = 1; a <= P; ++a) {
        CT v = ct_shfl_up(c[a], a);
        if (lane >= a) out = ct_add(out, v);
      }
      if (lane >= 32 - P) {
#pragma unroll
        for (int a = 1; a <= P; ++a) xch[it & 1][warp][a - 1][lane - (32 - P)] = c[a];
      }
      pend = out;
    }
    cp_async_wait<0>();
    __syncthreads();
    if (BULK && bfail) break;
    gbase += t1 - t0;
    if (t1 > t0) {
      const int pp = (t1 - 1) & 1;
      if (lane < P && warp > 0) {
#pragma unroll
        for (int a = 1; a <= P; ++a)
          if (a > lane) pend = ct_add(pend, xch[pp][warp - 1][a - 1][lane + P - a]);
      }
      if (t < nx) ct_store(yrow + (long long)(t1 - 1) * planeX + t, pend);
    }
    __syncthreads();   // the next segment reuses the rings and xch
  }
}

// Two values combined by one paired multiply-add: (a.x b.x + c.x, a.y b.y + c.y).
// FP32 pairs issue as one packed instruction (two FMAs per issue slot); FP64
// pairs are two scalar FMAs.
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
// FP64 pairs are computed in double-float arithmetic (GB300's FP64 rate is
// 1/64 of FP32): a pair of double-float values and two df multiply-adds.
struct df2 {
  df x, y;
};
__device__ __forceinline__ df2 pfma(df2 a, df2 b, df2 c) { return {df_fma(a.x, b.x, c.x), df_fma(a.y, b.y, c.y)}; }

// Pair<T>: the pair type of the Kronecker kernel, its compute type ct and
// the conversions and scalar operations in ct.
template <typename T> struct Pair;
template <> struct Pair<float> {
  typedef float2 type;
  typedef float ct;
  typedef float src;   // x as read by the Kronecker kernel
  static __device__ __forceinline__ float load(float v) { return v; }
  static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ float from(float v) { return v; }
  static __device__ __forceinline__ float to(float v) { return v; }
  static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
};
template <> struct Pair<double> {
  typedef df2 type;
  typedef df ct;
  typedef float2 src;   // x pre-split into double-float pairs (no FP64 work per read)
  static __device__ __forceinline__ df load(float2 v) { return {v.x, v.y}; }
  static __device__ __forceinline__ df2 make(df a, df b) { return {a, b}; }
  static __device__ __forceinline__ df from(double v) { return df_from(v); }
  static __device__ __forceinline__ double to(df v) { return df_to(v); }
  static __device__ __forceinline__ df mul(df a, df b) { return df_mul(a, b); }
  static __device__ __forceinline__ df fma(df a, df b, df c) { return df_fma(a, b, c); }
  static __device__ __forceinline__ df add(df a, df b) { return df_add(a, b); }
};

// Kronecker part of the operator for d = 2 (Sec. 3.1.1),
//   y = C_m (W_t (x) M_y (x) M_x) x + (M_t (x) (D_x M_y (x) K_x + D_y K_y (x) M_x)) x
//     = M_y r1 + D_y K_y r2,   r1 = C_m M_x xW + D_x K_x xM,  r2 = M_x xM,
// with xW = W_t x and xM = M_t x, in one pass.  Block = (32-column strip,
// time slice t):
//  1. (xW, xM) of the strip with a P-column halo, as pairs in shared memory,
//     from the 2P+1 planes of x around t (x is read from L2 by the blocks of
//     neighbouring slices; each plane comes from HBM about once);
//  2. the x bands in place (a warp owns whole rows; each lane one column);
//  3. the y bands down each column from a sliding register window.
// Every product of two bands' pairs is one paired multiply-add.  Bands
// [i][k] = A(i, i-P+k).  Shared memory: ny (32 + 2P + 2P + 1) pairs.
template <typename T, int P>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) kron2d_kernel(T *__restrict__ y, const typename Pair<T>::src *__restrict__ x,
                                                     const T *__restrict__ Wt, const T *__restrict__ Mt,
                                                     const T *__restrict__ Mx, const T *__restrict__ Kx,
                                                     const T *__restrict__ My, const T *__restrict__ Ky, int nx, int ny,
                                                     int Nt, T Cm, T Dx, T Dy) {
  typedef Pair<T> PT;
  typedef typename PT::type T2;
  typedef typename PT::ct CT;
  const CT z0 = PT::from(T(0));
  const T2 zz = PT::make(z0, z0);
  constexpr int B = 2 * P + 1, SW = 32, HW = SW + 2 * P;
  extern __shared__ __align__(16) unsigned char k2_raw[];
  T2 *S = reinterpret_cast<T2 *>(k2_raw);   // [ny][HW]: (xW, xM); after the x pass (r1, r2) in columns P..P+SW-1
  T2 *by = S + (size_t)ny * HW;             // [ny][B]: (M_y, D_y K_y) row pairs
  const int t = blockIdx.y, cx0 = blockIdx.x * SW;
  const long long Ns = (long long)nx * ny;
  const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5, nrg = blockDim.x >> 5;
  // row t of W_t and M_t as pairs; only the planes klo..khi exist
  const int klo = max(0, P - t), khi = min(B - 1, Nt - 1 - t + P);
  T2 tw[B];
#pragma unroll
  for (int k = 0; k < B; ++k)
    tw[k] = (k >= klo && k <= khi) ? PT::make(PT::from(Wt[(size_t)t * B + k]), PT::from(Mt[(size_t)t * B + k])) : zz;
  for (int e = threadIdx.x; e < ny * B; e += blockDim.x) {
    const int r = e / B, k = e - r * B, rr = r - P + k;
    const bool ok = rr >= 0 && rr < ny;
    by[e] = ok ? PT::make(PT::from(My[e]), PT::from(Dy * Ky[e])) : zz;
  }
  pdl_trigger();
  pdl_wait();   // the band rows above are staged before the previous kernel ends
  // 1. time bands of the strip (halo columns outside the plane are zero);
  // UE elements a round, all their loads issued before any product
  constexpr int UE = 4;
  const long long pofs = (long long)(t - P) * Ns;   // offset of plane t-P (negative near the start)
  const int nel = ny * HW;
  for (int e0 = threadIdx.x; e0 < nel; e0 += UE * blockDim.x) {
    typename PT::src v[UE][B];
#pragma unroll
    for (int u = 0; u < UE; ++u) {
      const int e = e0 + u * blockDim.x;
      const int r = e / HW, c = e - r * HW, cx = cx0 - P + c;
      const bool ok = e < nel && cx >= 0 && cx < nx;
      const long long o = pofs + (long long)r * nx + cx;
#pragma unroll
      for (int k = 0; k < B; ++k)
        v[u][k] = (ok && k >= klo && k <= khi) ? __ldg(x + (o + (long long)k * Ns)) : typename PT::src{};
    }
#pragma unroll
    for (int u = 0; u < UE; ++u) {
      const int e = e0 + u * blockDim.x;
      T2 acc = zz;
#pragma unroll
      for (int k = 0; k < B; ++k) {
        const CT cv = PT::load(v[u][k]);
        acc = pfma(tw[k], PT::make(cv, cv), acc);
      }
      if (e < nel) S[e] = acc;
    }
  }
  __syncthreads();
  // 2. x bands in place: all reads of a row precede the writes of its centre
  const int c = lane, cx = cx0 + c;
  T2 mx[B];
  CT kx[B];
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const bool ok = cx < nx && cx - P + k >= 0 && cx - P + k < nx;
    const CT m = PT::from(ok ? Mx[(size_t)cx * B + k] : T(0));
    mx[k] = PT::make(m, m);
    kx[k] = PT::from(ok ? Kx[(size_t)cx * B + k] : T(0));
  }
  const CT cm = PT::from(Cm), dx = PT::from(Dx);
  for (int r = rg; r < ny; r += nrg) {
    T2 *row = S + (size_t)r * HW + c;
    T2 a = zz;   // (M_x xW, M_x xM)
    CT b = z0;   // K_x xM
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const T2 v = row[k];
      a = pfma(mx[k], v, a);
      b = PT::fma(kx[k], v.y, b);
    }
    __syncwarp();
    row[P] = PT::make(PT::fma(cm, a.x, PT::mul(dx, b)), a.y);
    __syncwarp();
  }
  __syncthreads();
  if (cx >= nx) return;
  // 3. y bands: each warp a contiguous run of rows, (r1, r2) of rows r-P..r+P
  // in registers
  const T2 *R = S + P + c;   // row stride HW
  const int per = (ny + nrg - 1) / nrg, ra = rg * per, rb = min(ny, ra + per);
  if (ra >= rb) return;
  T2 w[B];
#pragma unroll
  for (int k = 0; k < B - 1; ++k) {
    const int rr = ra - P + k;
    w[k + 1] = (rr >= 0 && rr < ny) ? R[(size_t)rr * HW] : zz;
  }
  T *yo = y + (long long)t * Ns + (long long)ra * nx + cx;
  for (int r0 = ra; r0 < rb; r0 += B) {
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int r = r0 + u;
      if (r >= rb) break;
#pragma unroll
      for (int k = 0; k < B - 1; ++k) w[k] = w[k + 1];
      w[B - 1] = r + P < ny ? R[(size_t)(r + P) * HW] : zz;
      const T2 *br = by + (size_t)r * B;
      T2 acc = zz;
#pragma unroll
      for (int k = 0; k < B; ++k) acc = pfma(br[k], w[k], acc);
      *yo = PT::to(PT::add(acc.x, acc.y));
      yo += nx;
    }
  }
}

// Dense strided GEMM C[b](m, c) = sum_k A(m, k) X[b](k, c) with 64x64 tiles,
// 256 threads, 4x4 outputs per thread: the spatial transforms U_l, U_l^T of
// the fast-diagonalization preconditioner (Eq. factorized), the Gram matrix
// of Theta-hat and the products of the eigen-refinement.
struct GemmDesc {
  int M, N, K, batch;
  int splits = 1;                // K partitions; partial results go to C + split * M * N (scm, scc layout)
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
  int b = blockIdx.z % g.batch;
  int split = blockIdx.z / g.batch;
  int kchunk = ((g.K + g.splits - 1) / g.splits + BK - 1) / BK * BK;
  int kbeg = split * kchunk, kend = min(g.K, kbeg + kchunk);
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
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int l = tid; l < BM * BK; l += 256) {
      int mm, kk;
      if (a_k_fast) { kk = l % BK; mm = l / BK; } else { mm = l % BM; kk = l / BM; }
      int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < g.M && k < kend) ? A[m * g.sam + k * g.sak] : T(0);
    }
    for (int l = tid; l < BN * BK; l += 256) {
      int cc, kk;
      if (x_c_fast) { cc = l % BN; kk = l / BN; } else { kk = l % BK; cc = l / BK; }
      int c = c0 + cc, k = k0 + kk;
      Xs[kk][cc] = (c < g.N && k < kend) ? Xb[k * g.sbk + c * g.sbc] : T(0);
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
  T *Cb = C + (long long)b * g.scb + (long long)split * g.M * g.N;
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
// Banded forward/back substitution along time for every spatial eigen-index j
// (LU stored [it][k][j], 1/u_ii on the diagonal), one thread per j.  Only
// N_s time lines exist, so the sweep is bound by how many loads each thread
// keeps in flight: the operands of the next U steps are loaded before the
// current U steps are computed (two batches in flight).  Measured on the 2D
// workload against a warp-specialized cp.async ring, a per-thread cp.async
// ring, a blocked layout and 16-byte loads per thread, this is the fastest.
template <typename T, int P, int U>
__global__ void __launch_bounds__(128) tline_lu_kernel(T *__restrict__ z, const T *__restrict__ r,
                                                       const T *__restrict__ lu, int Nt, long long Ns) {
  pdl_trigger();
  pdl_wait();   // inputs and outputs are shared with the previous kernel
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= Ns) return;
  constexpr int B = 2 * P + 1;
  // forward substitution with the unit lower factor
  {
    T yw[P];
#pragma unroll
    for (int k = 0; k < P; ++k) yw[k] = T(0);
    T rv[U], lv[U][P], rn[U], ln[U][P];
    auto load = [&](int it0, T (&rr)[U], T (&ll)[U][P]) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int it = it0 + u;
        const bool ok = it < Nt;
        rr[u] = ok ? r[(long long)it * Ns + j] : T(0);
#pragma unroll
        for (int k = 1; k <= P; ++k)
          ll[u][k - 1] = (ok && it - k >= 0) ? lu[((long long)it * B + (P - k)) * Ns + j] : T(0);
      }
    };
    load(0, rv, lv);
    for (int it0 = 0; it0 < Nt; it0 += U) {
      if (it0 + U < Nt) load(it0 + U, rn, ln);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int it = it0 + u;
        if (it >= Nt) break;
        T v = rv[u];
#pragma unroll
        for (int k = P; k >= 1; --k) v -= lv[u][k - 1] * yw[P - k];
#pragma unroll
        for (int k = 0; k < P - 1; ++k) yw[k] = yw[k + 1];
        yw[P - 1] = v;
        z[(long long)it * Ns + j] = v;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        rv[u] = rn[u];
#pragma unroll
        for (int k = 0; k < P; ++k) lv[u][k] = ln[u][k];
      }
    }
  }
  // backward substitution with the upper factor (1/u_ii stored on the diagonal)
  {
    T zw[P];
#pragma unroll
    for (int k = 0; k < P; ++k) zw[k] = T(0);
    T yv[U], uv[U][P + 1], yn[U], un[U][P + 1];
    auto load = [&](int c0, T (&yy)[U], T (&ul)[U][P + 1]) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int it = Nt - 1 - (c0 + u);
        const bool ok = it >= 0;
        yy[u] = ok ? z[(long long)it * Ns + j] : T(0);
#pragma unroll
        for (int k = 0; k <= P; ++k) ul[u][k] = (ok && it + k < Nt) ? lu[((long long)it * B + (P + k)) * Ns + j] : T(0);
      }
    };
    load(0, yv, uv);
    for (int c0 = 0; c0 < Nt; c0 += U) {
      if (c0 + U < Nt) load(c0 + U, yn, un);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int it = Nt - 1 - (c0 + u);
        if (it < 0) break;
        T v = yv[u];
#pragma unroll
        for (int k = P; k >= 1; --k) v -= uv[u][k] * zw[k - 1];
        v *= uv[u][0];
#pragma unroll
        for (int k = P - 1; k > 0; --k) zw[k] = zw[k - 1];
        zw[0] = v;
        z[(long long)it * Ns + j] = v;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        yv[u] = yn[u];
#pragma unroll
        for (int k = 0; k <= P; ++k) uv[u][k] = un[u][k];
      }
    }
  }
}

// FP64 rows (n values each) into FP32 rows of stride `stride`, the padding zero.
__global__ void pad_d2f_kernel(float *__restrict__ out, const double *__restrict__ in, long long rows, long long n,
                               long long stride) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long rr = w0; rr < rows; rr += nw)
    for (long long k = lane; k < stride; k += 32) out[rr * stride + k] = k < n ? (float)in[rr * n + k] : 0.f;
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
  const VT *rowp[G];
#pragma unroll
  for (int g = 0; g < G; ++g) rowp[g] = reinterpret_cast<const VT *>(V + (long long)(i0 + min(g, cnt - 1)) * ldv);
  for (long long e = beg + threadIdx.x; e < end; e += blockDim.x) {
    VT x = wv[e];
    VT v[G];
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = rowp[g][e];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g].add(X::dot(v[g], x));
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

// out[i] = sum_b partial[i][b]: one warp per i, lanes take blocks in a fixed
// stride pattern and a fixed shuffle tree combines them (deterministic).
__global__ void reduce_blocks_kernel(double *__restrict__ out, const double *__restrict__ partial, int nblocks,
                                     int nv) {
  pdl_trigger();
  pdl_wait();   // inputs and outputs are shared with the previous kernel
  int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (i >= nv) return;
  const double *p = partial + (long long)i * nblocks;
  double t = 0.0;
  for (int b = lane; b < nblocks; b += 32) t += p[b];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
  if (lane == 0) out[i] = t;
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
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; e + stride < nvec; e += 2 * stride) {
    VT a = X::zero(), b = X::zero();
#pragma unroll 8
    for (int i = 0; i < nv; ++i) {
      const VT *vi = reinterpret_cast<const VT *>(V + (long long)i * ldv);
      a = X::fma(hs[i], vi[e], a);
      b = X::fma(hs[i], vi[e + stride], b);
    }
    wv[e] = X::upd(wv[e], a, s);
    wv[e + stride] = X::upd(wv[e + stride], b, s);
  }
  for (; e < nvec; e += stride) {
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

// Partial inner products of rows V_i (i < nv) with two vectors x1, x2 in one
// pass over the rows: partial[(2 i + c) * gridDim.x + b] = <V_i, x_c> over
// block b's chunk (Kahan FP32 / plain FP64 per thread, FP64 across threads in
// a fixed order), the dot pass of the delayed Gram-Schmidt below.
template <typename T, int G>
__global__ void __launch_bounds__(256) mdot2_kernel(double *__restrict__ partial, const T *__restrict__ V,
                                                    long long ldv, int nv, const T *__restrict__ x1,
                                                    const T *__restrict__ x2, long long n) {
  pdl_trigger();
  pdl_wait();   // inputs and outputs are shared with the previous kernel
  typedef V16<T> X;
  typedef typename X::type VT;
  constexpr int W = X::W;
  __shared__ double red[2 * G][8];
  const int i0 = blockIdx.y * G;
  const int cnt = min(G, nv - i0);
  const long long nvec = n / W;
  const long long chunk = (nvec + gridDim.x - 1) / gridDim.x;
  const long long beg = (long long)blockIdx.x * chunk, end = min(nvec, beg + chunk);
  T acc[G][2];
#pragma unroll
  for (int g = 0; g < G; ++g) { acc[g][0] = T(0); acc[g][1] = T(0); }
  const VT *y1 = reinterpret_cast<const VT *>(x1), *y2 = reinterpret_cast<const VT *>(x2);
  // rows past the group end repeat the last row (loads stay unconditional so
  // they are all in flight together); their sums are never written.  The
  // operands of the next element are loaded before the current one is used.
  const VT *rowp[G];
#pragma unroll
  for (int g = 0; g < G; ++g) rowp[g] = reinterpret_cast<const VT *>(V + (long long)(i0 + min(g, cnt - 1)) * ldv);
  long long e = beg + threadIdx.x;
  VT a, b, v[G];
  if (e < end) {
    a = y1[e]; b = y2[e];
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = rowp[g][e];
  }
  for (; e < end; e += blockDim.x) {
    const long long en = e + blockDim.x;
    VT an, bn, vn[G];
    if (en < end) {
      an = y1[en]; bn = y2[en];
#pragma unroll
      for (int g = 0; g < G; ++g) vn[g] = rowp[g][en];
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      acc[g][0] += X::dot(v[g], a);
      acc[g][1] += X::dot(v[g], b);
    }
    a = an; b = bn;
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = vn[g];
  }
  if (blockIdx.x == gridDim.x - 1)
    for (long long e = nvec * W + threadIdx.x; e < n; e += blockDim.x)
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (g < cnt) {
          T v = V[(long long)(i0 + g) * ldv + e];
          acc[g][0] += v * x1[e];
          acc[g][1] += v * x2[e];
        }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    if (g >= cnt) break;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      double t = (double)acc[g][c];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
      if (lane == 0) red[2 * g + c][warp] = t;
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < 2 * cnt) {
    double t = 0.0;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) t += red[threadIdx.x][wi];
    partial[(long long)(2 * i0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
  }
}

// Coefficients of the update pass of the delayed classical Gram-Schmidt (two
// passes over the basis per Arnoldi step instead of four).  Rows 0..j-1 of V
// are final; row j holds u_j (projected once), row j+1 holds w = A z_j.  From
// the dots D[2i+c] = <V_i, (u_j, w)_c> (i <= j+1) of the dot pass:
//   nu = sqrt(<u,u> - |a|^2), a_i = <V_i,u>   (Pythagoras: u is nearly orthogonal)
//   v_j = (u - sum a_i V_i) / nu              (reorthogonalized, normalized)
//   gam = <v_j, w> = (<u,w> - a.b) / nu,      b_i = <V_i, w>
//   u_{j+1} = sw (w - sum b_i V_i - gam v_j)  (projected once; sw scales it to
//             about unit norm, sw = 1/sqrt(<w,w> - |b|^2 - gam^2))
// One block: the sums over i in a fixed tree, then coef = [a_i / nu (j),
// b_i - a_i gam / nu (j), 1/nu, gam/nu, sw] in T and sc = (nu, gam, sw).
template <typename T>
__global__ void __launch_bounds__(256) dcgs2_coef_kernel(T *__restrict__ coef, double *__restrict__ sc,
                                                         const double *__restrict__ D, int j) {
  pdl_trigger();
  pdl_wait();   // inputs and outputs are shared with the previous kernel
  __shared__ double part[3][8];
  __shared__ double scal[2];
  double sa2 = 0.0, sab = 0.0, sb2 = 0.0;
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    const double a = D[2 * i], b = D[2 * i + 1];
    sa2 += a * a; sab += a * b; sb2 += b * b;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sa2 += __shfl_down_sync(0xffffffffu, sa2, off);
    sab += __shfl_down_sync(0xffffffffu, sab, off);
    sb2 += __shfl_down_sync(0xffffffffu, sb2, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { part[0][warp] = sa2; part[1][warp] = sab; part[2][warp] = sb2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    sa2 = sab = sb2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sa2 += part[0][w]; sab += part[1][w]; sb2 += part[2][w]; }
    const double uu = D[2 * j], uw = D[2 * j + 1], ww = D[2 * (j + 1) + 1];
    const double nu2 = uu - sa2;
    const double nu = nu2 > 0.0 ? sqrt(nu2) : 0.0;
    const double inu = nu > 0.0 ? 1.0 / nu : 0.0;
    const double gam = (uw - sab) * inu;
    const double q = ww - sb2 - gam * gam;
    const double sw = (q > 0.0 && q > 1e-30 * ww) ? 1.0 / sqrt(q) : (ww > 0.0 ? 1.0 / sqrt(ww) : 1.0);
    scal[0] = inu; scal[1] = gam * inu;
    coef[2 * j] = (T)inu; coef[2 * j + 1] = (T)(gam * inu); coef[2 * j + 2] = (T)sw;
    sc[0] = nu; sc[1] = gam; sc[2] = sw;
  }
  __syncthreads();
  const double inu = scal[0], gin = scal[1];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    coef[i] = (T)(D[2 * i] * inu);
    coef[j + i] = (T)(D[2 * i + 1] - D[2 * i] * gin);
  }
}

// The update pass itself, one read of rows 0..j+1, rows j and j+1 rewritten
// in place (16-byte aligned rows).
template <typename T>
__global__ void __launch_bounds__(256) dcgs2_update_kernel(T *__restrict__ V, long long ldv, int j,
                                                           const T *__restrict__ coef, long long n) {
  pdl_trigger();
  pdl_wait();   // inputs and outputs are shared with the previous kernel
  typedef V16<T> X;
  typedef typename X::type VT;
  constexpr int W = X::W;
  __shared__ T ca[512], cb[512];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    ca[i] = coef[i];
    cb[i] = coef[j + i];
  }
  const T tinu = coef[2 * j], tg = coef[2 * j + 1], tsw = coef[2 * j + 2];
  __syncthreads();
  T *U = V + (long long)j * ldv, *Wr = V + (long long)(j + 1) * ldv;
  const long long nvec = n / W;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nvec; e += stride) {
    VT aa = X::zero(), bb = X::zero();
#pragma unroll 8
    for (int i = 0; i < j; ++i) {
      const VT vi = reinterpret_cast<const VT *>(V + (long long)i * ldv)[e];
      aa = X::fma(ca[i], vi, aa);
      bb = X::fma(cb[i], vi, bb);
    }
    VT u = reinterpret_cast<VT *>(U)[e], w = reinterpret_cast<VT *>(Wr)[e];
    const T *ua = reinterpret_cast<const T *>(&u), *wa = reinterpret_cast<const T *>(&w);
    const T *aA = reinterpret_cast<const T *>(&aa), *bA = reinterpret_cast<const T *>(&bb);
    VT vo, wo;
    T *vA = reinterpret_cast<T *>(&vo), *woA = reinterpret_cast<T *>(&wo);
#pragma unroll
    for (int c = 0; c < W; ++c) {
      vA[c] = ua[c] * tinu - aA[c];
      woA[c] = tsw * (wa[c] - bA[c] - tg * ua[c]);
    }
    reinterpret_cast<VT *>(U)[e] = vo;
    reinterpret_cast<VT *>(Wr)[e] = wo;
  }
  if (blockIdx.x == 0)
    for (long long e = nvec * W + threadIdx.x; e < n; e += blockDim.x) {
      T a = T(0), b = T(0);
      for (int i = 0; i < j; ++i) {
        const T vi = V[(long long)i * ldv + e];
        a += ca[i] * vi;
        b += cb[i] * vi;
      }
      const T u = U[e], w = Wr[e];
      U[e] = u * tinu - a;
      Wr[e] = tsw * (w - b - tg * u);
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

// Blocks along the outer index so that the whole grid is about 16 blocks per
// SM (each thread then loops over several outer indices).
unsigned outer_blocks(long long outer, long long other_blocks) {
  long long target = 152LL * 16;
  long long g = std::max<long long>(1, target / std::max<long long>(1, other_blocks));
  return (unsigned)std::min<long long>(std::min<long long>(outer, g), 65535);
}

}  // namespace

// ---------------------------------------------------------------- launchers
template <typename T>
void launch_band_pass(cudaStream_t s, T *out, int nterms, const T *const *bands, const T *const *ins,
                      const double *coefs, int n, long long inner, long long outer, int p, bool accumulate) {
  TiledTerms<T> tt;
  tt.nterms = nterms;
  for (int t = 0; t < 3; ++t) {
    tt.in[t] = t < nterms ? ins[t] : nullptr;
    tt.tab[t] = t < nterms ? bands[t] : nullptr;
    tt.coef[t] = t < nterms ? (T)coefs[t] : T(0);
  }
  launch_tiled_p<T, OP_BAND>(s, p, out, tt, n, n, inner, outer, accumulate);
}

template <typename T>
void launch_interp_fwd(cudaStream_t s, T *out, const T *in, const T *tab, int nel, int p, int nq,
                       long long inner, long long outer) {
  (void)nq;
  TiledTerms<T> tt;
  tt.nterms = 1;
  tt.in[0] = in; tt.tab[0] = tab; tt.coef[0] = T(1);
  for (int t = 1; t < 3; ++t) { tt.in[t] = nullptr; tt.tab[t] = nullptr; tt.coef[t] = T(0); }
  launch_tiled_p<T, OP_FWD>(s, p, out, tt, nel + p, nel * (p + 1), inner, outer, false);
}

template <typename T>
void launch_interp_bwd(cudaStream_t s, T *out, const T *in, const T *tab, int nel, int p, int nq,
                       long long inner, long long outer, bool accumulate) {
  (void)nq;
  TiledTerms<T> tt;
  tt.nterms = 1;
  tt.in[0] = in; tt.tab[0] = tab; tt.coef[0] = T(1);
  for (int t = 1; t < 3; ++t) { tt.in[t] = nullptr; tt.tab[t] = nullptr; tt.coef[t] = T(0); }
  launch_tiled_p<T, OP_BWD>(s, p, out, tt, nel * (p + 1), nel + p, inner, outer, accumulate);
}

void launch_interp_fwd_pairs(cudaStream_t s, float2 *out, const float2 *in, const float2 *tab, int nel, int p,
                             long long inner, long long outer) {
  const int bx = (int)std::min<long long>(256, (inner + 31) / 32 * 32);
  const long long gx = (inner + bx - 1) / bx;
  const int nruns = (nel + kRunFwd - 1) / kRunFwd;
  dim3 grid((unsigned)gx, (unsigned)std::min<long long>(outer * nruns, 65535));
  st_count_launch();
  switch (p) {
    case 1: pdl_launch(ifwd_pairs_kernel<1>, grid, dim3(bx), 0, s, out, in, tab, nel, inner, outer, nruns); break;
    case 2: pdl_launch(ifwd_pairs_kernel<2>, grid, dim3(bx), 0, s, out, in, tab, nel, inner, outer, nruns); break;
    case 3: pdl_launch(ifwd_pairs_kernel<3>, grid, dim3(bx), 0, s, out, in, tab, nel, inner, outer, nruns); break;
    default: pdl_launch(ifwd_pairs_kernel<4>, grid, dim3(bx), 0, s, out, in, tab, nel, inner, outer, nruns); break;
  }
}

template <typename TO>
void launch_interp_bwd_pairs(cudaStream_t s, TO *out, const float2 *in, const float2 *tab, int nel, int p,
                             long long inner, long long outer, bool accumulate) {
  const int bx = (int)std::min<long long>(256, (inner + 31) / 32 * 32);
  const long long gx = (inner + bx - 1) / bx;
  const int nruns = (nel + p + kRunBwd - 1) / kRunBwd;
  dim3 grid((unsigned)gx, (unsigned)std::min<long long>(outer * nruns, 65535));
  const int acc = accumulate ? 1 : 0;
  st_count_launch();
  switch (p) {
    case 1: pdl_launch(ibwd_pairs_kernel<1, TO>, grid, dim3(bx), 0, s, out, in, tab, nel, inner, outer, nruns, acc); break;
    case 2: pdl_launch(ibwd_pairs_kernel<2, TO>, grid, dim3(bx), 0, s, out, in, tab, nel, inner, outer, nruns, acc); break;
    case 3: pdl_launch(ibwd_pairs_kernel<3, TO>, grid, dim3(bx), 0, s, out, in, tab, nel, inner, outer, nruns, acc); break;
    default: pdl_launch(ibwd_pairs_kernel<4, TO>, grid, dim3(bx), 0, s, out, in, tab, nel, inner, outer, nruns, acc); break;
  }
}
template void launch_interp_bwd_pairs<float2>(cudaStream_t, float2 *, const float2 *, const float2 *, int, int,
                                              long long, long long, bool);
template void launch_interp_bwd_pairs<double>(cudaStream_t, double *, const float2 *, const float2 *, int, int,
                                              long long, long long, bool);

template <typename T>
void launch_qband_apply(cudaStream_t s, T *z, const T *x, const float *bhi, const float *blo, int Nt, long long Qs,
                        int p) {
  int threads = 128;
  long long blocks = (Qs + threads - 1) / threads;
  switch (p) {
    case 1: st_count_launch(); qband_kernel<T, 1><<<(unsigned)blocks, threads, 0, s>>>(z, x, bhi, blo, Nt, Qs); break;
    case 2: st_count_launch(); qband_kernel<T, 2><<<(unsigned)blocks, threads, 0, s>>>(z, x, bhi, blo, Nt, Qs); break;
    case 3: st_count_launch(); qband_kernel<T, 3><<<(unsigned)blocks, threads, 0, s>>>(z, x, bhi, blo, Nt, Qs); break;
    default: st_count_launch(); qband_kernel<T, 4><<<(unsigned)blocks, threads, 0, s>>>(z, x, bhi, blo, Nt, Qs); break;
  }
}

int xband_fused_limit(size_t elem, int p) { return (elem == 8 || p >= 4) ? 256 : 512; }

template <typename T>
bool launch_xband_fused(cudaStream_t s, T *Y1, const T *X1, const float *bhi, const float *blo, const T *tab, int nel,
                        int Nt, long long rows, int p, int *err) {
  const int threads = (nel + p + 31) / 32 * 32;
  if (threads > xband_fused_limit(sizeof(T), p) || rows < 1) return false;
  // time segments so that the grid holds about 16 blocks per SM, each
  // segment at least 16 P steps long (its replay halo is P steps)
  long long want = (152LL * 16 + rows - 1) / rows;
  int nseg = (int)std::max<long long>(1, std::min<long long>(want, Nt / (16 * p)));
  int seglen = (Nt + nseg - 1) / nseg;
  nseg = (Nt + seglen - 1) / seglen;
  unsigned blocks = (unsigned)std::min<long long>(rows * nseg, 1LL << 30);
  constexpr int S = sizeof(T) == 4 ? 4 : 3;
  // every instance has the same function type, so this lambda has one
  // instantiation per T: the opt-in masks are kept per instance (P, BULK)
  auto go = [&](auto kern, int P, bool bulk_kern) {
    const int NB = sizeof(T) == 8 ? 2 : 1;
    size_t sh = (size_t)S * NB * (P + 1) * threads * (P + 1) * sizeof(float) + (size_t)S * threads * sizeof(T);
    static std::atomic<unsigned long long> attr[10] = {};
    smem_optin(kern, 200 * 1024, attr[2 * P + (bulk_kern ? 1 : 0)]);
    st_count_launch();
    pdl_launch(kern, dim3(blocks), dim3(threads), sh, s, Y1, X1, bhi, blo, tab, nel, Nt, rows, seglen, err);
  };
  // bulk band copies need 16-byte aligned slices: Q_x a multiple of 4 floats
  const bool bulk = (nel * (p + 1)) % 4 == 0 && ((uintptr_t)bhi % 16) == 0 && (!blo || ((uintptr_t)blo % 16) == 0);
  switch (p * 2 + (bulk ? 1 : 0)) {
    case 2: go(xband_fused_kernel<T, 1, S, false>, 1, false); break;
    case 3: go(xband_fused_kernel<T, 1, S, true>, 1, true); break;
    case 4: go(xband_fused_kernel<T, 2, S, false>, 2, false); break;
    case 5: go(xband_fused_kernel<T, 2, S, true>, 2, true); break;
    case 6: go(xband_fused_kernel<T, 3, S, false>, 3, false); break;
    case 7: go(xband_fused_kernel<T, 3, S, true>, 3, true); break;
    case 8: go(xband_fused_kernel<T, 4, S, false>, 4, false); break;
    default: go(xband_fused_kernel<T, 4, S, true>, 4, true); break;
  }
  return true;
}

// x split into double-float pairs for the FP64 instance of the Kronecker
// kernel (one conversion per value instead of one per read).
__global__ void split_df_kernel(float2 *__restrict__ out, const double *__restrict__ in, long long n) {
  pdl_trigger();
  pdl_wait();   // x is written by the previous kernel, out may still be read by it
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const df v = df_from(in[i]);
    out[i] = make_float2(v.hi, v.lo);
  }
}

template <typename T>
bool launch_kron2d(cudaStream_t s, T *y, const T *x, const void *split, const T *Wt, const T *Mt, const T *Mx,
                   const T *Kx, const T *My, const T *Ky, int nx, int ny, int Nt, int p, double Cm, double Dx,
                   double Dy) {
  const size_t sh = (size_t)ny * ((32 + 2 * p) + (2 * p + 1)) * 2 * sizeof(T);
  if (sh > 200 * 1024 || p > 4 || Nt > 65535) return false;
  dim3 g((unsigned)((nx + 31) / 32), (unsigned)Nt);
  const typename Pair<T>::src *xs;
  if constexpr (sizeof(T) == 8) xs = reinterpret_cast<const float2 *>(split);
  else xs = x;
  auto go = [&](auto k, int P) {
    static std::atomic<unsigned long long> attr[5] = {{0}, {0}, {0}, {0}, {0}};
    smem_optin(k, 200 * 1024, attr[P]);
    st_count_launch(); pdl_launch(k, g, dim3(256), sh, s, y, xs, Wt, Mt, Mx, Kx, My, Ky, nx, ny, Nt, (T)Cm, (T)Dx, (T)Dy);
  };
  switch (p) {
    case 1: go(kron2d_kernel<T, 1>, 1); break;
    case 2: go(kron2d_kernel<T, 2>, 2); break;
    case 3: go(kron2d_kernel<T, 3>, 3); break;
    default: go(kron2d_kernel<T, 4>, 4); break;
  }
  return true;
}

void launch_split_df(cudaStream_t s, float2 *out, const double *in, long long n) {
  st_count_launch();
  pdl_launch(split_df_kernel, dim3((unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16))),
             dim3(256), 0, s, out, in, n);
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

// Rotating transform out[(t nj + j) A + a] = sum_k M[j][k] in[(t A + a) nb + k]
// as a batched strided GEMM (batch t, rows j, columns a).
template <typename T>
void launch_rot_gemm(cudaStream_t s, T *out, const T *in, const T *M, int nb, int nj, long long Aa, long long Nt) {
  GemmDesc g;
  g.M = nj; g.N = (int)Aa; g.K = nb; g.batch = 1;
  g.sam = nb; g.sak = 1;
  g.sbb = Aa * nb; g.sbk = 1; g.sbc = nb;
  g.scb = (long long)nj * Aa; g.scm = Aa; g.scc = 1;
  const long long maxb = 65535;
  for (long long b0 = 0; b0 < Nt; b0 += maxb) {
    GemmDesc gb = g;
    gb.batch = (int)std::min<long long>(maxb, Nt - b0);
    launch_gemm<T>(s, out + b0 * g.scb, M, in + b0 * g.sbb, gb, 1.0, 0.0);
  }
}

template <typename T>
void launch_tline_lu_solve(cudaStream_t s, T *z, const T *r, const T *lu, int Nt, long long Ns, int p, int *err) {
  (void)err;
  constexpr int U = sizeof(T) == 4 ? 16 : 8;
  const unsigned blocks = (unsigned)((Ns + 127) / 128);
  switch (p) {
    case 1: st_count_launch(); pdl_launch(tline_lu_kernel<T, 1, U>, dim3(blocks), dim3(128), 0, s, z, r, lu, Nt, Ns); break;
    case 2: st_count_launch(); pdl_launch(tline_lu_kernel<T, 2, U>, dim3(blocks), dim3(128), 0, s, z, r, lu, Nt, Ns); break;
    case 3: st_count_launch(); pdl_launch(tline_lu_kernel<T, 3, U>, dim3(blocks), dim3(128), 0, s, z, r, lu, Nt, Ns); break;
    default: st_count_launch(); pdl_launch(tline_lu_kernel<T, 4, U>, dim3(blocks), dim3(128), 0, s, z, r, lu, Nt, Ns); break;
  }
}

void launch_pad_d2f(cudaStream_t s, float *out, const double *in, long long rows, long long n, long long stride) {
  long long blocks = std::min<long long>((rows + 7) / 8, 152LL * 32);
  st_count_launch(); pad_d2f_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, s>>>(out, in, rows, n, stride);
}

template <typename T>
void launch_multi_dot(cudaStream_t s, double *out, const T *V, long long ldv, int nv, const T *w, long long n,
                      double *scratch) {
  constexpr int G = 8;
  int groups = (nv + G - 1) / G;
  // enough blocks for about four waves in total, at least 8 vector steps per thread
  long long want = std::max<long long>(38, 4 * 304 / groups);
  long long cap = std::max<long long>(1, n / (V16<T>::W * 256 * 8));
  int bx = (int)std::max<long long>(1, std::min<long long>(std::min<long long>(want, cap), kDotBlocks));
  dim3 grid(bx, groups);
  // a single product (norms) takes the one-row instance: no repeated loads
  // of the same row and one accumulator per thread
  st_count_launch();
  if (nv == 1) mdot_kernel<T, 1><<<grid, 256, 0, s>>>(scratch, V, ldv, nv, w, n);
  else mdot_kernel<T, G><<<grid, 256, 0, s>>>(scratch, V, ldv, nv, w, n);
  st_count_launch(); reduce_blocks_kernel<<<(nv + 3) / 4, 128, 0, s>>>(out, scratch, bx, nv);
}

template <typename T>
void launch_multi_axpy(cudaStream_t s, T *w, const T *V, long long ldv, int nv, const double *h, long long n,
                       const double *nrm) {
  long long nvec = n / V16<T>::W;
  st_count_launch(); maxpy_kernel<T><<<grid_for(std::max<long long>(nvec / 2, 1)), kThreads, 0, s>>>(w, V, ldv, nv, h, n, nrm);
}

template <typename T>
void launch_multi_dot2(cudaStream_t s, double *out, const T *V, long long ldv, int nv, const T *x1, const T *x2,
                       long long n, double *scratch) {
  constexpr int G = 4;
  int groups = (nv + G - 1) / G;
  long long want = std::max<long long>(38, 4 * 304 / groups);
  long long cap = std::max<long long>(1, n / (V16<T>::W * 256 * 2));
  int bx = (int)std::max<long long>(1, std::min<long long>(std::min<long long>(want, cap), kDotBlocks));
  dim3 grid(bx, groups);
  st_count_launch(); pdl_launch(mdot2_kernel<T, G>, grid, dim3(256), 0, s, scratch, V, ldv, nv, x1, x2, n);
  st_count_launch(); pdl_launch(reduce_blocks_kernel, dim3((2 * nv + 3) / 4), dim3(128), 0, s, out, (const double *)scratch, bx, 2 * nv);
}

template <typename T>
void launch_dcgs2_update(cudaStream_t s, T *V, long long ldv, int j, const double *D, long long n, double *sc,
                         T *coef) {
  long long nvec = n / V16<T>::W;
  st_count_launch(); pdl_launch(dcgs2_coef_kernel<T>, dim3(1), dim3(256), 0, s, coef, sc, D, j);
  st_count_launch(); pdl_launch(dcgs2_update_kernel<T>, dim3(grid_for(std::max<long long>(nvec, 1))), dim3(kThreads), 0, s, V, ldv, j, (const T *)coef, n);
}

template <typename T>
void launch_scale_copy(cudaStream_t s, T *y, const T *x, double alpha, long long n) {
  st_count_launch(); scale_copy_kernel<T><<<grid_for(n), kThreads, 0, s>>>(y, x, alpha, n);
}

// out[r * stride + k] = in[r * n + k] (rows copied into 16-byte aligned rows):
// one warp per row, no index division.
__global__ void pad_rows_kernel(float *__restrict__ out, const float *__restrict__ in, long long rows, long long n,
                                long long stride) {
  pdl_trigger();
  pdl_wait();   // inputs and outputs are shared with the previous kernel
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = w0; r < rows; r += nw) {
    const float *src = in + r * n;
    float *dst = out + r * stride;
    for (long long k = lane; k < n; k += 32) dst[k] = src[k];
  }
}

void launch_pad_rows(cudaStream_t s, float *out, const float *in, long long rows, long long n, long long stride) {
  long long blocks = std::min<long long>((rows + 7) / 8, 152LL * 32);
  st_count_launch(); pdl_launch(pad_rows_kernel, dim3((unsigned)std::max<long long>(blocks, 1)), dim3(256), 0, s, out, in, rows, n, stride);
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
__global__ void f2d_kernel(double *__restrict__ y, const float *__restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
void launch_f2d(cudaStream_t s, double *y, const float *x, long long n) {
  st_count_launch(); f2d_kernel<<<grid_for(n), 256, 0, s>>>(y, x, n);
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

// C(m, c) = alpha sum_s P[s][m][c] + beta C(m, c): the fixed-order sum of split-K partials.
__global__ void splitk_reduce_kernel(double *C, const double *P, int M, int N, int S, long long scm, long long scc,
                                     double alpha, double beta) {
  long long total = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int m = (int)(e / N), c = (int)(e % N);
    double t = 0.0;
    for (int k = 0; k < S; ++k) t += P[(long long)k * total + e];
    double *dst = C + m * scm + c * scc;
    *dst = beta == 0.0 ? alpha * t : alpha * t + beta * *dst;
  }
}

// FP64 GEMM; with a workspace of at least `work_elems` doubles, small
// output grids with long K are split along K over more blocks (partials
// reduced in a fixed order, so results do not depend on the split).
void launch_gemm64(cudaStream_t s, double *C, const double *A, const double *X, int M, int N, int K,
                   long long sam, long long sak, long long sbk, long long sbc, long long scm, long long scc,
                   double alpha, double beta, double *work, long long work_elems) {
  GemmDesc g;
  g.M = M; g.N = N; g.K = K; g.batch = 1;
  g.sam = sam; g.sak = sak; g.sbb = 0; g.sbk = sbk; g.sbc = sbc; g.scb = 0; g.scm = scm; g.scc = scc;
  long long tiles = (long long)((M + 63) / 64) * ((N + 63) / 64);
  int S = 1;
  if (work && tiles < 2 * 152 && K >= 512) {
    S = (int)std::min<long long>(std::max<long long>(1, 4 * 152 / tiles), K / 256);
    while (S > 1 && (long long)S * M * N > work_elems) --S;
  }
  if (S <= 1) {
    launch_gemm<double>(s, C, A, X, g, alpha, beta);
    return;
  }
  GemmDesc gp = g;
  gp.splits = S;
  gp.scm = N; gp.scc = 1;          // partials are dense row-major M x N
  dim3 grid((N + 63) / 64, (M + 63) / 64, S);
  st_count_launch(); gemm_kernel<double><<<grid, 256, 0, s>>>(work, A, X, gp, 1.0, 0.0);
  st_count_launch(); splitk_reduce_kernel<<<grid_for((long long)M * N), kThreads, 0, s>>>(C, work, M, N, S, scm, scc, alpha, beta);
}

#define INST(T)                                                                                        \
  template void launch_band_pass<T>(cudaStream_t, T *, int, const T *const *, const T *const *,       \
                                    const double *, int, long long, long long, int, bool);            \
  template void launch_interp_fwd<T>(cudaStream_t, T *, const T *, const T *, int, int, int, long long, \
                                     long long);                                                      \
  template void launch_interp_bwd<T>(cudaStream_t, T *, const T *, const T *, int, int, int, long long, \
                                     long long, bool);                                                \
  template void launch_qband_apply<T>(cudaStream_t, T *, const T *, const float *, const float *, int, \
                                      long long, int);                                                  \
  template bool launch_kron2d<T>(cudaStream_t, T *, const T *, const void *, const T *, const T *,        \
                                 const T *, const T *, const T *, const T *, int, int, int, int, double, \
                                 double,                                                              \
                                 double);                                                              \
  template bool launch_xband_fused<T>(cudaStream_t, T *, const T *, const float *, const float *,       \
                                      const T *, int, int, long long, int, int *);                      \
  template void launch_mode_gemm<T>(cudaStream_t, T *, const T *, const T *, int, long long, long long); \
  template void launch_tline_lu_solve<T>(cudaStream_t, T *, const T *, const T *, int, long long, int,  \
                                          int *);                                                          \
  template void launch_rot_gemm<T>(cudaStream_t, T *, const T *, const T *, int, int, long long, long long); \
  template void launch_multi_dot<T>(cudaStream_t, double *, const T *, long long, int, const T *,      \
                                    long long, double *);                                             \
  template void launch_multi_axpy<T>(cudaStream_t, T *, const T *, long long, int, const double *,     \
                                     long long, const double *);                                      \
  template void launch_scale_copy<T>(cudaStream_t, T *, const T *, double, long long);              \
  template void launch_multi_dot2<T>(cudaStream_t, double *, const T *, long long, int, const T *,     \
                                     const T *, long long, double *);                                  \
  template void launch_dcgs2_update<T>(cudaStream_t, T *, long long, int, const double *, long long,   \
                                       double *, T *);
INST(float)
INST(double)
template bool launch_xband_fused<float2>(cudaStream_t, float2 *, const float2 *, const float *, const float *,
                                          const float2 *, int, int, long long, int, int *);
#undef INST
