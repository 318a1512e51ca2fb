// The reaction + SU part of the operator without stored time bands (the
// "lean" operator form).
//
// Sec. 3.1.1 writes A = C_m W_t (x) M_s + M_t (x) K_s + M_R + S-tilde, with
//   M_R x     = int int C(u^k, w^k) x v            (Eq. reaction; C_J for Newton)
//   S-tilde x = C_m sum_r R_rr sum_l int tau_l theta_{t,r} d_t^l x d_t^l v
//               * int theta_{s,r} x v              (Eq. tildeS).
// In the band form each spatial Gauss point q owns a symmetric N_t x N_t time
// band holding both terms, assembled once per linearization and streamed by
// every apply: (p+1) N_t values per spatial Gauss point, (p+1)^(d+1) values
// per unknown.  This kernel forms the same action without them:
//   * M_R is evaluated at the time Gauss points of each time element from
//     u^k and w^k, interpolated to the Gauss point in the kernel from their
//     coefficients at the Gauss rows of the other spatial axes (the arrays U1,
//     W1 of the same layout as X1 below), so C is recomputed, never stored;
//   * the SU term keeps its rank-R factors only: per spatial Gauss point the
//     R values d_r(q) = C_m sigma_r w_q theta_{s,r}(x_q) (formed once per
//     block from V by the d-linear interpolation on the spatial Greville
//     grid), and per rank the time band Tb[r][k][it] of sum_l tau_l
//     theta_{t,r} d^l b_it d^l b_{it+k}; the band of point q at row it is
//     sum_r d_r(q) Tb[r][.][it].
// The same kernel takes any list of such rank terms (scale cf[r], spatial
// factor V[:, r], time band Tb[r]).
//
// Layout and work split follow the fused x pass of the band form: X1, Y1 are
// [N_t][rows][n_x], the x coefficients of every Gauss row of the other axes;
// one block per (row, time segment), one thread per x element (its p+1
// Gauss points), the block rounded up to whole warps.  Thread e writes
// coefficient e of each output row; the thread of the last element also
// writes the p coefficients after it (a block of n_el + p threads would
// spend a whole warp on those p values when n_el is a multiple of 32).  The block
// sweeps its time segment with register windows of the rows it .. it+p of X,
// U and W at its Gauss points (new rows arrive through a cp.async ring in
// shared memory); at step it it
//   - applies the rank-term band of row it (upper part from the window, lower
//     part scattered into accumulators of the rows it+1 .. it+p),
//   - integrates time element it+1 (rows it .. it+p): C, x at its p+1 time
//     Gauss points, and the products back onto those rows,
//   - projects row it onto the x coefficients (warp shuffles, and across
//     warps through shared memory, in a fixed order) and stores it.
// A segment first replays the p steps before it, without output, to rebuild
// the accumulators.  The FP32 instance computes in float; the FP64 instance
// takes X1, Y1 as double-float pairs and computes in double-float arithmetic.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include "st_internal.h"
#include "df.cuh"
#include "pdl.cuh"

namespace {

template <typename T> struct LeanCT { typedef float type; };
template <> struct LeanCT<float2> { typedef df type; };

template <typename CT> __device__ __forceinline__ CT from_pair(float2 v);
template <> __device__ __forceinline__ float from_pair<float>(float2 v) { return v.x; }
template <> __device__ __forceinline__ df from_pair<df>(float2 v) { return {v.x, v.y}; }

template <int BYTES>
__device__ __forceinline__ void lean_cp_async(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void lean_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void lean_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int kLeanRing = 3;        // depth of the shared-memory ring of coefficient rows
constexpr int kLeanMaxThreads = 256;

template <typename T>
struct LeanArgs {
  T *Y1;
  const T *X1;
  const float2 *U1, *W1;        // u^k, w^k in the layout of X1 (double-float pairs); unused without M_R
  const T *tab;                 // x basis at the Gauss points [ex][g][a]
  const float2 *bt;             // time basis at the time Gauss points [e][gt][a], pairs
  const float2 *wt;             // time quadrature weights [e * nq + gt], pairs
  const double *ws[3];          // spatial quadrature weights per direction [e * nq + g]
  const int *hi[3];             // left Greville node of each 1D Gauss point
  const double *hl[3];          // weight of the right node
  const double *V;              // rank factors [N_s][Rt]
  const double *cf;             // scale of each rank term [Rt]
  const float2 *Tb;             // rank time bands [Rt][P+1][N_t], pairs
  int Rt;
  const double *V2, *cf2;       // a second list of rank terms ([N_s][R2], [R2]; the low-rank reaction)
  const float2 *Tb2;            // [R2][P+1][N_t]
  int R2;
  int exact;                    // M_R from u^k, w^k at the Gauss points
  int newton;                   // C_J instead of C_r
  double c1, c2, a;
  int d, nel, Nt, nel_t;
  int n[3], Q[3];
  long long rows;
  int seglen;
};

template <typename T, int P>
__global__ void __launch_bounds__(kLeanMaxThreads) xlean_kernel(LeanArgs<T> a) {
  typedef typename LeanCT<T>::type CT;
  constexpr int nq = P + 1, S = kLeanRing;
  __shared__ CT xch[2][kLeanMaxThreads / 32][P][P];   // [step parity][warp][a-1][lane-(32-P)]
  extern __shared__ __align__(16) unsigned char lean_raw[];
  const int nth = blockDim.x;
  const bool exact = a.exact != 0;
  const int nx = a.nel + P;
  const int rs = max(nth, (nx + 3) / 4 * 4);   // ring row stride: all n_x coefficients of a row
  T *xr = reinterpret_cast<T *>(lean_raw);                                    // [S][rs]
  float2 *ur = reinterpret_cast<float2 *>(lean_raw + (size_t)S * rs * sizeof(T));    // [S][rs]
  float2 *wr = ur + (exact ? (size_t)S * rs : 0);                             // [S][rs]
  CT *dsh = reinterpret_cast<CT *>(wr + (exact ? (size_t)S * rs : 0));        // [Rt][nq][nth]
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool owns = t < a.nel;
  const bool last = t == a.nel - 1;            // also writes coefficients n_el .. n_el + P - 1
  const int tail_warp = (a.nel - 1) >> 5;
  const CT zero = ct_zero<CT>();
  CT wv[nq][P + 1];
#pragma unroll
  for (int g = 0; g < nq; ++g)
#pragma unroll
    for (int k = 0; k <= P; ++k) wv[g][k] = owns ? ct_from<CT>(a.tab[((size_t)t * nq + g) * (P + 1) + k]) : zero;
  const CT c1 = ct_from<CT>(a.c1), c2 = ct_from<CT>(a.c2), aa = ct_from<CT>(a.a);
  const CT apl = ct_from<CT>(a.newton ? 2.0 * (1.0 + a.a) : 1.0 + a.a);
  const CT cu2 = ct_from<CT>(a.newton ? 3.0 : 1.0);
  pdl_trigger();
  pdl_wait();   // the tables above are set up before the previous kernel ends
  const long long planeX = a.rows * nx;
  const int nseg = (a.Nt + a.seglen - 1) / a.seglen;
  for (long long blk = blockIdx.x; blk < a.rows * nseg; blk += gridDim.x) {
    const long long o = blk % a.rows;
    const int t0 = (int)(blk / a.rows) * a.seglen, t1 = min(a.Nt, t0 + a.seglen);
    const int gy = a.d >= 2 ? (int)(o % a.Q[1]) : 0;
    const int gz = a.d >= 3 ? (int)(o / a.Q[1]) : 0;
    // quadrature weights and rank factors at this thread's Gauss points
    CT wq[nq];
    {
      double wrow = 1.0, ly = 0.0, lz = 0.0;
      int iy = 0, iz = 0;
      if (a.d >= 2) { wrow *= a.ws[1][gy]; iy = a.hi[1][gy]; ly = a.hl[1][gy]; }
      if (a.d >= 3) { wrow *= a.ws[2][gz]; iz = a.hi[2][gz]; lz = a.hl[2][gz]; }
      const int ncy = a.d >= 2 ? 2 : 1, ncz = a.d >= 3 ? 2 : 1;
#pragma unroll
      for (int g = 0; g < nq; ++g) {
        const int gx = t * nq + g;
        const double wqd = owns ? a.ws[0][gx] * wrow : 0.0;
        wq[g] = ct_from<CT>(wqd);
        const int ix = owns ? a.hi[0][gx] : 0;
        const double lx = owns ? a.hl[0][gx] : 0.0;
        for (int r = 0; r < a.Rt + a.R2; ++r) {
          const bool second = r >= a.Rt;
          const double *V = second ? a.V2 : a.V;
          const int Rl = second ? a.R2 : a.Rt, rl = second ? r - a.Rt : r;
          double th = 0.0;
          for (int cz = 0; cz < ncz; ++cz)
            for (int cy = 0; cy < ncy; ++cy)
              for (int cx = 0; cx < 2; ++cx) {
                const double wgt = (cx ? lx : 1.0 - lx) * (cy ? ly : 1.0 - ly) * (cz ? lz : 1.0 - lz);
                const long long idx = (ix + cx) + (long long)a.n[0] * ((iy + cy) + (long long)a.n[1] * (iz + cz));
                th += wgt * V[idx * Rl + rl];
              }
          const double scale = second ? a.cf2[rl] : a.cf[rl];
          dsh[((size_t)r * nq + g) * nth + t] = ct_from<CT>(owns ? scale * wqd * th : 0.0);
        }
      }
    }
    const int it0 = max(t0 - P, -1);   // replay from it0 (no output before t0)
    const T *xrow = a.X1 + o * nx;
    const float2 *urow = exact ? a.U1 + o * nx : nullptr;
    const float2 *wrow2 = exact ? a.W1 + o * nx : nullptr;
    T *yrow = a.Y1 + o * nx;
    auto interp = [&](const CT (&c)[P + 1], CT (&out)[nq]) {
#pragma unroll
      for (int g = 0; g < nq; ++g) {
        CT v = zero;
#pragma unroll
        for (int k = 0; k <= P; ++k) v = ct_fma(wv[g][k], c[k], v);
        out[g] = v;
      }
    };
    // windows: xw[k][g] = X(row it + k) at Gauss point g of this element
    CT xw[P + 1][nq], uw[P + 1][nq], ww[P + 1][nq];
#pragma unroll
    for (int k = 1; k <= P; ++k) {
      const int row = it0 + k - 1;
      const bool ok = owns && row >= 0 && row < a.Nt;
      CT c[P + 1];
#pragma unroll
      for (int j = 0; j <= P; ++j) c[j] = ok ? ct_from<CT>(xrow[(long long)row * planeX + t + j]) : zero;
      interp(c, xw[k]);
      if (exact) {
#pragma unroll
        for (int j = 0; j <= P; ++j) c[j] = ok ? from_pair<CT>(urow[(long long)row * planeX + t + j]) : zero;
        interp(c, uw[k]);
#pragma unroll
        for (int j = 0; j <= P; ++j) c[j] = ok ? from_pair<CT>(wrow2[(long long)row * planeX + t + j]) : zero;
        interp(c, ww[k]);
      } else {
#pragma unroll
        for (int g = 0; g < nq; ++g) uw[k][g] = ww[k][g] = zero;
      }
    }
    CT acc[P][nq];   // contributions owed to rows it+1 .. it+P
#pragma unroll
    for (int k = 0; k < P; ++k)
#pragma unroll
      for (int g = 0; g < nq; ++g) acc[k][g] = zero;
    // step it reads row it + P from ring slot (it - it0) % S
    auto issue = [&](int it) {
      const int row = it + P;
      if (it < t1 && row < a.Nt) {
        const int sl = (it - it0) % S;
        for (int cx = t; cx < nx; cx += nth) {
          lean_cp_async<(int)sizeof(T)>(xr + (size_t)sl * rs + cx, xrow + (long long)row * planeX + cx);
          if (exact) {
            lean_cp_async<8>(ur + (size_t)sl * rs + cx, urow + (long long)row * planeX + cx);
            lean_cp_async<8>(wr + (size_t)sl * rs + cx, wrow2 + (long long)row * planeX + cx);
          }
        }
      }
      lean_commit();
    };
#pragma unroll
    for (int u = 0; u < S - 1; ++u) issue(it0 + u);
    CT pend = zero;   // this thread's output of the previous step before its cross-warp part
    CT tail[P];       // the last element's thread: coefficients n_el - 1 + m, m = 1 .. P, likewise
#pragma unroll
    for (int m = 0; m < P; ++m) tail[m] = zero;
    auto flush = [&](int itf) {
      const int pp = itf & 1;
      if (lane < P && warp > 0) {
#pragma unroll
        for (int k = 1; k <= P; ++k)
          if (k > lane) pend = ct_add(pend, xch[pp][warp - 1][k - 1][lane + P - k]);
      }
      if (owns) ct_store(yrow + (long long)itf * planeX + t, pend);
      if (last) {
        // coefficient n_el - 1 + m takes c[k] of element n_el - 1 - (k - m), k >= m;
        // those in the previous warp are in its exchange slots
#pragma unroll
        for (int m = 1; m <= P; ++m) {
          CT v = tail[m - 1];
          if (warp > 0) {
#pragma unroll
            for (int k = m + 1; k <= P; ++k)
              if (k - m > lane) v = ct_add(v, xch[pp][warp - 1][k - 1][lane - (k - m) + P]);
          }
          ct_store(yrow + (long long)itf * planeX + a.nel - 1 + m, v);
        }
      }
    };
    for (int it = it0; it < t1; ++it) {
      lean_wait<S - 2>();
      __syncthreads();
      if (it > t0) flush(it - 1);
      issue(it + S - 1);
      // slide the windows and bring in row it + P
#pragma unroll
      for (int k = 0; k < P; ++k)
#pragma unroll
        for (int g = 0; g < nq; ++g) { xw[k][g] = xw[k + 1][g]; uw[k][g] = uw[k + 1][g]; ww[k][g] = ww[k + 1][g]; }
      {
        const int sl = (it - it0) % S;
        const bool ok = owns && it + P < a.Nt;
        CT c[P + 1];
#pragma unroll
        for (int j = 0; j <= P; ++j) c[j] = ok ? ct_from<CT>(xr[(size_t)sl * rs + t + j]) : zero;
        interp(c, xw[P]);
        if (exact) {
#pragma unroll
          for (int j = 0; j <= P; ++j) c[j] = ok ? from_pair<CT>(ur[(size_t)sl * rs + t + j]) : zero;
          interp(c, uw[P]);
#pragma unroll
          for (int j = 0; j <= P; ++j) c[j] = ok ? from_pair<CT>(wr[(size_t)sl * rs + t + j]) : zero;
          interp(c, ww[P]);
        }
      }
      CT yq[nq];
#pragma unroll
      for (int g = 0; g < nq; ++g) yq[g] = acc[0][g];
      if (a.Rt + a.R2 > 0 && it >= 0) {
        // band of row it: b[k][g] = T_q(it, it + k) = sum_r d_r(q) Tb[r][k][it]
        CT b[P + 1][nq];
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
          for (int g = 0; g < nq; ++g) b[k][g] = zero;
        for (int r = 0; r < a.Rt + a.R2; ++r) {
          const float2 *tb = r < a.Rt ? a.Tb + (size_t)r * (P + 1) * a.Nt : a.Tb2 + (size_t)(r - a.Rt) * (P + 1) * a.Nt;
          CT tk[P + 1];
#pragma unroll
          for (int k = 0; k <= P; ++k) tk[k] = from_pair<CT>(__ldg(tb + (size_t)k * a.Nt + it));
#pragma unroll
          for (int g = 0; g < nq; ++g) {
            const CT dv = dsh[((size_t)r * nq + g) * nth + t];
#pragma unroll
            for (int k = 0; k <= P; ++k) b[k][g] = ct_fma(dv, tk[k], b[k][g]);
          }
        }
#pragma unroll
        for (int g = 0; g < nq; ++g)
#pragma unroll
          for (int k = 0; k <= P; ++k) yq[g] = ct_fma(b[k][g], xw[k][g], yq[g]);
#pragma unroll
        for (int k = 0; k < P - 1; ++k)
#pragma unroll
          for (int g = 0; g < nq; ++g) acc[k][g] = ct_fma(b[k + 1][g], xw[0][g], acc[k + 1][g]);
#pragma unroll
        for (int g = 0; g < nq; ++g) acc[P - 1][g] = ct_fma(b[P][g], xw[0][g], zero);
      } else {
#pragma unroll
        for (int k = 0; k < P - 1; ++k)
#pragma unroll
          for (int g = 0; g < nq; ++g) acc[k][g] = acc[k + 1][g];
#pragma unroll
        for (int g = 0; g < nq; ++g) acc[P - 1][g] = zero;
      }
      // M_R on time element e = it + 1, whose local functions are rows it .. it + P
      const int e = it + 1;
      if (exact && e < a.nel_t) {
#pragma unroll
        for (int gt = 0; gt < nq; ++gt) {
          CT bv[P + 1];
#pragma unroll
          for (int k = 0; k <= P; ++k) bv[k] = from_pair<CT>(__ldg(a.bt + ((size_t)e * nq + gt) * (P + 1) + k));
          const CT wtt = from_pair<CT>(__ldg(a.wt + (size_t)e * nq + gt));
#pragma unroll
          for (int g = 0; g < nq; ++g) {
            CT xv = zero, uv = zero, wvv = zero;
#pragma unroll
            for (int k = 0; k <= P; ++k) {
              xv = ct_fma(bv[k], xw[k][g], xv);
              uv = ct_fma(bv[k], uw[k][g], uv);
              wvv = ct_fma(bv[k], ww[k][g], wvv);
            }
            // C_r = c1 ((u - (1 + a)) u + a) + c2 w, C_J = c1 ((3u - 2(1 + a)) u + a) + c2 w
            const CT C = ct_fma(c1, ct_fma(ct_fma(cu2, uv, ct_neg(apl)), uv, aa), ct_mul(c2, wvv));
            const CT sv = ct_mul(ct_mul(wtt, wq[g]), ct_mul(C, xv));
            yq[g] = ct_fma(bv[0], sv, yq[g]);
#pragma unroll
            for (int k = 1; k <= P; ++k) acc[k - 1][g] = ct_fma(bv[k], sv, acc[k - 1][g]);
          }
        }
      }
      // contributions of this element to the coefficients t .. t + P of row it
      CT c[P + 1];
#pragma unroll
      for (int k = 0; k <= P; ++k) {
        CT v = zero;
#pragma unroll
        for (int g = 0; g < nq; ++g) v = ct_fma(wv[g][k], yq[g], v);
        c[k] = v;
      }
      CT out = c[0];
#pragma unroll
      for (int k = 1; k <= P; ++k) {
        CT v = ct_shfl_up(c[k], k);
        if (lane >= k) out = ct_add(out, v);
      }
      if (warp == tail_warp) {   // warp-uniform: the shuffles below need the whole warp
#pragma unroll
        for (int m = 1; m <= P; ++m) {
          CT v = c[m];
#pragma unroll
          for (int k = m + 1; k <= P; ++k) {
            CT sv = ct_shfl_up(c[k], k - m);
            if (lane >= k - m) v = ct_add(v, sv);
          }
          tail[m - 1] = v;
        }
      }
      if (lane >= 32 - P) {
#pragma unroll
        for (int k = 1; k <= P; ++k) xch[it & 1][warp][k - 1][lane - (32 - P)] = c[k];
      }
      pend = out;
    }
    lean_wait<0>();
    __syncthreads();
    if (t1 > t0) flush(t1 - 1);
    __syncthreads();   // the next segment reuses the ring and xch
  }
}

// Dynamic shared memory of any lean launch (xlean_max_rank keeps it below):
// the opt-in is set once per device to this bound, so that every later launch
// of the instance fits whatever its rank.
constexpr int kLeanSmemMax = 200 * 1024;

template <typename T, int P>
st_status launch_p(cudaStream_t s, const LeanArgs<T> &a, int threads, size_t smem, unsigned grid) {
  static std::atomic<unsigned long long> optin{0};
  if (smem > (size_t)kLeanSmemMax) return ST_ERR_CAPACITY;
  cudaError_t e = smem_optin(xlean_kernel<T, P>, kLeanSmemMax, optin);
  if (e != cudaSuccess) {
    st_note_cuda_error(e, __FILE__, __LINE__);
    return ST_ERR_CUDA;
  }
  st_count_launch();
  e = pdl_launch(xlean_kernel<T, P>, dim3(grid), dim3(threads), smem, s, a);
  if (e != cudaSuccess) {
    st_note_cuda_error(e, __FILE__, __LINE__);
    return ST_ERR_CUDA;
  }
  return ST_OK;
}

}  // namespace

int xlean_threads(int nel, int p) { (void)p; return (nel + 31) / 32 * 32; }

bool xlean_feasible(int nel, int p) { return xlean_threads(nel, p) <= kLeanMaxThreads; }

size_t xlean_smem(int nel, int p, int rank, bool exact, bool pairs) {
  const size_t nth = (size_t)xlean_threads(nel, p);
  const size_t rs = std::max(nth, (size_t)(nel + p + 3) / 4 * 4);   // ring row stride, as in the kernel
  const size_t elem = pairs ? 8 : 4;
  return (size_t)kLeanRing * rs * (elem + (exact ? 16 : 0)) + (size_t)rank * (p + 1) * nth * elem;
}

int xlean_max_rank(int nel, int p, bool exact) {
  // the dynamic shared memory of a block stays within kLeanSmemMax in both precisions
  const size_t base = xlean_smem(nel, p, 0, exact, true);
  const size_t per = xlean_smem(nel, p, 1, exact, true) - base;
  const size_t lim = kLeanSmemMax;
  return base >= lim ? 0 : (int)((lim - base) / per);
}

template <typename T>
st_status launch_xlean(cudaStream_t s, const LeanTerms &L, T *Y1, const T *X1, const T *tab, long long rows) {
  LeanArgs<T> a;
  a.Y1 = Y1; a.X1 = X1;
  a.U1 = L.U1; a.W1 = L.W1;
  a.tab = tab;
  a.bt = L.bt; a.wt = L.wt;
  for (int l = 0; l < 3; ++l) { a.ws[l] = L.ws[l]; a.hi[l] = L.hi[l]; a.hl[l] = L.hl[l]; a.n[l] = L.n[l]; a.Q[l] = L.Q[l]; }
  a.V = L.V; a.cf = L.cf; a.Tb = L.Tb; a.Rt = L.Rt;
  a.V2 = L.V2; a.cf2 = L.cf2; a.Tb2 = L.Tb2; a.R2 = L.R2;
  a.exact = L.exact; a.newton = L.newton;
  a.c1 = L.c1; a.c2 = L.c2; a.a = L.a;
  a.d = L.d; a.nel = L.nel; a.Nt = L.Nt; a.nel_t = L.nel_t;
  a.rows = rows;
  const int p = L.p;
  const int threads = xlean_threads(L.nel, p);
  if (threads > kLeanMaxThreads || rows < 1) return ST_ERR_ARG;
  if (L.Rt + L.R2 > xlean_max_rank(L.nel, p, L.exact != 0)) return ST_ERR_CAPACITY;
  const size_t smem = xlean_smem(L.nel, p, L.Rt + L.R2, L.exact != 0, sizeof(T) == 8);
  // time segments: enough blocks for about four per SM, each at least 4p steps
  const long long want = 152LL * 4;
  int nseg = (int)std::max<long long>(1, std::min<long long>((want + rows - 1) / rows, L.Nt / std::max(4 * p, 1)));
  nseg = std::max(nseg, 1);
  a.seglen = (L.Nt + nseg - 1) / nseg;
  const long long total = rows * (long long)((L.Nt + a.seglen - 1) / a.seglen);
  const unsigned grid = (unsigned)std::min<long long>(total, 152LL * 64);
  switch (p) {
    case 1: return launch_p<T, 1>(s, a, threads, smem, grid);
    case 2: return launch_p<T, 2>(s, a, threads, smem, grid);
    case 3: return launch_p<T, 3>(s, a, threads, smem, grid);
    default: return launch_p<T, 4>(s, a, threads, smem, grid);
  }
}

template st_status launch_xlean<float>(cudaStream_t, const LeanTerms &, float *, const float *, const float *, long long);
template st_status launch_xlean<float2>(cudaStream_t, const LeanTerms &, float2 *, const float2 *, const float2 *,
                                        long long);
