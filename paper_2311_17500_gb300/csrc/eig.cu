// Symmetric (generalized) eigendecompositions on the device:
//  * the pencils (D_ll K_l, M_l) of the fast-diagonalization preconditioner
//    (Sec. 3.2: M_l-orthonormal generalized eigenvectors U_l, eigenvalues);
//  * the Gram matrix Theta-hat Theta-hat^T of the low-rank step (Eq. tol).
//
// Method: a parallel cyclic Jacobi method in FP32 on one thread block
// (round-robin pairing, all n/2 disjoint rotations of a round applied at
// once) gives eigenvectors to single precision; FP64 accuracy is then reached
// by the iterative refinement of Ogita and Aishima (Japan J. Indust. Appl.
// Math. 35, 2018), generalized to B-orthonormal eigenvectors:
//     R = I - X^T B X,  S = X^T A X,  lam_i = s_ii / (1 - r_ii),
//     E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i)  if |lam_i - lam_j| > delta,
//            r_ij / 2                                otherwise,
//     X <- X + X E,     delta = 2 (||S - diag(lam)|| + ||A|| ||R||),
// whose products run as FP64 GEMMs on the whole GPU.
#include <algorithm>
#include <cmath>
#include <vector>
#include <cooperative_groups.h>
#include "st_internal.h"

namespace cg = cooperative_groups;

void launch_gemm64(cudaStream_t s, double *C, const double *A, const double *X, int M, int N, int K,
                   long long sam, long long sak, long long sbk, long long sbc, long long scm, long long scc,
                   double alpha, double beta, double *work = nullptr, long long work_elems = 0);

namespace {

constexpr int kJacThreads = 1024;

// One-block cyclic Jacobi on the dense symmetric n x n matrix A (row-major,
// overwritten) accumulating eigenvectors in V (V[i*n + c] = i-th component of
// eigenvector c).  Rotations below `tol` * ||A||_F are skipped; the sweep loop
// stops after a sweep without rotations or after max_sweeps (bounded).
template <typename T>
__global__ void __launch_bounds__(kJacThreads) jacobi_kernel(T *A, T *V, int n, int max_sweeps, double tol,
                                                            int *sweeps_out) {
  extern __shared__ unsigned char smem_raw[];
  const int m = n + (n & 1);
  const int half = m / 2;
  T *cs = (T *)smem_raw;            // [half] cosines
  T *sn = cs + half;                // [half] sines
  int *pp = (int *)(sn + half);     // [half]
  int *qq = pp + half;              // [half]
  __shared__ int rotated;
  __shared__ double fro;
  int tid = threadIdx.x;
  for (int i = tid; i < n * n; i += blockDim.x) V[i] = (i / n == i % n) ? T(1) : T(0);
  if (tid == 0) fro = 0.0;
  __syncthreads();
  double loc = 0.0;
  for (int i = tid; i < n * n; i += blockDim.x) loc += (double)A[i] * (double)A[i];
  atomicAdd(&fro, loc);
  __syncthreads();
  const double thr = tol * sqrt(fro);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < m - 1; ++round) {
      // round-robin: position 0 fixed, positions 1..m-1 rotate by `round`
      for (int i = tid; i < half; i += blockDim.x) {
        int a = (i == 0) ? 0 : 1 + ((i - 1 + round) % (m - 1));
        int b = 1 + ((m - 2 - i + round) % (m - 1));
        int p = min(a, b), q = max(a, b);
        T c = T(1), s = T(0);
        if (q < n) {
          T apq = A[p * n + q];
          if (fabs((double)apq) > thr) {
            T app = A[p * n + p], aqq = A[q * n + q];
            T tau = (aqq - app) / (T(2) * apq);
            T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
            c = T(1) / sqrt(T(1) + t * t);
            s = t * c;
            rotated = 1;
          }
        }
        pp[i] = p; qq[i] = q; cs[i] = c; sn[i] = s;
      }
      __syncthreads();
      // rows p, q of A  (A <- J^T A)
      for (int idx = tid; idx < half * n; idx += blockDim.x) {
        int i = idx / n, k = idx % n;
        int p = pp[i], q = qq[i];
        if (q >= n || sn[i] == T(0)) continue;
        T c = cs[i], s = sn[i];
        T ap = A[p * n + k], aq = A[q * n + k];
        A[p * n + k] = c * ap - s * aq;
        A[q * n + k] = s * ap + c * aq;
      }
      __syncthreads();
      // columns p, q of A and V  (A <- A J, V <- V J)
      for (int idx = tid; idx < half * n; idx += blockDim.x) {
        int i = idx / n, k = idx % n;
        int p = pp[i], q = qq[i];
        if (q >= n || sn[i] == T(0)) continue;
        T c = cs[i], s = sn[i];
        T ap = A[k * n + p], aq = A[k * n + q];
        A[k * n + p] = c * ap - s * aq;
        A[k * n + q] = s * ap + c * aq;
        T vp = V[k * n + p], vq = V[k * n + q];
        V[k * n + p] = c * vp - s * vq;
        V[k * n + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// The same cyclic Jacobi spread over a thread-block cluster: every block
// computes the rotations of a round redundantly (identical data, identical
// results), then block r applies the row updates of the pairs i = r mod CL and
// the column updates of its slice of rows, the matrix staying in global
// memory (L2).  Three cluster barriers per round; the number of sweeps is
// bounded by max_sweeps.  `thr` is the absolute skip threshold.
template <typename T>
__global__ void __launch_bounds__(kJacThreads) jacobi_cluster_kernel(T *A, T *V, int n, int max_sweeps, double thr) {
  extern __shared__ unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int m = n + (n & 1);
  const int half = m / 2;
  T *cs = (T *)smem_raw;
  T *sn = cs + half;
  int *pp = (int *)(sn + half);
  int *qq = pp + half;
  __shared__ int rotated;
  const int tid = threadIdx.x;
  const int r0 = (int)((long long)n * rank / CL), r1 = (int)((long long)n * (rank + 1) / CL);
  for (int i = r0 * n + tid; i < r1 * n; i += blockDim.x) V[i] = (i / n == i % n) ? T(1) : T(0);
  cluster.sync();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < m - 1; ++round) {
      for (int i = tid; i < half; i += blockDim.x) {
        int a = (i == 0) ? 0 : 1 + ((i - 1 + round) % (m - 1));
        int b = 1 + ((m - 2 - i + round) % (m - 1));
        int p = min(a, b), q = max(a, b);
        T c = T(1), s = T(0);
        if (q < n) {
          T apq = A[p * n + q];
          if (fabs((double)apq) > thr) {
            T app = A[p * n + p], aqq = A[q * n + q];
            T tau = (aqq - app) / (T(2) * apq);
            T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
            c = T(1) / sqrt(T(1) + t * t);
            s = t * c;
            rotated = 1;
          }
        }
        pp[i] = p; qq[i] = q; cs[i] = c; sn[i] = s;
      }
      cluster.sync();   // everyone has read the pivots before rows change
      for (int idx = tid; idx < half * n; idx += blockDim.x) {
        int i = idx / n, k = idx % n;
        if (i % CL != rank) continue;
        int p = pp[i], q = qq[i];
        if (q >= n || sn[i] == T(0)) continue;
        T c = cs[i], s = sn[i];
        T ap = A[p * n + k], aq = A[q * n + k];
        A[p * n + k] = c * ap - s * aq;
        A[q * n + k] = s * ap + c * aq;
      }
      cluster.sync();
      int rows = r1 - r0;
      for (int idx = tid; idx < half * rows; idx += blockDim.x) {
        int i = idx / rows, k = r0 + idx % rows;
        int p = pp[i], q = qq[i];
        if (q >= n || sn[i] == T(0)) continue;
        T c = cs[i], s = sn[i];
        T ap = A[k * n + p], aq = A[k * n + q];
        A[k * n + p] = c * ap - s * aq;
        A[k * n + q] = s * ap + c * aq;
        T vp = V[k * n + p], vq = V[k * n + q];
        V[k * n + p] = c * vp - s * vq;
        V[k * n + q] = s * vp + c * vq;
      }
      cluster.sync();
    }
    if (!rotated) break;
    __syncthreads();
  }
}

__global__ void d2f_kernel(float *y, const double *x, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = (float)x[e];
}
__global__ void f2d_kernel(double *y, const float *x, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = (double)x[e];
}

// Dense symmetric matrix from a band (n x (2p+1)), times a scalar.
__global__ void band_to_dense_kernel(double *out, const double *band, int n, int p, double scale) {
  int B = 2 * p + 1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    int k = j - i + p;
    out[e] = (k >= 0 && k < B) ? scale * band[(size_t)i * B + k] : 0.0;
  }
}

// Banded Cholesky M = L L^T (one thread; n (p+1)^2 work); L stored as
// L[i][k] = L(i, i-p+k), k = 0..p.
__global__ void chol_band_kernel(double *L, const double *M, int n, int p, int *fail) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int B = 2 * p + 1, W = p + 1;
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k <= p; ++k) {
      int j = i - p + k;
      if (j < 0) { L[i * W + k] = 0.0; continue; }
      double s = M[(size_t)i * B + k];   // M(i, j), j <= i
      for (int m = max(0, i - p); m < j; ++m) {
        if (m < j - p) continue;
        s -= L[i * W + (m - i + p)] * L[j * W + (m - j + p)];
      }
      if (j < i) {
        L[i * W + k] = s / L[j * W + p];
      } else {
        if (!(s > 0.0)) { *fail = 1; s = 1.0; }
        L[i * W + p] = sqrt(s);
      }
    }
  }
}

// out[:, c] = L^{-1} v_c with v_c = in[:, c] (trans = 0) or in[c, :] (trans = 1).
__global__ void lower_solve_cols_kernel(double *out, const double *in, const double *L, int n, int p, int trans) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  int W = p + 1;
  for (int i = 0; i < n; ++i) {
    double s = trans ? in[(size_t)c * n + i] : in[(size_t)i * n + c];
    for (int m = max(0, i - p); m < i; ++m) s -= L[i * W + (m - i + p)] * out[(size_t)m * n + c];
    out[(size_t)i * n + c] = s / L[i * W + p];
  }
}

// out[:, c] = L^{-T} in[:, c]
__global__ void upper_solve_cols_kernel(double *out, const double *in, const double *L, int n, int p) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  int W = p + 1;
  for (int i = n - 1; i >= 0; --i) {
    double s = in[(size_t)i * n + c];
    for (int m = i + 1; m <= min(n - 1, i + p); ++m) s -= L[m * W + (i - m + p)] * out[(size_t)m * n + c];
    out[(size_t)i * n + c] = s / L[i * W + p];
  }
}

__global__ void symmetrize_kernel(double *A, int n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    if (i < j) {
      double v = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
      A[(size_t)i * n + j] = v;
      A[(size_t)j * n + i] = v;
    }
  }
}

// Norms for the refinement threshold: out[0] = ||S - diag(lam)||_F,
// out[1] = ||R||_F, with lam_i = s_ii / rm_ii and R = I - Rm.
__global__ void refine_norms_kernel(double *out, const double *S, const double *Rm, int n) {
  __shared__ double a[1024], b[1024];
  double sa = 0.0, sb = 0.0;
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    double r = (i == j ? 1.0 : 0.0) - Rm[e];
    sb += r * r;
    if (i != j) sa += S[e] * S[e];
  }
  a[threadIdx.x] = sa;
  b[threadIdx.x] = sb;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) { a[threadIdx.x] += a[threadIdx.x + off]; b[threadIdx.x] += b[threadIdx.x + off]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = sqrt(a[0]); out[1] = sqrt(b[0]); }
}

// E from S, Rm (see the file comment); lam written to lam_out.
__global__ void refine_E_kernel(double *E, const double *S, const double *Rm, double *lam_out, int n,
                                const double *norms, double normA) {
  double delta = 2.0 * (norms[0] + normA * norms[1]);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    double li = S[(size_t)i * n + i] / Rm[(size_t)i * n + i];
    double lj = S[(size_t)j * n + j] / Rm[(size_t)j * n + j];
    double r = (i == j ? 1.0 : 0.0) - Rm[e];
    double v;
    if (i != j && fabs(li - lj) > delta)
      v = (S[e] + lj * r) / (lj - li);
    else
      v = 0.5 * r;
    E[e] = v;
    if (i == j) lam_out[i] = li;
  }
}

__global__ void add_kernel(double *y, const double *x, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] += x[e];
}

// Descending order of lam (ties by index): rank[i]; then gather columns.
__global__ void sort_desc_kernel(double *lam_sorted, double *Xs, const double *lam, const double *X, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double li = lam[i];
    int r = 0;
    for (int j = 0; j < n; ++j) r += (lam[j] > li) || (lam[j] == li && j < i);
    lam_sorted[r] = li;
    for (int k = 0; k < n; ++k) Xs[(size_t)k * n + r] = X[(size_t)k * n + i];
  }
}

__global__ void transpose_kernel(double *out, const double *in, int n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    out[(size_t)j * n + i] = in[e];
  }
}

// One banded LU (no pivoting) of C_m W_t + (mu_j + a c1) M_t per spatial
// eigen-index j, row by row with the previous p U-rows in registers.
template <int P>
__global__ void fd_lu_kernel(double *lu, const double *Wt, const double *Mt, const double *mu, double Cm,
                             double shift, int Nt, long long Ns, int *fail) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= Ns) return;
  constexpr int B = 2 * P + 1;
  double sig = mu[j] + shift;
  double U[P][P + 1];   // U rows it-P .. it-1: U(row, row + c), c = 0..P
#pragma unroll
  for (int r = 0; r < P; ++r)
#pragma unroll
    for (int c = 0; c <= P; ++c) U[r][c] = 0.0;
  for (int it = 0; it < Nt; ++it) {
    double w[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      int col = it - P + k;
      w[k] = (col >= 0 && col < Nt) ? Cm * Wt[(size_t)it * B + k] + sig * Mt[(size_t)it * B + k] : 0.0;
    }
    // eliminate columns it-P .. it-1 using the stored U rows
#pragma unroll
    for (int k = 0; k < P; ++k) {
      int col = it - P + k;
      if (col < 0) continue;
      const double *urow = U[k];          // row `col` = it-P+k
      double l = w[k] * urow[0];          // urow[0] holds 1/u(col,col)
      w[k] = l;
#pragma unroll
      for (int c = 1; c <= P; ++c)
        if (k + c < B) w[k + c] -= l * urow[c];
    }
    double piv = w[P];
    if (!(fabs(piv) > 0.0) || piv != piv) { atomicExch(fail, 1); piv = 1.0; }
    w[P] = 1.0 / piv;
#pragma unroll
    for (int k = 0; k < B; ++k) lu[((long long)it * B + k) * Ns + j] = w[k];
#pragma unroll
    for (int r = 0; r < P - 1; ++r)
#pragma unroll
      for (int c = 0; c <= P; ++c) U[r][c] = U[r + 1][c];
#pragma unroll
    for (int c = 0; c <= P; ++c) U[P - 1][c] = w[P + c];
  }
}

// mu_j = sum_l lam_l[j_l]
__global__ void mu_kernel(double *mu, const double *l0, const double *l1, const double *l2, int n0, int n1,
                          int d, long long Ns) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < Ns; j += (long long)gridDim.x * blockDim.x) {
    int j0 = (int)(j % n0);
    double v = l0[j0];
    if (d > 1) v += l1[(j / n0) % n1];
    if (d > 2) v += l2[j / ((long long)n0 * n1)];
    mu[j] = v;
  }
}

inline int grid_for(long long total, int threads = 256) {
  long long g = (total + threads - 1) / threads;
  if (g > 152LL * 64) g = 152LL * 64;
  if (g < 1) g = 1;
  return (int)g;
}

// Dense or banded operand of the refinement products.
struct Op {
  const double *dense = nullptr;   // n x n
  const double *band = nullptr;    // n x (2p+1)
  double scale = 1.0;
};

void op_apply(cudaStream_t s, const Op &op, int n, int p, const double *X, double *Y) {
  if (op.dense) {
    launch_gemm64(s, Y, op.dense, X, n, n, n, n, 1, n, 1, n, 1, op.scale, 0.0);
  } else if (op.band) {
    const double *bands[1] = {op.band};
    const double *ins[1] = {X};
    double coefs[1] = {op.scale};
    launch_band_pass<double>(s, Y, 1, bands, ins, coefs, n, n, 1, p, false);
  } else {
    cudaMemcpyAsync(Y, X, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
}

// Refine X (n x n) in place for A x = lam B x; lam written to `lam`.
st_status refine(st_handle *h, const Op &A, const Op &B, int n, double normA, double *X, double *lam, int iters,
                 double *work) {
  cudaStream_t s = h->stream;
  size_t nn = (size_t)n * n;
  double *AX = work, *BX = work + nn, *S = work + 2 * nn, *Rm = work + 3 * nn, *E = work + 4 * nn,
         *XE = work + 5 * nn, *norms = work + 6 * nn;
  for (int it = 0; it < iters; ++it) {
    op_apply(s, A, n, h->p, X, AX);
    op_apply(s, B, n, h->p, X, BX);
    // S = X^T AX, Rm = X^T BX
    launch_gemm64(s, S, X, AX, n, n, n, 1, n, n, 1, n, 1, 1.0, 0.0);
    launch_gemm64(s, Rm, X, BX, n, n, n, 1, n, n, 1, n, 1, 1.0, 0.0);
    st_count_launch(); refine_norms_kernel<<<1, 1024, 0, s>>>(norms, S, Rm, n);
    st_count_launch(); refine_E_kernel<<<grid_for(nn), 256, 0, s>>>(E, S, Rm, lam, n, norms, normA);
    launch_gemm64(s, XE, X, E, n, n, n, n, 1, n, 1, n, 1, 1.0, 0.0);
    st_count_launch(); add_kernel<<<grid_for(nn), 256, 0, s>>>(X, XE, nn);
  }
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

double host_fro(cudaStream_t s, const double *A, size_t nn) {
  std::vector<double> hA(nn);
  cudaMemcpyAsync(hA.data(), A, nn * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  double f = 0.0;
  for (double v : hA) f += v * v;
  return std::sqrt(f);
}

st_status jacobi32(st_handle *h, const double *A64, int n, double *X64) {
  cudaStream_t s = h->stream;
  size_t nn = (size_t)n * n;
  float *A32 = h->eig32, *V32 = h->eig32 + nn;
  st_count_launch(); d2f_kernel<<<grid_for(nn), 256, 0, s>>>(A32, A64, nn);
  int m = n + (n & 1);
  size_t sh = (size_t)(m / 2) * (2 * sizeof(float) + 2 * sizeof(int));
  if (n < 96) {
    st_count_launch(); jacobi_kernel<float><<<1, kJacThreads, sh, s>>>(A32, V32, n, 30, 2e-7, nullptr);
  } else {
    double thr = 2e-7 * host_fro(s, A64, nn);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 8;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(8, 1, 1);
    cfg.blockDim = dim3(kJacThreads, 1, 1);
    cfg.dynamicSmemBytes = sh;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    st_count_launch();
    ST_CUDA(cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<float>, A32, V32, n, 30, thr));
  }
  st_count_launch(); f2d_kernel<<<grid_for(nn), 256, 0, s>>>(X64, V32, nn);
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}



// ---------------------------------------------------------------------------
// Lanczos with full reorthogonalization for the leading eigenpairs of the
// Gram matrix (symmetric positive semidefinite, FP64, one thread block, the
// matrix read from L2).  Steps j = j0 .. j1-1 extend the orthonormal basis
// Q (rows q_0 .. q_j1) and the tridiagonal T (alpha_j on the diagonal, beta_j
// coupling j and j+1); the new vector is orthogonalized against all earlier
// ones by classical Gram-Schmidt applied twice.  A step whose beta does not
// exceed `tiny` has found an invariant subspace: the run stops there and
// *kdone = j+1 (else j1).  All reductions are in a fixed order.
constexpr int kLzThreads = 1024;

__device__ __forceinline__ double lz_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; every thread receives the same value.
__device__ double lz_block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = lz_warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  return lz_warp_sum(lane < nw ? red[lane] : 0.0);
}

__global__ void __launch_bounds__(kLzThreads) lanczos_kernel(const double *__restrict__ G, int n, double *Q,
                                                             double *alpha, double *beta, int j0, int j1,
                                                             double tiny, int *kdone) {
  extern __shared__ double lz_sh[];
  double *w = lz_sh;        // [n]
  double *hc = lz_sh + n;   // [j1 + 1] Gram-Schmidt coefficients
  __shared__ double red[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = j0; j < j1; ++j) {
    const double *qj = Q + (size_t)j * n;
    for (int i = warp; i < n; i += nw) {
      const double *gr = G + (size_t)i * n;
      double v = 0.0;
      for (int c = lane; c < n; c += 32) v += gr[c] * qj[c];
      v = lz_warp_sum(v);
      if (lane == 0) w[i] = v;
    }
    __syncthreads();
    if (j > 0) {
      const double *qp = Q + (size_t)(j - 1) * n;
      const double b = beta[j - 1];
      for (int i = tid; i < n; i += blockDim.x) w[i] -= b * qp[i];
    }
    __syncthreads();
    double part = 0.0;
    for (int i = tid; i < n; i += blockDim.x) part += qj[i] * w[i];
    const double a = lz_block_sum(part, red);
    for (int i = tid; i < n; i += blockDim.x) w[i] -= a * qj[i];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int m = warp; m <= j; m += nw) {
        const double *qm = Q + (size_t)m * n;
        double v = 0.0;
        for (int i = lane; i < n; i += 32) v += qm[i] * w[i];
        v = lz_warp_sum(v);
        if (lane == 0) hc[m] = v;
      }
      __syncthreads();
      for (int i = tid; i < n; i += blockDim.x) {
        double v = w[i];
        for (int m = 0; m <= j; ++m) v -= hc[m] * Q[(size_t)m * n + i];
        w[i] = v;
      }
      __syncthreads();
    }
    part = 0.0;
    for (int i = tid; i < n; i += blockDim.x) part += w[i] * w[i];
    const double b = sqrt(lz_block_sum(part, red));
    if (tid == 0) { alpha[j] = a; beta[j] = b; }
    if (!(b > tiny)) {
      if (tid == 0) *kdone = j + 1;
      return;
    }
    double *qn = Q + (size_t)(j + 1) * n;
    const double inv = 1.0 / b;
    for (int i = tid; i < n; i += blockDim.x) qn[i] = w[i] * inv;
    __syncthreads();
  }
  if (tid == 0) *kdone = j1;
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x (Sturm
// sequence of the LDL^T pivots of T - x I).
int sturm_below(int k, const double *d, const double *e, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < k; ++i) {
    q = (d[i] - x) - (i > 0 ? e[i - 1] * e[i - 1] / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// r-th largest eigenvalue (r = 1..k) of the tridiagonal by bisection on the
// Sturm count, to full double precision.
double tridiag_eig_bisect(int k, const double *d, const double *e, int r, double lo, double hi) {
  for (int it = 0; it < 400 && hi - lo > 4e-16 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_below(k, d, e, mid) >= k - r + 1) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Eigenvector of the tridiagonal for the eigenvalue th by inverse iteration:
// three solves with T - th I, each followed by orthogonalization against
// `prev` (vectors of nearby eigenvalues) and normalization.  The solve is
// Gaussian elimination with partial pivoting, carried as one running row:
// row i of U has entries at columns i, i+1 and (after a row swap) i+2; a zero
// pivot is replaced by a tiny multiple of ||T||.
void tridiag_eigvec(int k, const double *d, const double *e, double th, double tnorm,
                    const std::vector<const double *> &prev, double *y) {
  std::vector<double> U0(k), U1(k), U2(k), z(k);
  const double small = 1e-300 + 1e-15 * tnorm;
  double nrm = 0.0;
  for (int i = 0; i < k; ++i) {
    y[i] = 1.0 + 0.1 * ((i * 7919) % 13);
    nrm += y[i] * y[i];
  }
  for (int i = 0; i < k; ++i) y[i] /= std::sqrt(nrm);
  for (int iter = 0; iter < 3; ++iter) {
    // running row: entries at columns i, i+1 (column i+2 is zero), rhs
    double c0 = d[0] - th, c1 = k > 1 ? e[0] : 0.0, cr = y[0];
    for (int i = 0; i + 1 < k; ++i) {
      const double n0 = e[i], n1 = d[i + 1] - th, n2 = i + 2 < k ? e[i + 1] : 0.0, nr = y[i + 1];
      double p0, p1, p2, pr, o0, o1, o2, orr;
      if (std::fabs(n0) > std::fabs(c0)) {
        p0 = n0; p1 = n1; p2 = n2; pr = nr;
        o0 = c0; o1 = c1; o2 = 0.0; orr = cr;
      } else {
        p0 = c0; p1 = c1; p2 = 0.0; pr = cr;
        o0 = n0; o1 = n1; o2 = n2; orr = nr;
      }
      if (p0 == 0.0) p0 = small;
      U0[i] = p0; U1[i] = p1; U2[i] = p2; z[i] = pr;
      const double m = o0 / p0;
      c0 = o1 - m * p1;
      c1 = o2 - m * p2;
      cr = orr - m * pr;
    }
    U0[k - 1] = c0 == 0.0 ? small : c0;
    U1[k - 1] = 0.0; U2[k - 1] = 0.0; z[k - 1] = cr;
    for (int i = k - 1; i >= 0; --i) {
      double v = z[i];
      if (i + 1 < k) v -= U1[i] * y[i + 1];
      if (i + 2 < k) v -= U2[i] * y[i + 2];
      y[i] = v / U0[i];
    }
    for (const double *pv : prev) {
      double dot = 0.0;
      for (int i = 0; i < k; ++i) dot += pv[i] * y[i];
      for (int i = 0; i < k; ++i) y[i] -= dot * pv[i];
    }
    nrm = 0.0;
    for (int i = 0; i < k; ++i) nrm += y[i] * y[i];
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return;
    for (int i = 0; i < k; ++i) y[i] /= nrm;
  }
}

}  // namespace

// Eigenpairs of the dense symmetric n x n matrix A (device), eigenvalues
// descending in eval, eigenvectors as columns of evec (row-major n x n).
st_status sym_eig_desc(st_handle *h, const double *A, int n, double *evec, double *eval) {
  cudaStream_t s = h->stream;
  size_t nn = (size_t)n * n;
  double *X = h->eig_work, *lam = h->eig_work + nn, *work = h->eig_work + nn + n;
  ST_TRY(jacobi32(h, A, n, X));
  Op opA, opB;
  opA.dense = A;
  double normA = host_fro(s, A, nn);
  ST_TRY(refine(h, opA, opB, n, normA, X, lam, 3, work));
  st_count_launch(); sort_desc_kernel<<<grid_for(n), 256, 0, s>>>(eval, evec, lam, X, n);
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

// Fast-diagonalization set-up (Sec. 3.2): for every spatial direction the
// generalized eigendecomposition of (D_ll K_l, M_l) with M_l-orthonormal
// eigenvectors, then one banded LU per spatial eigenvalue.
// Leading eigenpairs of the Gram matrix G (n x n, device) for the low-rank
// step (Eq. tol): Lanczos on the device, Rayleigh-Ritz on the tridiagonal on
// the host.  R is the smallest r with tr - sum_{i<=r} theta_i <= eps^2 tr over
// the Ritz values theta (which never exceed the eigenvalues they approach);
// the run extends the basis in batches until the Ritz pairs 1..R have
// residual estimates beta_k |s_{k,i}| <= 1e-14 theta_1, or the basis spans an
// invariant subspace.  On success Ur (n x R, row-major) holds the Ritz
// vectors and lam the Ritz values; ST_ERR_NOT_CONVERGED when kmax basis
// vectors did not suffice (the caller then takes the full decomposition).
st_status gram_top_eigs(st_handle *h, const double *G, int n, double tr, double eps, int cap, double *Ur, int *R_out,
                        std::vector<double> &lam) {
  cudaStream_t s = h->stream;
  const int kmax = std::min(n, 192);
  size_t shb = (size_t)(n + kmax + 2) * sizeof(double);
  if (shb > 200 * 1024) return ST_ERR_NOT_CONVERGED;
  static std::atomic<unsigned long long> attr{0};
  smem_optin(lanczos_kernel, 200 * 1024, attr);
  double *Q = h->eig_work;                       // (kmax + 1) x n
  double *ab = Q + (size_t)(kmax + 1) * n;       // alpha[kmax], beta[kmax]
  double *Sd = ab + 2 * kmax;                    // k x R coefficients of the Ritz vectors
  int *kd = (int *)(Sd + (size_t)kmax * kmax);
  // deterministic pseudo-random start vector (splitmix64), normalized
  std::vector<double> q0(n);
  unsigned long long st = 0x9e3779b97f4a7c15ull;
  double nrm = 0.0;
  for (int i = 0; i < n; ++i) {
    st += 0x9e3779b97f4a7c15ull;
    unsigned long long z = st;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    q0[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    nrm += q0[i] * q0[i];
  }
  nrm = std::sqrt(nrm);
  for (double &v : q0) v /= nrm;
  ST_CUDA(cudaMemcpyAsync(Q, q0.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  const double tiny = 1e-15 * tr;
  std::vector<double> al(kmax), be(kmax);
  int k = 0;
  while (k < kmax) {
    const int k1 = std::min(kmax, k + (k == 0 ? 24 : 16));
    size_t sh = (size_t)(n + k1 + 1) * sizeof(double);
    st_count_launch();
    lanczos_kernel<<<1, kLzThreads, sh, s>>>(G, n, Q, ab, ab + kmax, k, k1, tiny, kd);
    ST_CUDA(cudaGetLastError());
    int kdone = 0;
    ST_CUDA(cudaMemcpyAsync(&kdone, kd, sizeof(int), cudaMemcpyDeviceToHost, s));
    ST_CUDA(cudaMemcpyAsync(al.data(), ab, k1 * sizeof(double), cudaMemcpyDeviceToHost, s));
    ST_CUDA(cudaMemcpyAsync(be.data(), ab + kmax, k1 * sizeof(double), cudaMemcpyDeviceToHost, s));
    ST_CUDA(cudaStreamSynchronize(s));
    if (kdone < 1 || kdone > k1) return ST_ERR_CUDA;
    for (int i = 0; i < kdone; ++i)
      if (!std::isfinite(al[i]) || !std::isfinite(be[i])) return ST_ERR_NAN;
    k = kdone;
    const bool exact = kdone < k1 || k == n;   // invariant subspace, or the whole space
    // Ritz values, descending, until the kept energy reaches (1 - eps^2) tr
    double lo = al[0], hi = al[0], tnorm = 0.0;
    for (int i = 0; i < k; ++i) {
      double rad = (i > 0 ? std::fabs(be[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(be[i]) : 0.0);
      lo = std::min(lo, al[i] - rad);
      hi = std::max(hi, al[i] + rad);
      tnorm = std::max(tnorm, std::fabs(al[i]) + rad);
    }
    std::vector<double> theta;
    double kept = 0.0;
    int R = -1;
    double upper = hi;
    for (int r = 1; r <= k; ++r) {
      double th = tridiag_eig_bisect(k, al.data(), be.data(), r, lo, upper);
      theta.push_back(th);
      upper = th + 4e-16 * std::fabs(th) + 1e-300;
      kept += std::max(th, 0.0);
      if (tr - kept <= eps * eps * tr) { R = r; break; }
    }
    if (R < 0) {
      if (exact) R = k;
      else continue;
    }
    // Ritz vectors of T for the pairs 1..R and their residual estimates
    std::vector<double> Y((size_t)R * k);
    std::vector<const double *> prev;
    bool converged = true;
    for (int r = 0; r < R; ++r) {
      prev.clear();
      for (int q = 0; q < r; ++q)
        if (std::fabs(theta[q] - theta[r]) <= 1e-8 * tnorm) prev.push_back(&Y[(size_t)q * k]);
      tridiag_eigvec(k, al.data(), be.data(), theta[r], tnorm, prev, &Y[(size_t)r * k]);
      double res = std::fabs(be[k - 1] * Y[(size_t)r * k + k - 1]);
      if (!(res <= 1e-14 * theta[0])) converged = false;
    }
    if (!converged && !exact) continue;
    if (R > cap) R = cap;
    // Ur = Q^T S with S[m][r] = Y[r][m]  (n x R)
    std::vector<double> S((size_t)k * R);
    for (int m = 0; m < k; ++m)
      for (int r = 0; r < R; ++r) S[(size_t)m * R + r] = Y[(size_t)r * k + m];
    ST_CUDA(cudaMemcpyAsync(Sd, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_gemm64(s, Ur, Q, Sd, n, R, k, 1, n, R, 1, R, 1, 1.0, 0.0);
    ST_CUDA(cudaStreamSynchronize(s));   // S lives on the host stack of this call
    lam.assign(theta.begin(), theta.begin() + R);
    *R_out = R;
    return ST_OK;
  }
  return ST_ERR_NOT_CONVERGED;
}

st_status fd_setup(st_handle *h) {
  cudaStream_t s = h->stream;
  const st_problem_desc &D = h->desc;
  int p = h->p;
  int *fail = (int *)h->red;   // device int flag
  ST_CUDA(cudaMemsetAsync(fail, 0, sizeof(int), s));
  for (int l = 0; l < h->d; ++l) {
    int n = h->n[l];
    size_t nn = (size_t)n * n;
    double *L = h->eig_work;                      // n x (p+1)
    double *Kd = L + (size_t)n * (p + 1);         // dense D K
    double *T1 = Kd + nn, *C = T1 + nn, *X = C + nn, *lam = X + nn, *work = lam + n;
    st_count_launch(); chol_band_kernel<<<1, 1, 0, s>>>(L, h->Mb[l], n, p, fail);
    st_count_launch(); band_to_dense_kernel<<<grid_for(nn), 256, 0, s>>>(Kd, h->Kb[l], n, p, D.D[l]);
    st_count_launch(); lower_solve_cols_kernel<<<(n + 127) / 128, 128, 0, s>>>(T1, Kd, L, n, p, 0);   // T1 = L^-1 DK
    st_count_launch(); lower_solve_cols_kernel<<<(n + 127) / 128, 128, 0, s>>>(C, T1, L, n, p, 1);    // C = L^-1 T1^T
    st_count_launch(); symmetrize_kernel<<<grid_for(nn), 256, 0, s>>>(C, n);
    ST_TRY(jacobi32(h, C, n, T1));                                                   // T1 = Z
    st_count_launch(); upper_solve_cols_kernel<<<(n + 127) / 128, 128, 0, s>>>(X, T1, L, n, p);        // X = L^-T Z
    Op opA, opB;
    opA.band = h->Kb[l];
    opA.scale = D.D[l];
    opB.band = h->Mb[l];
    double normA = host_fro(s, Kd, nn);
    ST_TRY(refine(h, opA, opB, n, normA, X, lam, 3, work));
    ST_CUDA(cudaMemcpyAsync(h->U64[l], X, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    ST_CUDA(cudaMemcpyAsync(h->lam[l], lam, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    st_count_launch(); transpose_kernel<<<grid_for(nn), 256, 0, s>>>(h->UT64[l], h->U64[l], n);
    launch_band_to_f32(s, h->U32[l], h->U64[l], nn);
    launch_band_to_f32(s, h->UT32[l], h->UT64[l], nn);
  }
  st_count_launch(); mu_kernel<<<grid_for(h->Ns), 256, 0, s>>>(h->mu, h->lam[0], h->lam[1], h->lam[2], h->n[0], h->n[1], h->d, h->Ns);
  unsigned blocks = (unsigned)((h->Ns + 127) / 128);
  double shift = D.a * D.c1;
  switch (p) {
    case 1: st_count_launch(); fd_lu_kernel<1><<<blocks, 128, 0, s>>>(h->lu64, h->Wtb, h->Mtb, h->mu, D.C_m, shift, h->Nt, h->Ns, fail); break;
    case 2: st_count_launch(); fd_lu_kernel<2><<<blocks, 128, 0, s>>>(h->lu64, h->Wtb, h->Mtb, h->mu, D.C_m, shift, h->Nt, h->Ns, fail); break;
    case 3: st_count_launch(); fd_lu_kernel<3><<<blocks, 128, 0, s>>>(h->lu64, h->Wtb, h->Mtb, h->mu, D.C_m, shift, h->Nt, h->Ns, fail); break;
    default: st_count_launch(); fd_lu_kernel<4><<<blocks, 128, 0, s>>>(h->lu64, h->Wtb, h->Mtb, h->mu, D.C_m, shift, h->Nt, h->Ns, fail); break;
  }
  long long nlu = (long long)h->Nt * h->B * h->Ns;
  launch_band_to_f32(s, h->lu32, h->lu64, nlu);
  int hfail = 0;
  ST_CUDA(cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, s));
  ST_CUDA(cudaStreamSynchronize(s));
  ST_CUDA(cudaGetLastError());
  return hfail ? ST_ERR_BREAKDOWN : ST_OK;
}
