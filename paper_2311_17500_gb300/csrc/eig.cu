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
