// Internal declarations shared by the translation units of libst.so.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstddef>
#include <vector>
#include "st.h"

#define ST_MAXP 4
#define ST_MAXB (2 * ST_MAXP + 1)
// tile edge of the Gram matrix kernel of the low-rank steps
constexpr int kGramTile = 64;

// ---------------------------------------------------------------- host 1D data
// One parametric direction (space, or time with `scale` = T).  Tables are per
// knot span e (n_el spans, nq = p+1 Gauss points each); the local functions on
// span e are the global B-splines e .. e+p (open knots, maximal regularity).
struct Dir1D {
  int n_el = 0, p = 0, n = 0, nq = 0, kmax = 0;
  double scale = 1.0;
  std::vector<double> knots;      // parametric, n + p + 1
  std::vector<double> xq, wq;     // physical points / weights, [e*nq + q]
  std::vector<double> tab;        // [k][e][q][a]: k-th physical derivative of local fn a
  std::vector<double> greville;   // physical, n
  double at(int k, int e, int q, int a) const {
    return tab[(((size_t)k * n_el + e) * nq + q) * (p + 1) + a];
  }
};

struct HostSetup {
  Dir1D sdir[3];
  Dir1D tdir;
  // banded (n x (2p+1)), entry (i, i-p+k) at [i*(2p+1)+k]
  std::vector<double> M[3], K[3];   // spatial mass, stiffness (unscaled by D)
  std::vector<double> Mt, Wt;       // time, X_t indexing
  std::vector<double> tau_q;        // [l-1][e][q]
  std::vector<double> wlu;          // banded LU of W_t + b d_e M_t, no pivoting
};

st_status host_setup(const st_problem_desc &d, HostSetup &hs);
// M_t and LU(W_t + b d_e M_t) alone, both N_t x (2p+1) banded.
st_status host_time_bands(const st_problem_desc &d, std::vector<double> &Mt, std::vector<double> &wlu);
// The basis of `dr` at its Greville abscissae, banded: (i, j) = b_j(gamma_i);
// shift = 1 drops the first function (the time space X_t).
std::vector<double> greville_band(const Dir1D &dr, int shift);
// Banded LU without pivoting in place (n x (2p+1)); stores 1/u_ii on the diagonal.
int band_lu_inplace(double *a, int n, int p);

// ---------------------------------------------------------------- handle
struct st_handle {
  st_problem_desc desc;
  cudaStream_t stream = nullptr;
  int dev = 0;
  int d = 0, p = 0, nq = 0, B = 0;       // B = 2p+1
  int n[3] = {1, 1, 1}, nel[3] = {1, 1, 1}, Q[3] = {1, 1, 1};
  int Nt = 0, nel_t = 0, Qt = 0;
  long long Ns = 0, Ndof = 0, Qs = 0, Nel_s = 0, NtQs = 0, maxStage = 0;
  HostSetup hs;

  // 1D device data (FP64 and FP32 copies of the bands)
  double *Mb[3] = {}, *Kb[3] = {}, *Mtb = nullptr, *Wtb = nullptr;
  float *Mb32[3] = {}, *Kb32[3] = {}, *Mtb32 = nullptr, *Wtb32 = nullptr;
  double *Bq[3] = {}, *B2q[3] = {}, *wqs[3] = {};   // spatial tables [e][q][a], weights [e*nq+q]
  float2 *Bq2[3] = {}, *B2q2[3] = {};                 // the same tables as double-float pairs
  float *Bq32[3] = {};
  double *bt = nullptr;       // time tables [k][e][q][a], k = 0..p
  double *wt = nullptr;       // time weights [e*nq+q]
  double *xt = nullptr;       // time points [e*nq+q]
  int *tmask = nullptr;       // [e*nq+q]: bit b set if the time point lies in stimulus window b
  double *xs[3] = {};         // spatial points per direction [e*nq+q]
  double *tauq = nullptr;     // [l-1][e][q]
  double *bprod = nullptr;    // [e][q][pair] w_t b_i b_{i+k}, pairs (i, k) with k <= p - i
  float2 *bt2 = nullptr;      // bt for k = 0, 1 as double-float pairs (hi, lo)
  float2 *bprod2 = nullptr;   // bprod as double-float pairs
  float2 *Tr2 = nullptr;      // SU time bands (rank_cap x (p+1) N_t) as double-float pairs
  double *wlu = nullptr;      // LU of W_t + b d_e M_t
  // hat-function data of the Greville interpolation, per 1D Gauss point
  int *hat_i_t = nullptr, *hat_i_s[3] = {};
  double *hat_l_t = nullptr, *hat_l_s[3] = {};

  // fast diagonalization
  double *U64[3] = {}, *UT64[3] = {}, *lam[3] = {};
  float *U32[3] = {}, *UT32[3] = {};
  double *mu = nullptr;       // spatial eigenvalues mu_j, j over N_s
  float *UTp[3] = {}, *Up[3] = {};   // TF32 operands: U_l^T, U_l zero-padded to [Npad][Kpad]
  int Npad[3] = {}, Kpad[3] = {};
  bool use_tc = false;
  float *P32[2] = {};          // padded-row buffers of the tensor-core transforms
  int *tc_err = nullptr;
  double *lu64 = nullptr;     // [it][k][j], k = 0..2p
  long long Ns_pad = 0;       // spatial size with the innermost axis padded to a multiple of 4
  int nxp = 0;                // padded innermost axis
  float *lu32 = nullptr;

  // operator form: time bands stored per spatial Gauss point (band form), or
  // none (lean form: the reaction term is integrated from u^k, w^k in the
  // apply and the SU term kept as its rank factors; see kernels_lean.cu)
  bool lean = false;
  float2 *U1 = nullptr, *W1 = nullptr;   // lean: u^k, w^k at the Gauss rows of the other axes, [N_t][rows][n_x] pairs
  float2 *wt2 = nullptr;                 // time quadrature weights as double-float pairs
  double *cfr = nullptr;                 // lean: scale C_m sigma_r of each SU rank
  int lin_kind = ST_PICARD;              // linearization of the current operator
  bool inner_df = false;                 // the mixed inner solve applies the operator in double-float
  bool pre64 = false;                    // the mixed inner solve applies the FP64 preconditioner
  long long wcap = 0;                    // values per Gauss-point work buffer (W64 doubles, W32 floats)
  double *gpart = nullptr;               // Gram partial sums when the first work buffer is too small
  long long gpart_cap = 0;
  long long rows_x = 1;                  // Gauss rows of the axes other than x: prod_{l>=1} Q_l
  // linearization: symmetric time band per spatial Gauss point, [k][it][q], k = 0..p
  // time bands per spatial Gauss point [k][it][q] as double-float pairs:
  // band32 = high parts (the FP32 operator), band_lo = low parts
  float *band32 = nullptr;
  float *band_lo = nullptr;
  bool have_lin = false;
  double *f64 = nullptr;

  // ionic / low rank
  unsigned long long *emax = nullptr;   // [et][es] bit pattern of max |R| (non-negative double)
  double *stats = nullptr;              // [0] max|u| [1] max|d_t u| [2] max|R| (bit patterns)
  double *theta = nullptr;              // [Nt][Ns]
  double *gram = nullptr;               // [Nt][Nt]
  double *evec = nullptr, *eval = nullptr;
  double *eig_work = nullptr;
  float *eig32 = nullptr;
  int rank = 0;
  double *Ur = nullptr, *sr = nullptr, *Vr = nullptr;   // [Nt][R], [R], [Ns][R]
  double *th_t = nullptr;   // theta_{t,r} at time Gauss points [r][Qt]
  double *Tr = nullptr;     // SU time bands [r][k][it]
  int rank_cap = 0;
  double theta_fro = 0.0;
  // low-rank reaction coefficient (eps_reaction >= 0): Greville collocation
  // bands, the factors of the coefficient's Greville values, its time bands
  double *Gsb[3] = {}, *Gtb = nullptr;   // [n][2p+1] per direction, time on X_t
  int rankC = 0;
  double *UrC = nullptr, *srC = nullptr, *VrC = nullptr, *cfc = nullptr;   // [Nt][R], [R], [Ns][R], [R]
  double *thC = nullptr, *Tc = nullptr;  // rho_{t,r} at the time Gauss points [r][Qt]; bands [r][k][it]
  float2 *Tc2 = nullptr;                 // the bands as double-float pairs

  // workspaces
  double *W64[2] = {};
  float *W32[2] = {};
  double *K64[7] = {};
  float *K32[7] = {};
  double *U0 = nullptr, *L0 = nullptr, *Wq0 = nullptr;   // ionic fields at spatial qpts [Nt][Qs]
  double *red = nullptr;       // reduction scratch (device)
  double *red_host = nullptr;  // pinned host slots of the Arnoldi coefficients (two iterations)
  cudaEvent_t arn_ev[2] = {nullptr, nullptr};   // arrival of each slot
  // Krylov
  int m = 0;
  long long ldv = 0;          // Krylov basis leading dimension (16-byte aligned rows)
  double *V64 = nullptr; float *V32 = nullptr;
  double *Z64 = nullptr; float *Z32 = nullptr;   // preconditioned Krylov vectors (flexible GMRES)
  double *r64 = nullptr, *x64 = nullptr, *t64a = nullptr, *t64b = nullptr;
  double *z64 = nullptr, *b64 = nullptr;   // GMRES preconditioner output, Newton right-hand side
  float *r32 = nullptr, *t32a = nullptr, *t32b = nullptr, *d32 = nullptr;
  double *hcol = nullptr;      // device [2*(m+2)] Arnoldi coefficients
  double *gs_coef = nullptr;   // 2 (m + 2) values: Gram-Schmidt update coefficients (FP64 or FP32)
  std::vector<void *> allocs;
  // allocations come from the device's stream-ordered memory pool (allocated
  // and freed in the order of the handle's stream): freeing them then waits
  // for this stream only, where cudaFree would wait for the whole device
  bool pooled = false;
  // optional per-stage timing (CUDA events on the handle's stream)
  bool prof_on = false;
  struct ProfRec { int cat; cudaEvent_t a, b; double bytes, flops; };
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
};

// Opts `kernel` in to `bytes` of dynamic shared memory on the current device.
// The attribute is per device, so each call site keeps a mask of the devices
// it has set up, and a repeated call on the same device does nothing.
template <typename K>
inline cudaError_t smem_optin(K kernel, int bytes, std::atomic<unsigned long long> &devices_done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (devices_done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) devices_done.fetch_or(bit, std::memory_order_release);
  return e;
}

// Stage categories of the optional per-stage timing.
enum {
  PROF_KRON = 0,      // banded Kronecker passes of the operator
  PROF_INTERP = 1,    // sum-factorization passes (coefficients <-> Gauss points)
  PROF_QBAND = 2,     // time band per spatial Gauss point (reaction + SU)
  PROF_FD_GEMM = 3,   // preconditioner spatial transforms
  PROF_FD_LU = 4,     // preconditioner banded time solves
  PROF_ARNOLDI = 5,   // Gram-Schmidt inner products and updates, norms
  PROF_IONIC = 6,     // ionic quadrature and band assembly
  PROF_LOWRANK = 7,   // Theta-hat, Gram matrix, eigen-decomposition, SU band update
  PROF_APPLY64 = 8,   // the operator applied in FP64 (all of its passes)
  PROF_OTHER = 9,
  PROF_NCAT = 10
};

// Records events around the enclosed launches when profiling is on.
struct ProfScope {
  st_handle *h;
  size_t idx;
  ProfScope(st_handle *hh, int cat, double bytes, double flops = 0.0);
  ~ProfScope();
};

// ---------------------------------------------------------------- helpers
// Records the CUDA error behind an ST_ERR_CUDA / ST_ERR_OOM return, per calling
// thread (read back with st_last_cuda_error).
void st_note_cuda_error(cudaError_t e, const char *file, int line);
const char *st_cuda_detail();

#define ST_CUDA(call)                                                  \
  do {                                                                 \
    cudaError_t _e = (call);                                           \
    if (_e != cudaSuccess) {                                           \
      st_note_cuda_error(_e, __FILE__, __LINE__);                      \
      return _e == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA; \
    }                                                                  \
  } while (0)

#define ST_TRY(call)                    \
  do {                                  \
    st_status _s = (call);              \
    if (_s != ST_OK) return _s;         \
  } while (0)

// ---------------------------------------------------------------- kernels (launchers)
// generic tensor views: [outer][n][inner]
template <typename T>
void launch_band_pass(cudaStream_t s, T *out, int nterms, const T *const *bands, const T *const *ins,
                      const double *coefs, int n, long long inner, long long outer, int p, bool accumulate);
template <typename T>
void launch_interp_fwd(cudaStream_t s, T *out, const T *in, const T *tab, int nel, int p, int nq,
                       long long inner, long long outer);
template <typename T>
void launch_interp_bwd(cudaStream_t s, T *out, const T *in, const T *tab, int nel, int p, int nq,
                       long long inner, long long outer, bool accumulate);
template <typename T>
void launch_qband_apply(cudaStream_t s, T *z, const T *x, const float *bhi, const float *blo, int Nt, long long Qs,
                        int p);
// Fused x-axis reaction/SU pass Y1 = Bx^T band Bx X1 ([Nt][rows][nx] rows of
// x-coefficients at Gauss rows of the other axes); false when the x axis has
// too many elements for one block (then the caller takes the unfused path).
// Kronecker part of the operator for d = 2 (time pass into xW, xM, then the
// plane pass into y); false when a plane column does not fit shared memory.
template <typename T>
// 2D Kronecker part; for FP64, `split` holds x as double-float pairs
// (N_t n_y n_x float pairs, see launch_split_df), unused for FP32.
bool launch_kron2d(cudaStream_t s, T *y, const T *x, const void *split, const T *Wt, const T *Mt, const T *Mx,
                   const T *Kx, const T *My, const T *Ky, int nx, int ny, int Nt, int p, double Cm, double Dx,
                   double Dy);
// FP64 operator on double-float pairs: x split into (high, low) float pairs,
// and the strided interpolation passes with pair input (forward: pair output;
// backward: pair output, or FP64 output, optionally accumulated).
void launch_split_df(cudaStream_t s, float2 *out, const double *in, long long n);
void launch_interp_fwd_pairs(cudaStream_t s, float2 *out, const float2 *in, const float2 *tab, int nel, int p,
                             long long inner, long long outer);
template <typename TO>
void launch_interp_bwd_pairs(cudaStream_t s, TO *out, const float2 *in, const float2 *tab, int nel, int p,
                             long long inner, long long outer, bool accumulate);
// Lean form of the reaction + SU part (kernels_lean.cu): everything the
// kernel needs besides the x rows in and out.
struct LeanTerms {
  const float2 *U1 = nullptr, *W1 = nullptr;   // u^k, w^k rows (pairs); null without M_R
  const float2 *bt = nullptr, *wt = nullptr;   // time basis [e][gt][a] and weights [e*nq+gt], pairs
  const double *ws[3] = {};                    // spatial weights per direction
  const int *hi[3] = {};                       // Greville hat data per 1D Gauss point
  const double *hl[3] = {};
  const double *V = nullptr, *cf = nullptr;    // rank factors [N_s][Rt] and scales [Rt]
  const float2 *Tb = nullptr;                  // rank time bands [Rt][p+1][N_t], pairs
  int Rt = 0;
  const double *V2 = nullptr, *cf2 = nullptr;  // a second list of rank terms (the low-rank reaction)
  const float2 *Tb2 = nullptr;
  int R2 = 0;
  int exact = 0, newton = 0;
  double c1 = 0, c2 = 0, a = 0;
  int d = 1, p = 1, nel = 1, Nt = 1, nel_t = 1;
  int n[3] = {1, 1, 1}, Q[3] = {1, 1, 1};
};
// True when one block holds an x row of the lean kernel.
bool xlean_feasible(int nel, int p);
// Largest rank-term count the lean kernel takes (shared memory).
int xlean_max_rank(int nel, int p, bool exact);
// Y1 = (reaction + SU part along x and time) X1 for every Gauss row of the
// other axes; T = float (FP32) or float2 (double-float pairs).
template <typename T>
st_status launch_xlean(cudaStream_t s, const LeanTerms &L, T *Y1, const T *X1, const T *tab, long long rows);
LeanTerms lean_terms(st_handle *h);
// Largest block (threads) of the fused x pass for this element size and degree.
int xband_fused_limit(size_t elem, int p);
template <typename T>
bool launch_xband_fused(cudaStream_t s, T *Y1, const T *X1, const float *bhi, const float *blo, const T *tab, int nel,
                        int Nt, long long rows, int p, int *err);
template <typename T>
void launch_mode_gemm(cudaStream_t s, T *out, const T *in, const T *A, int n, long long inner, long long outer);
template <typename T>
void launch_tline_lu_solve(cudaStream_t s, T *z, const T *r, const T *lu, int Nt, long long Ns, int p, int *err);
template <typename T>
void launch_rot_gemm(cudaStream_t s, T *out, const T *in, const T *M, int nb, int nj, long long Aa, long long Nt);
st_status launch_tc_xform(cudaStream_t s, float *out, const float *X, long long R, int nb, long long in_stride,
                          const float *Mpad, int nj, int Npad, int Kpad, long long Aa, long long A_inner,
                          long long A_in_stride, int *err);
// FP64 rows of n values into zero-padded FP32 rows of `stride` values.
void launch_pad_d2f(cudaStream_t s, float *out, const double *in, long long rows, long long n, long long stride);
void launch_pad_rows(cudaStream_t s, float *out, const float *in, long long rows, long long n, long long stride);
// tensor-core transforms: process-wide self-test state (0 untested, 1 usable, -1 not usable)
int tc_state(cudaStream_t s, double *err_out);
template <typename T>
void launch_multi_dot(cudaStream_t s, double *out, const T *V, long long ldv, int nv, const T *w,
                      long long n, double *scratch);
// <V_i, x1>, <V_i, x2> for i < nv in one pass: out[2 i + c] (FP64).
template <typename T>
void launch_multi_dot2(cudaStream_t s, double *out, const T *V, long long ldv, int nv, const T *x1, const T *x2,
                       long long n, double *scratch);
// Update pass of the delayed classical Gram-Schmidt step j (rows j, j+1 of V
// rewritten in place from the dots D of launch_multi_dot2; (nu, gam, sw) -> sc;
// coef: 2j + 3 values of work space).
template <typename T>
void launch_dcgs2_update(cudaStream_t s, T *V, long long ldv, int j, const double *D, long long n, double *sc,
                         T *coef);
template <typename T>
void launch_multi_axpy(cudaStream_t s, T *w, const T *V, long long ldv, int nv, const double *h,
                       long long n, const double *nrm = nullptr);
template <typename T>
void launch_scale_copy(cudaStream_t s, T *y, const T *x, double alpha, long long n);
void launch_axpby64(cudaStream_t s, double *y, const double *x, double a, double b, long long n);
void launch_sub64(cudaStream_t s, double *r, const double *b, const double *ax, long long n);
void launch_d2f(cudaStream_t s, float *y, const double *x, double scale, long long n);
void launch_f2d_axpy(cudaStream_t s, double *y, const float *x, double scale, long long n);
void launch_f2d(cudaStream_t s, double *y, const float *x, long long n);
void launch_absmax64(cudaStream_t s, double *out, const double *x, const double *y, long long n, double *scratch);
void launch_norm2_64(cudaStream_t s, double *out, const double *x, long long n, double *scratch);
void launch_band_to_f32(cudaStream_t s, float *out, const double *in, long long n);

// ionic / stabilization
st_status ionic_run(st_handle *h, const double *u, const double *w, int kind, bool want_stats);
st_status theta_and_lowrank(st_handle *h, st_ionic_info *info);
st_status su_band_add(st_handle *h);
// The low-rank reaction coefficient at (u, w) for the linearization `kind`
// (eps_reaction >= 0): factors, time bands and scales.
st_status reaction_lowrank(st_handle *h, const double *u, const double *w, int kind);
st_status source_assemble(st_handle *h);
st_status wupdate_run(st_handle *h, const double *u, double *w);
// w-update with the time bands taken from host arrays and staged in the
// file-scope device scratch (no device allocation); Nt (2p+1) values each.
st_status wupdate_static_run(cudaStream_t s, const double *u, double *w, const double *Mt_host,
                             const double *lu_host, double bcoef, int Nt, long long Ns, int p);

// eigen / FD
st_status fd_setup(st_handle *h);
st_status sym_eig_desc(st_handle *h, const double *A, int n, double *evec, double *eval);
// Leading Ritz pairs of the Gram matrix by Lanczos (rank R of Eq. tol chosen
// from them); ST_ERR_NOT_CONVERGED when the full decomposition is needed.
st_status gram_top_eigs(st_handle *h, const double *G, int n, double tr, double eps, int cap, double *Ur, int *R_out,
                        std::vector<double> &lam);

// apply / precond
template <typename T>
st_status apply_T(st_handle *h, const T *x, T *y);
template <typename T>
st_status precond_T(st_handle *h, const T *r, T *z);

void *st_alloc(st_handle *h, size_t bytes, st_status *err);
// Process-wide count of kernel launches issued by this library, called just
// before each launch with the launch's source position.  An error found
// pending at that point (a launch refused by the runtime, or a runtime call
// after it) is attributed, per thread, to the launch before; the detail behind
// a later ST_ERR_CUDA names it.
void st_count_launch_at(const char *file, int line);
#define st_count_launch() st_count_launch_at(__FILE__, __LINE__)
