/*
 * st.h -- C ABI of the space-time isogeometric monodomain solver (libst.so).
 *
 * The library solves the monodomain equation coupled with the Rogers-McCulloch
 * ionic model (Sec. 3, eq. 3.1 of "Space-time Isogeometric Analysis of cardiac
 * electrophysiology") on the unit square or cube, with tensor-product B-splines
 * of degree p in space and time (Sec. 2) and optional Spline Upwind (SU)
 * stabilization (Sec. 3).  Everything after the 1D set-up runs in CUDA
 * kernels on the GPU of the calling thread's current device.
 *
 * Conventions shared by every entry point
 *   - Vectors of unknowns are device pointers to N_dof = N_t * N_s contiguous
 *     values in the colexicographic order of Sec. 2: x fastest, then y, z, and
 *     time slowest (index = i_t * N_s + i_x + n_x (i_y + n_y i_z)), with
 *     n_l = n_el[l] + p, N_s = prod n_l, N_t = n_el_t + p - 1 (the first time
 *     B-spline is removed to impose u = w = 0 at t = 0).
 *   - Pointers are owned by the caller and never freed by the library.  The
 *     handle owns all of its workspaces.
 *   - Work is enqueued on the stream passed to st_setup.  Calls that return
 *     host scalars (st_ionic, st_linsolve, st_solve, st_get) synchronize it;
 *     st_apply, st_precond, st_wupdate and st_rhs are asynchronous
 *     (st_wupdate_static is not: see there).
 *   - Errors are returned as st_status, never by aborting.  After ST_ERR_CUDA
 *     the handle must be destroyed; after any other error it stays usable.
 *   - A handle is not thread-safe; separate handles are independent.
 */
#ifndef ST_H
#define ST_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ST_OK = 0,
  ST_ERR_ARG = 1,            /* invalid argument or description */
  ST_ERR_OOM = 2,            /* device allocation failed */
  ST_ERR_CUDA = 3,           /* CUDA runtime error; destroy the handle */
  ST_ERR_NOT_CONVERGED = 4,  /* iteration cap reached; best iterate returned */
  ST_ERR_BREAKDOWN = 5,      /* zero pivot in a factorization */
  ST_ERR_NAN = 6,            /* NaN or Inf detected in a result */
  ST_ERR_TIMEOUT = 7,        /* a bounded device wait gave up */
  ST_ERR_STATE = 8,          /* call order violated (e.g. st_apply before st_ionic) */
  ST_ERR_CAPACITY = 9        /* problem too large for the fixed scratch of st_wupdate_static */
} st_status;

/* source kinds: f in eq. 3.1 */
enum { ST_SRC_ZERO = 0, ST_SRC_STIM = 1, ST_SRC_HEAT_MMS = 2, ST_SRC_E1_MMS = 3 };
/* stabilization (Sec. 3): plain Galerkin or the SU term S-tilde of Eq. (tildeS) */
enum { ST_GALERKIN = 0, ST_SU = 1 };
/* nonlinear iteration: fixed point of Sec. 3.1 or Newton on the u-equation */
enum { ST_PICARD = 0, ST_NEWTON = 1 };
/* arithmetic: FP64 throughout, or FP32 inner work with FP64 refinement */
enum { ST_FP64 = 0, ST_MIXED = 1 };
/* support extension of Eq. (suppext): literal (xi_{i-p}, xi_{i+p+1}) or the
 * symmetric union of neighbouring supports (xi_{i-p}, xi_{i+2p+1}) */
enum { ST_SUPPEXT_LITERAL = 0, ST_SUPPEXT_SYMMETRIC = 1 };
/* precision selector of st_apply / st_precond: ST_FP64 -> double*, ST_MIXED -> float* */
/* form of the reaction + SU part of the operator (Sec. 3.1.1, Eq. lin_sys_A):
 *  ST_FORM_BANDS: one symmetric time band per spatial Gauss point, assembled per
 *                 linearization and streamed by every apply ((p+1)^(d+1) values
 *                 per unknown of device memory);
 *  ST_FORM_LEAN:  no stored bands: the reaction term is integrated at the
 *                 space-time Gauss points from u^k, w^k inside the apply and the
 *                 SU term of Eq. (tildeS) is kept as its rank-R factors
 *                 (requires d >= 2 and n_el[0] + p <= 256);
 *  ST_FORM_AUTO:  the band form, faster per apply, unless its footprint
 *                 exceeds 160 GiB and the lean form applies. */
enum { ST_FORM_AUTO = 0, ST_FORM_BANDS = 1, ST_FORM_LEAN = 2 };
/* operator of the inner FP32 Krylov solve of the mixed mode (the Krylov
 * vectors and the preconditioner stay FP32):
 *  ST_INNER_FP32: the operator in FP32 arithmetic;
 *  ST_INNER_DF:   the operator in double-float arithmetic (FP64 accuracy on the
 *                 FP32 pipes), its input and output rounded to FP32;
 *  ST_INNER_AUTO: FP32 first; double-float for the rest of the handle's life
 *                 from a refinement step that fails with the FP64
 *                 preconditioner already in use (see ST_PRECOND_AUTO).
 * Either way an inner cycle cannot push the true residual of its correction d
 * below about u_32 ||A|| ||d|| / ||b|| (d is stored in FP32): on the 3D
 * 64^3 x 128 workload that level is near 4e-5 for every operator and
 * preconditioner choice.  Each FP32 cycle ends when it gets there (see
 * st_linsolve) and the FP64 refinement takes over. */
enum { ST_INNER_AUTO = 0, ST_INNER_FP32 = 1, ST_INNER_DF = 2 };
/* arithmetic of the preconditioner inside the FP32 Krylov solve (mixed mode):
 *  ST_PRECOND_TF32: spatial transforms on the tensor cores (tcgen05, TF32
 *                   inputs, FP32 accumulation) where every n_l <= 256 and the
 *                   once-per-process self-test passed, else on CUDA cores;
 *  ST_PRECOND_FP32: transforms on CUDA cores in FP32;
 *  ST_PRECOND_FP64: the FP64 preconditioner, its input and output rounded to
 *                   FP32;
 *  ST_PRECOND_AUTO: TF32 for d <= 2 and FP32 for d = 3, and FP64 from the
 *                   first refinement step on that fails (one that reduces the
 *                   true residual by less than a factor 2).
 * On the 3D workloads FP32 and FP64 preconditioners give the same residual
 * after the same number of iterations, the FP64 one at 4x the cost of an
 * iteration.  TF32 converges a little more slowly per iteration; on the
 * 64^3 x 128 workload it let a refinement step fail, after which the handle
 * ran the FP64 preconditioner and double-float operator at 4x the cost of
 * an FP64 solve (GB300 measurement).  Explicit TF32 stays available. */
enum { ST_PRECOND_AUTO = 0, ST_PRECOND_TF32 = 1, ST_PRECOND_FP32 = 2, ST_PRECOND_FP64 = 3 };

#define ST_MAX_STIM 8

/* Stimulus box: f += amp on the closed box [lo, hi] for t0 <= t < t1. */
typedef struct {
  double lo[3], hi[3];
  double t0, t1, amp;
} st_stim;

/* Problem description (plain data, copied by st_setup).
 * Model constants follow eq. 3.1 (dimensionless u, w); the numerical
 * parameters follow Sec. 3.1 and Sec. 4 of the paper. */
typedef struct {
  int d;                 /* spatial dimension, 1..3 */
  int p;                 /* spline degree in space and time, 1..4 (p_s = p_t, Sec. 4) */
  int n_el[3];           /* elements per spatial direction (unit interval, uniform), 1..1024 */
  int n_el_t;            /* time elements on [0, T] (uniform), 1..60000 */
  double T, C_m, D[3];   /* final time, membrane capacitance, diagonal conductivity */
  double a, b, c1, c2, d_e;   /* Rogers-McCulloch constants */
  int source_kind;       /* ST_SRC_* */
  int n_stim;            /* number of stimulus boxes (ST_SRC_STIM), <= ST_MAX_STIM */
  st_stim stim[ST_MAX_STIM];
  int stabilization;     /* ST_GALERKIN | ST_SU */
  int suppext;           /* ST_SUPPEXT_* */
  double eps_theta;      /* relative Frobenius tolerance of the low-rank theta, Eq. (tol) */
  int nonlinear;         /* ST_PICARD | ST_NEWTON */
  double alpha;          /* relaxation of the fixed point (Sec. 3.1) */
  double delta;          /* stop when ||u^{k+1} - u^k||_inf <= delta (Sec. 4) */
  int max_fp;            /* nonlinear iteration cap */
  int fix_w_zero;        /* 1: the recovery variable is held at zero (Sec. 4.1 test) */
  int precision;         /* ST_FP64 | ST_MIXED */
  int gmres_m;           /* Krylov basis size (restart length) */
  double rtol;           /* target true relative residual ||f - A u|| / ||f|| */
  int max_it;            /* cap on total inner GMRES iterations per linear solve */
  int operator_form;     /* ST_FORM_* */
  int inner_op;          /* ST_INNER_* (mixed mode) */
  double eps_reaction;   /* < 0: the reaction coefficient of Eq. (reaction) (C_J for
                          * Newton) exact at the Gauss points; >= 0: its values at
                          * the Greville grid, truncated to low rank at this
                          * relative Frobenius tolerance like Theta-hat (Eq. tol)
                          * and interpolated (d+1)-linearly, the low-rank reaction
                          * matrices of Sec. 4.2 */
  const double *breaks[3];   /* per spatial direction: NULL for a uniform mesh, else
                              * n_el[l] + 1 increasing breakpoints from 0 to 1 of the
                              * open knot vector (maximal regularity, Sec. 2); read by
                              * st_setup and st_footprint only (the caller keeps them) */
  const double *breaks_t;    /* the same for time, parametric on [0, 1] (scaled by T);
                              * e.g. knots clustered where the source switches (Sec. 4.2) */
  int precond_arith;         /* ST_PRECOND_* (mixed mode) */
} st_problem_desc;

typedef struct st_handle st_handle;

/* Sizes of the discrete problem. */
typedef struct {
  long long N_s, N_t, N_dof;
  long long Q_s;         /* spatial Gauss points: prod n_el[l] (p+1) */
  int n[3];              /* spatial basis functions per direction */
  int operator_form;     /* ST_FORM_BANDS or ST_FORM_LEAN: the form set-up chose */
  int precond_tc;        /* 1: the FP32 preconditioner's spatial transforms run on
                          * the tensor cores (tcgen05, TF32), 0: on CUDA cores */
} st_dims;

/* Output of st_ionic (Eq. theta_ce_u and Eq. tol). */
typedef struct {
  int rank;              /* R of the low-rank theta (0 when Theta-hat vanishes) */
  double u_max;          /* max |u| over the Gauss points */
  double ut_max;         /* max |d_t u| over the Gauss points */
  double den;            /* C_m (u_max / T + ut_max) */
  double r_max;          /* max |R| over the Gauss points */
  double theta_fro;      /* ||Theta-hat||_F */
  int rank_reaction;     /* rank of the low-rank reaction coefficient (eps_reaction >= 0), else 0 */
} st_ionic_info;

/* Per-solve statistics. */
typedef struct {
  int fp_iters;          /* nonlinear iterations taken (st_solve) */
  int gmres_iters;       /* inner Krylov iterations of the last linear solve */
  int outer_iters;       /* refinement steps of the last linear solve (mixed) */
  int total_gmres;       /* inner Krylov iterations summed over st_solve */
  int rank;              /* low-rank R of the last linearization */
  double rel_res;        /* true relative residual of the last linear solve (FP64) */
  double last_diff;      /* last ||u^{k+1} - u^k||_inf (st_solve) */
} st_stats;

/* Device bytes st_setup would allocate for this description (admission
 * control for the serving loop): an upper bound on the bytes that st_setup
 * and the later calls request from cudaMalloc for this handle (the runtime's
 * rounding of each allocation is not included).  ST_ERR_ARG on an invalid
 * description. */
st_status st_footprint(const st_problem_desc *desc, size_t *bytes);

/* Build a solver for `desc`: the 1D spline data of Sec. 2 and Sec. 3.1
 * (knots, Gauss tables, banded M_l, K_l, M_t, W_t, the tau_k of Eq. (tau),
 * Greville grids) on the host in FP64, then on the device the generalized
 * eigendecompositions of (D_ll K_l, M_l) and one banded LU of
 * C_m W_t + (mu_j + a c1) M_t per spatial eigenvalue mu_j (Sec. 3.2,
 * Eq. preconditioner, with the conductivity scaling of each direction), and the
 * right-hand side f of Eq. (rhsfun).  `cuda_stream` is a cudaStream_t (NULL =
 * legacy default stream).  On success *out owns every device buffer.  The
 * handle belongs to the device current at this call: every later call on it
 * runs there, whatever device the calling thread has current, and restores
 * the thread's device on return. */
st_status st_setup(const st_problem_desc *desc, void *cuda_stream, st_handle **out);

/* Release every resource of the handle (NULL is accepted). */
st_status st_destroy(st_handle *h);

/* Static description of a status code. */
const char *st_error_string(st_status s);

/* Diagnostics, no counterpart in the paper: the CUDA error behind the last
 * ST_ERR_CUDA or ST_ERR_OOM returned to the calling thread, as
 * "<error name> (<code>) at <file>:<line>", followed by ", pending since the
 * launch at <file>:<line>" when the error was already pending before a later
 * launch (a launch the runtime refused), else by ", last launch at
 * <file>:<line>"; "" if there was none.  The string is owned by the library
 * and stays valid until the thread's next such error. */
const char *st_last_cuda_error(void);

st_status st_get_dims(const st_handle *h, st_dims *out);

/* Linearize at (u, w) (device FP64 vectors): evaluate u, d_t u, the Laplacian
 * and w at every space-time Gauss point by sum factorization; form the
 * residual R of Eq. (theta_ce_u), its maxima over the support extensions and
 * Theta-hat; compute the low-rank U R V^T of Eq. (tol) (truncated SVD through
 * the Gram matrix); and assemble, for every spatial Gauss point, the time band
 * of the reaction term M_R (coefficient C_r of Eq. (reaction) for ST_PICARD,
 * its u-derivative for ST_NEWTON) plus the SU term of Eq. (tildeS).  After
 * this call st_apply applies the matrix A of Eq. (lin_sys_A). */
st_status st_ionic(st_handle *h, const double *u_dev, const double *w_dev, st_ionic_info *info);

/* Like st_ionic with an explicit linearization kind (ST_PICARD: C_r,
 * ST_NEWTON: C_J); keeps Theta-hat and the low-rank factors of the last
 * st_ionic call when `keep_theta` is 1 (theta frozen for Newton). */
st_status st_linearize(st_handle *h, const double *u_dev, const double *w_dev, int kind,
                       int keep_theta, st_ionic_info *info);

/* y = A x for the current linearization (Eq. lin_sys_A).  prec = ST_FP64:
 * x, y are double*; prec = ST_MIXED: float* (FP32 arithmetic).  x and y must
 * not overlap.  ST_ERR_STATE before the first st_ionic / st_linearize. */
st_status st_apply(st_handle *h, int prec, const void *x_dev, void *y_dev);

/* z = A-hat^{-1} r, the preconditioner of Eq. (preconditioner) applied by fast
 * diagonalization (Eq. factorized): spatial transforms with U_l^T, one banded
 * time solve per spatial eigenvalue, transforms with U_l.  Types as st_apply. */
st_status st_precond(st_handle *h, int prec, const void *r_dev, void *z_dev);

/* Solve A x = b_dev to ||b - A x||_2 / ||b||_2 <= desc.rtol (true residual in
 * FP64), starting from the x_dev passed in.  FP64 mode: flexible
 * right-preconditioned restarted GMRES in FP64.  Mixed mode: FP64 iterative
 * refinement around FP32 flexible GMRES (the FP32 preconditioner uses TF32
 * tensor cores, so it is kept as Z = M^{-1} V).  Arnoldi uses classical
 * Gram-Schmidt with one delayed reorthogonalization (two passes over the
 * basis per step) and FP64-accumulated inner products.  An FP32 cycle ends at
 * its tolerance, or where its iterate stops improving: when its Arnoldi
 * residual estimate first drops below 1e-3, 1e-4, ..., and every 10 columns
 * after that, it forms its iterate (one extra operator application) and ends
 * if the true residual is above twice the estimate.
 * ST_ERR_NOT_CONVERGED after desc.max_it inner iterations (x holds the best
 * iterate). */
st_status st_linsolve(st_handle *h, const double *b_dev, double *x_dev, st_stats *stats);

/* w_dev = L^{-1} g(u) (Eq. lin_sys_L): by the exact elimination of Sec. 3.2,
 * w = b (W_t + b d_e M_t)^{-1} M_t applied along time at every spatial index. */
st_status st_wupdate(st_handle *h, const double *u_dev, double *w_dev);

/* Allocation-free w-update.  The paper has no counterpart: this is the
 * operation of st_wupdate (Sec. 3.2, w = b (W_t + b d_e M_t)^{-1} M_t applied
 * along time at every spatial index) without a handle, for callers that
 * cannot allocate device memory -- e.g. a serving process whose device memory
 * is committed to admitted requests (admission by st_footprint) or owned by
 * another allocator, where cudaMalloc may fail and cudaFree would synchronize
 * the whole device and stall the other requests' streams.
 *
 * desc: the problem (only d, p, n_el, n_el_t, T, b, d_e are used; the whole
 * description must pass the checks of st_setup).  u_dev, w_dev: device
 * vectors of N_dof FP64 values in the layout above, u_dev != w_dev; w_dev is
 * overwritten.  cuda_stream: the stream the work is enqueued on (0 = legacy
 * default stream).  Result: the same values as st_wupdate on a handle set up
 * from the same description.
 *
 * Synchronization: the call is not fully asynchronous.  The two bands are
 * copied from ordinary (pageable) host memory that the call owns only while
 * it runs; a copy from pageable memory first waits for the work already
 * queued on cuda_stream, so the call returns only after that earlier work
 * has finished and the bands have been handed to the device.  The w kernel
 * itself is queued behind the copies and may still be running on return.
 *
 * Memory: no device memory is allocated (no cudaMalloc, cudaFree or
 * allocating library call).  The two time bands M_t and LU(W_t + b d_e M_t),
 * 2 N_t (2p+1) FP64 values, are built on the host (ordinary heap vectors)
 * and copied into one file-scope __device__ array of ST_WUPDATE_STATIC_CAPACITY
 * doubles (576 KiB; N_t <= 4096 at p = 4) per device.  Larger problems return
 * ST_ERR_CAPACITY before any work.  Nothing in that array has to start at
 * zero: each call writes both bands in full before its kernel reads them.
 * The first call on each device (that device current) looks up the array's
 * device address with cudaGetSymbolAddress and caches it; make that first
 * call before any stream capture.
 *
 * Concurrency: the array is shared by every call on a device, so calls that
 * overlap in time (other streams or host threads) race on it; serialize them
 * on one stream. */
#define ST_WUPDATE_STATIC_CAPACITY 73728
st_status st_wupdate_static(const st_problem_desc *desc, const double *u_dev, double *w_dev, void *cuda_stream);

/* Copy the assembled right-hand side f of Eq. (rhsfun) to f_dev (FP64). */
st_status st_rhs(st_handle *h, double *f_dev);

/* The nonlinear loop from the (u_dev, w_dev) passed in (u^0 = w^0 = 0 in the
 * paper): ST_PICARD runs the relaxed fixed point of Sec. 3.1; ST_NEWTON
 * runs Newton on the u-equation with w lagged and theta frozen per step.
 * Stops when ||u^{k+1} - u^k||_inf <= delta; ST_ERR_NOT_CONVERGED after max_fp. */
st_status st_solve(st_handle *h, double *u_dev, double *w_dev, st_stats *stats);

/* Copy internal arrays to HOST memory for inspection; `bytes` must equal the
 * array's size.  what: */
enum {
  ST_GET_THETA_HAT = 0,  /* double[N_t * N_s], row-major (time, space) */
  ST_GET_LOWRANK_S = 1,  /* double[R]          singular values */
  ST_GET_LOWRANK_U = 2,  /* double[N_t * R]    row-major */
  ST_GET_LOWRANK_V = 3,  /* double[N_s * R]    row-major */
  ST_GET_TAU_Q = 4,      /* double[p * n_el_t * (p+1)]  tau_k at time Gauss points */
  ST_GET_FD_EIG = 5,     /* double[sum_l n_l]  generalized eigenvalues of (D_ll K_l, M_l) */
  ST_GET_BANDS_1D = 6,   /* double[(sum_l 2 n_l + 2 N_t) (2p+1)]: M_l, K_l per direction, M_t, W_t */
  ST_GET_REACTION_S = 7, /* double[rank_reaction]  singular values of the low-rank reaction coefficient */
  ST_GET_REACTION_U = 8, /* double[N_t * rank_reaction]  its time factors, row-major */
  ST_GET_REACTION_V = 9, /* double[N_s * rank_reaction]  its space factors, row-major */
  ST_GET_REACTION_TB = 10 /* double[rank_reaction * (p+1) * N_t]  its time mass bands [r][k][it] */
};
st_status st_get(st_handle *h, int what, void *dst_host, size_t bytes);

/* Optional per-stage timing, for measurement only (no part of the method):
 * st_profile(h, 1) clears the record and brackets every later launch group
 * of a stage with CUDA events on the handle's stream; st_profile(h, 0) stops.
 * st_profile_read sums, for one stage, the event-timed milliseconds, the
 * algorithmic bytes moved (the compulsory HBM traffic of the launch group:
 * each input read once, each output written once), the flops, and the number
 * of launch groups.  Stages: */
enum {
  ST_STAGE_KRON = 0,     /* banded Kronecker passes of A */
  ST_STAGE_INTERP = 1,   /* sum-factorization passes between coefficients and Gauss points */
  ST_STAGE_QBAND = 2,    /* time band per spatial Gauss point (reaction + SU terms) */
  ST_STAGE_FD_GEMM = 3,  /* preconditioner spatial transforms */
  ST_STAGE_FD_LU = 4,    /* preconditioner banded time solves */
  ST_STAGE_ARNOLDI = 5,  /* Gram-Schmidt inner products, updates and norms */
  ST_STAGE_IONIC = 6,    /* ionic quadrature and reaction band assembly */
  ST_STAGE_LOWRANK = 7,  /* Theta-hat, Gram matrix, eigen-decomposition, SU bands */
  ST_STAGE_APPLY64 = 8,  /* the operator in FP64 (outer residuals; stages 0-2 then hold FP32 work only) */
  ST_STAGE_COUNT = 10
};
st_status st_profile(st_handle *h, int enable);
/* Self-test of the tensor-core (tcgen05, TF32) spatial transforms of the
 * preconditioner against the CUDA-core transform, run once per process on a
 * ragged problem; *usable = 1 when the FP32 preconditioner uses them, and
 * *max_rel_err is the largest difference relative to the largest value. */
st_status st_tc_selftest(int *usable, double *max_rel_err);
/* Number of kernel launches this library has issued in the process so far. */
long long st_launch_count(void);
st_status st_profile_read(st_handle *h, int stage, double *ms, double *bytes, double *flops, long long *launches);

#ifdef __cplusplus
}
#endif
#endif /* ST_H */
