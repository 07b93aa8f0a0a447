/*
 * hkgeneo.h - C ABI of the GB300 (sm_103a) solver for the indefinite Helmholtz
 * problem  -div(A grad u) - k^2 u = f in Omega,  u = 0 on the boundary
 * (Eq. 1.1 of arXiv 2406.06283), discretised by P1 finite elements
 * (Sec. 2.1, Eq. 2.11-2.12) and solved by right-preconditioned flexible GMRES
 * with the two-level additive Schwarz preconditioner (Eq. 2.22-2.23) whose
 * coarse space is the H_k-GenEO space (Eq. 5.12, Def. 5.1).
 *
 * Conventions shared by every call:
 *  - Every function returns an hk_status; 0 (HK_OK) is success.  No call
 *    throws, aborts or exits.  hk_last_error() gives a one-line message for
 *    the most recent failure on the calling thread.
 *  - Pointers are HOST pointers unless the parameter name ends in _dev
 *    (device pointers on the handle's device).  Input arrays are read during
 *    the call only; the caller keeps ownership of every pointer it passes.
 *  - The library owns every device allocation it makes and frees it in
 *    hk_destroy.  A handle is bound to the device that was current at
 *    hk_setup and to the CUDA stream passed there (NULL = the legacy default
 *    stream).  Calls on one handle must not overlap in time.
 *  - Degrees of freedom (dofs) are the non-Dirichlet nodes in increasing
 *    node index; every dof vector (rhs, u, z, ...) is laid out in that order,
 *    n_rhs vectors one after another (rhs[r * n_dofs + l]).
 *  - Arrays are 0-based; int32_t for indices, double for values.
 */
#ifndef HKGENEO_H
#define HKGENEO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HK_OK = 0,
  HK_BAD_ARG = 1,          /* inconsistent sizes, tau <= 0, overlap < 1, NULL pointer, ... */
  HK_SINGULAR_LOCAL = 2,   /* a local Dirichlet matrix B_i is singular (Remark after Lemma 3.4) */
  HK_SINGULAR_COARSE = 3,  /* the coarse matrix Z^T B Z is singular */
  HK_EIG_FAIL = 4,         /* a local eigenproblem could not be reduced or solved */
  HK_NO_CONVERGENCE = 5,   /* max_iters reached; outputs hold the last iterate */
  HK_OOM = 6,              /* device allocation failed */
  HK_TIMEOUT = 7,          /* a bounded device wait ran out */
  HK_CUDA_ERROR = 8,       /* a CUDA runtime call failed */
  HK_UNSUPPORTED = 9,      /* input outside the library's limits (e.g. a level set wider than 256 dofs) */
  HK_PENDING = 10          /* hk_server_poll: the request has not finished yet */
} hk_status;

enum { HK_FP64 = 0, HK_FP32_PRECOND = 1, HK_SPLIT_BF16_PRECOND = 2 };  /* hk_params.precision */
enum { HK_TWO_LEVEL = 0, HK_ONE_LEVEL = 1, HK_COARSE_ONLY = 2 };  /* hk_params.levels */
enum { HK_AS = 0, HK_RAS_POU = 1 };                            /* hk_params.weighting */

/* Simplicial mesh (Sec. 2.1: any shape-regular triangulation, d = 2 or 3). */
typedef struct {
  int dim;                     /* 2 (triangles) or 3 (tetrahedra) */
  int n_nodes;
  const double* xyz;           /* n_nodes * dim coordinates, node-major */
  int n_elems;
  const int32_t* elems;        /* n_elems * (dim + 1) node ids */
  const uint8_t* is_boundary;  /* n_nodes flags; 1 = Dirichlet node (not a dof) */
} hk_mesh;

/* Decomposition and solver parameters. */
typedef struct {
  int n_sub;                   /* number of subdomains N */
  const int32_t* elem_to_sub;  /* n_elems: non-overlapping element partition {Omega_i'} */
  int overlap_layers;          /* applications of the one-layer extension of Def. 2.3 (>= 1) */
  double tau;                  /* keep local eigenvalues lambda < tau (> 0); Def. 5.1 */
  int precision;               /* HK_FP64: whole solver in FP64.  HK_FP32_PRECOND: the
                                  preconditioner (local and coarse solves) applied in FP32 from
                                  factors computed in FP64; Krylov vectors, matvec and Arnoldi FP64.
                                  HK_SPLIT_BF16_PRECOND: as HK_FP32_PRECOND, with the local block sweeps
                                  (Eq. 2.22) as tensor-core products: every level record R and vector x
                                  split into BF16 pairs (R = R_hi + R_lo, x = x_hi + x_lo) and
                                  R_hi x_hi + R_hi x_lo + R_lo x_hi accumulated in FP32, x kept as the
                                  BF16 pair between levels (about 16 significant bits); where those
                                  sweeps are unavailable (a level wider than 256 dofs, or a subdomain
                                  whose vectors do not fit shared memory) or measured slower for a batch
                                  size, the FP32 sweeps run instead (hk_set_sweep_path). */
  int levels;                  /* HK_TWO_LEVEL (Eq. 2.23), HK_ONE_LEVEL (Eq. 2.22), HK_COARSE_ONLY */
  int weighting;               /* HK_AS: unweighted sum of local solves (Eq. 2.22);
                                  HK_RAS_POU: local solves weighted by 1/mu (variant) */
  int restart;                 /* FGMRES restart length m (1 .. 256) */
  int max_iters;               /* total inner iterations allowed per right-hand side */
} hk_params;

typedef struct hk_handle hk_handle;

/* Setup: device assembly of B = K - k^2 M and D_k = K + k^2 M (Sec. 2.1,
 * Prop. 2.6), the overlapping subdomains by Def. 2.3 applied overlap_layers
 * times, dof/ovdof (Def. 3.2) and mu (Def. 2.7), the local Dirichlet factors
 * of B_i = R_i B R_i^T (Eq. 2.22), the H_k-GenEO eigenproblems (Eq. 5.12) with
 * the eigenvectors below tau, the coarse basis Z = [E_i Xi_i p_l] (Def. 5.1)
 * and the coarse matrix E = Z^T B Z with its inverse (Eq. 2.23).
 *   mesh, elem_coeff (n_elems scalars a_T > 0), k >= 0, params: host inputs.
 *   cuda_stream: a cudaStream_t (may be NULL).  *out receives the handle.
 * Errors: HK_BAD_ARG, HK_UNSUPPORTED, HK_SINGULAR_LOCAL, HK_EIG_FAIL,
 * HK_SINGULAR_COARSE, HK_OOM, HK_CUDA_ERROR; *out is NULL on any error. */
hk_status hk_setup(const hk_mesh* mesh, const double* elem_coeff, double k,
                   const hk_params* params, void* cuda_stream, hk_handle** out);

/* Same as hk_setup, with every array of `mesh`, `elem_coeff` and `params->elem_to_sub` in
 * device memory of the current device (the library copies them; the caller keeps ownership). */
hk_status hk_setup_device(const hk_mesh* mesh_dev, const double* elem_coeff_dev, double k,
                          const hk_params* params, void* cuda_stream, hk_handle** out);

/* Setup with the two nested decompositions of Sec. 2.3.  Coarse: the subdomains of params
 * (elem_to_sub extended overlap_layers times, Def. 2.3), on which the H_k-GenEO eigenproblems, the
 * partition of unity Xi^c and the coarse space are built (Def. 5.1).  Fine: inside every coarse
 * subdomain Omega_i^c, its elements grouped by elem_to_fine (labels 0 .. n_fine_labels-1, e.g. a finer
 * box partition), each group extended fine_overlap_layers times by Def. 2.3 within Omega_i^c, so that
 * Omega_i^c is the union of its Q_i fine subdomains (groups whose subdomain holds no dof are left out).
 * The one-level part of the preconditioner sums the local solves over all fine subdomains (Eq. 2.22);
 * the coarse correction is that of Eq. 2.23.  Every dof must lie in some fine dof set (so
 * fine_overlap_layers >= 1 in practice), else HK_BAD_ARG.  params->levels must be HK_TWO_LEVEL.
 * The handle serves hk_solve, hk_solve_left_dk, hk_apply_precond and hk_theory (Lambda and H^f of the
 * fine subdomains); hk_apply_precond_noalloc and the serving calls do not take it (HK_UNSUPPORTED).
 * Other errors as hk_setup. */
hk_status hk_setup_nested(const hk_mesh* mesh, const double* elem_coeff, double k, const hk_params* params,
                          int n_fine_labels, const int32_t* elem_to_fine, int fine_overlap_layers,
                          void* cuda_stream, hk_handle** out);
/* Same as hk_setup_nested with every array in device memory (as hk_setup_device). */
hk_status hk_setup_nested_device(const hk_mesh* mesh_dev, const double* elem_coeff_dev, double k,
                                 const hk_params* params, int n_fine_labels, const int32_t* elem_to_fine_dev,
                                 int fine_overlap_layers, void* cuda_stream, hk_handle** out);

/* Solve B u = rhs for n_rhs right-hand sides (load vectors) with FGMRES
 * preconditioned on the right by the setup's preconditioner, x_0 = 0, until
 * the relative residual ||rhs - B u|| / ||rhs|| <= tol (checked on the true
 * residual) or max_iters inner iterations.
 *   rhs: n_rhs * n_dofs (host).  u: n_rhs * n_dofs (host, written).
 *   iters: n_rhs (written).  res_hist: NULL or n_rhs * max_iters, written with
 *   the recurrence estimates |g_{j+1}| / ||rhs|| of each inner step (unused
 *   tail left untouched).  final_true_rel_res: NULL or n_rhs.
 * Returns HK_NO_CONVERGENCE (outputs still written) if any rhs did not
 * converge.  The host copies in and out are part of the call. */
hk_status hk_solve(hk_handle* h, int n_rhs, const double* rhs, double tol, double* u,
                   int32_t* iters, double* res_hist, double* final_true_rel_res);

/* Same as hk_solve with rhs_dev and u_dev in device memory (n_rhs * n_dofs
 * doubles each).  iters, res_hist and final_true_rel_res are host arrays. */
hk_status hk_solve_device(hk_handle* h, int n_rhs, const double* rhs_dev, double tol, double* u_dev,
                          int32_t* iters, double* res_hist, double* final_true_rel_res);

/* Left-preconditioned GMRES(m) in the D_k inner product: the Krylov method of Thm. 3.1, on the
 * preconditioned system M^{-1} B u = M^{-1} f of Eq. 2.24 (M^{-1} the setup's preconditioner, in its
 * precision form), with <x, y>_D = y^T D_k x, D_k = A + k^2 S (Prop. 2.6), in the Arnoldi process and
 * the residual minimisation.  x_0 = 0; restart and max_iters from the parameters.  A right-hand side
 * has converged when ||M^{-1}(rhs - B u)||_{D_k} <= tol ||M^{-1} rhs||_{D_k} (the residual of Eq. 4.22).
 *   rhs, u: n_rhs * n_dofs (host).  iters: n_rhs (written).  res_hist: NULL or n_rhs * max_iters,
 *   the recurrence estimates ||M^{-1} r_j||_{D_k} / ||M^{-1} rhs||_{D_k} of each inner step (unused tail
 *   untouched).  final_true_rel_res: NULL or n_rhs, ||rhs - B u|| / ||rhs||.  final_pc_rel_res: NULL or
 *   n_rhs, the D_k-norm ratio at the end.
 * Returns HK_NO_CONVERGENCE (outputs still written) if any rhs did not converge.  The loop is driven
 * from the host (one small device-to-host copy per inner step); results do not depend on n_rhs. */
hk_status hk_solve_left_dk(hk_handle* h, int n_rhs, const double* rhs, double tol, double* u, int32_t* iters,
                           double* res_hist, double* final_true_rel_res, double* final_pc_rel_res);
/* Same with rhs_dev and u_dev in device memory (n_rhs * n_dofs doubles each). */
hk_status hk_solve_left_dk_device(hk_handle* h, int n_rhs, const double* rhs_dev, double tol, double* u_dev,
                                  int32_t* iters, double* res_hist, double* final_true_rel_res,
                                  double* final_pc_rel_res);

/* The quantities of Thm. 3.1 for this handle (two-level preconditioner). */
typedef struct {
  double Lambda;          /* most subdomains sharing one element (the fine subdomains are the subdomains) */
  double tau;             /* min_i lambda_{m_i+1}: the smallest local eigenvalue left out of the coarse space
                             (the FP64-refined value next above the kept ones; not certified by an inertia
                             count) */
  int tau_is_lower_bound; /* 1: no subdomain had a refined value above its kept ones below tau + 0.05, and
                             tau holds that bound */
  double Theta;           /* 1 / tau */
  double k;               /* wavenumber */
  double H_f;             /* largest subdomain diameter used (given, or the largest bounding-box diagonal of
                             a subdomain's dof nodes when the caller passes H_f <= 0) */
  double c_stab;          /* the stability constant C_stab of the problem (caller's value) */
  double s;               /* Eq. 4.3 */
  double gamma;           /* Eq. 4.5: ||r^(m)||_D^2 <= (1 - gamma^2)^m ||r^(0)||_D^2 when s < 1 */
  int guaranteed;         /* s < 1 */
} hk_theory_t;
/* Errors: HK_BAD_ARG; HK_UNSUPPORTED for a one-level or coarse-only handle. */
hk_status hk_theory(const hk_handle* h, double c_stab, double H_f, hk_theory_t* out);

typedef struct {
  int dim, n_nodes, n_elems, n_dofs, n_sub;
  int n0;                      /* coarse dimension sum_i m_i */
  int max_mu;                  /* largest multiplicity mu_l (Def. 2.7) */
  int lambda_elems;            /* Lambda: most subdomains sharing one element */
  int max_level;               /* widest level set of any local factor */
  int max_dof;                 /* largest |dof(Omega_i)| */
  int nnz;                     /* nonzeros of B */
  int precision, levels;
  size_t bytes_resident;       /* device bytes held by the handle */
  long long factor_elems;      /* entries of all local factor blocks (FP64, setup only): the inverse of each
                                  level's Schur complement and its coupling product of the twisted
                                  block factorisation, each padded to 4 entries */
  long long dof_total;         /* sum_i |dof(Omega_i)| */
  long long coarse_elems;      /* entries of all Z_i, sum_i |dof(Omega_i)| m_i */
  long long lower_nnz;         /* couplings L_j between consecutive level sets, sum over subdomains */
  double setup_ms[8];          /* phases: assembly, decomposition, local factors, eigen, coarse,
                                  total; [6], [7] 0 (unused) */
  size_t bytes_peak;           /* most device bytes the handle held at once (setup temporaries included) */
  long long graph_solves;      /* solves run as one CUDA graph (device-side loops); the others were
                                  driven from the host (kernel timing on, graph capture unavailable, or
                                  graphs switched off by hk_set_solve_graphs) */
  double eigen_kernel_ms[4];   /* setup kernels of the eigenproblems: [0] FP64 inertia count below tau,
                                  [1] FP32 Lanczos candidates, [2] FP64 refinement, [3] 0 */
  double eigen_kernel_gflop[4]; /* their algorithmic work in GFLOP (2 per multiply-add of the dense level
                                  operations: factorisations, sweeps, Gram-Schmidt, projections) */
  long long tc_record_bytes;   /* device bytes of the split-BF16 level records of the tensor-core sweeps
                                  (0: not built, i.e. another precision form or sweeps unavailable) */
  int last_sweeps;             /* local sweeps of the last preconditioner apply: HK_SWEEPS_CUDA_CORE or
                                  HK_SWEEPS_TENSOR_CORE (0 before the first apply) */
  int twist_moved;             /* subdomains whose block factorisation meets at a level other than the
                                  middle one (chosen for a smaller pivot growth, see local_growth) */
  double local_growth[2];      /* largest pivot growth ||pivot block inverse||_inf x ||B_i||_inf over the
                                  local factorisations: [0] as factored (a subdomain whose growth towards
                                  its middle level exceeds 1000 and 50x the median, or which meets a
                                  pivot below 1e-10 max|B_i| there, is factored towards another level),
                                  [1] had every subdomain been factored towards its middle level (inf
                                  where a level block was singular in floating point) */
  int fine_subdomains;         /* nested decompositions (hk_setup_nested): number of fine subdomains
                                  (sum_i Q_i), else 0; the local solves, max_level, twist_moved,
                                  local_growth, tc_record_bytes, last_sweeps and levels_merged then
                                  refer to them */
  int fine_lambda_elems;       /* Lambda over the fine subdomains (Sec. 2.4), else 0 */
  int fine_max_dof;            /* largest |dof(Omega^f_{i,j})|, else 0 */
  long long fine_dof_total;    /* sum of |dof(Omega^f_{i,j})|, else 0 */
  int levels_merged;           /* level boundaries removed from the local factorisations: where no twist
                                  level avoids a singular (or outlying) leading or trailing level block,
                                  the first such level of each one-sided elimination is merged with its
                                  successor (wider blocks, fewer levels; see max_level) */
} hk_info_t;

hk_status hk_info(const hk_handle* h, hk_info_t* info);

/* Frees every device allocation of the handle.  NULL is accepted. */
hk_status hk_destroy(hk_handle* h);

const char* hk_status_string(hk_status s);
const char* hk_last_error(void);

/* ---- Kernel timing (CUDA events on the handle's stream) ---- */
enum {
  HK_T_LOCAL_APPLY = 0,  /* gather, coarse restriction and local block sweeps (Eq. 2.22) */
  HK_T_COARSE_SOLVE = 1, /* E^{-1} c (Eq. 2.23) */
  HK_T_SCATTER = 2,      /* pull-form sum of local and coarse corrections */
  HK_T_SPMV = 3,         /* B z */
  HK_T_ARNOLDI = 4,      /* Gram-Schmidt passes, Givens update, normalisation */
  HK_T_CYCLE = 5,        /* cycle end: least squares, x update, true residual */
  HK_T_NCAT = 6
};
/* on != 0 starts recording the solve kernels of later calls (and clears earlier records). */
hk_status hk_set_timing(hk_handle* h, int on);
/* Sums the recorded launches per category: ms[HK_T_NCAT] milliseconds, count[HK_T_NCAT] launches. */
hk_status hk_kernel_times(hk_handle* h, double* ms, int32_t* count);

/* on != 0 (the default): each hk_solve runs as one CUDA graph whose FGMRES cycle and inner-step loops
 * are device-side conditional WHILE nodes (one launch, one synchronisation per solve).  on == 0: the
 * same kernels with the loops driven from the host (one synchronisation per inner step).  The results
 * are bitwise the same.  Graphs pay off for a handle solved alone; handles whose solves overlap with
 * other handles' on other streams (the serving calls) run faster without them. */
hk_status hk_set_solve_graphs(hk_handle* h, int on);

/* Local sweeps of the split-BF16 form (hk_params.precision == HK_SPLIT_BF16_PRECOND):
 * HK_SWEEPS_AUTO (the default) runs the tensor-core sweeps unless the handle's autotuner, which times
 * both on the first solve of each batch size, measured the FP32 CUDA-core sweeps faster;
 * HK_SWEEPS_CUDA_CORE always runs the FP32 sweeps; HK_SWEEPS_TENSOR_CORE always runs the tensor-core
 * sweeps.  Pinning a path makes results reproducible bit for bit across processes (the automatic
 * choice depends on timings).  Errors: HK_BAD_ARG (unknown path), HK_UNSUPPORTED (tensor-core sweeps
 * asked for in another precision form, or unavailable for this handle's subdomains). */
enum { HK_SWEEPS_AUTO = 0, HK_SWEEPS_CUDA_CORE = 1, HK_SWEEPS_TENSOR_CORE = 2 };
hk_status hk_set_sweep_path(hk_handle* h, int path);

/* Waits for the handle's device work and reports a failure that a kernel recorded since the last
 * check: a bounded device wait that ran out (HK_TIMEOUT) or a failed pivot.  The record is cleared
 * by this call (and by every call that reports it: hk_solve, hk_solve_device, hk_apply_precond),
 * so each failure is reported once.  Callers of hk_apply_precond_noalloc use it after their work,
 * since that call does not synchronise. */
hk_status hk_check_status(hk_handle* h);

/* Test hook of the failure path: the number of polls a grid barrier of the cooperative
 * Gram-Schmidt step makes before it gives up and records HK_TIMEOUT (default 2^25, about a second;
 * 0 restores the default).  With a small limit a solve ends after the inner step whose barrier gave
 * up, returns HK_TIMEOUT and leaves the handle usable.  Other waits keep their limits. */
hk_status hk_set_wait_limit(hk_handle* h, int grid_barrier_polls);

/* Number of CUDA kernels the library has launched in this process so far (all handles). */
long long hk_kernel_launches(void);

/* ---- Inspection and single-step calls (same data the solve uses) ---- */

/* CSR of B (which = 0) or D_k (which = 1): rowptr n_dofs+1, col/val nnz. */
hk_status hk_get_matrix(const hk_handle* h, int which, int32_t* rowptr, int32_t* col, double* val);

/* Subdomain i: sizes[0] = |dof(Omega_i)|, sizes[1] = |ovdof \ dof|, sizes[2] = number of
 * level sets, sizes[3] = m_i.  Any of the arrays may be NULL:
 * dof: |dof| global dof ids in the factor's level order; gamma: |ovdof \ dof| ids, increasing;
 * level_ptr: level sets + 1 offsets into dof. */
hk_status hk_get_subdomain(const hk_handle* h, int i, int32_t* sizes, int32_t* dof, int32_t* gamma,
                           int32_t* level_ptr);

/* mu_l for every dof (n_dofs). */
hk_status hk_get_mu(const hk_handle* h, int32_t* mu);

/* Kept eigenvalues of subdomain i (m_i, ascending) and the coarse vectors Z_i
 * (|dof| x m_i row-major, rows in the level order of hk_get_subdomain's dof). */
hk_status hk_get_eigen(const hk_handle* h, int i, double* lam, double* Z);

/* E = Z^T B Z and its inverse (n0 x n0 row-major each; either may be NULL). */
hk_status hk_get_coarse(const hk_handle* h, double* E, double* Einv);

/* z = M^{-1} v (one preconditioner apply, Eq. 2.23 / 2.22) for n_rhs host vectors. */
hk_status hk_apply_precond(hk_handle* h, int n_rhs, const double* v, double* z);

/* Allocation-free variant of hk_apply_precond (the paper has no counterpart: this is a service
 * for callers that may not allocate device memory, such as code recording a CUDA graph or a
 * framework that forbids allocations on its hot path).  z_dev = M^{-1} v_dev for n_rhs device
 * vectors (n_rhs * n_dofs doubles each, caller-owned).  Intermediate vectors live in one fixed
 * 8 MiB device array per device, held from library load until process exit; a request that
 * needs more (n_rhs * (2 sum_i |dof(Omega_i)| + 2 (n0 + 1)) elements of 4 bytes in the FP32 form,
 * 8 in the FP64 form, each part rounded up to 256 bytes) returns HK_UNSUPPORTED before any
 * launch.  The first call on a device looks the array's address up and raises the apply kernels'
 * shared-memory limits (call it before any stream capture).  All calls share the array: calls
 * that overlap on the GPU race.  Ordered on the handle's stream (the coarse part runs on a
 * second, high-priority stream of the handle, forked from and joined back into it); calls no
 * cudaMalloc/cudaFree or allocating library routine.  Like the other apply calls, a bounded
 * device wait that runs out is recorded on the handle: hk_check_status reports it. */
hk_status hk_apply_precond_noalloc(hk_handle* h, int n_rhs, const double* v_dev, double* z_dev);

/* y = B x for n_rhs host vectors. */
hk_status hk_matvec(hk_handle* h, int n_rhs, const double* x, double* y);

/* Load vector (f, phi_l) of the P1 interpolant of nodal values f_nodal (n_nodes), written to
 * rhs (n_dofs); exact for piecewise-linear f (Eq. 2.12's right-hand side). */
hk_status hk_assemble_load(hk_handle* h, const double* f_nodal, double* rhs);

/* ---- Serving: a request loop over cached operators ----
 *
 * A server owns a set of operators (problem descriptions: mesh, coefficients, k,
 * parameters) and answers solve requests on them.  The method has no serving
 * layer; this is the deployment form of the same setup (hk_setup) and solve
 * (hk_solve), with three properties:
 *  - Operator cache.  An operator's setup (factors, coarse space, E^{-1}) is
 *    built on its first request and kept resident, keyed by the operator's
 *    content (a 64-bit FNV-1a hash of every input array and parameter), so
 *    later right-hand sides skip setup.  Adding identical content twice
 *    returns the same id.
 *  - Admission by device memory.  The resident operators (their
 *    hk_info_t.bytes_resident, solve workspaces included) plus reservations for
 *    setups and solves in flight stay within `device_mem_budget`.  A setup
 *    reserves its peak: 24 KiB per dof (2D) or 64 KiB per dof (3D) before the
 *    operator's first setup, 1.25 x the measured hk_info_t.bytes_peak after it.
 *    A solve of s right-hand sides on n dofs reserves the workspace it lacks, for
 *    S = s rounded up to a power of two (the handle's workspace capacity):
 *    8 S ((2 restart + 6) n + (restart + 1)(restart + 4) + max_iters) bytes plus
 *    the preconditioner's buffers and 1 MiB.  When a batch does not fit, idle
 *    operators are evicted, least recently used first; a request waits while
 *    the memory is held by work in flight.  A request whose operator cannot fit
 *    even in an empty server fails with HK_OOM.
 *  - Continuous batching.  `n_slots` worker threads each drive their own CUDA
 *    stream.  A free slot takes the oldest waiting request whose operator is
 *    not in use, together with every other waiting request on that operator
 *    with the same tol (up to `max_batch_rhs` right-hand sides), and solves
 *    them as one multi-right-hand-side FGMRES.  Work on different operators
 *    overlaps on the device.  Each right-hand side's arithmetic is the same
 *    alone and in a batch: results do not depend on the mix.
 * All calls are thread-safe.  Times are milliseconds since hk_server_create. */
typedef struct hk_server hk_server;

/* device_mem_budget: bytes (> 0) on the current device; n_slots: worker threads/streams (1..64);
 * max_batch_rhs: most right-hand sides solved together (1..64). */
hk_status hk_server_create(size_t device_mem_budget, int n_slots, int max_batch_rhs, hk_server** out);

/* Registers an operator (arguments as hk_setup; the arrays are copied).  No device work happens
 * here.  *op_id receives the operator's id. */
hk_status hk_server_add_operator(hk_server* srv, const hk_mesh* mesh, const double* elem_coeff, double k,
                                 const hk_params* params, uint64_t* op_id);

/* Queues n_rhs right-hand sides (n_rhs * n_dofs doubles, copied) on operator op_id.
 * *ticket identifies the request for hk_server_poll. */
hk_status hk_server_submit(hk_server* srv, uint64_t op_id, int n_rhs, const double* rhs, double tol,
                           uint64_t* ticket);

typedef struct {
  double submit_ms, start_ms, end_ms; /* queued, taken by a slot, finished */
  int32_t batch_rhs;                  /* right-hand sides in the solve that served the request */
  int32_t setup_ran;                  /* 1 if the operator's setup ran for this batch (cache miss) */
  int32_t slot;                       /* worker slot */
  int32_t n_rhs;
} hk_request_info;

/* Waits up to wait_ms (0 = do not wait, < 0 = without limit) for request `ticket`.  While it
 * runs: HK_PENDING.  Once finished: writes the outputs as hk_solve does (u: n_rhs * n_dofs,
 * iters: n_rhs, res_hist: NULL or n_rhs * max_iters, final_true_rel_res: NULL or n_rhs,
 * info: NULL or one record), forgets the ticket and returns the request's status.  An unknown
 * ticket gives HK_BAD_ARG. */
hk_status hk_server_poll(hk_server* srv, uint64_t ticket, int wait_ms, double* u, int32_t* iters,
                         double* res_hist, double* final_true_rel_res, hk_request_info* info);

typedef struct {
  long long submitted, completed, failed; /* requests */
  long long setups, evictions, batches, cache_hits;
  int resident_ops, n_ops, queued;
  size_t bytes_in_use, bytes_peak, budget;
} hk_server_stats;

hk_status hk_server_get_stats(hk_server* srv, hk_server_stats* out);

/* Finishes the work in flight, fails the queued requests (their tickets are dropped), frees every
 * operator and the server.  NULL is accepted. */
hk_status hk_server_destroy(hk_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* HKGENEO_H */
