// Internal declarations of the hkgeneo CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <string>
#include <map>
#include <vector>

#include "hkgeneo.h"

// Library limits (checked at setup, HK_UNSUPPORTED beyond them).
#define HK_MAXB 256        // widest level set of a local block-tridiagonal factor
#define HK_MAXM 256        // most eigenvectors kept on one subdomain
#define HK_MAXROW 64       // most nonzeros in one row of B
#define HK_MAXSTAR 64      // most elements around one node
#define HK_MAXRESTART 256  // longest FGMRES cycle

// Device error record written by kernels (first nonzero code wins).
struct DevStatus {
  int code;     // hk_status
  int where;    // subdomain / row / step that failed
  double value; // offending value (pivot, ...)
};

__device__ __forceinline__ void dev_fail(DevStatus* st, int code, int where, double value) {
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->where = where;
    st->value = value;
  }
}

void hk_set_error(const char* fmt, ...);

// Every kernel launch of the library bumps this process-wide counter (hk_kernel_launches()).
extern std::atomic<long long> g_hk_launches;
// >= 0 while this thread captures a CUDA graph: captured kernels are counted here, and the graph's
// executions are added to g_hk_launches after each replay.
extern thread_local int g_hk_capture_count;
inline void hk_count_launch() {
  if (g_hk_capture_count >= 0) ++g_hk_capture_count;
  else g_hk_launches.fetch_add(1, std::memory_order_relaxed);
}
#define HK_COUNT_LAUNCH() hk_count_launch()

#define HK_TRY(expr)                         \
  do {                                       \
    hk_status s_ = (expr);                   \
    if (s_ != HK_OK) return s_;              \
  } while (0)

#define HK_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      hk_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));   \
      return e_ == cudaErrorMemoryAllocation ? HK_OOM : HK_CUDA_ERROR;                     \
    }                                                                                      \
  } while (0)

#define HK_LAUNCH_CHECK() HK_CUDA(cudaGetLastError())

// A device array with its element count.
template <typename T>
struct DArr {
  T* p = nullptr;
  size_t n = 0;
};

// The preconditioner is applied in FP32 arithmetic (FP32 and split-BF16 forms).
inline bool precond_f32(const hk_params& p) { return p.precision != HK_FP64; }

// Per-subdomain Krylov / apply workspace sizes are derived from these.
struct Sub {
  int nI, nG, L;        // |dof|, |ovdof \ dof|, number of level sets
  int I_off;            // offset of the subdomain's dof rows in concatenated arrays
  int G_off;            // offset into concatenated Gamma lists
  int lev_off;          // offset of its level pointer array (L + 1 entries)
  long long f_off;      // offset of its factor blocks (elements)
  long long csr_off;    // offset of its local CSR entries
  int m;                // kept eigenvectors
  int c_off;            // offset in the coarse vector
  long long z_off;      // offset of Z_i (nI * m)
  int bw;               // half bandwidth of D_II in level order
  int M;                // twist level of its local factorisation (see hk_local.cu)
};

struct hk_handle {
  int dev = 0;
  cudaStream_t stream = nullptr;
  int dim = 0, nv = 0, n_nodes = 0, n_elems = 0, n = 0, n_sub = 0;
  double k = 0;
  hk_params p{};
  // sizes
  int nnz = 0, n0 = 0, max_mu = 0, lambda_elems = 0, max_level = 0, max_dof = 0, max_L = 0, n_sm = 0;
  long long I_total = 0, G_total = 0, f_total = 0, csr_total = 0, z_total = 0, lower_nnz = 0;
  std::vector<Sub> subs;
  double setup_ms[8] = {0};
  double eigen_ms[4] = {0};     // inertia, Lanczos, refinement (hk_info_t.eigen_kernel_ms)
  double eigen_gflop[4] = {0};  // their algorithmic GFLOP (hk_info_t.eigen_kernel_gflop)

  // ---- device data kept for the solve ----
  DevStatus* d_status = nullptr;
  double* d_xyz = nullptr;
  int* d_elems = nullptr;
  double* d_coeff = nullptr;
  int* d_dof_of_node = nullptr;   // n_nodes, -1 on Dirichlet nodes
  int* d_node_of_dof = nullptr;   // n
  int* d_ne_ptr = nullptr;        // node -> element CSR
  int* d_ne_idx = nullptr;
  int* d_rowptr = nullptr;        // CSR of B / D_k over dofs
  int* d_col = nullptr;
  double* d_valB = nullptr;
  double* d_valD = nullptr;
  int* d_mu = nullptr;            // n
  // subdomain lists
  int* d_sub_info = nullptr;      // per subdomain: nI, nG, L, I_off, G_off, lev_off, m, c_off (8 ints)
  long long* d_sub_off = nullptr; // per subdomain: f_off, csr_off, z_off (3 long long)
  int* d_I = nullptr;             // I_total: global dof ids, level order
  int* d_Isorted = nullptr;       // I_total: global dof ids, increasing
  int* d_perm = nullptr;          // I_total: position in level order of each Isorted entry
  int* d_G = nullptr;             // G_total: Gamma ids, increasing
  int* d_lev = nullptr;           // level pointers
  // local CSR (rows in level order): capacity per row = global row length
  int* d_lrow = nullptr;          // I_total + n_sub row starts (per subdomain: nI + 1)
  int* d_lcntI = nullptr;         // I_total: entries inside dof
  int* d_lcntG = nullptr;         // I_total: entries on Gamma
  int* d_lcol = nullptr;          // csr_total
  double* d_lvalB = nullptr;      // csr_total
  double* d_lvalD = nullptr;      // csr_total
  // pull map
  int* d_pull_ptr = nullptr;      // n + 1
  int* d_pull_row = nullptr;      // entries: global row in concatenated level-ordered arrays
  int* d_pull_sub = nullptr;      // entries: subdomain id
  // local factors: per level S_j^{-1} (b_j x b_j) then G_j (b_j x b_{j+1}), row-major (setup only)
  double* d_F64 = nullptr;
  // level records streamed by the apply (see hk_local.cu), their table and the largest record
  unsigned char* d_pack = nullptr;
  long long* d_lvtab = nullptr;
  long long* d_lvfo = nullptr;    // setup only: per level, offset of its blocks in the FP64 factors
  long long pack_bytes = 0, pack_stage = 0;
  // split-BF16 form: level records of the tensor-core sweeps (see hk_tc.cu), their table, the ring
  // stage size, the widest padded level-ordered vector and whether the sweeps are available
  unsigned char* d_pack_tc = nullptr;
  long long* d_lvtab_tc = nullptr;
  int* d_tc_prow = nullptr;     // per local dof (level order): its row in the padded level order
  long long tc_bytes = 0;
  int tc_stage = 0, tc_max_apad = 0;
  bool tc_ok = false;
  int sweep_path = 0;           // hk_set_sweep_path
  int last_sweeps = 0;          // HK_SWEEPS_* of the last apply
  std::map<int, int> tc_tuned;  // per batch size: 1 if the tensor-core sweeps measured faster
  // coarse space
  double* d_lam = nullptr;        // per subdomain kept eigenvalues (HK_MAXM each)
  double* d_Z64 = nullptr;        // z_total, per subdomain nI x m row-major
  void* d_Zt = nullptr;           // Z in the apply's type, per subdomain m x nI (restriction and prolongation)
  double* d_E = nullptr;          // n0 x n0
  double* d_Einv64 = nullptr;
  float* d_Einv32 = nullptr;

  // ---- solve workspace (grown on demand) ----
  int ws_rhs = 0, ws_m = 0;
  double* d_V = nullptr;          // (m + 1) x s x n
  double* d_Zk = nullptr;         // m x s x n
  double* d_w = nullptr;          // s x n
  double* d_x = nullptr;          // s x n
  double* d_f = nullptr;          // s x n
  double* d_ybuf64 = nullptr;     // s x I_total local solutions (FP64 form)
  float* d_ybuf32 = nullptr;      // s x I_total (FP32 form)
  double* d_c64 = nullptr;        // s x n0 coarse rhs
  double* d_cc64 = nullptr;       // s x n0 coarse solution
  float* d_c32 = nullptr;
  float* d_cc32 = nullptr;
  double* d_part = nullptr;       // reduction partials
  unsigned* d_counter = nullptr;  // last-block counters
  double* d_H = nullptr;          // s x (m+1) x m Hessenberg
  double* d_cs = nullptr;         // s x m
  double* d_sn = nullptr;
  double* d_g = nullptr;          // s x (m+1)
  double* d_hcol = nullptr;       // s x 2 x (m+1) Gram-Schmidt coefficients
  int* d_state = nullptr;         // s x 8 per-rhs control words
  double* d_rstate = nullptr;     // s x 8 per-rhs scalars (||f||, beta, residual, ...)
  double* d_hist = nullptr;       // s x max_iters
  int* h_state = nullptr;         // pinned host mirror of d_state
  double* h_rstate = nullptr;
  int h_code = 0;                 // host copy of d_status->code (host-driven solve loop)
  unsigned wait_polls = 1u << 25; // polls of a grid barrier before it gives up (hk_set_wait_limit)

  std::vector<std::pair<void*, size_t>> allocs;  // live allocations and their sizes
  size_t bytes_peak = 0;
  size_t bytes = 0;
  bool dev_inputs = false;  // setup arrays are device pointers
  // FGMRES solve as one CUDA graph per (right-hand sides, tol), its cycle and inner-step loops run on
  // the device by conditional WHILE nodes (see hk_krylov.cu)
  struct SolveGraph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    int iter_kernels = 0, cycle_kernels = 0;
  };
  std::map<std::pair<int, double>, SolveGraph> graphs;
  bool graphs_ok = true;        // false after a failed graph build: the host-driven loop is used
  int coop_state = 0;           // cooperative Gram-Schmidt launch: 0 unknown, 1 usable, -1 not
  bool use_graphs = true;       // hk_set_solve_graphs
  long long graph_solves = 0;
  std::map<int, int> nr_tuned;  // right-hand sides per apply CTA chosen by apply_autotune, per batch size
  cudaStream_t cap_stream = nullptr;  // blocking stream for graphs when the handle's stream is the legacy one
  cudaStream_t aux_stream = nullptr;  // setup: local factors overlapping the eigenproblems
  cudaEvent_t ev_lf = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;  // apply: coarse path beside the local sweeps
  cudaStream_t co_stream = nullptr;                    // apply: the coarse path's stream (high priority)
  bool lf_pending = false;
  int lf_stage = 0;             // local factors: 1 growth pass launched, 2 factors launched
  std::vector<int> lev_host;    // setup only: host copy of the level pointers
  double* d_gF = nullptr;       // setup only: growth pass scratch factors, offsets, results
  long long* d_gfo = nullptr;
  double* d_gval = nullptr;
  int* d_twist = nullptr;       // per subdomain: twist level M of its factorisation
  double growth_twist = 0, growth_mid = 0;  // max over subdomains of the pivot growth (chosen M; M = (L-1)/2)
  int twist_moved = 0;          // subdomains whose twist level is not the middle one
  int levels_merged = 0;        // level boundaries removed where no twist level avoided a singular block
  // nested decompositions (Sec. 2.3): this handle holds the coarse subdomains (eigenproblems, coarse
  // space) and child the fine ones (local solves, a one-level handle that only applies); fine_parent: the
  // coarse subdomain of each fine one
  hk_handle* child = nullptr;
  bool apply_only = false;
  std::vector<int> fine_parent;
  double tau_next = INFINITY;   // min over subdomains of the first local eigenvalue not kept (Thm. 3.1 tau)
  bool tau_next_lb = false;     // tau_next is only the lower bound tau + delta (no candidate above the kept)
  int* d_ctl = nullptr;         // [0] inner step j, [1] cycles run, [2] inner steps run
  const int* g_jp = nullptr;    // while an inner step is captured: the device word holding j
  long long g_jstride = 0;      // ... and the distance between consecutive Krylov vectors

  // kernel timing
  bool timing = false;
  struct TL { int cat; cudaEvent_t a, b; };
  std::vector<TL> tl;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
};

cudaEvent_t hk_event(hk_handle* h);
// Wraps a launch in two recorded events when timing is on.
#define HK_TIMED(h, cat, ...)                                        \
  do {                                                               \
    cudaEvent_t ta_ = nullptr;                                       \
    if ((h)->timing) {                                               \
      ta_ = hk_event(h);                                             \
      cudaEventRecord(ta_, (h)->stream);                             \
    }                                                                \
    __VA_ARGS__;                                                     \
    if ((h)->timing) {                                               \
      cudaEvent_t tb_ = hk_event(h);                                 \
      cudaEventRecord(tb_, (h)->stream);                             \
      (h)->tl.push_back({(cat), ta_, tb_});                          \
    }                                                                \
  } while (0)

// Allocation helper: zero-initialised device memory tracked by the handle, from the device's
// stream-ordered memory pool (hk_pool_init keeps freed blocks cached in the pool, so repeated setups
// and solves do not go back to the driver).
void hk_pool_init(int dev);
template <typename T>
hk_status dalloc(hk_handle* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  hk_pool_init(h->dev);
  cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), h->stream);
  if (e != cudaSuccess) {
    hk_set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    return HK_OOM;
  }
  h->allocs.emplace_back((void*)*p, count * sizeof(T));
  h->bytes += count * sizeof(T);
  if (h->bytes > h->bytes_peak) h->bytes_peak = h->bytes;
  e = cudaMemsetAsync(*p, 0, count * sizeof(T), h->stream);
  if (e != cudaSuccess) {
    hk_set_error("cudaMemset failed: %s", cudaGetErrorString(e));
    return HK_CUDA_ERROR;
  }
  return HK_OK;
}

void dfree(hk_handle* h, void* p);

// Raises a kernel's dynamic shared-memory limit once, to the device's opt-in maximum minus the
// kernel's static shared memory.  The limit is a per-kernel global setting: raising it to the maximum
// once (instead of to each launch's size) keeps concurrent setups on other host threads from
// lowering it under a launch.  The launch still asks for exactly the bytes it uses.
hk_status hk_allow_smem_fn(const void* fn);
hk_status hk_max_carveout_fn(const void* fn);
template <typename F>
hk_status hk_max_carveout(F* fn) {
  return hk_max_carveout_fn(reinterpret_cast<const void*>(fn));
}
template <typename F>
hk_status hk_allow_smem(F* fn) {
  return hk_allow_smem_fn(reinterpret_cast<const void*>(fn));
}

// Reads the device status record (synchronising the handle's stream) and clears it; returns its code
// with a message naming the phase.
hk_status check_device_status(hk_handle* h, const char* phase);

// Sparse H_k-GenEO pencil (B^N, C) over ovdof(Omega_i) of every subdomain, rows in the level order of
// ovdof (built in hk_eigen.cu; used by the eigenvalue kernels of hk_lanczos.cu and the refinement).
struct OvdofPencil {
  const int* o_off = nullptr;     // device: first row of each subdomain
  const int* levptr = nullptr;    // device: per subdomain L + 1 level pointers, at o_off[s] + s
  const int* L = nullptr;         // device: level count per subdomain
  const int* cnt = nullptr;       // device: row lengths
  const int* col = nullptr;       // device: maxrow columns per row
  const double* B = nullptr;      // device: B^N values
  const double* C = nullptr;      // device: C values
  const int* o2i = nullptr;       // device: dof level position of each row (-1 on Gamma)
  int maxrow = 0, max_b = 0, max_nO = 0;
  std::vector<int> h_off, h_nO, h_L;   // host copies: first row, rows, levels per subdomain
  std::vector<int> h_levptr;           // host copy of the level pointers
};
// #{lambda < tau} per subdomain (FP64 inertia of B^N - tau C), into d_neg, on stream st (which must
// follow the setup stream's work up to the pencil).
hk_status eigen_inertia(hk_handle* h, const OvdofPencil& op, double tau, int* d_neg, cudaStream_t st);
// Candidate eigenvalues below lam_cut (FP32 shift-invert block Lanczos), ascending, into d_lamhat (HK_MAXM
// per subdomain) and their number into d_cnt, for every subdomain s with cols[s] > 0 (the largest Krylov
// basis; the others are left as they are).  The basis starts at cols0 columns and grows to 4 c + 48 (c the
// candidates counted) when that is larger.  *ms: the kernel's time.
hk_status eigen_lanczos(hk_handle* h, const OvdofPencil& op, const std::vector<int>& cols, int cols0, double lam_cut,
                        double* d_lamhat, int* d_cnt, float* ms);

// ---- phases (each file implements one) ----
hk_status phase_assembly(hk_handle* h, const hk_mesh* mesh, const double* coeff);
hk_status phase_decomposition(hk_handle* h, const int32_t* elem_to_sub, uint8_t** d_elem_in_out);
// The rest of the decomposition from an element membership elem_in[s * n_elems + e] of h->n_sub subdomains.
hk_status decomposition_from_membership(hk_handle* h, const uint8_t* d_elem_in);
// Nested decompositions (Sec. 2.3): the membership of the fine subdomains inside the coarse subdomains of h
// (coarse membership d_cin), allocated in h; their number and parent coarse subdomain.
hk_status nested_fine_membership(hk_handle* h, const uint8_t* d_cin, int nlab, const int32_t* elem_to_fine,
                                 int fine_overlap, uint8_t** d_fin_out, int* nf_out, std::vector<int>* parent_out);
hk_status phase_local_factors_begin(hk_handle* h);
hk_status phase_local_factors_mid(hk_handle* h);
hk_status phase_local_factors_end(hk_handle* h);
hk_status phase_eigen(hk_handle* h, const uint8_t* d_elem_in);
hk_status phase_coarse(hk_handle* h);

// ---- solve-time operations ----
hk_status ensure_workspace(hk_handle* h, int s);
// Destroys the cached solve graphs (their kernels hold workspace pointers).
void hk_drop_graphs(hk_handle* h);
// Raises the shared-memory limit of every apply kernel instantiation (before any graph capture).
hk_status apply_prepare(hk_handle* h);
// Times the apply for every admissible number of right-hand sides per CTA (1, 2, 4, 8, 16) at batch size s
// and keeps the fastest (the arithmetic per right-hand side is the same for all of them); in the split-BF16
// form also the tensor-core sweeps against the fastest of those.
hk_status apply_autotune(hk_handle* h, int s);
// True when apply_autotune has not yet run for batch size s.
bool apply_needs_tuning(const hk_handle* h, int s);

// ---- tensor-core sweeps of the split-BF16 form (hk_tc.cu) ----
// Host part of the record layout: the level table, the records' size and the launch limits, from the
// level pointers `lev` (host copy); sets h->tc_ok.  Allocates the records and the table.
hk_status tc_plan(hk_handle* h, const std::vector<int>& lev);
// Packs the records from the FP64 factors h->d_F64 (per-level offsets h->d_lvfo) on stream st.
hk_status tc_pack(hk_handle* h, cudaStream_t st);
// The local sweeps of s right-hand sides (gather of v, block sweeps, local solutions into ybuf).
hk_status tc_launch(hk_handle* h, int s, const double* v, const int* active, float* ybuf);
hk_status tc_prepare();
// z = M^{-1} v for s vectors (v, z: s x n device arrays, FP64).  `active` is NULL or
// the per-rhs state words (8 ints per rhs, word 0 nonzero = process this rhs).
hk_status op_apply(hk_handle* h, int s, const double* v, double* z, const int* active);
// y = B x for s vectors.
hk_status op_matvec(hk_handle* h, int s, const double* x, double* y, const int* active);
// y = A x for s vectors, A with the sparsity of B and the values val (h->d_valB or h->d_valD).
hk_status op_spmv_values(hk_handle* h, int s, const double* val, const double* x, double* y, const int* active);
// Left-preconditioned GMRES in the D_k inner product (hk_dkgmres.cu); device vectors.
hk_status run_left_dk_gmres(hk_handle* h, int s, const double* rhs_dev, double tol, double* u_dev, int32_t* iters,
                            double* res_hist, double* final_true, double* final_pc);
hk_status op_load(hk_handle* h, const double* f_nodal_dev, double* rhs_dev);
hk_status run_fgmres(hk_handle* h, int s, const double* rhs_dev, double tol, double* u_dev,
                     int32_t* iters, double* res_hist, double* final_res);

// ---- shared device helpers ----
// Exclusive scan of n ints in one CTA (setup sizes); total written to *total.
void launch_scan_exclusive(const int* in, int* out, int n, int* total, cudaStream_t st);
void launch_to_f32(const double* a, float* b, long long n, cudaStream_t st);
hk_status upload_sub_info(hk_handle* h);
hk_status build_apply_z(hk_handle* h);
hk_status build_levels(hk_handle* h, const std::vector<int>& counts, const std::vector<int>& offsets,
                       const int* d_nodes, int* d_levptr, int* d_perm, int* d_nodes_lev, std::vector<int>& L_out,
                       int* max_width);

// Geometry of a P1 simplex: volume and barycentric gradients g[v][d].
__device__ __forceinline__ double simplex_geometry(int dim, const double* __restrict__ xyz,
                                                   const int* __restrict__ vid, double g[4][3]) {
  if (dim == 2) {
    double x0 = xyz[2 * vid[0]], y0 = xyz[2 * vid[0] + 1];
    double a = xyz[2 * vid[1]] - x0, c = xyz[2 * vid[1] + 1] - y0;   // edge 1 = (a, c)
    double b = xyz[2 * vid[2]] - x0, d = xyz[2 * vid[2] + 1] - y0;   // edge 2 = (b, d)
    double det = a * d - b * c;                                        // columns (a,c), (b,d)
    double inv = 1.0 / det;
    // inverse of [[a, b], [c, d]] rows: grad lambda_1 = ( d, -b)/det, grad lambda_2 = (-c, a)/det
    g[1][0] = d * inv;  g[1][1] = -b * inv;
    g[2][0] = -c * inv; g[2][1] = a * inv;
    g[0][0] = -g[1][0] - g[2][0];
    g[0][1] = -g[1][1] - g[2][1];
    return fabs(det) * 0.5;
  } else {
    double p0[3] = {xyz[3 * vid[0]], xyz[3 * vid[0] + 1], xyz[3 * vid[0] + 2]};
    double E[3][3];  // E[r][c] = component r of edge c
    for (int c = 0; c < 3; ++c)
      for (int r = 0; r < 3; ++r) E[r][c] = xyz[3 * vid[c + 1] + r] - p0[r];
    double C00 = E[1][1] * E[2][2] - E[1][2] * E[2][1];
    double C01 = E[1][2] * E[2][0] - E[1][0] * E[2][2];
    double C02 = E[1][0] * E[2][1] - E[1][1] * E[2][0];
    double det = E[0][0] * C00 + E[0][1] * C01 + E[0][2] * C02;
    double inv = 1.0 / det;
    // rows of E^{-1} are the gradients of lambda_1..3: E^{-1} = adj(E)^T... adj(E)[c][r] = cofactor(r,c)
    double Inv[3][3];
    Inv[0][0] = C00 * inv;
    Inv[1][0] = C01 * inv;
    Inv[2][0] = C02 * inv;
    Inv[0][1] = (E[0][2] * E[2][1] - E[0][1] * E[2][2]) * inv;
    Inv[1][1] = (E[0][0] * E[2][2] - E[0][2] * E[2][0]) * inv;
    Inv[2][1] = (E[0][1] * E[2][0] - E[0][0] * E[2][1]) * inv;
    Inv[0][2] = (E[0][1] * E[1][2] - E[0][2] * E[1][1]) * inv;
    Inv[1][2] = (E[0][2] * E[1][0] - E[0][0] * E[1][2]) * inv;
    Inv[2][2] = (E[0][0] * E[1][1] - E[0][1] * E[1][0]) * inv;
    for (int v = 0; v < 3; ++v)
      for (int d = 0; d < 3; ++d) g[v + 1][d] = Inv[v][d];
    for (int d = 0; d < 3; ++d) g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
    return fabs(det) / 6.0;
  }
}

__device__ __forceinline__ int bsearch_int(const int* __restrict__ a, int n, int key) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int v = a[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sumi(int v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of a double (all threads get the result). `sh` has >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0;
  if (w == 0) {
    t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) sh[0] = t;
  }
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}
__device__ __forceinline__ int block_sumi(int v, int* sh) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sumi(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int t = 0;
  if (w == 0) {
    t = lane < nw ? sh[lane] : 0;
    t = warp_sumi(t);
    if (lane == 0) sh[0] = t;
  }
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

// In-place Gauss-Jordan inverse of the b x b row-major matrix A (shared
// memory) with partial pivoting; returns through *minpiv the smallest |pivot|.
// A pivot with |p| < pivot_floor is replaced by +-pivot_floor (inverse iteration on a nearly singular
// shifted matrix wants a large, finite solution); pivot_floor = 0 keeps the pivots as they are.
__device__ inline void gauss_jordan_inverse(double* A, int b, int* piv, double* red_v, int* red_i, double* minpiv,
                                            double pivot_floor = 0.0) {
  int tid = threadIdx.x, T = blockDim.x;
  for (int k = 0; k < b; ++k) {
    // pivot search in column k, rows k..b-1 (ties -> smallest row)
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < b; i += T) {
      double v = fabs(A[i * b + k]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = red_v[0];
      int bj = red_i[0];
      for (int w = 1; w < (T >> 5); ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bj)) { bv = red_v[w]; bj = red_i[w]; }
      piv[k] = bj;
      if (bv < *minpiv) *minpiv = bv;
    }
    __syncthreads();
    int p = piv[k];
    if (p != k)
      for (int c = tid; c < b; c += T) {
        double t = A[k * b + c];
        A[k * b + c] = A[p * b + c];
        A[p * b + c] = t;
      }
    __syncthreads();
    // the reciprocal pivot once, by thread 0 (an FP64 division per thread would fill the FP64 pipe)
    if (tid == 0) {
      double pv = A[k * b + k];
      if (fabs(pv) < pivot_floor) pv = pv < 0 ? -pivot_floor : pivot_floor;
      red_v[0] = pv != 0.0 ? 1.0 / pv : 0.0;
      A[k * b + k] = 1.0;
    }
    __syncthreads();
    double inv = red_v[0];
    for (int c = tid; c < b; c += T) A[k * b + c] *= inv;
    __syncthreads();
    // eliminate column k from every other row: a warp per row, lanes over the columns (column k and
    // row k are only read here)
    {
      int lane = tid & 31, nwarp = T >> 5;
      for (int i = tid >> 5; i < b; i += nwarp) {
        if (i == k) continue;
        double g = A[i * b + k];
        for (int c = lane; c < b; c += 32)
          if (c != k) A[i * b + c] -= g * A[k * b + c];
      }
    }
    __syncthreads();
    for (int i = tid; i < b; i += T)
      if (i != k) A[i * b + k] = -A[i * b + k] * A[k * b + k];
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, in reverse order
  for (int k = b - 1; k >= 0; --k) {
    int p = piv[k];
    if (p != k)
      for (int r = tid; r < b; r += T) {
        double t = A[r * b + k];
        A[r * b + k] = A[r * b + p];
        A[r * b + p] = t;
      }
    __syncthreads();
  }
}

