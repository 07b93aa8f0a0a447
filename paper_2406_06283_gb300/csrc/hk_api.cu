// C ABI of the hkgeneo library: argument checks, phase orchestration,
// host/device copies, inspection calls.  All arithmetic of the method runs in
// the kernels of the other translation units.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>

#include <algorithm>
#include <cmath>
#include <vector>
#include "hk_internal.cuh"

static thread_local char g_err[512] = "";
std::atomic<long long> g_hk_launches{0};
thread_local int g_hk_capture_count = -1;

extern "C" long long hk_kernel_launches(void) { return g_hk_launches.load(); }

void hk_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char* hk_last_error(void) { return g_err; }

extern "C" const char* hk_status_string(hk_status s) {
  switch (s) {
    case HK_OK: return "HK_OK";
    case HK_BAD_ARG: return "HK_BAD_ARG";
    case HK_SINGULAR_LOCAL: return "HK_SINGULAR_LOCAL";
    case HK_SINGULAR_COARSE: return "HK_SINGULAR_COARSE";
    case HK_EIG_FAIL: return "HK_EIG_FAIL";
    case HK_NO_CONVERGENCE: return "HK_NO_CONVERGENCE";
    case HK_OOM: return "HK_OOM";
    case HK_TIMEOUT: return "HK_TIMEOUT";
    case HK_CUDA_ERROR: return "HK_CUDA_ERROR";
    case HK_UNSUPPORTED: return "HK_UNSUPPORTED";
    case HK_PENDING: return "HK_PENDING";
  }
  return "unknown";
}

void hk_pool_init(int dev) {
  static std::once_flag done[64];
  if (dev < 0 || dev >= 64) return;
  std::call_once(done[dev], [dev] {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      unsigned long long keep = ~0ULL;  // keep freed blocks in the pool
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
  });
}

hk_status hk_allow_smem_fn(const void* fn) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  HK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({fn, dev})) return HK_OK;
  int optin = 0;
  HK_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  HK_CUDA(cudaFuncGetAttributes(&fa, fn));
  HK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
  done.insert({fn, dev});
  return HK_OK;
}

// The setup kernels that run beside the eigensolver's Lanczos blocks ask for the largest shared-memory
// carveout: an SM configured for a small one takes no block that needs a large one until it drains.
hk_status hk_max_carveout_fn(const void* fn) {
  HK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared));
  return HK_OK;
}

void dfree(hk_handle* h, void* p) {
  if (!p) return;
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->allocs[i].first == p) {
      h->bytes -= h->allocs[i].second;
      h->allocs[i] = h->allocs.back();
      h->allocs.pop_back();
      break;
    }
  cudaFreeAsync(p, h->stream);
}

hk_status check_device_status(hk_handle* h, const char* phase) {
  DevStatus st;
  cudaError_t e = cudaMemcpyAsync(&st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    hk_set_error("%s: %s", phase, cudaGetErrorString(e));
    return HK_CUDA_ERROR;
  }
  if (st.code != HK_OK) {
    hk_set_error("%s: %s at index %d (value %.6g)", phase, hk_status_string((hk_status)st.code), st.where, st.value);
    // cleared, so that a later phase or call is not blamed for this failure
    cudaMemsetAsync(h->d_status, 0, sizeof(DevStatus), h->stream);
    cudaStreamSynchronize(h->stream);
    return (hk_status)st.code;
  }
  return HK_OK;
}

extern "C" hk_status hk_check_status(hk_handle* h) {
  if (!h) return HK_BAD_ARG;
  int cur = -1;
  HK_CUDA(cudaGetDevice(&cur));
  if (cur != h->dev) HK_CUDA(cudaSetDevice(h->dev));
  hk_status s = check_device_status(h, "device work");
  if (cur != h->dev) cudaSetDevice(cur);
  return s;
}

extern "C" hk_status hk_set_wait_limit(hk_handle* h, int grid_barrier_polls) {
  if (!h || grid_barrier_polls < 0) return HK_BAD_ARG;
  unsigned polls = grid_barrier_polls == 0 ? (1u << 25) : (unsigned)grid_barrier_polls;
  if (polls != h->wait_polls) {
    // the limit is a kernel argument: cached solve graphs hold the old one
    HK_CUDA(cudaStreamSynchronize(h->stream));
    hk_drop_graphs(h);
    h->wait_polls = polls;
  }
  return HK_OK;
}

static void destroy_all(hk_handle* h) {
  if (!h) return;
  if (h->child) {
    destroy_all(h->child);
    h->child = nullptr;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->dev);
  cudaStreamSynchronize(h->stream);
  hk_drop_graphs(h);
  if (h->aux_stream) {
    cudaStreamSynchronize(h->aux_stream);
    cudaStreamDestroy(h->aux_stream);
    h->aux_stream = nullptr;
  }
  if (h->ev_lf) cudaEventDestroy(h->ev_lf);
  h->ev_lf = nullptr;
  if (h->co_stream) {
    cudaStreamSynchronize(h->co_stream);
    cudaStreamDestroy(h->co_stream);
    h->co_stream = nullptr;
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  h->ev_fork = h->ev_join = nullptr;
  if (h->cap_stream) {
    cudaStreamSynchronize(h->cap_stream);
    cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
  }
  for (auto& a : h->allocs) cudaFreeAsync(a.first, h->stream);
  h->allocs.clear();
  cudaStreamSynchronize(h->stream);
  if (h->h_state) cudaFreeHost(h->h_state);
  if (h->h_rstate) cudaFreeHost(h->h_rstate);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  cudaSetDevice(cur);
  delete h;
}

extern "C" hk_status hk_destroy(hk_handle* h) {
  destroy_all(h);
  return HK_OK;
}

struct PhaseTimer {
  cudaEvent_t a, b;
  cudaStream_t st;
  explicit PhaseTimer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  double stop() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventRecord(a, st);
    return ms;
  }
  ~PhaseTimer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// Nested decompositions (Sec. 2.3): the fine label of every element and the fine overlap layers.
struct NestedArgs {
  int n_labels;
  const int32_t* elem_to_fine;
  int fine_overlap;
};

static hk_status setup_impl(hk_handle* h, const hk_mesh* mesh, const double* coeff, const hk_params* prm,
                            const NestedArgs* nest = nullptr) {
  HK_TRY(dalloc(h, &h->d_status, 1));
  PhaseTimer t(h->stream);
  HK_TRY(phase_assembly(h, mesh, coeff));
  h->setup_ms[0] = t.stop();
  uint8_t* d_elem_in = nullptr;
  HK_TRY(phase_decomposition(h, prm->elem_to_sub, &d_elem_in));
  hk_handle* c = nullptr;
  if (nest) {
    // the fine subdomains and their local solves in a child handle (one level, apply only); this handle
    // keeps the coarse subdomains for the eigenproblems and the coarse space
    c = new hk_handle();
    h->child = c;
    c->dev = h->dev;
    c->stream = h->stream;
    c->dim = h->dim;
    c->nv = h->nv;
    c->n_nodes = h->n_nodes;
    c->n_elems = h->n_elems;
    c->k = h->k;
    c->p = h->p;
    c->p.levels = HK_ONE_LEVEL;
    c->dev_inputs = h->dev_inputs;
    c->apply_only = true;
    HK_TRY(dalloc(c, &c->d_status, 1));
    HK_TRY(phase_assembly(c, mesh, coeff));
    uint8_t* d_fin = nullptr;
    int nf = 0;
    HK_TRY(nested_fine_membership(h, d_elem_in, nest->n_labels, nest->elem_to_fine, nest->fine_overlap, &d_fin, &nf,
                                  &h->fine_parent));
    c->n_sub = c->p.n_sub = nf;
    hk_status ds = decomposition_from_membership(c, d_fin);
    dfree(h, d_fin);
    HK_TRY(ds);
  }
  h->setup_ms[1] = t.stop();
  if (c) HK_TRY(phase_local_factors_begin(c));
  HK_TRY(phase_local_factors_begin(h));
  if (h->p.levels != HK_ONE_LEVEL) {
    // the factor kernels run on the auxiliary stream meanwhile; setup_ms[2] is their host part
    h->setup_ms[2] = t.stop();
    HK_TRY(phase_eigen(h, d_elem_in));
    h->setup_ms[3] = t.stop();
    HK_TRY(phase_local_factors_mid(h));
    if (c) HK_TRY(phase_local_factors_mid(c));
    HK_TRY(phase_coarse(h));
    HK_TRY(phase_local_factors_end(h));
    if (c) HK_TRY(phase_local_factors_end(c));
    h->setup_ms[4] = t.stop();
  } else {
    HK_TRY(phase_local_factors_end(h));
    h->setup_ms[2] = t.stop();
  }
  dfree(h, d_elem_in);
  h->setup_ms[5] = h->setup_ms[0] + h->setup_ms[1] + h->setup_ms[2] + h->setup_ms[3] + h->setup_ms[4];
  return HK_OK;
}

static hk_status setup_common(const hk_mesh* mesh, const double* elem_coeff, double k, const hk_params* prm,
                              void* cuda_stream, hk_handle** out, bool dev_inputs, const NestedArgs* nest = nullptr) {
  if (!out) {
    hk_set_error("out is NULL");
    return HK_BAD_ARG;
  }
  *out = nullptr;
  if (!mesh || !elem_coeff || !prm || !mesh->xyz || !mesh->elems || !mesh->is_boundary || !prm->elem_to_sub) {
    hk_set_error("NULL argument");
    return HK_BAD_ARG;
  }
  if ((mesh->dim != 2 && mesh->dim != 3) || mesh->n_nodes <= 0 || mesh->n_elems <= 0 || prm->n_sub <= 0 ||
      prm->overlap_layers < 1 || !(prm->tau > 0) || !(k >= 0) || prm->restart < 1 ||
      prm->restart > HK_MAXRESTART || prm->max_iters < 1 || prm->precision < HK_FP64 ||
      prm->precision > HK_SPLIT_BF16_PRECOND || prm->levels < HK_TWO_LEVEL || prm->levels > HK_COARSE_ONLY ||
      prm->weighting < HK_AS || prm->weighting > HK_RAS_POU) {
    hk_set_error("invalid sizes or parameters (dim %d, n_sub %d, overlap %d, tau %g, restart %d)", mesh->dim,
                 prm->n_sub, prm->overlap_layers, prm->tau, prm->restart);
    return HK_BAD_ARG;
  }
  hk_handle* h = new hk_handle();
  cudaGetDevice(&h->dev);
  h->stream = (cudaStream_t)cuda_stream;
  h->dim = mesh->dim;
  h->nv = mesh->dim + 1;
  h->n_nodes = mesh->n_nodes;
  h->n_elems = mesh->n_elems;
  h->n_sub = prm->n_sub;
  h->k = k;
  h->p = *prm;
  h->p.elem_to_sub = nullptr;
  h->dev_inputs = dev_inputs;
  if (nest) h->p.levels = HK_COARSE_ONLY;  // its own apply is the coarse correction; the child adds the local part
  hk_status s = setup_impl(h, mesh, elem_coeff, prm, nest);
  if (s != HK_OK) {
    cudaGetLastError();
    destroy_all(h);
    return s;
  }
  *out = h;
  return HK_OK;
}

extern "C" hk_status hk_setup(const hk_mesh* mesh, const double* elem_coeff, double k, const hk_params* prm,
                              void* cuda_stream, hk_handle** out) {
  return setup_common(mesh, elem_coeff, k, prm, cuda_stream, out, false);
}

static hk_status setup_nested_common(const hk_mesh* mesh, const double* elem_coeff, double k, const hk_params* prm,
                                     int n_fine_labels, const int32_t* elem_to_fine, int fine_overlap,
                                     void* cuda_stream, hk_handle** out, bool dev_inputs) {
  if (out) *out = nullptr;
  if (!prm || prm->levels != HK_TWO_LEVEL || n_fine_labels < 1 || !elem_to_fine || fine_overlap < 0) {
    hk_set_error("hk_setup_nested: needs the two-level preconditioner, fine labels and fine_overlap >= 0");
    return HK_BAD_ARG;
  }
  NestedArgs nest{n_fine_labels, elem_to_fine, fine_overlap};
  return setup_common(mesh, elem_coeff, k, prm, cuda_stream, out, dev_inputs, &nest);
}

extern "C" hk_status hk_setup_nested(const hk_mesh* mesh, const double* elem_coeff, double k, const hk_params* prm,
                                     int n_fine_labels, const int32_t* elem_to_fine, int fine_overlap_layers,
                                     void* cuda_stream, hk_handle** out) {
  return setup_nested_common(mesh, elem_coeff, k, prm, n_fine_labels, elem_to_fine, fine_overlap_layers, cuda_stream,
                             out, false);
}

extern "C" hk_status hk_setup_nested_device(const hk_mesh* mesh_dev, const double* elem_coeff_dev, double k,
                                            const hk_params* prm, int n_fine_labels, const int32_t* elem_to_fine_dev,
                                            int fine_overlap_layers, void* cuda_stream, hk_handle** out) {
  return setup_nested_common(mesh_dev, elem_coeff_dev, k, prm, n_fine_labels, elem_to_fine_dev, fine_overlap_layers,
                             cuda_stream, out, true);
}

extern "C" hk_status hk_setup_device(const hk_mesh* mesh_dev, const double* elem_coeff_dev, double k,
                                     const hk_params* prm, void* cuda_stream, hk_handle** out) {
  return setup_common(mesh_dev, elem_coeff_dev, k, prm, cuda_stream, out, true);
}

cudaEvent_t hk_event(hk_handle* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

extern "C" hk_status hk_set_timing(hk_handle* h, int on) {
  if (!h) return HK_BAD_ARG;
  HK_CUDA(cudaStreamSynchronize(h->stream));
  h->tl.clear();
  h->ev_used = 0;
  h->timing = on != 0;
  if (h->child) {
    h->child->tl.clear();
    h->child->ev_used = 0;
    h->child->timing = on != 0;
  }
  return HK_OK;
}

extern "C" hk_status hk_set_solve_graphs(hk_handle* h, int on) {
  if (!h) return HK_BAD_ARG;
  h->use_graphs = on != 0;
  return HK_OK;
}

extern "C" hk_status hk_set_sweep_path(hk_handle* h, int path) {
  if (!h || path < HK_SWEEPS_AUTO || path > HK_SWEEPS_TENSOR_CORE) {
    hk_set_error("hk_set_sweep_path: invalid arguments");
    return HK_BAD_ARG;
  }
  if (h->child) {  // nested decompositions: the local sweeps are the fine handle's
    HK_TRY(hk_set_sweep_path(h->child, path));
    HK_CUDA(cudaStreamSynchronize(h->stream));
    hk_drop_graphs(h);
    return HK_OK;
  }
  if (path == HK_SWEEPS_TENSOR_CORE && !h->tc_ok) {
    hk_set_error(h->p.precision == HK_SPLIT_BF16_PRECOND
                     ? "tensor-core sweeps unavailable for this handle's subdomains"
                     : "tensor-core sweeps need the split-BF16 precision form");
    return HK_UNSUPPORTED;
  }
  if (path != h->sweep_path) {
    HK_CUDA(cudaStreamSynchronize(h->stream));
    hk_drop_graphs(h);  // captured solves hold the launches of the old path
  }
  h->sweep_path = path;
  return HK_OK;
}

extern "C" hk_status hk_kernel_times(hk_handle* h, double* ms, int32_t* count) {
  if (!h || !ms || !count) return HK_BAD_ARG;
  HK_CUDA(cudaStreamSynchronize(h->stream));
  for (int c = 0; c < HK_T_NCAT; ++c) {
    ms[c] = 0;
    count[c] = 0;
  }
  for (const hk_handle* q = h; q; q = q->child)  // a nested handle's local sweeps are its child's
    for (auto& t : q->tl) {
      float e = 0;
      HK_CUDA(cudaEventElapsedTime(&e, t.a, t.b));
      ms[t.cat] += e;
      count[t.cat] += 1;
    }
  return HK_OK;
}

extern "C" hk_status hk_solve_device(hk_handle* h, int n_rhs, const double* rhs_dev, double tol, double* u_dev,
                                     int32_t* iters, double* res_hist, double* final_true_rel_res) {
  if (!h || n_rhs < 1 || !rhs_dev || !u_dev || !iters || !(tol > 0)) {
    hk_set_error("invalid solve arguments");
    return HK_BAD_ARG;
  }
  return run_fgmres(h, n_rhs, rhs_dev, tol, u_dev, iters, res_hist, final_true_rel_res);
}

extern "C" hk_status hk_solve_left_dk_device(hk_handle* h, int n_rhs, const double* rhs_dev, double tol,
                                             double* u_dev, int32_t* iters, double* res_hist, double* final_true,
                                             double* final_pc) {
  if (!h || n_rhs < 1 || !rhs_dev || !u_dev || !iters || !(tol > 0)) {
    hk_set_error("invalid solve arguments");
    return HK_BAD_ARG;
  }
  return run_left_dk_gmres(h, n_rhs, rhs_dev, tol, u_dev, iters, res_hist, final_true, final_pc);
}

extern "C" hk_status hk_solve_left_dk(hk_handle* h, int n_rhs, const double* rhs, double tol, double* u,
                                      int32_t* iters, double* res_hist, double* final_true, double* final_pc) {
  if (!h || n_rhs < 1 || !rhs || !u || !iters || !(tol > 0)) {
    hk_set_error("invalid solve arguments");
    return HK_BAD_ARG;
  }
  size_t bytes = sizeof(double) * (size_t)n_rhs * h->n;
  double *d_in = nullptr, *d_out = nullptr;
  if (dalloc(h, &d_in, bytes / sizeof(double)) != HK_OK || dalloc(h, &d_out, bytes / sizeof(double)) != HK_OK) {
    if (d_in) dfree(h, d_in);
    return HK_OOM;
  }
  hk_status s = HK_OK;
  if (cudaMemcpyAsync(d_in, rhs, bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) s = HK_CUDA_ERROR;
  if (s == HK_OK) s = run_left_dk_gmres(h, n_rhs, d_in, tol, d_out, iters, res_hist, final_true, final_pc);
  if (s == HK_OK || s == HK_NO_CONVERGENCE) {
    cudaError_t e = cudaMemcpyAsync(u, d_out, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      hk_set_error("copy-out: %s", cudaGetErrorString(e));
      s = HK_CUDA_ERROR;
    }
  }
  dfree(h, d_in);
  dfree(h, d_out);
  return s;
}

extern "C" hk_status hk_theory(const hk_handle* h, double c_stab, double H_f, hk_theory_t* out) {
  if (!h || !out || !(c_stab >= 0)) {
    hk_set_error("hk_theory: invalid arguments");
    return HK_BAD_ARG;
  }
  if (h->p.levels != HK_TWO_LEVEL && !h->child) {
    hk_set_error("hk_theory: the theorem is stated for the two-level preconditioner");
    return HK_UNSUPPORTED;
  }
  // Lambda and H^f are those of the fine subdomains (the subdomains themselves with one decomposition)
  const hk_handle* f = h->child ? h->child : h;
  if (!(H_f > 0)) {
    // largest bounding-box diagonal of a subdomain's dof nodes
    std::vector<double> xyz((size_t)h->n_nodes * h->dim);
    std::vector<int> node(f->n), I(f->I_total);
    HK_CUDA(cudaMemcpy(xyz.data(), f->d_xyz, sizeof(double) * xyz.size(), cudaMemcpyDeviceToHost));
    HK_CUDA(cudaMemcpy(node.data(), f->d_node_of_dof, sizeof(int) * node.size(), cudaMemcpyDeviceToHost));
    HK_CUDA(cudaMemcpy(I.data(), f->d_I, sizeof(int) * I.size(), cudaMemcpyDeviceToHost));
    H_f = 0;
    for (const Sub& u : f->subs) {
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int a = 0; a < u.nI; ++a) {
        const double* p = &xyz[(size_t)node[I[(size_t)u.I_off + a]] * h->dim];
        for (int d = 0; d < h->dim; ++d) lo[d] = std::min(lo[d], p[d]), hi[d] = std::max(hi[d], p[d]);
      }
      double d2 = 0;
      for (int d = 0; d < h->dim; ++d) d2 += (hi[d] - lo[d]) * (hi[d] - lo[d]);
      if (u.nI > 0) H_f = std::max(H_f, std::sqrt(d2));
    }
  }
  double Lam = f->lambda_elems, tau = h->tau_next, k = h->k;
  double Theta = 1.0 / tau, a = 2.0 + 3.0 * std::pow(Lam, 4) * Theta;
  out->Lambda = Lam;
  out->tau = tau;
  out->tau_is_lower_bound = h->tau_next_lb ? 1 : 0;
  out->Theta = Theta;
  out->k = k;
  out->H_f = H_f;
  out->c_stab = c_stab;
  out->s = 2.0 * Lam * Lam * a * (2.0 * k * std::sqrt(Theta) * (1.0 + c_stab) + 3.0 * k * H_f);
  out->gamma = (1.0 - out->s) / (a * (18.0 + 8.0 * Lam * Lam * Lam));
  out->guaranteed = out->s < 1.0 ? 1 : 0;
  return HK_OK;
}

extern "C" hk_status hk_solve(hk_handle* h, int n_rhs, const double* rhs, double tol, double* u, int32_t* iters,
                              double* res_hist, double* final_true_rel_res) {
  if (!h || n_rhs < 1 || !rhs || !u || !iters || !(tol > 0)) {
    hk_set_error("invalid solve arguments");
    return HK_BAD_ARG;
  }
  size_t bytes = sizeof(double) * (size_t)n_rhs * h->n;
  double *d_in = nullptr, *d_out = nullptr;
  HK_CUDA(cudaMallocAsync(&d_in, bytes, h->stream));
  cudaError_t e = cudaMallocAsync(&d_out, bytes, h->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(d_in, h->stream);
    hk_set_error("cudaMallocAsync: %s", cudaGetErrorString(e));
    return HK_OOM;
  }
  hk_status s = HK_OK;
  e = cudaMemcpyAsync(d_in, rhs, bytes, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) s = HK_CUDA_ERROR;
  if (s == HK_OK) s = run_fgmres(h, n_rhs, d_in, tol, d_out, iters, res_hist, final_true_rel_res);
  if (s == HK_OK || s == HK_NO_CONVERGENCE) {
    e = cudaMemcpyAsync(u, d_out, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      hk_set_error("copy-out: %s", cudaGetErrorString(e));
      s = HK_CUDA_ERROR;
    }
  }
  cudaFreeAsync(d_in, h->stream);
  cudaFreeAsync(d_out, h->stream);
  cudaStreamSynchronize(h->stream);
  return s;
}

extern "C" hk_status hk_info(const hk_handle* h, hk_info_t* info) {
  if (!h || !info) return HK_BAD_ARG;
  memset(info, 0, sizeof(*info));
  info->dim = h->dim;
  info->n_nodes = h->n_nodes;
  info->n_elems = h->n_elems;
  info->n_dofs = h->n;
  info->n_sub = h->n_sub;
  info->n0 = h->n0;
  info->max_mu = h->max_mu;
  info->lambda_elems = h->lambda_elems;
  info->max_level = h->max_level;
  info->max_dof = h->max_dof;
  info->nnz = h->nnz;
  info->precision = h->p.precision;
  info->levels = h->child ? HK_TWO_LEVEL : h->p.levels;
  info->bytes_resident = h->bytes + (h->child ? h->child->bytes : 0);
  info->factor_elems = h->f_total;
  info->dof_total = h->I_total;
  info->coarse_elems = h->z_total;
  info->lower_nnz = h->lower_nnz;
  for (int i = 0; i < 8; ++i) info->setup_ms[i] = h->setup_ms[i];
  info->bytes_peak = h->bytes_peak;
  info->graph_solves = h->graph_solves;
  for (int i = 0; i < 4; ++i) info->eigen_kernel_ms[i] = h->eigen_ms[i];
  for (int i = 0; i < 4; ++i) info->eigen_kernel_gflop[i] = h->eigen_gflop[i];
  info->tc_record_bytes = h->tc_ok ? h->tc_bytes : 0;
  info->last_sweeps = h->last_sweeps;
  info->twist_moved = h->twist_moved;
  info->levels_merged = h->levels_merged;
  info->local_growth[0] = h->growth_twist;
  info->local_growth[1] = h->growth_mid;
  const hk_handle* c = h->child;
  info->fine_subdomains = c ? c->n_sub : 0;
  info->fine_lambda_elems = c ? c->lambda_elems : 0;
  info->fine_max_dof = c ? c->max_dof : 0;
  info->fine_dof_total = c ? c->I_total : 0;
  if (c) {
    info->max_level = c->max_level;
    info->twist_moved = c->twist_moved;
    info->levels_merged = c->levels_merged;
    info->local_growth[0] = c->growth_twist;
    info->local_growth[1] = c->growth_mid;
    info->tc_record_bytes = c->tc_ok ? c->tc_bytes : 0;
    info->last_sweeps = c->last_sweeps;
  }
  return HK_OK;
}

extern "C" hk_status hk_get_matrix(const hk_handle* h, int which, int32_t* rowptr, int32_t* col, double* val) {
  if (!h || which < 0 || which > 1) return HK_BAD_ARG;
  cudaStream_t st = h->stream;
  if (rowptr) HK_CUDA(cudaMemcpyAsync(rowptr, h->d_rowptr, sizeof(int) * (h->n + 1), cudaMemcpyDeviceToHost, st));
  if (col) HK_CUDA(cudaMemcpyAsync(col, h->d_col, sizeof(int) * h->nnz, cudaMemcpyDeviceToHost, st));
  if (val)
    HK_CUDA(cudaMemcpyAsync(val, which == 0 ? h->d_valB : h->d_valD, sizeof(double) * h->nnz, cudaMemcpyDeviceToHost,
                            st));
  HK_CUDA(cudaStreamSynchronize(st));
  return HK_OK;
}

extern "C" hk_status hk_get_subdomain(const hk_handle* h, int i, int32_t* sizes, int32_t* dof, int32_t* gamma,
                                      int32_t* level_ptr) {
  if (!h || i < 0 || i >= h->n_sub) return HK_BAD_ARG;
  const Sub& u = h->subs[i];
  cudaStream_t st = h->stream;
  if (sizes) {
    sizes[0] = u.nI;
    sizes[1] = u.nG;
    sizes[2] = u.L;
    sizes[3] = u.m;
  }
  if (dof) HK_CUDA(cudaMemcpyAsync(dof, h->d_I + u.I_off, sizeof(int) * u.nI, cudaMemcpyDeviceToHost, st));
  if (gamma && u.nG)
    HK_CUDA(cudaMemcpyAsync(gamma, h->d_G + u.G_off, sizeof(int) * u.nG, cudaMemcpyDeviceToHost, st));
  if (level_ptr)
    HK_CUDA(cudaMemcpyAsync(level_ptr, h->d_lev + u.lev_off, sizeof(int) * (u.L + 1), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  return HK_OK;
}

extern "C" hk_status hk_get_mu(const hk_handle* h, int32_t* mu) {
  if (!h || !mu) return HK_BAD_ARG;
  HK_CUDA(cudaMemcpyAsync(mu, h->d_mu, sizeof(int) * h->n, cudaMemcpyDeviceToHost, h->stream));
  HK_CUDA(cudaStreamSynchronize(h->stream));
  return HK_OK;
}

extern "C" hk_status hk_get_eigen(const hk_handle* h, int i, double* lam, double* Z) {
  if (!h || i < 0 || i >= h->n_sub) return HK_BAD_ARG;
  const Sub& u = h->subs[i];
  if (u.m == 0) return HK_OK;
  cudaStream_t st = h->stream;
  if (lam) HK_CUDA(cudaMemcpyAsync(lam, h->d_lam + (size_t)i * HK_MAXM, sizeof(double) * u.m, cudaMemcpyDeviceToHost, st));
  if (Z) HK_CUDA(cudaMemcpyAsync(Z, h->d_Z64 + u.z_off, sizeof(double) * u.nI * u.m, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  return HK_OK;
}

extern "C" hk_status hk_get_coarse(const hk_handle* h, double* E, double* Einv) {
  if (!h) return HK_BAD_ARG;
  size_t b = sizeof(double) * (size_t)h->n0 * h->n0;
  if (h->n0 == 0) return HK_OK;
  if (E) HK_CUDA(cudaMemcpyAsync(E, h->d_E, b, cudaMemcpyDeviceToHost, h->stream));
  if (Einv) HK_CUDA(cudaMemcpyAsync(Einv, h->d_Einv64, b, cudaMemcpyDeviceToHost, h->stream));
  HK_CUDA(cudaStreamSynchronize(h->stream));
  return HK_OK;
}

static hk_status with_device_vectors(hk_handle* h, int n_in, int n_out, int s, const double* in, double* out,
                                     hk_status (*fn)(hk_handle*, int, const double*, double*)) {
  size_t bi = sizeof(double) * (size_t)s * n_in, bo = sizeof(double) * (size_t)s * n_out;
  double *d_in = nullptr, *d_out = nullptr;
  HK_CUDA(cudaMalloc(&d_in, bi));
  cudaError_t e = cudaMalloc(&d_out, bo);
  if (e != cudaSuccess) {
    cudaFree(d_in);
    return HK_OOM;
  }
  hk_status s_ = HK_OK;
  if (cudaMemcpyAsync(d_in, in, bi, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) s_ = HK_CUDA_ERROR;
  if (s_ == HK_OK) s_ = fn(h, s, d_in, d_out);
  if (s_ == HK_OK && cudaMemcpyAsync(out, d_out, bo, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    s_ = HK_CUDA_ERROR;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) s_ = HK_CUDA_ERROR;
  cudaFree(d_in);
  cudaFree(d_out);
  return s_;
}

static hk_status apply_fn(hk_handle* h, int s, const double* v, double* z) { return op_apply(h, s, v, z, nullptr); }
static hk_status matvec_fn(hk_handle* h, int s, const double* x, double* y) {
  return op_matvec(h, s, x, y, nullptr);
}
static hk_status load_fn(hk_handle* h, int, const double* f, double* r) { return op_load(h, f, r); }

extern "C" hk_status hk_apply_precond(hk_handle* h, int n_rhs, const double* v, double* z) {
  if (!h || n_rhs < 1 || !v || !z) return HK_BAD_ARG;
  HK_TRY(ensure_workspace(h, n_rhs));
  HK_TRY(with_device_vectors(h, h->n, h->n, n_rhs, v, z, apply_fn));
  // a bounded wait of the apply that ran out leaves z untrusted
  return check_device_status(h, "preconditioner apply");
}

extern "C" hk_status hk_matvec(hk_handle* h, int n_rhs, const double* x, double* y) {
  if (!h || n_rhs < 1 || !x || !y) return HK_BAD_ARG;
  return with_device_vectors(h, h->n, h->n, n_rhs, x, y, matvec_fn);
}

extern "C" hk_status hk_assemble_load(hk_handle* h, const double* f_nodal, double* rhs) {
  if (!h || !f_nodal || !rhs) return HK_BAD_ARG;
  size_t bi = sizeof(double) * (size_t)h->n_nodes;
  double *d_in = nullptr, *d_out = nullptr;
  HK_CUDA(cudaMalloc(&d_in, bi));
  HK_CUDA(cudaMalloc(&d_out, sizeof(double) * h->n));
  hk_status s = HK_OK;
  if (cudaMemcpyAsync(d_in, f_nodal, bi, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) s = HK_CUDA_ERROR;
  if (s == HK_OK) s = load_fn(h, 1, d_in, d_out);
  if (s == HK_OK &&
      cudaMemcpyAsync(rhs, d_out, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    s = HK_CUDA_ERROR;
  cudaStreamSynchronize(h->stream);
  cudaFree(d_in);
  cudaFree(d_out);
  return s;
}
