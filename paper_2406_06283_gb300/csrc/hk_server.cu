// Serving layer: cached operators, admission by a device-memory budget and continuous batching of
// solve requests over worker slots (one host thread and one CUDA stream per operator in use).
// All arithmetic stays in the setup and solve of the other translation units: the server only
// decides what runs when, copies right-hand sides in and solutions out, and keeps the books.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "hk_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct SrvOp {
  uint64_t id = 0, key = 0;
  hk_mesh mesh{};
  std::vector<double> xyz, coeff;
  std::vector<int32_t> elems, e2s;
  std::vector<uint8_t> bnd;
  double k = 0;
  hk_params prm{};
  int n_dofs = 0;
  hk_handle* h = nullptr;
  cudaStream_t stream = nullptr;
  size_t bytes = 0;        // device bytes held while resident (hk_info_t.bytes_resident)
  size_t est_setup = 0;    // bytes a setup may hold at its peak
  bool busy = false;
  uint64_t last_use = 0;
  int queued = 0;          // waiting requests on this operator
};

struct SrvReq {
  uint64_t ticket = 0, op = 0;
  int n_rhs = 0;
  double tol = 0;
  std::vector<double> rhs, u, hist, true_res;
  std::vector<int32_t> iters;
  hk_status status = HK_OK;
  bool done = false;
  std::string err;
  hk_request_info info{};
};

}  // namespace

struct hk_server {
  int dev = 0;
  size_t budget = 0;
  int n_slots = 1, max_batch = 16;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<uint64_t, SrvOp*> ops;
  std::unordered_map<uint64_t, uint64_t> by_key;
  std::unordered_map<uint64_t, SrvReq*> reqs;
  std::deque<uint64_t> queue;  // waiting tickets in arrival order
  size_t in_use = 0, peak = 0;
  uint64_t next_op = 1, next_ticket = 1, use_clock = 0;
  long long submitted = 0, completed = 0, failed = 0, setups = 0, evictions = 0, batches = 0, hits = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  Clock::time_point t0 = Clock::now();
  double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

static uint64_t fnv1a(uint64_t hsh, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    hsh ^= b[i];
    hsh *= 1099511628211ULL;
  }
  return hsh;
}

// Bytes reserved for a solve of s right-hand sides: the FGMRES workspace ensure_workspace allocates
// (Krylov and flexible bases, vectors, Hessenberg and Givens data, histories), hk_solve's staging of
// rhs and u, the preconditioner's local and coarse buffers, and 1 MiB of slack.
static size_t solve_workspace_bytes(const SrvOp* o, const hk_handle* h, int s) {
  int cap = 1;  // the handle allocates for a power of two right-hand sides
  while (cap < s) cap <<= 1;
  s = cap;
  size_t m = (size_t)o->prm.restart, n = (size_t)o->n_dofs;
  size_t pf = precond_f32(o->prm) ? 4 : 8;
  size_t b = 8 * (size_t)s * ((2 * m + 6) * n + (m + 1) * (m + 4) + (size_t)o->prm.max_iters);
  if (h) b += pf * (size_t)s * ((size_t)h->I_total + 2 * ((size_t)h->n0 + 1));
  return b + (1 << 20);
}

static void fail_request(hk_server* S, SrvReq* r, hk_status st, const char* msg) {
  r->status = st;
  r->err = msg ? msg : "";
  r->done = true;
  r->info.end_ms = S->now_ms();
  S->failed++;
}

// Evicts idle resident operators (least recently used first, those with no waiting request before
// the others) until `need` more bytes fit.  Caller holds the lock.
static bool make_room(hk_server* S, size_t need, const SrvOp* keep) {
  while (S->in_use + need > S->budget) {
    SrvOp* victim = nullptr;
    for (auto& kv : S->ops) {
      SrvOp* o = kv.second;
      if (!o->h || o->busy || o == keep) continue;
      if (!victim || (o->queued == 0 && victim->queued > 0) ||
          ((o->queued == 0) == (victim->queued == 0) && o->last_use < victim->last_use))
        victim = o;
    }
    if (!victim) return false;
    hk_destroy(victim->h);
    victim->h = nullptr;
    S->in_use -= victim->bytes;
    victim->bytes = 0;
    S->evictions++;
  }
  return true;
}

struct Batch {
  SrvOp* op = nullptr;
  std::vector<SrvReq*> reqs;
  int s = 0;
  bool setup = false;
  size_t reserved = 0;
};

// Picks the next batch (caller holds the lock).  Returns false when nothing can start now.
static bool pick_batch(hk_server* S, Batch& b) {
  for (size_t qi = 0; qi < S->queue.size(); ++qi) {
    SrvReq* r = S->reqs[S->queue[qi]];
    SrvOp* o = S->ops[r->op];
    if (o->busy) continue;
    bool setup = o->h == nullptr;
    // gather every waiting request on this operator with the same tol, oldest first
    b = Batch{};
    b.op = o;
    b.setup = setup;
    for (size_t qj = qi; qj < S->queue.size() && b.s < S->max_batch; ++qj) {
      SrvReq* q = S->reqs[S->queue[qj]];
      if (q->op != o->id || q->tol != r->tol) continue;
      if (b.s > 0 && b.s + q->n_rhs > S->max_batch) break;
      b.reqs.push_back(q);
      b.s += q->n_rhs;
    }
    // memory: a setup reserves its peak estimate; a solve reserves workspace beyond what the handle holds
    auto need_for = [&](int s_) {
      size_t ws = solve_workspace_bytes(o, o->h, s_);
      size_t have = (!setup && o->h->ws_rhs >= s_) ? ws : 0;
      return (setup ? o->est_setup : 0) + (ws > have ? ws - have : 0);
    };
    size_t own = setup ? 0 : o->bytes;  // the operator's own resident bytes cannot be evicted for it
    while (b.reqs.size() > 1 && own + need_for(b.s) > S->budget) {
      b.s -= b.reqs.back()->n_rhs;
      b.reqs.pop_back();
    }
    size_t need = need_for(b.s);
    if (own + need > S->budget) {  // cannot run even in an otherwise empty server
      S->queue.erase(S->queue.begin() + qi);
      o->queued--;
      fail_request(S, r, HK_OOM, "operator does not fit in the server's device-memory budget");
      S->cv_done.notify_all();
      --qi;
      continue;
    }
    if (S->in_use + need > S->budget && !make_room(S, need, o)) continue;  // wait for memory
    for (SrvReq* q : b.reqs) {
      for (size_t qj = 0; qj < S->queue.size(); ++qj)
        if (S->queue[qj] == q->ticket) {
          S->queue.erase(S->queue.begin() + qj);
          break;
        }
      o->queued--;
    }
    b.reserved = need;
    S->in_use += need;
    S->peak = std::max(S->peak, S->in_use);
    o->busy = true;
    return true;
  }
  b = Batch{};
  return false;
}

static void run_batch(hk_server* S, Batch& b, int slot) {
  SrvOp* o = b.op;
  double t_start = S->now_ms();
  hk_status st = HK_OK;
  std::string err;
  if (b.setup) {
    if (!o->stream) cudaStreamCreateWithFlags(&o->stream, cudaStreamNonBlocking);
    hk_params prm = o->prm;
    prm.elem_to_sub = o->e2s.data();
    st = hk_setup(&o->mesh, o->coeff.data(), o->k, &prm, o->stream, &o->h);
    if (st != HK_OK) err = hk_last_error();
    // solves of different operators overlap through their streams; launched loops overlap better there
    // than concurrent graphs with device-side loops (measured: 90 vs 46 solves/s on the serving stream)
    else hk_set_solve_graphs(o->h, 0);
  }
  std::vector<double> rhs((size_t)b.s * o->n_dofs), u((size_t)b.s * o->n_dofs), hist, tres(b.s);
  std::vector<int32_t> iters(b.s, 0);
  hist.assign((size_t)b.s * o->prm.max_iters, 0.0);
  if (st == HK_OK) {
    size_t off = 0;
    for (SrvReq* q : b.reqs) {
      memcpy(rhs.data() + off, q->rhs.data(), sizeof(double) * q->rhs.size());
      off += q->rhs.size();
    }
    st = hk_solve(o->h, b.s, rhs.data(), b.reqs[0]->tol, u.data(), iters.data(), hist.data(), tres.data());
    if (st != HK_OK && st != HK_NO_CONVERGENCE) err = hk_last_error();
  }
  std::lock_guard<std::mutex> lk(S->mu);
  double t_end = S->now_ms();
  S->in_use -= b.reserved;
  if (b.setup) {
    if (st == HK_OK || st == HK_NO_CONVERGENCE) S->setups++;
  } else {
    S->hits++;
  }
  if (o->h) {
    // a failed solve keeps the operator; a failed setup left no handle
    hk_info_t inf;
    hk_info(o->h, &inf);
    S->in_use -= o->bytes;
    o->bytes = inf.bytes_resident;
    S->in_use += o->bytes;
    o->est_setup = inf.bytes_peak + inf.bytes_peak / 4;
  }
  S->peak = std::max(S->peak, S->in_use);
  S->batches++;
  o->busy = false;
  o->last_use = ++S->use_clock;
  size_t off = 0;
  int r0 = 0;
  for (SrvReq* q : b.reqs) {
    q->info.start_ms = t_start;
    q->info.end_ms = t_end;
    q->info.batch_rhs = b.s;
    q->info.setup_ran = b.setup ? 1 : 0;
    q->info.slot = slot;
    q->status = st;
    q->err = err;
    if (o->h && (st == HK_OK || st == HK_NO_CONVERGENCE)) {
      size_t nn = (size_t)q->n_rhs * o->n_dofs;
      q->u.assign(u.begin() + off, u.begin() + off + nn);
      q->iters.assign(iters.begin() + r0, iters.begin() + r0 + q->n_rhs);
      q->true_res.assign(tres.begin() + r0, tres.begin() + r0 + q->n_rhs);
      q->hist.assign(hist.begin() + (size_t)r0 * o->prm.max_iters,
                     hist.begin() + (size_t)(r0 + q->n_rhs) * o->prm.max_iters);
    }
    off += (size_t)q->n_rhs * o->n_dofs;
    r0 += q->n_rhs;
    q->done = true;
    if (st == HK_OK || st == HK_NO_CONVERGENCE) S->completed++;
    else S->failed++;
  }
  S->cv_done.notify_all();
  S->cv_work.notify_all();
}

static void worker_main(hk_server* S, int slot) {
  cudaSetDevice(S->dev);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    Batch b;
    S->cv_work.wait(lk, [&] { return S->stop || pick_batch(S, b); });
    if (!b.op) {
      if (S->stop) return;
      continue;
    }
    lk.unlock();
    run_batch(S, b, slot);
    lk.lock();
    if (S->stop && S->queue.empty()) return;
  }
}

extern "C" hk_status hk_server_create(size_t budget, int n_slots, int max_batch_rhs, hk_server** out) {
  if (!out || budget == 0 || n_slots < 1 || n_slots > 64 || max_batch_rhs < 1 || max_batch_rhs > 64) {
    hk_set_error("invalid server arguments");
    return HK_BAD_ARG;
  }
  hk_server* S = new hk_server();
  cudaGetDevice(&S->dev);
  hk_pool_init(S->dev);
  S->budget = budget;
  S->n_slots = n_slots;
  S->max_batch = max_batch_rhs;
  for (int i = 0; i < n_slots; ++i) S->workers.emplace_back(worker_main, S, i);
  *out = S;
  return HK_OK;
}

extern "C" hk_status hk_server_add_operator(hk_server* S, const hk_mesh* mesh, const double* coeff, double k,
                                           const hk_params* prm, uint64_t* op_id) {
  if (!S || !mesh || !coeff || !prm || !op_id || !mesh->xyz || !mesh->elems || !mesh->is_boundary ||
      !prm->elem_to_sub || (mesh->dim != 2 && mesh->dim != 3) || mesh->n_nodes <= 0 || mesh->n_elems <= 0 ||
      prm->max_iters < 1 || prm->restart < 1) {
    hk_set_error("invalid operator arguments");
    return HK_BAD_ARG;
  }
  SrvOp* o = new SrvOp();
  int nv = mesh->dim + 1;
  o->xyz.assign(mesh->xyz, mesh->xyz + (size_t)mesh->dim * mesh->n_nodes);
  o->elems.assign(mesh->elems, mesh->elems + (size_t)nv * mesh->n_elems);
  o->bnd.assign(mesh->is_boundary, mesh->is_boundary + mesh->n_nodes);
  o->coeff.assign(coeff, coeff + mesh->n_elems);
  o->e2s.assign(prm->elem_to_sub, prm->elem_to_sub + mesh->n_elems);
  o->k = k;
  o->prm = *prm;
  o->prm.elem_to_sub = nullptr;
  o->mesh = *mesh;
  o->mesh.xyz = o->xyz.data();
  o->mesh.elems = o->elems.data();
  o->mesh.is_boundary = o->bnd.data();
  for (uint8_t f : o->bnd) o->n_dofs += f ? 0 : 1;
  uint64_t key = 1469598103934665603ULL;
  key = fnv1a(key, &mesh->dim, sizeof(int));
  key = fnv1a(key, o->xyz.data(), sizeof(double) * o->xyz.size());
  key = fnv1a(key, o->elems.data(), sizeof(int32_t) * o->elems.size());
  key = fnv1a(key, o->bnd.data(), o->bnd.size());
  key = fnv1a(key, o->coeff.data(), sizeof(double) * o->coeff.size());
  key = fnv1a(key, o->e2s.data(), sizeof(int32_t) * o->e2s.size());
  key = fnv1a(key, &k, sizeof(double));
  int ints[7] = {prm->n_sub, prm->overlap_layers, prm->precision, prm->levels, prm->weighting, prm->restart,
                 prm->max_iters};
  key = fnv1a(key, ints, sizeof(ints));
  key = fnv1a(key, &prm->tau, sizeof(double));
  o->key = key;
  // estimate of a setup's peak device bytes until one has been measured
  o->est_setup = (size_t)o->n_dofs * (mesh->dim == 2 ? 24576 : 65536);
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->by_key.find(key);
  if (it != S->by_key.end()) {
    delete o;
    *op_id = it->second;
    return HK_OK;
  }
  o->id = S->next_op++;
  S->ops[o->id] = o;
  S->by_key[key] = o->id;
  *op_id = o->id;
  return HK_OK;
}

extern "C" hk_status hk_server_submit(hk_server* S, uint64_t op_id, int n_rhs, const double* rhs, double tol,
                                     uint64_t* ticket) {
  if (!S || !rhs || !ticket || n_rhs < 1 || !(tol > 0)) {
    hk_set_error("invalid submit arguments");
    return HK_BAD_ARG;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->ops.find(op_id);
  if (it == S->ops.end() || S->stop) {
    hk_set_error("unknown operator %llu", (unsigned long long)op_id);
    return HK_BAD_ARG;
  }
  if (n_rhs > S->max_batch) {
    hk_set_error("request of %d right-hand sides exceeds the server's batch limit %d", n_rhs, S->max_batch);
    return HK_BAD_ARG;
  }
  SrvOp* o = it->second;
  lk.unlock();
  SrvReq* r = new SrvReq();
  r->op = op_id;
  r->n_rhs = n_rhs;
  r->tol = tol;
  r->rhs.assign(rhs, rhs + (size_t)n_rhs * o->n_dofs);
  r->info.n_rhs = n_rhs;
  lk.lock();
  r->ticket = S->next_ticket++;
  r->info.submit_ms = S->now_ms();
  S->reqs[r->ticket] = r;
  S->queue.push_back(r->ticket);
  o->queued++;
  S->submitted++;
  *ticket = r->ticket;
  S->cv_work.notify_one();
  return HK_OK;
}

extern "C" hk_status hk_server_poll(hk_server* S, uint64_t ticket, int wait_ms, double* u, int32_t* iters,
                                   double* res_hist, double* final_true_rel_res, hk_request_info* info) {
  if (!S) return HK_BAD_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    hk_set_error("unknown ticket %llu", (unsigned long long)ticket);
    return HK_BAD_ARG;
  }
  SrvReq* r = it->second;
  if (!r->done) {
    if (wait_ms < 0)
      S->cv_done.wait(lk, [&] { return r->done; });
    else if (wait_ms > 0)
      S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return r->done; });
    if (!r->done) return HK_PENDING;
  }
  S->reqs.erase(it);
  lk.unlock();
  if (!r->u.empty()) {
    if (u) memcpy(u, r->u.data(), sizeof(double) * r->u.size());
    if (iters) memcpy(iters, r->iters.data(), sizeof(int32_t) * r->iters.size());
    if (res_hist) memcpy(res_hist, r->hist.data(), sizeof(double) * r->hist.size());
    if (final_true_rel_res) memcpy(final_true_rel_res, r->true_res.data(), sizeof(double) * r->true_res.size());
  }
  if (info) *info = r->info;
  hk_status st = r->status;
  if (st != HK_OK && !r->err.empty()) hk_set_error("%s", r->err.c_str());
  delete r;
  return st;
}

extern "C" hk_status hk_server_get_stats(hk_server* S, hk_server_stats* out) {
  if (!S || !out) return HK_BAD_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->setups = S->setups;
  out->evictions = S->evictions;
  out->batches = S->batches;
  out->cache_hits = S->hits;
  out->n_ops = (int)S->ops.size();
  for (auto& kv : S->ops) out->resident_ops += kv.second->h ? 1 : 0;
  out->queued = (int)S->queue.size();
  out->bytes_in_use = S->in_use;
  out->bytes_peak = S->peak;
  out->budget = S->budget;
  return HK_OK;
}

extern "C" hk_status hk_server_destroy(hk_server* S) {
  if (!S) return HK_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (uint64_t t : S->queue) {
      SrvReq* r = S->reqs[t];
      S->ops[r->op]->queued--;
      fail_request(S, r, HK_BAD_ARG, "server destroyed before the request ran");
    }
    S->queue.clear();
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  for (auto& t : S->workers) t.join();
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(S->dev);
  for (auto& kv : S->ops) {
    SrvOp* o = kv.second;
    if (o->h) hk_destroy(o->h);
    if (o->stream) cudaStreamDestroy(o->stream);
    delete o;
  }
  for (auto& kv : S->reqs) delete kv.second;
  cudaSetDevice(cur);
  delete S;
  return HK_OK;
}
