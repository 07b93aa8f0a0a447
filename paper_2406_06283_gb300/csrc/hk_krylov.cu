// Right-preconditioned flexible GMRES(m) on the device (the Krylov solver the
// paper analyses for Eq. 2.24, Thm. 3.1, used here with the preconditioner on
// the right and the Euclidean inner product), for s right-hand sides at once.
//
// Per inner step j and right-hand side r:
//   z_j = M^{-1} v_j (op_apply), w = B z_j (op_matvec),
//   classical Gram-Schmidt applied twice (CGS2): h = V^T w, w -= V h, twice,
//   h_{j+1,j} = ||w||, Givens rotations on the Hessenberg column, v_{j+1} = w / h_{j+1,j}.
// A right-hand side stops its cycle when |g_{j+1}| <= tol ||f||, at the cycle
// length, on breakdown, or at max_iters; at cycle end x += Z_m y with R y = g
// and the true residual f - B x decides between done and a new cycle.
// Reductions are two-stage: per-CTA partial sums, then the last CTA to
// finish adds them in CTA order, so every run gives the same bits.
#include "hk_internal.cuh"

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

#define RED_BLOCKS 304
#define RED_THREADS 256

// state words per rhs
enum { ST_ACTIVE = 0, ST_DONE = 1, ST_ITERS = 2, ST_JD = 3, ST_CONV = 4 };
// real state per rhs
enum { RS_NF = 0, RS_HNEXT = 1, RS_EST = 2, RS_TRUE = 3, RS_BETA = 4 };

__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ bool amlast;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    amlast = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (amlast) __threadfence();
  return amlast;
}

__global__ void k_spmv(int n, int s, const int* __restrict__ rowptr, const int* __restrict__ col,
                       const double* __restrict__ val, const double* __restrict__ x, double* y,
                       const int* __restrict__ active) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  int q0 = rowptr[l], q1 = rowptr[l + 1];
  for (int r = 0; r < s; ++r) {
    if (active && !active[8 * r + ST_ACTIVE]) continue;
    const double* xr = x + (long long)r * n;
    double acc = 0;
    for (int q = q0; q < q1; ++q) acc += val[q] * xr[col[q]];
    y[(long long)r * n + l] = acc;
  }
}

hk_status op_matvec(hk_handle* h, int s, const double* x, double* y, const int* active) {
  k_spmv<<<nblk(h->n, 256), 256, 0, h->stream>>>(h->n, s, h->d_rowptr, h->d_col, h->d_valB, x, y, active); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  return HK_OK;
}

// Gram-Schmidt pass.  MODE 0: w = B z_j on the CTA's rows (the matvec, fused), then
// h1 = V^T w.  MODE 1: w -= V h1, then h2 = V^T w.
// MODE 2: w -= V h2, ||w||^2, then (last CTA) the Hessenberg column, Givens
// rotation, residual estimate and stopping decision of every active rhs.
template <int MODE>
__global__ void k_gs(int n, int s, int m, int j, const double* __restrict__ V, double* w, int* state,
                     double* rstate, double* hcoef, double* part, unsigned* counter, double* H, double* cs,
                     double* sn, double* g, double* hist, int max_iters, double tol,
                     const int* __restrict__ rowptr, const int* __restrict__ col, const double* __restrict__ val,
                     const double* __restrict__ zj) {
  int chunk = (n + gridDim.x - 1) / gridDim.x;
  int l0 = blockIdx.x * chunk, l1 = min(n, l0 + chunk);
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int nc = MODE == 2 ? 1 : j + 1;  // values per rhs
  __shared__ double red[32];
  for (int r = 0; r < s; ++r) {
    if (!state[8 * r + ST_ACTIVE]) continue;
    double* wr = w + (long long)r * n;
    if (MODE == 0) {
      const double* zr = zj + (long long)r * n;
      for (int l = l0 + tid; l < l1; l += blockDim.x) {
        double acc = 0;
        for (int q = rowptr[l]; q < rowptr[l + 1]; ++q) acc += val[q] * zr[col[q]];
        wr[l] = acc;
      }
      __syncthreads();
    }
    if (MODE >= 1) {
      const double* hc = hcoef + (long long)r * 2 * (m + 1) + (MODE == 1 ? 0 : m + 1);
      for (int l = l0 + tid; l < l1; l += blockDim.x) {
        double acc = wr[l];
        for (int i = 0; i <= j; ++i) acc -= hc[i] * V[((long long)i * s + r) * n + l];
        wr[l] = acc;
      }
      __syncthreads();
    }
    double* pr = part + ((long long)blockIdx.x * s + r) * (m + 2);
    if (MODE <= 1) {
      for (int i = warp; i <= j; i += nw) {
        const double* vi = V + ((long long)i * s + r) * n;
        double acc = 0;
        for (int l = l0 + lane; l < l1; l += 32) acc += wr[l] * vi[l];
        acc = warp_sum(acc);
        if (lane == 0) pr[i] = acc;
      }
    } else {
      double acc = 0;
      for (int l = l0 + tid; l < l1; l += blockDim.x) acc += wr[l] * wr[l];
      acc = block_sum(acc, red);
      if (tid == 0) pr[0] = acc;
    }
  }
  if (!last_block(counter)) return;
  // final reduction: one warp per value, lanes over CTAs in a fixed order
  for (int e = warp; e < s * nc; e += nw) {
    int r = e / nc, i = e % nc;
    if (!state[8 * r + ST_ACTIVE]) continue;
    double acc = 0;
    for (int b = lane; b < gridDim.x; b += 32) acc += part[((long long)b * s + r) * (m + 2) + i];
    acc = warp_sum(acc);
    if (lane == 0) {
      if (MODE == 0) hcoef[(long long)r * 2 * (m + 1) + i] = acc;
      else if (MODE == 1) hcoef[(long long)r * 2 * (m + 1) + (m + 1) + i] = acc;
      else rstate[8 * r + RS_HNEXT] = sqrt(acc);
    }
  }
  if (MODE == 2) {
    __syncthreads();
    for (int r = tid; r < s; r += blockDim.x) {
      if (!state[8 * r + ST_ACTIVE]) continue;
      double* Hr = H + (long long)r * (m + 1) * m;  // H[i][jj] at i * m + jj
      const double* h1 = hcoef + (long long)r * 2 * (m + 1);
      const double* h2 = h1 + (m + 1);
      double* csr = cs + (long long)r * m;
      double* snr = sn + (long long)r * m;
      double* gr = g + (long long)r * (m + 1);
      for (int i = 0; i <= j; ++i) Hr[i * m + j] = h1[i] + h2[i];
      double hn = rstate[8 * r + RS_HNEXT];
      Hr[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        double a = Hr[i * m + j], b = Hr[(i + 1) * m + j];
        Hr[i * m + j] = csr[i] * a + snr[i] * b;
        Hr[(i + 1) * m + j] = -snr[i] * a + csr[i] * b;
      }
      double a = Hr[j * m + j], b = Hr[(j + 1) * m + j];
      double den = hypot(a, b);
      csr[j] = a / den;
      snr[j] = b / den;
      Hr[j * m + j] = den;
      Hr[(j + 1) * m + j] = 0.0;
      gr[j + 1] = -snr[j] * gr[j];
      gr[j] = csr[j] * gr[j];
      int it = ++state[8 * r + ST_ITERS];
      double nf = rstate[8 * r + RS_NF];
      double est = fabs(gr[j + 1]);
      rstate[8 * r + RS_EST] = est;
      if (hist && it <= max_iters) hist[(long long)r * max_iters + it - 1] = est / nf;
      state[8 * r + ST_JD] = j + 1;
      bool stop = est <= tol * nf || it >= max_iters || hn == 0.0 || j + 1 == m;
      if (stop) state[8 * r + ST_ACTIVE] = 0;
    }
  }
  __syncthreads();
  if (tid == 0) *counter = 0u;
}

__global__ void k_normalize(int n, int s, int j, double* V, const double* __restrict__ w,
                            const int* __restrict__ state, const double* __restrict__ rstate) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  for (int r = 0; r < s; ++r) {
    if (!state[8 * r + ST_ACTIVE]) continue;
    double inv = 1.0 / rstate[8 * r + RS_HNEXT];
    V[((long long)(j + 1) * s + r) * n + l] = w[(long long)r * n + l] * inv;
  }
}

// ||u_r||^2 for every rhs flagged in `mask` (word ST_DONE == 0), into rstate[slot].
__global__ void k_norm2(int n, int s, const double* __restrict__ u, const int* __restrict__ state, double* rstate,
                        int slot, double* part, unsigned* counter, int sqrt_it) {
  int chunk = (n + gridDim.x - 1) / gridDim.x;
  int l0 = blockIdx.x * chunk, l1 = min(n, l0 + chunk);
  __shared__ double red[32];
  for (int r = 0; r < s; ++r) {
    if (state[8 * r + ST_DONE]) continue;
    const double* ur = u + (long long)r * n;
    double acc = 0;
    for (int l = l0 + threadIdx.x; l < l1; l += blockDim.x) acc += ur[l] * ur[l];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) part[(long long)blockIdx.x * s + r] = acc;
  }
  if (!last_block(counter)) return;
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < s; r += nw) {
    if (state[8 * r + ST_DONE]) continue;
    double acc = 0;
    for (int b = lane; b < gridDim.x; b += 32) acc += part[(long long)b * s + r];
    acc = warp_sum(acc);
    if (lane == 0) rstate[8 * r + slot] = sqrt_it ? sqrt(acc) : acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

// Starts a cycle for every rhs not done: beta = ||r||, v_0 = r / beta, g = beta e_1.
__global__ void k_start_cycle(int n, int s, int m, const double* __restrict__ rvec, double* V, int* state,
                              const double* __restrict__ rstate, double* g) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  for (int r = 0; r < s; ++r) {
    if (state[8 * r + ST_DONE]) continue;
    double beta = rstate[8 * r + RS_BETA];
    if (l < n) V[(long long)r * n + l] = rvec[(long long)r * n + l] / beta;
    if (l == 0) {
      double* gr = g + (long long)r * (m + 1);
      gr[0] = beta;
      for (int i = 1; i <= m; ++i) gr[i] = 0.0;
    }
  }
}

__global__ void k_activate(int s, int* state) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < s) state[8 * r + ST_ACTIVE] = state[8 * r + ST_DONE] ? 0 : 1;
}

// y = R^{-1} g (upper triangular jd x jd), stored over g.
__global__ void k_cycle_solve(int s, int m, const int* __restrict__ state, const double* __restrict__ H, double* g) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s || state[8 * r + ST_DONE]) return;
  int jd = state[8 * r + ST_JD];
  const double* Hr = H + (long long)r * (m + 1) * m;
  double* gr = g + (long long)r * (m + 1);
  for (int i = jd - 1; i >= 0; --i) {
    double v = gr[i];
    for (int c = i + 1; c < jd; ++c) v -= Hr[i * m + c] * gr[c];
    gr[i] = v / Hr[i * m + i];
  }
}

// x += Zk y, then w = f (the matvec that follows turns it into f - B x).
__global__ void k_xupdate(int n, int s, int m, const int* __restrict__ state, const double* __restrict__ Zk,
                          const double* __restrict__ g, double* x) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  for (int r = 0; r < s; ++r) {
    if (state[8 * r + ST_DONE]) continue;
    int jd = state[8 * r + ST_JD];
    const double* gr = g + (long long)r * (m + 1);
    double acc = x[(long long)r * n + l];
    for (int i = 0; i < jd; ++i) acc += gr[i] * Zk[((long long)i * s + r) * n + l];
    x[(long long)r * n + l] = acc;
  }
}

__global__ void k_residual(int n, int s, const int* __restrict__ state, const double* __restrict__ f,
                           double* w) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  for (int r = 0; r < s; ++r) {
    if (state[8 * r + ST_DONE]) continue;
    w[(long long)r * n + l] = f[(long long)r * n + l] - w[(long long)r * n + l];
  }
}

// After the true residual: done if ||r|| <= tol ||f|| or out of iterations.
__global__ void k_cycle_decide(int s, int* state, double* rstate, double tol, int max_iters) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s || state[8 * r + ST_DONE]) return;
  double nf = rstate[8 * r + RS_NF];
  double tr = rstate[8 * r + RS_BETA] / nf;
  rstate[8 * r + RS_TRUE] = tr;
  if (tr <= tol) {
    state[8 * r + ST_DONE] = 1;
    state[8 * r + ST_CONV] = 1;
  } else if (state[8 * r + ST_ITERS] >= max_iters) {
    state[8 * r + ST_DONE] = 1;
  }
}

__global__ void k_zero_rhs_init(int s, int* state, double* rstate) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  double nf = rstate[8 * r + RS_BETA];
  rstate[8 * r + RS_NF] = nf;
  for (int q = 0; q < 8; ++q) state[8 * r + q] = 0;
  if (nf == 0.0) {
    state[8 * r + ST_DONE] = 1;
    state[8 * r + ST_CONV] = 1;
    rstate[8 * r + RS_TRUE] = 0.0;
  }
}

hk_status ensure_workspace(hk_handle* h, int s) {
  int m = h->p.restart;
  if (h->ws_rhs >= s && h->ws_m == m) return HK_OK;
  void* old[] = {h->d_V, h->d_Zk, h->d_w, h->d_x, h->d_f, h->d_ybuf64, h->d_ybuf32, h->d_c64, h->d_cc64,
                 h->d_c32, h->d_cc32, h->d_part, h->d_counter, h->d_H, h->d_cs, h->d_sn, h->d_g, h->d_hcol,
                 h->d_state, h->d_rstate, h->d_hist};
  for (void* p : old)
    if (p) dfree(h, p);
  if (h->h_state) cudaFreeHost(h->h_state);
  if (h->h_rstate) cudaFreeHost(h->h_rstate);
  long long n = h->n;
  HK_TRY(dalloc(h, &h->d_V, (size_t)(m + 1) * s * n));
  HK_TRY(dalloc(h, &h->d_Zk, (size_t)m * s * n));
  HK_TRY(dalloc(h, &h->d_w, (size_t)s * n));
  HK_TRY(dalloc(h, &h->d_x, (size_t)s * n));
  HK_TRY(dalloc(h, &h->d_f, (size_t)s * n));
  if (h->p.precision == HK_FP32_PRECOND) {
    HK_TRY(dalloc(h, &h->d_ybuf32, (size_t)s * h->I_total));
    HK_TRY(dalloc(h, &h->d_c32, (size_t)s * (h->n0 + 1)));
    HK_TRY(dalloc(h, &h->d_cc32, (size_t)s * (h->n0 + 1)));
    h->d_ybuf64 = nullptr; h->d_c64 = nullptr; h->d_cc64 = nullptr;
  } else {
    HK_TRY(dalloc(h, &h->d_ybuf64, (size_t)s * h->I_total));
    HK_TRY(dalloc(h, &h->d_c64, (size_t)s * (h->n0 + 1)));
    HK_TRY(dalloc(h, &h->d_cc64, (size_t)s * (h->n0 + 1)));
    h->d_ybuf32 = nullptr; h->d_c32 = nullptr; h->d_cc32 = nullptr;
  }
  HK_TRY(dalloc(h, &h->d_part, (size_t)RED_BLOCKS * s * (m + 2)));
  HK_TRY(dalloc(h, &h->d_counter, 8));
  HK_TRY(dalloc(h, &h->d_H, (size_t)s * (m + 1) * m));
  HK_TRY(dalloc(h, &h->d_cs, (size_t)s * m));
  HK_TRY(dalloc(h, &h->d_sn, (size_t)s * m));
  HK_TRY(dalloc(h, &h->d_g, (size_t)s * (m + 1)));
  HK_TRY(dalloc(h, &h->d_hcol, (size_t)s * 2 * (m + 1)));
  HK_TRY(dalloc(h, &h->d_state, (size_t)s * 8));
  HK_TRY(dalloc(h, &h->d_rstate, (size_t)s * 8));
  HK_TRY(dalloc(h, &h->d_hist, (size_t)s * h->p.max_iters));
  HK_CUDA(cudaMallocHost(&h->h_state, sizeof(int) * s * 8));
  HK_CUDA(cudaMallocHost(&h->h_rstate, sizeof(double) * s * 8));
  h->ws_rhs = s;
  h->ws_m = m;
  return HK_OK;
}

hk_status run_fgmres(hk_handle* h, int s, const double* rhs_dev, double tol, double* u_dev, int32_t* iters,
                     double* res_hist, double* final_res) {
  HK_TRY(ensure_workspace(h, s));
  cudaStream_t st = h->stream;
  int n = h->n, m = h->p.restart, mi = h->p.max_iters;
  long long sn_ = (long long)s * n;
  HK_CUDA(cudaMemcpyAsync(h->d_f, rhs_dev, sizeof(double) * sn_, cudaMemcpyDeviceToDevice, st));
  HK_CUDA(cudaMemsetAsync(h->d_x, 0, sizeof(double) * sn_, st));
  HK_CUDA(cudaMemsetAsync(h->d_hist, 0, sizeof(double) * (size_t)s * mi, st));
  HK_CUDA(cudaMemsetAsync(h->d_state, 0, sizeof(int) * s * 8, st));
  HK_CUDA(cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned) * 8, st));
  // ||f|| into RS_BETA, then initialise the per-rhs state from it
  k_norm2<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, h->d_f, h->d_state, h->d_rstate, RS_BETA, h->d_part,
                                              h->d_counter, 1); HK_COUNT_LAUNCH();
  k_zero_rhs_init<<<nblk(s, 64), 64, 0, st>>>(s, h->d_state, h->d_rstate); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  const double* rvec = h->d_f;  // residual of x = 0
  int* act = h->d_state;        // ST_ACTIVE is word 0 of each rhs's 8 words
  while (true) {
    k_start_cycle<<<nblk(n, 256), 256, 0, st>>>(n, s, m, rvec, h->d_V, h->d_state, h->d_rstate, h->d_g); HK_COUNT_LAUNCH();
    k_activate<<<nblk(s, 64), 64, 0, st>>>(s, h->d_state); HK_COUNT_LAUNCH();
    HK_LAUNCH_CHECK();
    for (int j = 0; j < m; ++j) {
      double* vj = h->d_V + (long long)j * sn_;
      double* zj = h->d_Zk + (long long)j * sn_;
      HK_TRY(op_apply(h, s, vj, zj, act));
      cudaEvent_t ga = nullptr;
      if (h->timing) {
        ga = hk_event(h);
        cudaEventRecord(ga, st);
      }
      k_gs<0><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, m, j, h->d_V, h->d_w, h->d_state, h->d_rstate, h->d_hcol,
                                                  h->d_part, h->d_counter, h->d_H, h->d_cs, h->d_sn, h->d_g,
                                                  h->d_hist, mi, tol, h->d_rowptr, h->d_col, h->d_valB, zj); HK_COUNT_LAUNCH();
      k_gs<1><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, m, j, h->d_V, h->d_w, h->d_state, h->d_rstate, h->d_hcol,
                                                  h->d_part, h->d_counter, h->d_H, h->d_cs, h->d_sn, h->d_g,
                                                  h->d_hist, mi, tol, h->d_rowptr, h->d_col, h->d_valB, zj); HK_COUNT_LAUNCH();
      k_gs<2><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, m, j, h->d_V, h->d_w, h->d_state, h->d_rstate, h->d_hcol,
                                                  h->d_part, h->d_counter, h->d_H, h->d_cs, h->d_sn, h->d_g,
                                                  h->d_hist, mi, tol, h->d_rowptr, h->d_col, h->d_valB, zj); HK_COUNT_LAUNCH();
      k_normalize<<<nblk(n, 256), 256, 0, st>>>(n, s, j, h->d_V, h->d_w, h->d_state, h->d_rstate); HK_COUNT_LAUNCH();
      if (h->timing) {
        cudaEvent_t gb = hk_event(h);
        cudaEventRecord(gb, st);
        h->tl.push_back({HK_T_ARNOLDI, ga, gb});
      }
      HK_LAUNCH_CHECK();
      HK_CUDA(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(int) * 8 * s, cudaMemcpyDeviceToHost, st));
      HK_CUDA(cudaStreamSynchronize(st));
      bool any = false;
      for (int r = 0; r < s; ++r) any |= h->h_state[8 * r + ST_ACTIVE] != 0;
      if (!any) break;
    }
    // cycle end: x += Zk y, true residual
    cudaEvent_t ca = nullptr;
    if (h->timing) {
      ca = hk_event(h);
      cudaEventRecord(ca, st);
    }
    k_cycle_solve<<<nblk(s, 64), 64, 0, st>>>(s, m, h->d_state, h->d_H, h->d_g); HK_COUNT_LAUNCH();
    k_xupdate<<<nblk(n, 256), 256, 0, st>>>(n, s, m, h->d_state, h->d_Zk, h->d_g, h->d_x); HK_COUNT_LAUNCH();
    k_spmv<<<nblk(n, 256), 256, 0, st>>>(n, s, h->d_rowptr, h->d_col, h->d_valB, h->d_x, h->d_w, nullptr); HK_COUNT_LAUNCH();
    k_residual<<<nblk(n, 256), 256, 0, st>>>(n, s, h->d_state, h->d_f, h->d_w); HK_COUNT_LAUNCH();
    k_norm2<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, h->d_w, h->d_state, h->d_rstate, RS_BETA, h->d_part,
                                                h->d_counter, 1); HK_COUNT_LAUNCH();
    k_cycle_decide<<<nblk(s, 64), 64, 0, st>>>(s, h->d_state, h->d_rstate, tol, mi); HK_COUNT_LAUNCH();
    if (h->timing) {
      cudaEvent_t cb = hk_event(h);
      cudaEventRecord(cb, st);
      h->tl.push_back({HK_T_CYCLE, ca, cb});
    }
    HK_LAUNCH_CHECK();
    HK_CUDA(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(int) * 8 * s, cudaMemcpyDeviceToHost, st));
    HK_CUDA(cudaStreamSynchronize(st));
    bool all_done = true;
    for (int r = 0; r < s; ++r) all_done &= h->h_state[8 * r + ST_DONE] != 0;
    if (all_done) break;
    rvec = h->d_w;
  }
  HK_CUDA(cudaMemcpyAsync(u_dev, h->d_x, sizeof(double) * sn_, cudaMemcpyDeviceToDevice, st));
  HK_CUDA(cudaMemcpyAsync(h->h_rstate, h->d_rstate, sizeof(double) * 8 * s, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(int) * 8 * s, cudaMemcpyDeviceToHost, st));
  if (res_hist)
    HK_CUDA(cudaMemcpyAsync(res_hist, h->d_hist, sizeof(double) * (size_t)s * mi, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  bool allconv = true;
  for (int r = 0; r < s; ++r) {
    if (iters) iters[r] = h->h_state[8 * r + ST_ITERS];
    if (final_res) final_res[r] = h->h_rstate[8 * r + RS_TRUE];
    allconv &= h->h_state[8 * r + ST_CONV] != 0;
  }
  return allconv ? HK_OK : HK_NO_CONVERGENCE;
}
