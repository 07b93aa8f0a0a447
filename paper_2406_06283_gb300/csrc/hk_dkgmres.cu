// Left-preconditioned GMRES(m) in the D_k inner product: the Krylov method of Thm. 3.1, applied to the
// preconditioned system of Eq. 2.24, M^{-1} B u = M^{-1} f, with <x, y>_D = y^T D_k x (D_k = A + k^2 S,
// Prop. 2.6) in the Arnoldi process and in the residual minimisation.
//
// For s right-hand sides together (each with its own Krylov space; converged ones drop out):
//   cycle start: r = M^{-1}(f - B x), beta = ||r||_D (beta_0 of the first cycle is the reference);
//   step j: w = M^{-1} B v_j; classical Gram-Schmidt twice in the D_k inner product, with the basis
//     kept beside its image under D_k (dv_i = D_k v_i), so that <w, v_i>_D = dv_i^T w is a Euclidean dot:
//       h = DV_j^T w, w -= V_j h, h' = DV_j^T w, w -= V_j h'  (column h + h' of the Hessenberg matrix);
//     dw = D_k w, h_{j+1,j} = (w^T dw)^{1/2}, v_{j+1} = w / h_{j+1,j}, dv_{j+1} = dw / h_{j+1,j};
//     Givens rotations and the residual estimate |g_{j+1}| = ||M^{-1}(f - B x_j)||_D on the host;
//   stop a right-hand side when |g_{j+1}| <= tol beta_0, the cycle is full, or max_iters; at the end
//   of the cycle x += V y (H y = g) and the preconditioned residual is recomputed; the solve ends when
//   its D_k norm is <= tol beta_0.
// The sums over the rows are deterministic: each CTA of a fixed grid adds its row chunk in order and
// the partial sums are added in CTA order, so a right-hand side gives the same bits alone and in a
// batch.  The loop is driven from the host (one small copy per step), the matvecs and the
// preconditioner are those of the right-preconditioned solver (op_matvec, op_apply).
#include <algorithm>
#include <cmath>
#include <vector>

#include "hk_internal.cuh"

#define DK_BLOCKS 148
#define DK_THREADS 256

static inline int dk_nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// part[(b * s + r) * ld + i] = sum over the CTA's rows l of A_i[r][l] w[r][l], i < nv
// (A_i = A + i * astride, vectors of n entries per right-hand side).
__global__ void __launch_bounds__(DK_THREADS) k_dk_dots(int n, int s, int nv, const double* __restrict__ A,
                                                        long long astride, const double* __restrict__ w,
                                                        const int* __restrict__ act, double* part, int ld) {
  __shared__ double red[DK_THREADS / 32];
  int r = blockIdx.y;
  if (!act[8 * r]) return;
  long long chunk = ((long long)n + gridDim.x - 1) / gridDim.x;
  long long l0 = blockIdx.x * chunk, l1 = min((long long)n, l0 + chunk);
  const double* wr = w + (long long)r * n;
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i < nv; ++i) {
    const double* ar = A + i * astride + (long long)r * n;
    double acc = 0;
    for (long long l = l0 + threadIdx.x; l < l1; l += blockDim.x) acc += ar[l] * wr[l];
    acc = warp_sum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int q = 0; q < DK_THREADS / 32; ++q) t += red[q];
      part[((long long)blockIdx.x * s + r) * ld + i] = t;
    }
    __syncthreads();
  }
}

// out[r * ld + i] = sum over CTAs b (in order) of part[(b * s + r) * ld + i]
__global__ void k_dk_reduce(int s, int nv, int nb, const double* __restrict__ part, const int* __restrict__ act,
                            double* out, int ld) {
  int r = blockIdx.x, i = threadIdx.x;
  if (i >= nv || !act[8 * r]) return;
  double t = 0;
  for (int b = 0; b < nb; ++b) t += part[((long long)b * s + r) * ld + i];
  out[(long long)r * ld + i] = t;
}

// w[r] += sign * sum_{i < nv} coef[r * ld + i] A_i[r]
__global__ void k_dk_axpy(int n, int s, int nv, const double* __restrict__ A, long long astride,
                          const double* __restrict__ coef, int ld, double sign, double* w,
                          const int* __restrict__ act) {
  int r = blockIdx.y;
  if (!act[8 * r]) return;
  long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  const double* c = coef + (long long)r * ld;
  double acc = 0;
  for (int i = 0; i < nv; ++i) acc += c[i] * A[i * astride + (long long)r * n + l];
  w[(long long)r * n + l] += sign * acc;
}

// dst[r] = src[r] * sc[r]  and  dst2[r] = src2[r] * sc[r]
__global__ void k_dk_scale2(int n, int s, const double* __restrict__ sc, const double* __restrict__ src,
                            double* dst, const double* __restrict__ src2, double* dst2, const int* __restrict__ act) {
  int r = blockIdx.y;
  if (!act[8 * r]) return;
  long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  long long o = (long long)r * n + l;
  dst[o] = src[o] * sc[r];
  dst2[o] = src2[o] * sc[r];
}

// t = f - t  (t held B x)
__global__ void k_dk_resid(long long tot, const double* __restrict__ f, double* t) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < tot) t[e] = f[e] - t[e];
}

namespace {
struct DkState {  // host side of one right-hand side's GMRES
  std::vector<double> H, cs, sn, g;
  double beta0 = 0, nf = 0, pc_rel = 1, true_rel = 1;
  int iters = 0, jd = 0;
  bool conv = false, done = false, step = false;
};
}  // namespace

hk_status run_left_dk_gmres(hk_handle* h, int s, const double* f, double tol, double* u, int32_t* iters_out,
                            double* res_hist, double* final_true, double* final_pc) {
  HK_TRY(ensure_workspace(h, s));
  if (h->child) {
    HK_TRY(ensure_workspace(h->child, s));
    if (apply_needs_tuning(h->child, s)) HK_TRY(apply_autotune(h->child, s));
  }
  if (apply_needs_tuning(h, s)) HK_TRY(apply_autotune(h, s));
  cudaStream_t st = h->stream;
  int n = h->n, m = h->p.restart, mi = h->p.max_iters, ld = m + 2;
  long long sn = (long long)s * n;
  double *V = nullptr, *DV = nullptr, *W = nullptr, *DW = nullptr, *T = nullptr, *part = nullptr, *cf = nullptr;
  double* sc = nullptr;
  int* act = nullptr;
  HK_TRY(dalloc(h, &V, (size_t)(m + 1) * sn));
  HK_TRY(dalloc(h, &DV, (size_t)(m + 1) * sn));
  HK_TRY(dalloc(h, &W, (size_t)sn));
  HK_TRY(dalloc(h, &DW, (size_t)sn));
  HK_TRY(dalloc(h, &T, (size_t)sn));
  HK_TRY(dalloc(h, &part, (size_t)DK_BLOCKS * s * ld));
  HK_TRY(dalloc(h, &cf, (size_t)3 * s * ld));  // Gram-Schmidt passes 1, 2 and the norm
  HK_TRY(dalloc(h, &sc, (size_t)s));
  HK_TRY(dalloc(h, &act, (size_t)8 * s));
  auto release = [&]() {
    void* fr[] = {V, DV, W, DW, T, part, cf, sc, act};
    for (void* p : fr) dfree(h, p);
  };
  std::vector<DkState> R(s);
  std::vector<int> hact(8 * (size_t)s, 0);
  std::vector<double> hc(3 * (size_t)s * ld), hs(s);
  auto upload_act = [&](auto pred) -> hk_status {
    for (int r = 0; r < s; ++r) hact[8 * r] = pred(r) ? 1 : 0;
    HK_CUDA(cudaMemcpyAsync(act, hact.data(), sizeof(int) * hact.size(), cudaMemcpyHostToDevice, st));
    return HK_OK;
  };
  // cf[slot] (s x ld) = sum_i < nv of A_i^T w per right-hand side
  auto dots = [&](int nv, const double* A, long long astride, const double* w, int slot) -> hk_status {
    k_dk_dots<<<dim3(DK_BLOCKS, s), DK_THREADS, 0, st>>>(n, s, nv, A, astride, w, act, part, ld);
    HK_COUNT_LAUNCH();
    k_dk_reduce<<<s, std::max(32, (nv + 31) / 32 * 32), 0, st>>>(s, nv, DK_BLOCKS, part, act,
                                                                 cf + (size_t)slot * s * ld, ld);
    HK_COUNT_LAUNCH();
    HK_LAUNCH_CHECK();
    return HK_OK;
  };
  auto fetch = [&]() -> hk_status {
    HK_CUDA(cudaMemcpyAsync(hc.data(), cf, sizeof(double) * hc.size(), cudaMemcpyDeviceToHost, st));
    HK_CUDA(cudaStreamSynchronize(st));
    HK_TRY(check_device_status(h, "solve"));
    return HK_OK;
  };
  auto hcol = [&](int slot, int r, int i) { return hc[((size_t)slot * s + r) * ld + i]; };
  dim3 gv(dk_nblk(n, 256), s);
  hk_status rc = HK_OK;
  auto body = [&]() -> hk_status {
    HK_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * sn, st));
    HK_TRY(upload_act([](int) { return true; }));
    HK_TRY(dots(1, f, 0, f, 0));
    HK_TRY(fetch());
    for (int r = 0; r < s; ++r) {
      R[r].nf = std::sqrt(hcol(0, r, 0));
      R[r].H.assign((size_t)(m + 1) * m, 0.0);
      R[r].cs.assign(m, 0.0);
      R[r].sn.assign(m, 0.0);
      R[r].g.assign(m + 1, 0.0);
      if (R[r].nf == 0) R[r].done = R[r].conv = true, R[r].pc_rel = R[r].true_rel = 0;
    }
    bool first = true;
    for (;;) {
      // cycle start: r = M^{-1}(f - B x) for every right-hand side still running
      HK_TRY(upload_act([&](int r) { return !R[r].done; }));
      HK_TRY(op_matvec(h, s, u, T, act));
      k_dk_resid<<<dk_nblk(sn, 256), 256, 0, st>>>(sn, f, T);
      HK_COUNT_LAUNCH();
      HK_TRY(op_apply(h, s, T, V, act));
      HK_TRY(op_spmv_values(h, s, h->d_valD, V, DV, act));
      HK_TRY(dots(1, V, 0, DV, 0));
      HK_TRY(fetch());
      bool any = false;
      for (int r = 0; r < s; ++r) {
        DkState& q = R[r];
        if (q.done) continue;
        double beta = std::sqrt(std::max(hcol(0, r, 0), 0.0));
        if (first) q.beta0 = beta;
        q.pc_rel = q.beta0 > 0 ? beta / q.beta0 : 0;
        if (!first && q.pc_rel <= tol) q.done = q.conv = true;
        else if (q.iters >= mi || beta == 0) q.done = true, q.conv = beta == 0;
        if (q.done) continue;
        q.g.assign(m + 1, 0.0);
        q.g[0] = beta;
        q.jd = 0;
        q.step = true;
        hs[r] = 1.0 / beta;
        any = true;
      }
      first = false;
      if (!any) break;
      HK_TRY(upload_act([&](int r) { return R[r].step; }));
      HK_CUDA(cudaMemcpyAsync(sc, hs.data(), sizeof(double) * s, cudaMemcpyHostToDevice, st));
      k_dk_scale2<<<gv, 256, 0, st>>>(n, s, sc, V, V, DV, DV, act);
      HK_COUNT_LAUNCH();
      for (int j = 0; j < m; ++j) {
        double* Vj = V + (size_t)j * sn;
        HK_TRY(op_matvec(h, s, Vj, T, act));
        HK_TRY(op_apply(h, s, T, W, act));
        // classical Gram-Schmidt, twice, in the D_k inner product
        HK_TRY(dots(j + 1, DV, sn, W, 0));
        k_dk_axpy<<<gv, 256, 0, st>>>(n, s, j + 1, V, sn, cf, ld, -1.0, W, act);
        HK_COUNT_LAUNCH();
        HK_TRY(dots(j + 1, DV, sn, W, 1));
        k_dk_axpy<<<gv, 256, 0, st>>>(n, s, j + 1, V, sn, cf + (size_t)s * ld, ld, -1.0, W, act);
        HK_COUNT_LAUNCH();
        HK_TRY(op_spmv_values(h, s, h->d_valD, W, DW, act));
        HK_TRY(dots(1, W, 0, DW, 2));
        HK_TRY(fetch());
        bool cont = false;
        for (int r = 0; r < s; ++r) {
          DkState& q = R[r];
          if (!q.step) continue;
          double* Hc = &q.H[0];
          auto Hij = [&](int i) -> double& { return Hc[(size_t)i * m + j]; };
          for (int i = 0; i <= j; ++i) Hij(i) = hcol(0, r, i) + hcol(1, r, i);
          double hn = std::sqrt(std::max(hcol(2, r, 0), 0.0));
          Hij(j + 1) = hn;
          for (int i = 0; i < j; ++i) {
            double t = q.cs[i] * Hij(i) + q.sn[i] * Hij(i + 1);
            Hij(i + 1) = -q.sn[i] * Hij(i) + q.cs[i] * Hij(i + 1);
            Hij(i) = t;
          }
          double den = std::hypot(Hij(j), Hij(j + 1));
          q.cs[j] = Hij(j) / den;
          q.sn[j] = Hij(j + 1) / den;
          Hij(j) = den;
          Hij(j + 1) = 0;
          q.g[j + 1] = -q.sn[j] * q.g[j];
          q.g[j] = q.cs[j] * q.g[j];
          if (res_hist && q.iters < mi) res_hist[(size_t)r * mi + q.iters] = std::fabs(q.g[j + 1]) / q.beta0;
          ++q.iters;
          q.jd = j + 1;
          bool stop = std::fabs(q.g[j + 1]) <= tol * q.beta0 || q.iters >= mi || hn == 0 || j == m - 1;
          if (stop) q.step = false;
          else hs[r] = 1.0 / hn, cont = true;
        }
        if (!cont) break;
        HK_TRY(upload_act([&](int r) { return R[r].step; }));
        HK_CUDA(cudaMemcpyAsync(sc, hs.data(), sizeof(double) * s, cudaMemcpyHostToDevice, st));
        k_dk_scale2<<<gv, 256, 0, st>>>(n, s, sc, W, V + (size_t)(j + 1) * sn, DW, DV + (size_t)(j + 1) * sn,
                                        act);
        HK_COUNT_LAUNCH();
      }
      // cycle end: x += V y with H y = g (upper triangular, jd columns) per right-hand side
      std::vector<double> y((size_t)s * ld, 0.0);
      for (int r = 0; r < s; ++r) {
        DkState& q = R[r];
        if (q.done || q.jd == 0) continue;
        for (int i = q.jd - 1; i >= 0; --i) {
          double t = q.g[i];
          for (int c = i + 1; c < q.jd; ++c) t -= q.H[(size_t)i * m + c] * y[(size_t)r * ld + c];
          y[(size_t)r * ld + i] = t / q.H[(size_t)i * m + i];
        }
      }
      HK_TRY(upload_act([&](int r) { return !R[r].done && R[r].jd > 0; }));
      HK_CUDA(cudaMemcpyAsync(cf, y.data(), sizeof(double) * y.size(), cudaMemcpyHostToDevice, st));
      int jmax = 0;
      for (int r = 0; r < s; ++r)
        if (!R[r].done) jmax = std::max(jmax, R[r].jd);
      k_dk_axpy<<<gv, 256, 0, st>>>(n, s, jmax, V, sn, cf, ld, 1.0, u, act);
      HK_COUNT_LAUNCH();
      HK_LAUNCH_CHECK();
    }
    // true residual ||f - B x|| / ||f||
    HK_TRY(upload_act([&](int r) { return R[r].nf > 0; }));
    HK_TRY(op_matvec(h, s, u, T, act));
    k_dk_resid<<<dk_nblk(sn, 256), 256, 0, st>>>(sn, f, T);
    HK_COUNT_LAUNCH();
    HK_TRY(dots(1, T, 0, T, 0));
    HK_TRY(fetch());
    for (int r = 0; r < s; ++r)
      if (R[r].nf > 0) R[r].true_rel = std::sqrt(std::max(hcol(0, r, 0), 0.0)) / R[r].nf;
    return HK_OK;
  };
  rc = body();
  release();
  HK_TRY(rc);
  bool all = true;
  for (int r = 0; r < s; ++r) {
    if (iters_out) iters_out[r] = R[r].iters;
    if (final_true) final_true[r] = R[r].true_rel;
    if (final_pc) final_pc[r] = R[r].pc_rel;
    all &= R[r].conv;
  }
  return all ? HK_OK : HK_NO_CONVERGENCE;
}
