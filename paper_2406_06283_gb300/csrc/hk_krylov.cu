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

#define RED_BLOCKS 152
#define RED_THREADS 512

// state words per rhs
enum { ST_ACTIVE = 0, ST_DONE = 1, ST_ITERS = 2, ST_JD = 3, ST_CONV = 4 };
// real state per rhs
enum { RS_NF = 0, RS_HNEXT = 1, RS_EST = 2, RS_TRUE = 3, RS_BETA = 4, RS_HINV = 5 };

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

// New Hessenberg column j of rhs r (h1 + h2 above the diagonal, hn below), the previous
// rotations applied to it, the new rotation, the residual estimate and the stopping decision.
// Called by every thread of one CTA: the column and the previous rotations are first staged in
// shared memory (sc, 3 (m + 1) + 1 doubles).  Applying rotation i to the pair (x_i, b_{i+1}),
// x_0 = b_0, gives H[i][j] = c_i x_i + s_i b_{i+1} and x_{i+1} = -s_i x_i + c_i b_{i+1}: an affine
// recurrence x_{i+1} = alpha_i x_i + beta_i, so warp 0 composes the maps of consecutive rotations
// with a shuffle scan (each lane a run of ceil(j / 32) rotations) instead of one chain of j
// dependent FP64 steps; lane 0 then forms the new rotation from (x_j, hn).
__device__ void givens_column(int r, int j, int m, double hn, int* state, double* rstate, const double* hcoef,
                              double* H, double* cs, double* sn, double* g, double* hist, int max_iters,
                              double tol, double* sc) {
  const double* h1 = hcoef + (long long)r * 2 * (m + 1);
  const double* h2 = h1 + (m + 1);
  double* csr = cs + (long long)r * m;
  double* snr = sn + (long long)r * m;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) sc[i] = h1[i] + h2[i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    sc[(m + 1) + i] = csr[i];
    sc[2 * (m + 1) + i] = snr[i];
  }
  double* xj = sc + 3 * (m + 1);  // x_j, passed from the lane holding the last rotation to lane 0
  __syncthreads();
  if (threadIdx.x < 32) {
    int lane = threadIdx.x;
    double* Hr = H + (long long)r * (m + 1) * m;  // H[i][jj] at i * m + jj
    const double* c_ = sc + (m + 1);
    const double* s_ = sc + 2 * (m + 1);
    double b0 = sc[0];
    int E = (j + 31) / 32, i0 = lane * E, i1 = min(j, i0 + E);
    // this lane's run of maps composed: x -> A x + B
    double A = 1.0, B = 0.0;
    for (int i = i0; i < i1; ++i) {
      double al = -s_[i], be = c_[i] * sc[i + 1];
      A = al * A;
      B = al * B + be;
    }
    // inclusive scan over the lanes (earlier runs applied first), then the exclusive prefix
    for (int d = 1; d < 32; d <<= 1) {
      double Ao = __shfl_up_sync(0xffffffffu, A, d), Bo = __shfl_up_sync(0xffffffffu, B, d);
      if (lane >= d) {
        B = A * Bo + B;
        A = A * Ao;
      }
    }
    double Ae = __shfl_up_sync(0xffffffffu, A, 1), Be = __shfl_up_sync(0xffffffffu, B, 1);
    if (lane == 0) Ae = 1.0, Be = 0.0;
    double x = Ae * b0 + Be;  // x_{i0}
    for (int i = i0; i < i1; ++i) {
      double b = sc[i + 1];
      Hr[i * m + j] = c_[i] * x + s_[i] * b;
      x = -s_[i] * x + c_[i] * b;
    }
    if (j == 0 ? lane == 0 : (i0 < j && i1 == j)) *xj = j == 0 ? b0 : x;
    __syncwarp();
    if (lane == 0) {
      double* gr = g + (long long)r * (m + 1);
      double a = *xj, b = hn;
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
}

// out[i] = sum over CTAs b (lanes over b in order, then the shuffle tree) of
// part[(b * s + r) * (m + 2) + i] for i < nc: a warp per value, four values of a warp in flight
// together.
#define RED_VPW 4
__device__ __forceinline__ void reduce_parts(const double* part, int s, int r, int m, int nc, double* out) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i0 = warp; i0 < nc; i0 += nw * RED_VPW) {
    double acc[RED_VPW];
#pragma unroll
    for (int u = 0; u < RED_VPW; ++u) acc[u] = 0;
    for (int b = lane; b < gridDim.x; b += 32) {
      const double* pb = part + ((long long)b * s + r) * (m + 2);
#pragma unroll
      for (int u = 0; u < RED_VPW; ++u)
        if (i0 + u * nw < nc) acc[u] += pb[i0 + u * nw];
    }
#pragma unroll
    for (int u = 0; u < RED_VPW; ++u) {
      double a = warp_sum(acc[u]);
      if (lane == 0 && i0 + u * nw < nc) out[i0 + u * nw] = a;
    }
  }
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

// y = A x for s vectors with the sparsity of B and the values `val` (B or D_k); active as for op_apply.
hk_status op_spmv_values(hk_handle* h, int s, const double* val, const double* x, double* y, const int* active) {
  k_spmv<<<nblk(h->n, 256), 256, 0, h->stream>>>(h->n, s, h->d_rowptr, h->d_col, val, x, y, active); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  return HK_OK;
}

hk_status op_matvec(hk_handle* h, int s, const double* x, double* y, const int* active) {
  k_spmv<<<nblk(h->n, 256), 256, 0, h->stream>>>(h->n, s, h->d_rowptr, h->d_col, h->d_valB, x, y, active); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  return HK_OK;
}

// Gram-Schmidt pass.  MODE 0: w = B z_j on the CTA's rows (the matvec, fused), then
// h1 = V^T w.  MODE 1: w -= V h1, then h2 = V^T w.
// MODE 2: w -= V h2, ||w||^2, then (last CTA) the Hessenberg column, Givens
// rotation, residual estimate and stopping decision.
// Grid (RED_BLOCKS, s): blockIdx.y is the right-hand side, so the right-hand sides of a
// batch run side by side; each has its own completion counter, and the last CTA of a
// right-hand side adds its partials in CTA order.  The partition into row chunks does not
// depend on the batch size, so a right-hand side gives the same bits alone and in a batch.
template <int MODE>
__global__ void k_gs(int n, int s, int m, int j, const int* __restrict__ jp, const double* __restrict__ V,
                     double* w, int* state, double* rstate, double* hcoef, double* part, unsigned* counter,
                     double* H, double* cs, double* sn, double* g, double* hist, int max_iters, double tol,
                     const int* __restrict__ rowptr, const int* __restrict__ col, const double* __restrict__ val,
                     const double* __restrict__ Zk) {
  int r = blockIdx.y;
  if (!state[8 * r + ST_ACTIVE]) return;  // uniform over the CTAs of this right-hand side
  if (jp) j = *jp;  // captured inner step: j read on the device
  const double* zj = Zk + (long long)j * s * n;
  int chunk = (n + gridDim.x - 1) / gridDim.x;
  int l0 = blockIdx.x * chunk, l1 = min(n, l0 + chunk);
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int nc = MODE == 2 ? 1 : j + 1;  // values
  __shared__ double red[32];
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
  if (!last_block(counter + 8 + r)) return;
  // final reduction in the fixed CTA order
  __shared__ double fin[HK_MAXRESTART + 1];
  reduce_parts(part, s, r, m, nc, fin);
  __syncthreads();
  for (int i = tid; i < nc; i += blockDim.x) {
    if (MODE == 0) hcoef[(long long)r * 2 * (m + 1) + i] = fin[i];
    else if (MODE == 1) hcoef[(long long)r * 2 * (m + 1) + (m + 1) + i] = fin[i];
  }
  if (MODE == 2) {
    __shared__ double gsc[3 * (HK_MAXRESTART + 1) + 1];
    double hn = sqrt(fin[0]);
    if (tid == 0) {
      rstate[8 * r + RS_HNEXT] = hn;
      rstate[8 * r + RS_HINV] = hn > 0.0 ? 1.0 / hn : 0.0;  // once here, not per entry in k_normalize
    }
    givens_column(r, j, m, hn, state, rstate, hcoef, H, cs, sn, g, hist, max_iters, tol, gsc);
  }
  __syncthreads();
  if (tid == 0) counter[8 + r] = 0u;
}

// ---- one inner step's Gram-Schmidt as a single cooperative launch (batches of at most
// HK_COOP_RHS right-hand sides).  The same arithmetic as k_gs<0..2> + k_normalize in the same
// order (row chunks of RED_BLOCKS CTAs, warp-per-value reductions with lanes over CTAs), so
// both forms give the same bits; the four dependent passes are separated by grid barriers
// instead of kernel boundaries, and every CTA reduces the partial sums it needs itself.
#define HK_COOP_RHS 4

// Grid-wide barrier of a cooperative launch: arrival counter and generation word; the spin is
// bounded (`polls` polls, about a second at the default 2^25), after which HK_TIMEOUT is recorded and
// the CTA goes on.  The solve then stops at the end of the inner step and reports HK_TIMEOUT; the
// barrier words are zeroed at the start of every solve.
__device__ __forceinline__ void grid_barrier(unsigned* count, unsigned* gen, DevStatus* st, unsigned polls) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vg = gen;
    unsigned g0 = *vg;
    __threadfence();
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned it = 0;
      while (*vg == g0) {
        if (++it > polls) {
          dev_fail(st, HK_TIMEOUT, -2, 0.0);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

__global__ void __launch_bounds__(RED_THREADS) k_arnoldi_coop(
    int n, int s, int m, int j, const int* __restrict__ jp, double* V, double* w, int* state, double* rstate,
    double* hcoef, double* partA, double* partB, unsigned* bar, double* H, double* cs, double* sn, double* g,
    double* hist, int max_iters, double tol, const int* __restrict__ rowptr, const int* __restrict__ col,
    const double* __restrict__ val, const double* __restrict__ Zk, DevStatus* st, unsigned polls) {
  __shared__ double red[32];
  __shared__ double hsh[HK_COOP_RHS][HK_MAXRESTART + 1];
  __shared__ int act[HK_COOP_RHS];
  if (jp) j = *jp;
  const double* zj = Zk + (long long)j * s * n;
  int chunk = (n + gridDim.x - 1) / gridDim.x;
  int l0 = blockIdx.x * chunk, l1 = min(n, l0 + chunk);
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid < s) act[tid] = state[8 * tid + ST_ACTIVE];
  __syncthreads();
  // A: w = B z_j, h1 partials
  for (int r = 0; r < s; ++r) {
    if (!act[r]) continue;
    double* wr = w + (long long)r * n;
    const double* zr = zj + (long long)r * n;
    for (int l = l0 + tid; l < l1; l += blockDim.x) {
      double acc = 0;
      for (int q = rowptr[l]; q < rowptr[l + 1]; ++q) acc += val[q] * zr[col[q]];
      wr[l] = acc;
    }
    __syncthreads();
    double* pr = partA + ((long long)blockIdx.x * s + r) * (m + 2);
    for (int i = warp; i <= j; i += nw) {
      const double* vi = V + ((long long)i * s + r) * n;
      double acc = 0;
      for (int l = l0 + lane; l < l1; l += 32) acc += wr[l] * vi[l];
      acc = warp_sum(acc);
      if (lane == 0) pr[i] = acc;
    }
  }
  grid_barrier(bar, bar + 1, st, polls);
  // B: h1, w -= V h1, h2 partials;  C: h2, w -= V h2, ||w||^2 partials
  for (int pass = 0; pass < 2; ++pass) {
    const double* pin = pass == 0 ? partA : partB;
    double* pout = pass == 0 ? partB : partA;
    for (int r = 0; r < s; ++r) {
      if (!act[r]) continue;
      double* hr = hsh[r];
      reduce_parts(pin, s, r, m, j + 1, hr);
      __syncthreads();
      if (blockIdx.x == 0)
        for (int i = tid; i <= j; i += blockDim.x) hcoef[(long long)r * 2 * (m + 1) + pass * (m + 1) + i] = hr[i];
      double* wr = w + (long long)r * n;
      for (int l = l0 + tid; l < l1; l += blockDim.x) {
        double acc = wr[l];
        for (int i = 0; i <= j; ++i) acc -= hr[i] * V[((long long)i * s + r) * n + l];
        wr[l] = acc;
      }
      __syncthreads();
      double* pr = pout + ((long long)blockIdx.x * s + r) * (m + 2);
      if (pass == 0) {
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
      __syncthreads();
    }
    grid_barrier(bar, bar + 1, st, polls);
  }
  // D: ||w||, v_{j+1} = w / ||w|| on the CTA's rows; CTA 0: Hessenberg column, Givens, stop test
  for (int r = 0; r < s; ++r) {
    if (!act[r]) continue;
    reduce_parts(partA, s, r, m, 1, &hsh[r][0]);
    __syncthreads();
    double hn = sqrt(hsh[r][0]);
    double hinv = hn > 0.0 ? 1.0 / hn : 0.0;
    const double* wr = w + (long long)r * n;
    double* vn = V + ((long long)(j + 1) * s + r) * n;
    for (int l = l0 + tid; l < l1; l += blockDim.x) vn[l] = wr[l] * hinv;
    if (blockIdx.x == 0) {
      if (tid == 0) {
        rstate[8 * r + RS_HNEXT] = hn;
        rstate[8 * r + RS_HINV] = hinv;
      }
      // the staging area reuses hsh: every thread has read hsh[r][0] (hn) above
      __syncthreads();
      givens_column(r, j, m, hn, state, rstate, hcoef, H, cs, sn, g, hist, max_iters, tol, &hsh[0][0]);
    }
  }
}

__global__ void k_normalize(int n, int s, int j, const int* __restrict__ jp, double* V,
                            const double* __restrict__ w, const int* __restrict__ state,
                            const double* __restrict__ rstate) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  if (jp) j = *jp;
  for (int r = 0; r < s; ++r) {
    if (!state[8 * r + ST_ACTIVE]) continue;
    double inv = rstate[8 * r + RS_HINV];
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

// ---- device-side loop control of the graph form.  ctl[0] = inner step j of the cycle, ctl[1] = cycles
// run, ctl[2] = inner steps run.  Both loops are bounded by counters that only grow: the inner one by
// j < m, the outer one by the cycle count; both end at once when a kernel has recorded a failure (a
// bounded wait that ran out).
__global__ void k_ctl_cycle_begin(int* ctl, cudaGraphConditionalHandle inner) {
  ctl[0] = 0;
  cudaGraphSetConditional(inner, 1u);  // a nested condition keeps its last value: re-arm it every cycle
}

__global__ void k_ctl_step_end(int s, const int* __restrict__ state, int* ctl, int m,
                               const DevStatus* __restrict__ st, cudaGraphConditionalHandle inner) {
  int j = ++ctl[0];
  ++ctl[2];
  int any = 0;
  for (int r = 0; r < s; ++r) any |= state[8 * r + ST_ACTIVE];
  cudaGraphSetConditional(inner, (any && j < m && st->code == 0) ? 1u : 0u);
}

__global__ void k_ctl_cycle_end(int s, const int* __restrict__ state, int* ctl, int max_cycles,
                                const DevStatus* __restrict__ st, cudaGraphConditionalHandle outer) {
  int c = ++ctl[1];
  int all = 1;
  for (int r = 0; r < s; ++r) all &= state[8 * r + ST_DONE] != 0;
  cudaGraphSetConditional(outer, (!all && c < max_cycles && st->code == 0) ? 1u : 0u);
}

void hk_drop_graphs(hk_handle* h) {
  for (auto& kv : h->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.g) cudaGraphDestroy(kv.second.g);
  }
  h->graphs.clear();
}

hk_status ensure_workspace(hk_handle* h, int s) {
  int m = h->p.restart;
  if (h->ws_rhs >= s && h->ws_m == m) return HK_OK;
  // capacity rounded up to a power of two right-hand sides, so a sequence of growing batches
  // reallocates a few times only (the layouts use the actual count, a prefix of the arrays)
  int cap = 1;
  while (cap < s) cap <<= 1;
  s = cap;
  hk_drop_graphs(h);
  HK_TRY(apply_prepare(h));
  if (h->apply_only) {
    // the fine handle of a nested pair: the preconditioner's buffers only (and an input and an output block
    // for the autotuner)
    void* oldb[] = {h->d_V, h->d_Zk, h->d_ybuf64, h->d_ybuf32, h->d_c64, h->d_cc64, h->d_c32, h->d_cc32};
    for (void* p : oldb)
      if (p) dfree(h, p);
    h->d_V = h->d_Zk = h->d_ybuf64 = h->d_c64 = h->d_cc64 = nullptr;
    h->d_ybuf32 = h->d_c32 = h->d_cc32 = nullptr;
    HK_TRY(dalloc(h, &h->d_V, (size_t)s * h->n));
    HK_TRY(dalloc(h, &h->d_Zk, (size_t)s * h->n));
    if (precond_f32(h->p)) {
      HK_TRY(dalloc(h, &h->d_ybuf32, 2 * (size_t)s * h->I_total));
      HK_TRY(dalloc(h, &h->d_c32, (size_t)s * (h->n0 + 1)));
      HK_TRY(dalloc(h, &h->d_cc32, (size_t)s * (h->n0 + 1)));
    } else {
      HK_TRY(dalloc(h, &h->d_ybuf64, 2 * (size_t)s * h->I_total));
      HK_TRY(dalloc(h, &h->d_c64, (size_t)s * (h->n0 + 1)));
      HK_TRY(dalloc(h, &h->d_cc64, (size_t)s * (h->n0 + 1)));
    }
    HK_CUDA(cudaMemsetAsync(h->d_V, 0, sizeof(double) * (size_t)s * h->n, h->stream));
    h->ws_rhs = s;
    h->ws_m = m;
    h->nr_tuned.clear();
    h->tc_tuned.clear();
    return HK_OK;
  }
  void* old[] = {h->d_V, h->d_Zk, h->d_w, h->d_x, h->d_f, h->d_ybuf64, h->d_ybuf32, h->d_c64, h->d_cc64,
                 h->d_c32, h->d_cc32, h->d_part, h->d_counter, h->d_H, h->d_cs, h->d_sn, h->d_g, h->d_hcol,
                 h->d_state, h->d_rstate, h->d_hist, h->d_ctl};
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
  if (precond_f32(h->p)) {
    HK_TRY(dalloc(h, &h->d_ybuf32, 2 * (size_t)s * h->I_total));  // local solutions | coarse prolongation
    HK_TRY(dalloc(h, &h->d_c32, (size_t)s * (h->n0 + 1)));
    HK_TRY(dalloc(h, &h->d_cc32, (size_t)s * (h->n0 + 1)));
    h->d_ybuf64 = nullptr; h->d_c64 = nullptr; h->d_cc64 = nullptr;
  } else {
    HK_TRY(dalloc(h, &h->d_ybuf64, 2 * (size_t)s * h->I_total));  // local solutions | coarse prolongation
    HK_TRY(dalloc(h, &h->d_c64, (size_t)s * (h->n0 + 1)));
    HK_TRY(dalloc(h, &h->d_cc64, (size_t)s * (h->n0 + 1)));
    h->d_ybuf32 = nullptr; h->d_c32 = nullptr; h->d_cc32 = nullptr;
  }
  HK_TRY(dalloc(h, &h->d_part, 2 * (size_t)RED_BLOCKS * s * (m + 2)));  // two buffers (cooperative step)
  HK_TRY(dalloc(h, &h->d_counter, 8 + (size_t)s));  // [0]: norms; [8 + r]: Gram-Schmidt of rhs r
  HK_TRY(dalloc(h, &h->d_H, (size_t)s * (m + 1) * m));
  HK_TRY(dalloc(h, &h->d_cs, (size_t)s * m));
  HK_TRY(dalloc(h, &h->d_sn, (size_t)s * m));
  HK_TRY(dalloc(h, &h->d_g, (size_t)s * (m + 1)));
  HK_TRY(dalloc(h, &h->d_hcol, (size_t)s * 2 * (m + 1)));
  HK_TRY(dalloc(h, &h->d_state, (size_t)s * 8));
  HK_TRY(dalloc(h, &h->d_rstate, (size_t)s * 8));
  HK_TRY(dalloc(h, &h->d_hist, (size_t)s * h->p.max_iters));
  HK_TRY(dalloc(h, &h->d_ctl, 4));
  HK_CUDA(cudaMallocHost(&h->h_state, sizeof(int) * s * 8));
  HK_CUDA(cudaMallocHost(&h->h_rstate, sizeof(double) * s * 8));
  h->ws_rhs = s;
  h->ws_m = m;
  h->nr_tuned.clear();
  h->tc_tuned.clear();
  return HK_OK;
}

// Residual of x = 0 and per-rhs state; w = f so that every cycle starts from w.
static hk_status fgmres_init(hk_handle* h, int s, const double* rhs_dev) {
  cudaStream_t st = h->stream;
  int n = h->n, mi = h->p.max_iters;
  long long sn_ = (long long)s * n;
  HK_CUDA(cudaMemcpyAsync(h->d_f, rhs_dev, sizeof(double) * sn_, cudaMemcpyDeviceToDevice, st));
  HK_CUDA(cudaMemcpyAsync(h->d_w, rhs_dev, sizeof(double) * sn_, cudaMemcpyDeviceToDevice, st));
  HK_CUDA(cudaMemsetAsync(h->d_x, 0, sizeof(double) * sn_, st));
  HK_CUDA(cudaMemsetAsync(h->d_hist, 0, sizeof(double) * (size_t)s * mi, st));
  HK_CUDA(cudaMemsetAsync(h->d_state, 0, sizeof(int) * s * 8, st));
  HK_CUDA(cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned) * (8 + (size_t)s), st));
  HK_CUDA(cudaMemsetAsync(h->d_ctl, 0, sizeof(int) * 4, st));
  // ||f|| into RS_BETA, then initialise the per-rhs state from it
  k_norm2<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, h->d_f, h->d_state, h->d_rstate, RS_BETA, h->d_part,
                                              h->d_counter, 1); HK_COUNT_LAUNCH();
  k_zero_rhs_init<<<nblk(s, 64), 64, 0, st>>>(s, h->d_state, h->d_rstate); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  return HK_OK;
}

// beta = ||r||, v_0 = r / beta, g = beta e_1 for every rhs not done; activate them.
static hk_status fgmres_cycle_start(hk_handle* h, int s) {
  cudaStream_t st = h->stream;
  int n = h->n, m = h->p.restart;
  k_start_cycle<<<nblk(n, 256), 256, 0, st>>>(n, s, m, h->d_w, h->d_V, h->d_state, h->d_rstate, h->d_g); HK_COUNT_LAUNCH();
  k_activate<<<nblk(s, 64), 64, 0, st>>>(s, h->d_state); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  return HK_OK;
}

// Whether the cooperative Gram-Schmidt launch fits on this device (RED_BLOCKS CTAs resident).
static bool coop_ready(hk_handle* h) {
  if (h->coop_state == 0) {
    int coop = 0, nsm = 0, per = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_arnoldi_coop, RED_THREADS, 0);
    h->coop_state = (coop && (long long)nsm * per >= RED_BLOCKS) ? 1 : -1;
    cudaGetLastError();
  }
  return h->coop_state > 0;
}

// Inner step j: z_j = M^{-1} v_j, w = B z_j, CGS2, Givens, v_{j+1}.  With jp != NULL every kernel reads
// j from *jp (the captured form); otherwise j is passed by value.
static hk_status fgmres_step(hk_handle* h, int s, double tol, int j, const int* jp) {
  cudaStream_t st = h->stream;
  int n = h->n, m = h->p.restart, mi = h->p.max_iters;
  long long sn_ = (long long)s * n;
  const double* vj = h->d_V + (jp ? 0 : (long long)j * sn_);
  double* zj = h->d_Zk + (jp ? 0 : (long long)j * sn_);
  h->g_jp = jp;
  h->g_jstride = sn_;
  hk_status rc = op_apply(h, s, vj, zj, h->d_state);
  h->g_jp = nullptr;
  HK_TRY(rc);
  cudaEvent_t ga = nullptr;
  if (h->timing) {
    ga = hk_event(h);
    cudaEventRecord(ga, st);
  }
  if (s <= HK_COOP_RHS && coop_ready(h)) {
    double* partB = h->d_part + (size_t)RED_BLOCKS * s * (m + 2);
    unsigned* bar = h->d_counter + 2;
    double* V = h->d_V;
    const double* Zk = h->d_Zk;
    void* args[] = {&n, &s, &m, &j, (void*)&jp, &V, &h->d_w, &h->d_state, &h->d_rstate, &h->d_hcol, &h->d_part,
                    &partB, &bar, &h->d_H, &h->d_cs, &h->d_sn, &h->d_g, &h->d_hist, &mi, &tol, &h->d_rowptr,
                    &h->d_col, &h->d_valB, (void*)&Zk, &h->d_status, &h->wait_polls};
    HK_CUDA(cudaLaunchCooperativeKernel((const void*)k_arnoldi_coop, dim3(RED_BLOCKS), dim3(RED_THREADS), args, 0, st));
    HK_COUNT_LAUNCH();
    if (h->timing) {
      cudaEvent_t gb = hk_event(h);
      cudaEventRecord(gb, st);
      h->tl.push_back({HK_T_ARNOLDI, ga, gb});
    }
    return HK_OK;
  }
  k_gs<0><<<dim3(RED_BLOCKS, s), RED_THREADS, 0, st>>>(n, s, m, j, jp, h->d_V, h->d_w, h->d_state, h->d_rstate, h->d_hcol,
                                              h->d_part, h->d_counter, h->d_H, h->d_cs, h->d_sn, h->d_g, h->d_hist,
                                              mi, tol, h->d_rowptr, h->d_col, h->d_valB, h->d_Zk); HK_COUNT_LAUNCH();
  k_gs<1><<<dim3(RED_BLOCKS, s), RED_THREADS, 0, st>>>(n, s, m, j, jp, h->d_V, h->d_w, h->d_state, h->d_rstate, h->d_hcol,
                                              h->d_part, h->d_counter, h->d_H, h->d_cs, h->d_sn, h->d_g, h->d_hist,
                                              mi, tol, h->d_rowptr, h->d_col, h->d_valB, h->d_Zk); HK_COUNT_LAUNCH();
  k_gs<2><<<dim3(RED_BLOCKS, s), RED_THREADS, 0, st>>>(n, s, m, j, jp, h->d_V, h->d_w, h->d_state, h->d_rstate, h->d_hcol,
                                              h->d_part, h->d_counter, h->d_H, h->d_cs, h->d_sn, h->d_g, h->d_hist,
                                              mi, tol, h->d_rowptr, h->d_col, h->d_valB, h->d_Zk); HK_COUNT_LAUNCH();
  k_normalize<<<nblk(n, 256), 256, 0, st>>>(n, s, j, jp, h->d_V, h->d_w, h->d_state, h->d_rstate); HK_COUNT_LAUNCH();
  if (h->timing) {
    cudaEvent_t gb = hk_event(h);
    cudaEventRecord(gb, st);
    h->tl.push_back({HK_T_ARNOLDI, ga, gb});
  }
  HK_LAUNCH_CHECK();
  return HK_OK;
}

// Cycle end: x += Zk y, w = f - B x, ||w||, done / new cycle decision.
static hk_status fgmres_cycle_end(hk_handle* h, int s, double tol) {
  cudaStream_t st = h->stream;
  int n = h->n, m = h->p.restart, mi = h->p.max_iters;
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
  return HK_OK;
}

// Captures the whole solve (after fgmres_init) into one graph:
//   WHILE (not all done, cycles < max_iters + 2) {            outer, handle c_out
//     cycle start; j = 0; re-arm c_in
//     WHILE (some rhs active and j < m) { inner step j; j++ } inner, handle c_in
//     cycle end
//   }
static hk_status build_solve_graph(hk_handle* h, int s, double tol, hk_handle::SolveGraph& G) {
  cudaStream_t st = h->stream;
  int m = h->p.restart, max_cycles = h->p.max_iters + 2;
  cudaGraph_t g = nullptr;
  HK_CUDA(cudaGraphCreate(&g, 0));
  G.g = g;
  cudaGraphConditionalHandle c_out, c_in;
  HK_CUDA(cudaGraphConditionalHandleCreate(&c_out, g, 1, cudaGraphCondAssignDefault));
  HK_CUDA(cudaGraphConditionalHandleCreate(&c_in, g, 0, 0));
  cudaGraphNodeParams po = {};
  po.type = cudaGraphNodeTypeConditional;
  po.conditional.handle = c_out;
  po.conditional.type = cudaGraphCondTypeWhile;
  po.conditional.size = 1;
  cudaGraphNode_t n_out;
  HK_CUDA(cudaGraphAddNode(&n_out, g, nullptr, nullptr, 0, &po));
  cudaGraph_t body_out = po.conditional.phGraph_out[0];
  cudaGraph_t body_in = nullptr;
  hk_status rc = HK_OK;
  cudaError_t e = cudaStreamBeginCaptureToGraph(st, body_out, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    hk_set_error("graph capture: %s", cudaGetErrorString(e));
    return HK_CUDA_ERROR;
  }
  g_hk_capture_count = 0;
  rc = fgmres_cycle_start(h, s);
  if (rc == HK_OK) {
    k_ctl_cycle_begin<<<1, 1, 0, st>>>(h->d_ctl, c_in);
    HK_COUNT_LAUNCH();
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd);
    cudaGraphNodeParams pi = {};
    pi.type = cudaGraphNodeTypeConditional;
    pi.conditional.handle = c_in;
    pi.conditional.type = cudaGraphCondTypeWhile;
    pi.conditional.size = 1;
    cudaGraphNode_t n_in = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&n_in, body_out, deps, nullptr, nd, &pi);
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(st, &n_in, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
      body_in = pi.conditional.phGraph_out[0];
      rc = fgmres_cycle_end(h, s, tol);
      k_ctl_cycle_end<<<1, 1, 0, st>>>(s, h->d_state, h->d_ctl, max_cycles, h->d_status, c_out);
      HK_COUNT_LAUNCH();
    } else {
      hk_set_error("graph capture: %s", cudaGetErrorString(e));
      rc = HK_CUDA_ERROR;
    }
  }
  G.cycle_kernels = g_hk_capture_count;
  cudaGraph_t tmp = nullptr;
  e = cudaStreamEndCapture(st, &tmp);
  if (rc == HK_OK && e != cudaSuccess) {
    hk_set_error("graph capture: %s", cudaGetErrorString(e));
    rc = HK_CUDA_ERROR;
  }
  if (rc == HK_OK) {
    e = cudaStreamBeginCaptureToGraph(st, body_in, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      hk_set_error("graph capture: %s", cudaGetErrorString(e));
      rc = HK_CUDA_ERROR;
    } else {
      g_hk_capture_count = 0;
      rc = fgmres_step(h, s, tol, 0, h->d_ctl);
      k_ctl_step_end<<<1, 1, 0, st>>>(s, h->d_state, h->d_ctl, m, h->d_status, c_in);
      HK_COUNT_LAUNCH();
      G.iter_kernels = g_hk_capture_count;
      e = cudaStreamEndCapture(st, &tmp);
      if (rc == HK_OK && e != cudaSuccess) {
        hk_set_error("graph capture: %s", cudaGetErrorString(e));
        rc = HK_CUDA_ERROR;
      }
    }
  }
  g_hk_capture_count = -1;
  if (rc == HK_OK) {
    e = cudaGraphInstantiate(&G.exec, g, 0);
    if (e != cudaSuccess) {
      hk_set_error("graph instantiate: %s", cudaGetErrorString(e));
      rc = HK_CUDA_ERROR;
    }
  }
  cudaGetLastError();
  return rc;
}

static hk_status fgmres_results(hk_handle* h, int s, double* u_dev, int32_t* iters, double* res_hist,
                                double* final_res, int* ctl_out) {
  cudaStream_t st = h->stream;
  int n = h->n, mi = h->p.max_iters;
  long long sn_ = (long long)s * n;
  HK_CUDA(cudaMemcpyAsync(u_dev, h->d_x, sizeof(double) * sn_, cudaMemcpyDeviceToDevice, st));
  HK_CUDA(cudaMemcpyAsync(h->h_rstate, h->d_rstate, sizeof(double) * 8 * s, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(int) * 8 * s, cudaMemcpyDeviceToHost, st));
  if (ctl_out) HK_CUDA(cudaMemcpyAsync(ctl_out, h->d_ctl, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
  if (res_hist)
    HK_CUDA(cudaMemcpyAsync(res_hist, h->d_hist, sizeof(double) * (size_t)s * mi, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  // a bounded device wait that ran out during the solve (apply or Gram-Schmidt): the outputs are
  // written but not trusted
  HK_TRY(check_device_status(h, "solve"));
  bool allconv = true;
  for (int r = 0; r < s; ++r) {
    if (iters) iters[r] = h->h_state[8 * r + ST_ITERS];
    if (final_res) final_res[r] = h->h_rstate[8 * r + RS_TRUE];
    allconv &= h->h_state[8 * r + ST_CONV] != 0;
  }
  return allconv ? HK_OK : HK_NO_CONVERGENCE;
}

hk_status run_fgmres(hk_handle* h, int s, const double* rhs_dev, double tol, double* u_dev, int32_t* iters,
                     double* res_hist, double* final_res) {
  HK_TRY(ensure_workspace(h, s));
  if (h->child) {
    HK_TRY(ensure_workspace(h->child, s));
    if (apply_needs_tuning(h->child, s)) HK_TRY(apply_autotune(h->child, s));
  }
  if (apply_needs_tuning(h, s)) HK_TRY(apply_autotune(h, s));
  cudaStream_t st = h->stream;
  int m = h->p.restart;
  HK_TRY(fgmres_init(h, s, rhs_dev));
  if (!h->timing && h->graphs_ok && h->use_graphs) {
    // one graph launch for the whole solve; the loops run on the device.  The legacy default stream
    // cannot be captured: then the graph is captured and launched on a private blocking stream, which
    // the legacy stream orders with the work before and after it.
    cudaStream_t gs = h->stream;
    if (gs == nullptr || gs == cudaStreamLegacy) {
      if (!h->cap_stream) HK_CUDA(cudaStreamCreate(&h->cap_stream));
      gs = h->cap_stream;
    }
    auto key = std::make_pair(s, tol);
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
      hk_handle::SolveGraph G;
      cudaStream_t user = h->stream;
      h->stream = gs;
      hk_status brc = build_solve_graph(h, s, tol, G);
      h->stream = user;
      if (brc != HK_OK) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        if (G.g) cudaGraphDestroy(G.g);
        h->graphs_ok = false;  // keep the kernels, drive the loops from the host
      } else {
        it = h->graphs.emplace(key, G).first;
      }
    }
    if (h->graphs_ok) {
      HK_CUDA(cudaGraphLaunch(it->second.exec, gs));
      h->graph_solves++;
      int ctl[4] = {0, 0, 0, 0};
      hk_status rs = fgmres_results(h, s, u_dev, iters, res_hist, final_res, ctl);
      g_hk_launches.fetch_add((long long)it->second.cycle_kernels * ctl[1] + (long long)it->second.iter_kernels * ctl[2],
                              std::memory_order_relaxed);
      return rs;
    }
  }
  // host-driven loops (kernel timing on, or no graph support): the same kernels
  while (true) {
    HK_TRY(fgmres_cycle_start(h, s));
    for (int j = 0; j < m; ++j) {
      HK_TRY(fgmres_step(h, s, tol, j, nullptr));
      HK_CUDA(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(int) * 8 * s, cudaMemcpyDeviceToHost, st));
      HK_CUDA(cudaMemcpyAsync(&h->h_code, &h->d_status->code, sizeof(int), cudaMemcpyDeviceToHost, st));
      HK_CUDA(cudaStreamSynchronize(st));
      if (h->h_code != 0) return fgmres_results(h, s, u_dev, iters, res_hist, final_res, nullptr);
      bool any = false;
      for (int r = 0; r < s; ++r) any |= h->h_state[8 * r + ST_ACTIVE] != 0;
      if (!any) break;
    }
    HK_TRY(fgmres_cycle_end(h, s, tol));
    HK_CUDA(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(int) * 8 * s, cudaMemcpyDeviceToHost, st));
    HK_CUDA(cudaStreamSynchronize(st));
    bool all_done = true;
    for (int r = 0; r < s; ++r) all_done &= h->h_state[8 * r + ST_DONE] != 0;
    if (all_done) break;
  }
  return fgmres_results(h, s, u_dev, iters, res_hist, final_res, nullptr);
}
