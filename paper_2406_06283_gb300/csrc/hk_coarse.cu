// Coarse operator of Eq. 2.23: E = Z^T B Z (the Galerkin matrix of
// B_0 = R_0 B E_0 with R_0 = Z^T) and its inverse, both FP64 on the device.
// Z_i is supported on dof(Omega_i), so the block E_ij is nonzero only when
// some dof of Omega_i is coupled by B to a dof of Omega_j; those pairs are
// found from the pull map and each pair's block is computed by one CTA in a
// fixed summation order.  E^{-1} is formed by Gauss-Jordan elimination with
// partial pivoting (one column per step); a pivot below 1e-10 max|E| reports
// HK_SINGULAR_COARSE.
#include <algorithm>

#include <cooperative_groups.h>

#include "hk_internal.cuh"

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

__global__ void k_coarse_pairs(int n, int n_sub, const int* __restrict__ rowptr, const int* __restrict__ col,
                               const int* __restrict__ pull_ptr, const int* __restrict__ pull_sub, uint8_t* pair) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  for (int q = rowptr[l]; q < rowptr[l + 1]; ++q) {
    int c = col[q];
    for (int p = pull_ptr[l]; p < pull_ptr[l + 1]; ++p)
      for (int r = pull_ptr[c]; r < pull_ptr[c + 1]; ++r)
        pair[(long long)pull_sub[p] * n_sub + pull_sub[r]] = 1;
  }
}

// E_ij = Z_i^T (B Z_j)|_{dof(Omega_i)}, rows of dof(Omega_i) taken in chunks.
#define HK_ECHUNK 32
__global__ void k_coarse_block(const int* __restrict__ pairs, int n0, const int* __restrict__ sub_info,
                               const long long* __restrict__ sub_off, const int* __restrict__ Ilev,
                               const int* __restrict__ Isorted, const int* __restrict__ perm,
                               const int* __restrict__ rowptr, const int* __restrict__ col,
                               const double* __restrict__ valB, const double* __restrict__ Z, double* E) {
  extern __shared__ double sm[];  // HK_ECHUNK x mj
  int i = pairs[2 * blockIdx.x], j = pairs[2 * blockIdx.x + 1];
  const int* si = sub_info + 8 * i;
  const int* sj = sub_info + 8 * j;
  int nIi = si[0], offi = si[3], mi = si[6], ci = si[7];
  int nIj = sj[0], offj = sj[3], mj = sj[6], cj = sj[7];
  if (mi == 0 || mj == 0) return;
  const double* Zi = Z + sub_off[3 * i + 2];
  const double* Zj = Z + sub_off[3 * j + 2];
  for (int e = threadIdx.x; e < mi * mj; e += blockDim.x)
    E[(long long)(ci + e / mj) * n0 + cj + e % mj] = 0.0;
  __syncthreads();
  for (int a0 = 0; a0 < nIi; a0 += HK_ECHUNK) {
    int na = min(HK_ECHUNK, nIi - a0);
    for (int e = threadIdx.x; e < na * mj; e += blockDim.x) {
      int a = a0 + e / mj, lj = e % mj;
      int g = Ilev[offi + a];
      double acc = 0;
      for (int q = rowptr[g]; q < rowptr[g + 1]; ++q) {
        int idx = bsearch_int(Isorted + offj, nIj, col[q]);
        if (idx < 0) continue;
        int b = perm[offj + idx];
        acc += valB[q] * Zj[(long long)b * mj + lj];
      }
      sm[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < mi * mj; e += blockDim.x) {
      int li = e / mj, lj = e % mj;
      double acc = 0;
      for (int a = 0; a < na; ++a) acc += Zi[(long long)(a0 + a) * mi + li] * sm[a * mj + lj];
      E[(long long)(ci + li) * n0 + cj + lj] += acc;
    }
    __syncthreads();
  }
}

__global__ void k_absmax(const double* __restrict__ a, long long n, double* out) {
  __shared__ double red[32];
  double m = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    // monotone max on a non-negative double through its bit pattern
    atomicMax((unsigned long long*)out, (unsigned long long)__double_as_longlong(t));
  }
}

// Blocked in-place Gauss-Jordan inverse of the n0 x n0 matrix A with partial pivoting and implicit row
// interchanges.  Unblocked, step k picks the unused row p_k with the largest |A[p][k]|, scales it, and
// eliminates column k from every other row; column k then holds column p_k of the accumulated
// transform, and the inverse is Inv[k][j] = A[p_k][q_j] with q the inverse of p (k_gj_unpermute).
// Blocked, the steps of a panel of HK_GJ_NB columns touch only the panel's columns (k_gj_panel); the
// panel's composite row transform is then I + sum_j (C_j - e_{p_j}) e_{p_j}^T, C_j the panel's final
// column j, so every other column gets the rank-HK_GJ_NB update A[:, c] += (C - E_P) A[P, c] with the
// pivot rows P read before it (k_gj_update).  Same pivots as the unblocked form, FP64 throughout.
#define HK_GJ_NB 32

// Panel steps k0 .. k1-1 on columns k0 .. k1-1 (k1 - k0 <= HK_GJ_NB) by one thread-block cluster of G
// CTAs.  Row i is owned by CTA i mod G, which keeps the row's panel entries (and its used flag) in
// shared memory for the whole panel: Ps[r][j] holds A[i][k0 + j] for i = me + G r.  Each step reduces
// the per-CTA maxima through distributed shared memory, every CTA reads the unscaled pivot row from its
// owner's shared memory and scales its own copy, eliminates its rows and searches its rows for the next
// pivot; the step ends at the cluster barrier, after which the owner overwrites the pivot row with the
// scaled one (no CTA reads it any more).  Ties go to the smallest row index.
__global__ void k_gj_panel(double* A, int n0, int k0, int k1, int* piv, int* used, double* minpiv) {
  extern __shared__ double Ps[];  // nloc x HK_GJ_NB, then nloc used flags
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ double cmax_v[2];  // this CTA's maximum for the next column (double buffered)
  __shared__ int cmax_i[2];
  __shared__ int sh_p;
  __shared__ double sh_f;
  __shared__ double prow[HK_GJ_NB];  // the scaled pivot row
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  int nb = k1 - k0;
  int G = (int)cl.num_blocks(), me = (int)cl.block_rank();
  int nloc = me < n0 ? (n0 - me + G - 1) / G : 0;
  int nloc_max = (n0 + G - 1) / G;
  int* uloc = reinterpret_cast<int*>(Ps + (long long)nloc_max * HK_GJ_NB);
  for (int e = tid; e < nloc * nb; e += T) {
    int r = e / nb, j = e % nb;
    Ps[r * HK_GJ_NB + j] = A[(long long)(me + G * r) * n0 + k0 + j];
  }
  for (int r = tid; r < nloc; r += T) uloc[r] = used[me + G * r];
  __syncthreads();
  auto local_max = [&](int jc, int buf) {
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int r = tid; r < nloc; r += T) {
      if (uloc[r]) continue;
      double v = fabs(Ps[r * HK_GJ_NB + jc]);
      int i = me + G * r;
      if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = rv[0];
      int bj = ri[0];
      for (int w = 1; w < nw; ++w)
        if (rv[w] > bv || (rv[w] == bv && ri[w] < bj)) { bv = rv[w]; bj = ri[w]; }
      cmax_v[buf] = bv;
      cmax_i[buf] = bj;
    }
  };
  local_max(0, k0 & 1);
  cl.sync();
  int pprev = -1;
  for (int k = k0; k < k1; ++k) {
    int jk = k - k0;
    if (pprev >= 0 && me == pprev % G) {  // deferred: the scaled previous pivot row into its owner's rows
      int rp = pprev / G;
      for (int j = tid; j < nb; j += T) Ps[rp * HK_GJ_NB + j] = prow[j];
    }
    __syncthreads();
    int buf = k & 1;
    if (warp == 0) {
      double bv = -1.0;
      int bj = 0x7fffffff;
      if (lane < G) {
        bv = *cl.map_shared_rank(&cmax_v[buf], lane);
        bj = *cl.map_shared_rank(&cmax_i[buf], lane);
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ov > bv || (ov == bv && oi < bj)) { bv = ov; bj = oi; }
      }
      if (lane == 0) sh_p = bj;
    }
    __syncthreads();
    int p = sh_p, owner = p % G, rp = p / G;
    const double* prem = cl.map_shared_rank(Ps + (long long)rp * HK_GJ_NB, owner);  // unscaled pivot row
    if (tid == 0) {
      double pv = prem[jk];
      sh_f = pv != 0.0 ? 1.0 / pv : 0.0;
      if (me == 0) {
        piv[k] = p;
        if (fabs(pv) < *minpiv) *minpiv = fabs(pv);
      }
    }
    __syncthreads();
    double f = sh_f;
    double pj_ = tid < nb ? prem[tid] : 0.0;
    __syncthreads();  // prow of the previous step was consumed above
    if (tid < nb) prow[tid] = tid == jk ? f : pj_ * f;
    __syncthreads();
    // eliminate column k from the owned rows other than p
    for (int r = warp; r < nloc; r += nw) {
      if (me + G * r == p) continue;
      double* ar = Ps + r * HK_GJ_NB;
      double g = ar[jk];
      __syncwarp();
      if (g != 0.0 && lane < nb) ar[lane] = lane == jk ? -g * f : ar[lane] - g * prow[lane];
    }
    if (me == owner && tid == 0) uloc[rp] = 1;
    __syncthreads();
    if (k + 1 < k1) local_max(jk + 1, (k + 1) & 1);
    cl.sync();
    pprev = p;
  }
  if (pprev >= 0 && me == pprev % G) {
    int rp = pprev / G;
    for (int j = tid; j < nb; j += T) Ps[rp * HK_GJ_NB + j] = prow[j];
  }
  __syncthreads();
  for (int e = tid; e < nloc * nb; e += T) {
    int r = e / nb, j = e % nb;
    A[(long long)(me + G * r) * n0 + k0 + j] = Ps[r * HK_GJ_NB + j];
  }
  for (int r = tid; r < nloc; r += T) used[me + G * r] = uloc[r];
}

// Q[j][c] = A[p_{k0+j}][c] for the panel's pivot rows (read before the update changes them).
__global__ void k_gj_pivot_rows(const double* __restrict__ A, int n0, int k0, int nb, const int* __restrict__ piv,
                                double* Q) {
  int j = blockIdx.y;
  const double* src = A + (long long)piv[k0 + j] * n0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n0; c += gridDim.x * blockDim.x)
    Q[(long long)j * n0 + c] = src[c];
}

// A[i][c] += sum_j (A[i][k0+j] - [i == p_j]) Q[j][c] for every column c outside the panel: a 64 x 64
// output tile per CTA, 256 threads with 4 x 4 outputs each, the panel slice and Q slice in shared memory.
__global__ void __launch_bounds__(256) k_gj_update(double* A, int n0, int k0, int nb, const int* __restrict__ piv,
                                                   const double* __restrict__ Q) {
  __shared__ double Cs[64][HK_GJ_NB + 1];
  __shared__ double Qs[HK_GJ_NB][64];
  __shared__ int pj[HK_GJ_NB];
  int i0 = blockIdx.y * 64, c0 = blockIdx.x * 64, tid = threadIdx.x;
  if (tid < nb) pj[tid] = piv[k0 + tid];
  __syncthreads();
  for (int e = tid; e < 64 * HK_GJ_NB; e += 256) {
    int r = e / HK_GJ_NB, j = e % HK_GJ_NB;
    int i = i0 + r;
    double v = 0.0;
    if (i < n0 && j < nb) v = A[(long long)i * n0 + k0 + j] - (i == pj[j] ? 1.0 : 0.0);
    Cs[r][j] = v;
  }
  for (int e = tid; e < HK_GJ_NB * 64; e += 256) {
    int j = e / 64, c = e % 64;
    Qs[j][c] = (j < nb && c0 + c < n0) ? Q[(long long)j * n0 + c0 + c] : 0.0;
  }
  __syncthreads();
  int tr = (tid / 16) * 4, tc = (tid % 16) * 4;
  double acc[4][4] = {};
  for (int j = 0; j < nb; ++j) {
    double a[4], q[4];
    for (int u = 0; u < 4; ++u) a[u] = Cs[tr + u][j];
    for (int u = 0; u < 4; ++u) q[u] = Qs[j][tc + u];
    for (int u = 0; u < 4; ++u)
      for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * q[v];
  }
  for (int u = 0; u < 4; ++u) {
    int i = i0 + tr + u;
    if (i >= n0) continue;
    for (int v = 0; v < 4; ++v) {
      int c = c0 + tc + v;
      if (c >= n0 || (c >= k0 && c < k0 + nb)) continue;
      A[(long long)i * n0 + c] += acc[u][v];
    }
  }
}

// Inv[k][j] = A[p_k][q_j], q = p^{-1}.
__global__ void k_gj_unpermute(const double* __restrict__ A, double* Inv, int n0, const int* __restrict__ piv,
                               const int* __restrict__ qinv) {
  int k = blockIdx.x;
  const double* ar = A + (long long)piv[k] * n0;
  for (int j = threadIdx.x; j < n0; j += blockDim.x) Inv[(long long)k * n0 + j] = ar[qinv[j]];
}

__global__ void k_invert_perm(const int* __restrict__ piv, int* qinv, int n0) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n0) qinv[piv[k]] = k;
}

hk_status phase_coarse(hk_handle* h) {
  cudaStream_t st = h->stream;
  int ns = h->n_sub, n0 = h->n0, n = h->n;
  if (n0 == 0) return HK_OK;
  uint8_t* d_pair = nullptr;
  HK_TRY(dalloc(h, &d_pair, (size_t)ns * ns));
  k_coarse_pairs<<<nblk(n, 256), 256, 0, st>>>(n, ns, h->d_rowptr, h->d_col, h->d_pull_ptr, h->d_pull_sub, d_pair); HK_COUNT_LAUNCH();
  std::vector<uint8_t> pair((size_t)ns * ns);
  HK_CUDA(cudaMemcpyAsync(pair.data(), d_pair, pair.size(), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  std::vector<int> plist;
  for (int i = 0; i < ns; ++i)
    for (int j = 0; j < ns; ++j)
      if (pair[(size_t)i * ns + j] && h->subs[i].m > 0 && h->subs[j].m > 0) {
        plist.push_back(i);
        plist.push_back(j);
      }
  int np = (int)plist.size() / 2;
  int* d_plist = nullptr;
  HK_TRY(dalloc(h, &d_plist, plist.size()));
  HK_CUDA(cudaMemcpyAsync(d_plist, plist.data(), sizeof(int) * plist.size(), cudaMemcpyHostToDevice, st));
  HK_TRY(dalloc(h, &h->d_E, (size_t)n0 * n0));
  HK_TRY(dalloc(h, &h->d_Einv64, (size_t)n0 * n0));
  int maxm = 0;
  for (auto& u : h->subs) maxm = u.m > maxm ? u.m : maxm;
  size_t shm = sizeof(double) * HK_ECHUNK * maxm;
  HK_TRY(hk_allow_smem(k_coarse_block));
  if (np > 0) {
    k_coarse_block<<<np, 256, shm, st>>>(d_plist, n0, h->d_sub_info, h->d_sub_off, h->d_I, h->d_Isorted,
                                         h->d_perm, h->d_rowptr, h->d_col, h->d_valB, h->d_Z64, h->d_E);
    HK_COUNT_LAUNCH();
  }
  HK_LAUNCH_CHECK();
  HK_CUDA(cudaMemcpyAsync(h->d_Einv64, h->d_E, sizeof(double) * n0 * n0, cudaMemcpyDeviceToDevice, st));
  double* d_sc = nullptr;  // [0] max|E|, [1] min pivot
  int* d_piv = nullptr;
  HK_TRY(dalloc(h, &d_sc, 2));
  HK_TRY(dalloc(h, &d_piv, n0));
  k_absmax<<<304, 256, 0, st>>>(h->d_E, (long long)n0 * n0, d_sc);
  HK_COUNT_LAUNCH();
  double big = 1e300;
  HK_CUDA(cudaMemcpyAsync(d_sc + 1, &big, sizeof(double), cudaMemcpyHostToDevice, st));
  {
    // blocked: per panel one launch of one thread-block cluster, then the rank-HK_GJ_NB update
    int threads = 256;  // a panel step is short: cheap barriers matter more than threads
    // cluster size: enough CTAs that each holds its rows' panel entries in shared memory
    auto panel_smem = [&](int g) { return (size_t)((n0 + g - 1) / g) * (HK_GJ_NB * sizeof(double) + sizeof(int)); };
    int G = std::min(8, std::max(1, n0 / 64));
    while (G < 8 && panel_smem(G) > 200 * 1024) G *= 2;
    if (panel_smem(G) > 200 * 1024) G = 16;  // non-portable cluster size
    if (panel_smem(G) > 200 * 1024) {
      hk_set_error("coarse dimension %d too large for the shared-memory panel factorisation", n0);
      return HK_UNSUPPORTED;
    }
    HK_TRY(hk_allow_smem(k_gj_panel));
    if (G > 8) HK_CUDA(cudaFuncSetAttribute(k_gj_panel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    int *d_used = nullptr, *d_q = nullptr;
    double* d_Q = nullptr;
    double* d_work = h->d_Einv64;  // A, then unpermuted into a copy
    double* d_tmp = nullptr;
    HK_TRY(dalloc(h, &d_used, n0));
    HK_TRY(dalloc(h, &d_q, n0));
    HK_TRY(dalloc(h, &d_Q, (size_t)HK_GJ_NB * n0));
    HK_TRY(dalloc(h, &d_tmp, (size_t)n0 * n0));
    double* minp = d_sc + 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = panel_smem(G);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = G;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    for (int k0 = 0; k0 < n0; k0 += HK_GJ_NB) {
      int k1 = std::min(n0, k0 + HK_GJ_NB), nb = k1 - k0;
      HK_CUDA(cudaLaunchKernelEx(&cfg, k_gj_panel, d_work, n0, k0, k1, d_piv, d_used, minp));
      HK_COUNT_LAUNCH();
      if (nb < n0) {
        k_gj_pivot_rows<<<dim3(nblk(n0, 256), nb), 256, 0, st>>>(d_work, n0, k0, nb, d_piv, d_Q);
        HK_COUNT_LAUNCH();
        k_gj_update<<<dim3(nblk(n0, 64), nblk(n0, 64)), 256, 0, st>>>(d_work, n0, k0, nb, d_piv, d_Q);
        HK_COUNT_LAUNCH();
      }
    }
    HK_LAUNCH_CHECK();
    HK_TRY(check_device_status(h, "coarse inverse"));
    k_invert_perm<<<nblk(n0, 256), 256, 0, st>>>(d_piv, d_q, n0);
    HK_COUNT_LAUNCH();
    k_gj_unpermute<<<n0, 256, 0, st>>>(d_work, d_tmp, n0, d_piv, d_q);
    HK_COUNT_LAUNCH();
    HK_CUDA(cudaMemcpyAsync(h->d_Einv64, d_tmp, sizeof(double) * (size_t)n0 * n0, cudaMemcpyDeviceToDevice, st));
    HK_LAUNCH_CHECK();
    HK_CUDA(cudaStreamSynchronize(st));
    void* fr[] = {d_used, d_q, d_tmp, d_Q};
    for (void* q : fr) dfree(h, q);
  }
  double sc[2];
  HK_CUDA(cudaMemcpyAsync(sc, d_sc, sizeof(sc), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  if (!(sc[1] > 1e-10 * sc[0])) {
    hk_set_error("coarse matrix singular: pivot %.3e, max|E| %.3e", sc[1], sc[0]);
    return HK_SINGULAR_COARSE;
  }
  if (precond_f32(h->p)) {
    HK_TRY(dalloc(h, &h->d_Einv32, (size_t)n0 * n0));
    launch_to_f32(h->d_Einv64, h->d_Einv32, (long long)n0 * n0, st);
    HK_LAUNCH_CHECK();
  }
  HK_TRY(build_apply_z(h));
  HK_CUDA(cudaStreamSynchronize(st));
  dfree(h, d_pair);
  dfree(h, d_plist);
  dfree(h, d_sc);
  dfree(h, d_piv);
  return HK_OK;
}
