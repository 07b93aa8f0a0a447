// Coarse operator of Eq. 2.23: E = Z^T B Z (the Galerkin matrix of
// B_0 = R_0 B E_0 with R_0 = Z^T) and its inverse, both FP64 on the device.
// Z_i is supported on dof(Omega_i), so the block E_ij is nonzero only when
// some dof of Omega_i is coupled by B to a dof of Omega_j; those pairs are
// found from the pull map and each pair's block is computed by one CTA in a
// fixed summation order.  E^{-1} is formed by Gauss-Jordan elimination with
// partial pivoting (one column per step); a pivot below 1e-10 max|E| reports
// HK_SINGULAR_COARSE.
#include <algorithm>

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

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  The wait is bounded: after
// ~2^24 polls the barrier gives up, records HK_TIMEOUT and returns false.
struct GridBar {
  unsigned count;
  unsigned gen;
};

__device__ bool grid_barrier(GridBar* gb, unsigned nblocks, unsigned& my_gen, DevStatus* st, int* sh_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned g = my_gen;
    __threadfence();
    unsigned arrived = atomicAdd(&gb->count, 1u) + 1u;
    if (arrived == nblocks) {
      gb->count = 0u;
      __threadfence();
      atomicExch(&gb->gen, g + 1u);
    } else {
      unsigned spins = 0;
      while (atomicAdd(&gb->gen, 0u) == g) {
        if (++spins > (1u << 24)) {
          ok = 0;
          dev_fail(st, HK_TIMEOUT, blockIdx.x, 0);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    *sh_ok = ok;
  }
  my_gen += 1u;
  __syncthreads();
  return *sh_ok != 0;
}

// In-place Gauss-Jordan inverse of the n0 x n0 matrix A with partial pivoting and implicit row
// interchanges: step k picks the unused row p_k with the largest |A[p][k]|, scales it, and eliminates
// column k from every other row; column k then holds column p_k of the accumulated transform.  The
// inverse is Inv[k][j] = A[p_k][q_j] with q the inverse of p (applied by k_gj_unpermute).  Rows are
// owned by CTAs (row i by CTA i mod gridDim); the pivot search of step k+1 is fused into the
// elimination of step k (per-CTA maxima, reduced redundantly by every CTA after the barrier), so each
// step costs one grid barrier.  Ties go to the smallest row index.
__global__ void k_gj_persistent(double* A, int n0, int* piv, int* used, double* pmax_v, int* pmax_i,
                                GridBar* gb, double* minpiv, DevStatus* st) {
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ int sh_ok, sh_p;
  __shared__ double sh_f;
  extern __shared__ double prow[];  // the scaled pivot row
  int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  unsigned G = gridDim.x, my_gen = 0;
  // initial pivot search for column 0 (every CTA over its rows)
  auto local_max = [&](int col, int buf) {
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = blockIdx.x + G * tid; i < n0; i += G * T) {
      if (used[i]) continue;
      double v = fabs(A[(long long)i * n0 + col]);
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
      pmax_v[buf * G + blockIdx.x] = bv;
      pmax_i[buf * G + blockIdx.x] = bj;
    }
    __syncthreads();
  };
  local_max(0, 0);
  if (!grid_barrier(gb, G, my_gen, st, &sh_ok)) return;
  int pprev = -1;  // pivot row of the previous step, written back by its owner after the barrier
  for (int k = 0; k < n0; ++k) {
    if (pprev >= 0 && blockIdx.x == (unsigned)(pprev % (int)G)) {
      for (int j = tid; j < n0; j += T) A[(long long)pprev * n0 + j] = prow[j];
      __syncthreads();
    }
    int buf = k & 1;
    // every CTA reduces the per-CTA maxima the same way (warp 0, lanes over CTAs)
    if (warp == 0) {
      double bv = -1.0;
      int bj = 0x7fffffff;
      for (unsigned b = lane; b < G; b += 32) {
        double v = pmax_v[buf * G + b];
        int i = pmax_i[buf * G + b];
        if (v > bv || (v == bv && i < bj)) { bv = v; bj = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ov > bv || (ov == bv && oi < bj)) { bv = ov; bj = oi; }
      }
      if (lane == 0) {
        sh_p = bj;
        double pv = A[(long long)bj * n0 + k];
        sh_f = pv != 0.0 ? 1.0 / pv : 0.0;
        if (blockIdx.x == 0) {
          piv[k] = bj;
          if (fabs(pv) < *minpiv) *minpiv = fabs(pv);
        }
      }
    }
    __syncthreads();
    int p = sh_p;
    double f = sh_f;
    // scaled pivot row (column k of it becomes f)
    for (int j = tid; j < n0; j += T) prow[j] = j == k ? f : A[(long long)p * n0 + j] * f;
    __syncthreads();
    // eliminate column k from the owned rows other than p (row p is rewritten after the barrier,
    // once no CTA reads its unscaled values any more)
    for (int i = blockIdx.x + G * warp; i < n0; i += G * nw) {
      double* ai = A + (long long)i * n0;
      if (i == p) continue;
      double g = ai[k];
      __syncwarp();
      if (g != 0.0)
        for (int j = lane; j < n0; j += 32) ai[j] = j == k ? -g * f : ai[j] - g * prow[j];
    }
    if (blockIdx.x == (unsigned)(p % G) && tid == 0) used[p] = 1;
    __syncthreads();
    if (k + 1 < n0) local_max(k + 1, (k + 1) & 1);
    if (!grid_barrier(gb, G, my_gen, st, &sh_ok)) return;
    pprev = p;
  }
  if (pprev >= 0 && blockIdx.x == (unsigned)(pprev % (int)G))
    for (int j = tid; j < n0; j += T) A[(long long)pprev * n0 + j] = prow[j];
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
    // one cooperative launch; grid = co-resident CTAs (at most one per SM here)
    int threads = 512, nsm = 0, per_sm = 0, dev = h->dev;
    size_t pshm = sizeof(double) * (size_t)n0;
    HK_TRY(hk_allow_smem(k_gj_persistent));
    HK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    HK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_persistent, threads, pshm));
    if (per_sm < 1) {
      hk_set_error("coarse inverse: no co-resident CTA possible (n0 = %d)", n0);
      return HK_UNSUPPORTED;
    }
    // each step costs one grid barrier plus n0^2 / G FP64 updates per CTA: 64 CTAs balance the two
    int G = std::min(std::min(nsm, 64), std::max(1, n0 / 8));
    int *d_used = nullptr, *d_pi = nullptr, *d_q = nullptr;
    double* d_pv = nullptr;
    GridBar* d_gb = nullptr;
    double* d_work = h->d_Einv64;  // A, then unpermuted into a copy
    double* d_tmp = nullptr;
    HK_TRY(dalloc(h, &d_used, n0));
    HK_TRY(dalloc(h, &d_pi, 2 * G));
    HK_TRY(dalloc(h, &d_pv, 2 * G));
    HK_TRY(dalloc(h, &d_q, n0));
    HK_TRY(dalloc(h, &d_gb, 1));
    HK_TRY(dalloc(h, &d_tmp, (size_t)n0 * n0));
    void* args[] = {&d_work, &n0, &d_piv, &d_used, &d_pv, &d_pi, &d_gb, &d_sc, &h->d_status};
    double* minp = d_sc + 1;
    args[7] = &minp;
    HK_CUDA(cudaLaunchCooperativeKernel((void*)k_gj_persistent, dim3(G), dim3(threads), args, pshm, st));
    HK_COUNT_LAUNCH();
    HK_LAUNCH_CHECK();
    HK_TRY(check_device_status(h, "coarse inverse"));
    k_invert_perm<<<nblk(n0, 256), 256, 0, st>>>(d_piv, d_q, n0);
    HK_COUNT_LAUNCH();
    k_gj_unpermute<<<n0, 256, 0, st>>>(d_work, d_tmp, n0, d_piv, d_q);
    HK_COUNT_LAUNCH();
    HK_CUDA(cudaMemcpyAsync(h->d_Einv64, d_tmp, sizeof(double) * (size_t)n0 * n0, cudaMemcpyDeviceToDevice, st));
    HK_LAUNCH_CHECK();
    HK_CUDA(cudaStreamSynchronize(st));
    void* fr[] = {d_used, d_pi, d_pv, d_q, d_gb, d_tmp};
    for (void* q : fr) dfree(h, q);
  }
  double sc[2];
  HK_CUDA(cudaMemcpyAsync(sc, d_sc, sizeof(sc), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  if (!(sc[1] > 1e-10 * sc[0])) {
    hk_set_error("coarse matrix singular: pivot %.3e, max|E| %.3e", sc[1], sc[0]);
    return HK_SINGULAR_COARSE;
  }
  if (h->p.precision == HK_FP32_PRECOND) {
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
