// Coarse operator of Eq. 2.23: E = Z^T B Z (the Galerkin matrix of
// B_0 = R_0 B E_0 with R_0 = Z^T) and its inverse, both FP64 on the device.
// Z_i is supported on dof(Omega_i), so the block E_ij is nonzero only when
// some dof of Omega_i is coupled by B to a dof of Omega_j; those pairs are
// found from the pull map and each pair's block is computed by one CTA in a
// fixed summation order.  E^{-1} is formed by Gauss-Jordan elimination with
// partial pivoting (one column per step); a pivot below 1e-10 max|E| reports
// HK_SINGULAR_COARSE.
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

// Step k, part 1 (one CTA): pivot search in column k, row swap, scaling of row k.
__global__ void k_gj_pivot(double* A, int n0, int k, int* piv, double* minpiv) {
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ int p_s;
  __shared__ double inv_s;
  int tid = threadIdx.x;
  double best = -1;
  int bi = k;
  for (int i = k + tid; i < n0; i += blockDim.x) {
    double v = fabs(A[(long long)i * n0 + k]);
    if (v > best) { best = v; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, best, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
  }
  if ((tid & 31) == 0) { rv[tid >> 5] = best; ri[tid >> 5] = bi; }
  __syncthreads();
  if (tid == 0) {
    double bv = rv[0];
    int bj = ri[0];
    for (int w = 1; w < (blockDim.x >> 5); ++w)
      if (rv[w] > bv || (rv[w] == bv && ri[w] < bj)) { bv = rv[w]; bj = ri[w]; }
    p_s = bj;
    piv[k] = bj;
    if (bv < *minpiv) *minpiv = bv;
  }
  __syncthreads();
  int p = p_s;
  if (p != k)
    for (int c = tid; c < n0; c += blockDim.x) {
      double t = A[(long long)k * n0 + c];
      A[(long long)k * n0 + c] = A[(long long)p * n0 + c];
      A[(long long)p * n0 + c] = t;
    }
  __syncthreads();
  if (tid == 0) {
    double pv = A[(long long)k * n0 + k];
    inv_s = pv != 0.0 ? 1.0 / pv : 0.0;
    A[(long long)k * n0 + k] = 1.0;
  }
  __syncthreads();
  double inv = inv_s;
  for (int c = tid; c < n0; c += blockDim.x) A[(long long)k * n0 + c] *= inv;
}

// Step k, part 2: eliminate column k from every other row (one warp per row).
__global__ void k_gj_elim(double* A, int n0, int k) {
  int lane = threadIdx.x & 31;
  int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n0 || i == k) return;
  double* ri = A + (long long)i * n0;
  const double* rk = A + (long long)k * n0;
  double f = 0;
  if (lane == 0) f = ri[k];
  f = __shfl_sync(0xffffffffu, f, 0);
  if (f == 0.0) return;
  for (int c = lane; c < n0; c += 32)
    if (c != k) ri[c] -= f * rk[c];
  __syncwarp();
  if (lane == 0) ri[k] = -f * rk[k];
}

__global__ void k_gj_unscramble(double* A, int n0, const int* __restrict__ piv) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n0) return;
  double* row = A + (long long)r * n0;
  for (int k = n0 - 1; k >= 0; --k) {
    int p = piv[k];
    if (p != k) {
      double t = row[k];
      row[k] = row[p];
      row[p] = t;
    }
  }
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
  HK_CUDA(cudaFuncSetAttribute(k_coarse_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
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
  k_absmax<<<304, 256, 0, st>>>(h->d_E, (long long)n0 * n0, d_sc); HK_COUNT_LAUNCH();
  double big = 1e300;
  HK_CUDA(cudaMemcpyAsync(d_sc + 1, &big, sizeof(double), cudaMemcpyHostToDevice, st));
  for (int k = 0; k < n0; ++k) {
    k_gj_pivot<<<1, 1024, 0, st>>>(h->d_Einv64, n0, k, d_piv, d_sc + 1); HK_COUNT_LAUNCH();
    k_gj_elim<<<nblk((long long)n0 * 32, 256), 256, 0, st>>>(h->d_Einv64, n0, k); HK_COUNT_LAUNCH();
  }
  k_gj_unscramble<<<nblk(n0, 128), 128, 0, st>>>(h->d_Einv64, n0, d_piv); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
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
