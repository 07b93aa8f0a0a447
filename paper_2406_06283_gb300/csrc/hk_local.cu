// Local Dirichlet factors of B_i = R_i B R_i^T (Eq. 2.22) and their use in
// the preconditioner apply (Eq. 2.22-2.23).
//
// In level order B_i is block tridiagonal: diagonal blocks D_j, couplings
// L_j = B[level j, level j-1] and U_j = B[level j, level j+1] = L_{j+1}^T.
// Its block LU uses the Schur complements
//     S_0 = D_0,   S_j = D_j - L_j S_{j-1}^{-1} U_{j-1},
// and a solve B_i x = r is the pair of sweeps
//     forward   y_j = S_j^{-1} (r_j - L_j y_{j-1})
//     backward  x_j = y_j - G_j x_{j+1},   G_j = S_j^{-1} U_j.
// Setup stores S_j^{-1} (b_j x b_j) and G_j (b_j x b_{j+1}) densely, row-major,
// each block starting on a 4-element boundary; the sparse L_j is read from
// the local CSR.  S_j^{-1} is formed in FP64 by Gauss-Jordan elimination with
// partial pivoting; a pivot below 1e-10 max|B_i| reports HK_SINGULAR_LOCAL.
#include "hk_internal.cuh"

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }
__host__ __device__ __forceinline__ long long pad4(long long x) { return (x + 3) & ~3LL; }

// Element count of the factor blocks of one subdomain.
long long factor_elems(const int* lp, int L) {
  long long t = 0;
  for (int j = 0; j < L; ++j) {
    long long b = lp[j + 1] - lp[j];
    long long bn = j + 1 < L ? lp[j + 2] - lp[j + 1] : 0;
    t += pad4(b * b) + pad4(b * bn);
  }
  return t;
}

// In-place Gauss-Jordan inverse of the b x b row-major matrix A (shared
// memory) with partial pivoting; returns through *minpiv the smallest |pivot|.
__device__ void gauss_jordan_inverse(double* A, int b, int* piv, double* red_v, int* red_i, double* minpiv) {
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
    double pv = A[k * b + k];
    double inv = pv != 0.0 ? 1.0 / pv : 0.0;
    __syncthreads();
    if (tid == 0) A[k * b + k] = 1.0;
    __syncthreads();
    for (int c = tid; c < b; c += T) A[k * b + c] *= inv;
    __syncthreads();
    // eliminate column k from every other row
    for (int e = tid; e < b * b; e += T) {
      int i = e / b, c = e % b;
      if (i == k || c == k) continue;
      A[i * b + c] -= A[i * b + k] * A[k * b + c];
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

__global__ void k_block_lu(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                           const int* __restrict__ levptr, const int* __restrict__ lrow,
                           const int* __restrict__ lcntI, const int* __restrict__ lcol,
                           const double* __restrict__ lval, double* F, DevStatus* st) {
  extern __shared__ double smem[];
  __shared__ int piv[HK_MAXB];
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ double minpiv;
  int s = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], L = si[2], off = si[3], loff = si[5];
  long long foff = sub_off[3 * s], coff = sub_off[3 * s + 1];
  const int* lp = levptr + loff;
  const int* lr = lrow + off + s;
  double* S = smem;
  // scale for the singularity test: max |B_i| entry
  double mx = 0;
  for (int a = tid; a < nI; a += T)
    for (int q = 0; q < lcntI[off + a]; ++q) mx = fmax(mx, fabs(lval[coff + lr[a] + q]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) red_v[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    double m2 = 0;
    for (int w = 0; w < (T >> 5); ++w) m2 = fmax(m2, red_v[w]);
    red_v[0] = m2;
    minpiv = 1e300;
  }
  __syncthreads();
  double scale = red_v[0];
  __syncthreads();
  long long bo = foff, prev_go = -1;
  int prev_r0 = 0;
  for (int j = 0; j < L; ++j) {
    int r0 = lp[j], b = lp[j + 1] - r0;
    int r1 = lp[j + 1];
    int bn = j + 1 < L ? lp[j + 2] - r1 : 0;
    // S = D_j - L_j G_{j-1}
    for (int e = tid; e < b * b; e += T) {
      int qa = e / b, t = e % b;
      int a = r0 + qa;
      const int* cl = lcol + coff + lr[a];
      const double* cv = lval + coff + lr[a];
      int cnt = lcntI[off + a];
      double v = 0;
      for (int q = 0; q < cnt; ++q) {
        int c = cl[q];
        if (c == r0 + t) v += cv[q];
        else if (j > 0 && c >= prev_r0 && c < r0) v -= cv[q] * F[prev_go + (long long)(c - prev_r0) * b + t];
      }
      S[e] = v;
    }
    __syncthreads();
    gauss_jordan_inverse(S, b, piv, red_v, red_i, &minpiv);
    for (int e = tid; e < b * b; e += T) F[bo + e] = S[e];
    long long go = bo + pad4((long long)b * b);
    // G_j = S_j^{-1} U_j, with U_j[a, c] = B[c, a] read from the rows of level j+1
    for (int e = tid; e < b * bn; e += T) {
      int qt = e / bn, cc = e % bn;
      int c = r1 + cc;
      const int* cl = lcol + coff + lr[c];
      const double* cv = lval + coff + lr[c];
      int cnt = lcntI[off + c];
      double v = 0;
      for (int q = 0; q < cnt; ++q) {
        int a = cl[q];
        if (a >= r0 && a < r1) v += S[qt * b + (a - r0)] * cv[q];
      }
      F[go + e] = v;
    }
    __syncthreads();
    prev_go = go;
    prev_r0 = r0;
    bo = go + pad4((long long)b * bn);
  }
  if (tid == 0 && !(minpiv > 1e-10 * scale)) dev_fail(st, HK_SINGULAR_LOCAL, s, minpiv / scale);
}

// Number of couplings L_j (row in level j, column in level j-1) of every subdomain.
__global__ void k_count_lower(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                              const int* __restrict__ levptr, const int* __restrict__ lrow,
                              const int* __restrict__ lcntI, const int* __restrict__ lcol,
                              unsigned long long* out) {
  int s = blockIdx.x;
  const int* si = sub_info + 8 * s;
  int L = si[2], off = si[3], loff = si[5];
  long long coff = sub_off[3 * s + 1];
  const int* lp = levptr + loff;
  const int* lr = lrow + off + s;
  unsigned long long c = 0;
  for (int j = 1; j < L; ++j)
    for (int a = lp[j] + threadIdx.x; a < lp[j + 1]; a += blockDim.x)
      for (int q = 0; q < lcntI[off + a]; ++q) c += lcol[coff + lr[a] + q] < lp[j];
  atomicAdd(out, c);
}

__global__ void k_to_f32(const double* __restrict__ a, float* b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

void launch_to_f32(const double* a, float* b, long long n, cudaStream_t st) {
  if (n > 0) k_to_f32<<<nblk(n, 256), 256, 0, st>>>(a, b, n);
}

hk_status phase_local_factors(hk_handle* h) {
  cudaStream_t st = h->stream;
  int ns = h->n_sub;
  std::vector<int> lev(h->I_total + ns);
  HK_CUDA(cudaMemcpyAsync(lev.data(), h->d_lev, sizeof(int) * lev.size(), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  long long fo = 0;
  for (int s = 0; s < ns; ++s) {
    Sub& u = h->subs[s];
    u.f_off = fo;
    fo += factor_elems(&lev[u.lev_off], u.L);
  }
  h->f_total = fo;
  HK_TRY(upload_sub_info(h));
  if (h->p.levels == HK_COARSE_ONLY) return HK_OK;
  {
    unsigned long long* d_cnt = nullptr;
    HK_TRY(dalloc(h, &d_cnt, 1));
    k_count_lower<<<ns, 128, 0, st>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI, h->d_lcol,
                                      d_cnt);
    unsigned long long c = 0;
    HK_CUDA(cudaMemcpyAsync(&c, d_cnt, sizeof(c), cudaMemcpyDeviceToHost, st));
    HK_CUDA(cudaStreamSynchronize(st));
    h->lower_nnz = (long long)c;
    dfree(h, d_cnt);
  }
  HK_TRY(dalloc(h, &h->d_F64, fo));
  size_t shm = sizeof(double) * (size_t)h->max_level * h->max_level;
  HK_CUDA(cudaFuncSetAttribute(k_block_lu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  k_block_lu<<<ns, 256, shm, st>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI, h->d_lcol,
                                   h->d_lvalB, h->d_F64, h->d_status);
  HK_LAUNCH_CHECK();
  HK_TRY(check_device_status(h, "local factors"));
  if (h->p.precision == HK_FP32_PRECOND) {
    HK_TRY(dalloc(h, &h->d_F32, fo));
    launch_to_f32(h->d_F64, h->d_F32, fo, st);
    HK_TRY(dalloc(h, &h->d_lvalB32, h->csr_total));
    launch_to_f32(h->d_lvalB, h->d_lvalB32, h->csr_total, st);
    HK_LAUNCH_CHECK();
    HK_CUDA(cudaStreamSynchronize(st));
    dfree(h, h->d_F64);
    h->d_F64 = nullptr;
  }
  return HK_OK;
}

// ====================================================================== apply
// One CTA per (subdomain, group of NR right-hand sides):
//   gather r_i = v[dof(Omega_i)] (R_i of Eq. 2.22), coarse restriction
//   c_i = Z_i^T r_i (R_0 = Z^T, Eq. 2.23), then the two block sweeps, and
//   the local solution y_i written to ybuf.  T is the arithmetic type
//   (float in the FP32 form, double in the FP64 form).
template <typename T, int NR>
__global__ void k_local_apply(int n, int s_tot, const double* __restrict__ v, const int* __restrict__ active,
                              const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                              const int* __restrict__ levptr, const int* __restrict__ Ilev,
                              const int* __restrict__ lrow, const int* __restrict__ lcntI,
                              const int* __restrict__ lcol, const T* __restrict__ lval, const T* __restrict__ F,
                              const T* __restrict__ Z, int do_local, int do_coarse, long long I_total, int n0,
                              T* ybuf, T* cvec) {
  extern __shared__ unsigned char smem_raw[];
  T* x = reinterpret_cast<T*>(smem_raw);  // nI x NR
  int s = blockIdx.x, r_base = blockIdx.y * NR;
  int tid = threadIdx.x, T_ = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T_ >> 5;
  const int* si = sub_info + 8 * s;
  int nI = si[0], L = si[2], off = si[3], loff = si[5], m = si[6], c_off = si[7];
  long long foff = sub_off[3 * s], coff = sub_off[3 * s + 1], zoff = sub_off[3 * s + 2];
  T* tmp = x + (size_t)nI * NR;           // HK_MAXB x NR
  int nr = s_tot - r_base < NR ? s_tot - r_base : NR;
  bool act[NR];
  for (int r = 0; r < NR; ++r) act[r] = r < nr && (active == nullptr || active[8 * (r_base + r)]);
  // gather
  for (int e = tid; e < nI * NR; e += T_) {
    int a = e / NR, r = e % NR;
    x[e] = act[r] ? (T)v[(long long)(r_base + r) * n + Ilev[off + a]] : (T)0;
  }
  __syncthreads();
  // coarse restriction c_i = Z_i^T r_i
  if (do_coarse) {
    for (int e = tid; e < m * NR; e += T_) {
      int l = e / NR, r = e % NR;
      if (!act[r]) continue;
      T acc = 0;
      const T* zc = Z + zoff + l;
      for (int a = 0; a < nI; ++a) acc += zc[(long long)a * m] * x[a * NR + r];
      cvec[(long long)(r_base + r) * n0 + c_off + l] = acc;
    }
  }
  if (!do_local) return;
  const int* lp = levptr + loff;
  const int* lr = lrow + off + s;
  long long bo = foff;
  // forward sweep
  for (int j = 0; j < L; ++j) {
    int r0 = lp[j], b = lp[j + 1] - r0, bn = j + 1 < L ? lp[j + 2] - lp[j + 1] : 0;
    if (j > 0) {
      for (int e = tid; e < b * NR; e += T_) {
        int a = r0 + e / NR, r = e % NR;
        const int* cl = lcol + coff + lr[a];
        const T* cv = lval + coff + lr[a];
        int cnt = lcntI[off + a];
        T acc = x[a * NR + r];
        for (int q = 0; q < cnt; ++q)
          if (cl[q] < r0) acc -= cv[q] * x[cl[q] * NR + r];
        x[a * NR + r] = acc;
      }
      __syncthreads();
    }
    const T* Sinv = F + bo;
    for (int q = warp; q < b; q += nw) {
      T acc[NR];
      for (int r = 0; r < NR; ++r) acc[r] = 0;
      for (int t = lane; t < b; t += 32) {
        T sv = Sinv[q * b + t];
        for (int r = 0; r < NR; ++r) acc[r] += sv * x[(r0 + t) * NR + r];
      }
      for (int r = 0; r < NR; ++r) {
        T a = acc[r];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) tmp[q * NR + r] = a;
      }
    }
    __syncthreads();
    for (int e = tid; e < b * NR; e += T_) x[r0 * NR + e] = tmp[e];
    __syncthreads();
    bo += pad4((long long)b * b) + pad4((long long)b * bn);
  }
  // backward sweep: x_j -= G_j x_{j+1}; bo walks back over the blocks
  {
    int bl = lp[L] - lp[L - 1];
    bo -= pad4((long long)bl * bl);  // level L-1 has no G block
  }
  for (int j = L - 2; j >= 0; --j) {
    int r0 = lp[j], b = lp[j + 1] - r0, r1 = lp[j + 1], bn = lp[j + 2] - r1;
    bo -= pad4((long long)b * b) + pad4((long long)b * bn);
    const T* Gj = F + bo + pad4((long long)b * b);
    for (int q = warp; q < b; q += nw) {
      T acc[NR];
      for (int r = 0; r < NR; ++r) acc[r] = 0;
      for (int t = lane; t < bn; t += 32) {
        T gv = Gj[q * bn + t];
        for (int r = 0; r < NR; ++r) acc[r] += gv * x[(r1 + t) * NR + r];
      }
      for (int r = 0; r < NR; ++r) {
        T a = acc[r];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) x[(r0 + q) * NR + r] -= a;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < nI * NR; e += T_) {
    int a = e / NR, r = e % NR;
    if (act[r]) ybuf[(long long)(r_base + r) * I_total + off + a] = x[e];
  }
}

// cc = E^{-1} c for s vectors (E^{-1} dense n0 x n0 row-major): one warp per row.
template <typename T>
__global__ void k_coarse_solve(int n0, int s, const T* __restrict__ Einv, const T* __restrict__ c, T* cc,
                               const int* __restrict__ active) {
  int lane = threadIdx.x & 31;
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n0) return;
  const T* er = Einv + (long long)row * n0;
  for (int r = 0; r < s; ++r) {
    if (active && !active[8 * r]) continue;
    const T* cr = c + (long long)r * n0;
    T acc = 0;
    for (int t = lane; t < n0; t += 32) acc += er[t] * cr[t];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) cc[(long long)r * n0 + row] = acc;
  }
}

// z_l = sum over (i, a) holding l of  w * y_i[a] + (Z_i cc_i)[a]   (pull form of
// the sums in Eq. 2.22-2.23; w = 1, or 1/mu_l for the RAS variant).
template <typename T>
__global__ void k_scatter(int n, int s, const int* __restrict__ pull_ptr, const int* __restrict__ pull_row,
                          const int* __restrict__ pull_sub, const int* __restrict__ sub_info,
                          const long long* __restrict__ sub_off, const T* __restrict__ ybuf,
                          const T* __restrict__ Z, const T* __restrict__ cc, long long I_total, int n0,
                          int do_local, int do_coarse, int ras, const int* __restrict__ mu, double* z,
                          const int* __restrict__ active) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  int p0 = pull_ptr[l], p1 = pull_ptr[l + 1];
  T wl = ras ? (T)1 / (T)mu[l] : (T)1;
  for (int r = 0; r < s; ++r) {
    if (active && !active[8 * r]) continue;
    T acc = 0;
    for (int p = p0; p < p1; ++p) {
      int row = pull_row[p];
      if (do_local) acc += wl * ybuf[(long long)r * I_total + row];
      if (do_coarse) {
        int sb = pull_sub[p];
        const int* si = sub_info + 8 * sb;
        int m = si[6], c_off = si[7], a = row - si[3];
        const T* zr = Z + sub_off[3 * sb + 2] + (long long)a * m;
        const T* cr = cc + (long long)r * n0 + c_off;
        for (int q = 0; q < m; ++q) acc += zr[q] * cr[q];
      }
    }
    z[(long long)r * n + l] = (double)acc;
  }
}

template <typename T, int NR>
static hk_status launch_local(hk_handle* h, int s, const double* v, const int* active, const T* lval, const T* F,
                              const T* Z, T* ybuf, T* cvec, int do_local, int do_coarse) {
  size_t shm = sizeof(T) * ((size_t)h->max_dof * NR + (size_t)HK_MAXB * NR);
  static bool attr_set = false;
  if (!attr_set) {
    HK_CUDA(cudaFuncSetAttribute(k_local_apply<T, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  if (shm > 200 * 1024) {
    hk_set_error("subdomain too large for the shared-memory apply (%d dofs)", h->max_dof);
    return HK_UNSUPPORTED;
  }
  dim3 grid(h->n_sub, (s + NR - 1) / NR);
  HK_TIMED(h, HK_T_LOCAL_APPLY,
           (k_local_apply<T, NR><<<grid, 256, shm, h->stream>>>(h->n, s, v, active, h->d_sub_info, h->d_sub_off,
                                                               h->d_lev, h->d_I, h->d_lrow, h->d_lcntI, h->d_lcol,
                                                               lval, F, Z, do_local, do_coarse, h->I_total, h->n0,
                                                               ybuf, cvec)));
  HK_LAUNCH_CHECK();
  return HK_OK;
}

template <typename T>
static hk_status apply_t(hk_handle* h, int s, const double* v, double* z, const int* active, const T* lval,
                         const T* F, const T* Z, const T* Einv, T* ybuf, T* c, T* cc) {
  int do_local = h->p.levels != HK_COARSE_ONLY;
  int do_coarse = h->p.levels != HK_ONE_LEVEL && h->n0 > 0;
  int NRmax = sizeof(T) == 4 ? 8 : 4;
  if (h->max_dof > 6000) NRmax = 1;
  else if (h->max_dof > 3000) NRmax = NRmax > 2 ? 2 : NRmax;
  int nr = s >= 8 && NRmax >= 8 ? 8 : s >= 4 && NRmax >= 4 ? 4 : s >= 2 && NRmax >= 2 ? 2 : 1;
  hk_status rc;
  switch (nr) {
    case 8: rc = launch_local<T, 8>(h, s, v, active, lval, F, Z, ybuf, c, do_local, do_coarse); break;
    case 4: rc = launch_local<T, 4>(h, s, v, active, lval, F, Z, ybuf, c, do_local, do_coarse); break;
    case 2: rc = launch_local<T, 2>(h, s, v, active, lval, F, Z, ybuf, c, do_local, do_coarse); break;
    default: rc = launch_local<T, 1>(h, s, v, active, lval, F, Z, ybuf, c, do_local, do_coarse); break;
  }
  HK_TRY(rc);
  if (do_coarse) {
    int rows_per_block = 8;
    HK_TIMED(h, HK_T_COARSE_SOLVE,
             (k_coarse_solve<T><<<nblk(h->n0, rows_per_block), 32 * rows_per_block, 0, h->stream>>>(
                 h->n0, s, Einv, c, cc, active)));
  }
  HK_TIMED(h, HK_T_SCATTER,
           (k_scatter<T><<<nblk(h->n, 128), 128, 0, h->stream>>>(
               h->n, s, h->d_pull_ptr, h->d_pull_row, h->d_pull_sub, h->d_sub_info, h->d_sub_off, ybuf, Z, cc,
               h->I_total, h->n0, do_local, do_coarse, h->p.weighting == HK_RAS_POU, h->d_mu, z, active)));
  HK_LAUNCH_CHECK();
  return HK_OK;
}

hk_status op_apply(hk_handle* h, int s, const double* v, double* z, const int* active) {
  HK_TRY(ensure_workspace(h, s));
  if (h->p.precision == HK_FP32_PRECOND)
    return apply_t<float>(h, s, v, z, active, h->d_lvalB32, h->d_F32, h->d_Z32, h->d_Einv32, h->d_ybuf32, h->d_c32,
                          h->d_cc32);
  return apply_t<double>(h, s, v, z, active, h->d_lvalB, h->d_F64, h->d_Z64, h->d_Einv64, h->d_ybuf64, h->d_c64,
                         h->d_cc64);
}

// ======================================================= allocation-free apply
// Some callers cannot allocate device memory when they apply the
// preconditioner: code running while a stream is being captured into a CUDA
// graph (cudaMalloc is not allowed there), or a host framework that owns all
// device memory through its own allocator and forbids allocations on its hot
// path.  hk_apply_precond_noalloc serves them: it runs the same three kernels
// as hk_apply_precond on caller-provided device vectors, and keeps its
// intermediate vectors (local solutions, coarse right-hand side and coarse
// solution) in the fixed device array below instead of allocating.
//
// The array is HK_NOALLOC_SCRATCH_BYTES per device and stays allocated on
// every device that loads the library until the process exits.  Its device
// address is looked up once per device (host code may not use the symbol
// itself as a pointer: it is only a host-side stand-in), on the first call
// made on that device; that first call should happen before any stream
// capture.  Every call uses the same array, so calls whose kernels overlap on
// the GPU race with each other.  The array keeps the contents of the last
// call; each call writes every scratch element it reads before reading it, so
// nothing has to be cleared.
#include <mutex>

#define HK_NOALLOC_SCRATCH_BYTES (8u << 20)
#define HK_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[HK_NOALLOC_SCRATCH_BYTES];
static void* g_noalloc_ptr[HK_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

static hk_status noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= HK_NOALLOC_MAX_DEVICES) {
    hk_set_error("device %d outside the %d devices the allocation-free apply supports", dev,
                 HK_NOALLOC_MAX_DEVICES);
    return HK_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // the device `dev` is current here
    if (e != cudaSuccess || !p) {
      hk_set_error("cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
      return HK_CUDA_ERROR;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return HK_OK;
}

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" hk_status hk_apply_precond_noalloc(hk_handle* h, int n_rhs, const double* v_dev, double* z_dev) {
  if (!h || n_rhs < 1 || !v_dev || !z_dev) {
    hk_set_error("hk_apply_precond_noalloc: invalid arguments");
    return HK_BAD_ARG;
  }
  size_t esz = h->p.precision == HK_FP32_PRECOND ? sizeof(float) : sizeof(double);
  size_t ylen = align256(esz * (size_t)n_rhs * (size_t)h->I_total);
  size_t clen = align256(esz * (size_t)n_rhs * (size_t)(h->n0 + 1));
  size_t need = ylen + 2 * clen;
  if (need > HK_NOALLOC_SCRATCH_BYTES) {
    hk_set_error("hk_apply_precond_noalloc needs %zu scratch bytes for %d right-hand sides; the fixed array "
                 "holds %u (use fewer right-hand sides per call)", need, n_rhs, HK_NOALLOC_SCRATCH_BYTES);
    return HK_UNSUPPORTED;
  }
  int cur = -1;
  HK_CUDA(cudaGetDevice(&cur));
  if (cur != h->dev) HK_CUDA(cudaSetDevice(h->dev));
  void* base = nullptr;
  hk_status s = noalloc_scratch(h->dev, &base);
  if (s == HK_OK) {
    unsigned char* b = static_cast<unsigned char*>(base);
    if (h->p.precision == HK_FP32_PRECOND)
      s = apply_t<float>(h, n_rhs, v_dev, z_dev, nullptr, h->d_lvalB32, h->d_F32, h->d_Z32, h->d_Einv32,
                         reinterpret_cast<float*>(b), reinterpret_cast<float*>(b + ylen),
                         reinterpret_cast<float*>(b + ylen + clen));
    else
      s = apply_t<double>(h, n_rhs, v_dev, z_dev, nullptr, h->d_lvalB, h->d_F64, h->d_Z64, h->d_Einv64,
                          reinterpret_cast<double*>(b), reinterpret_cast<double*>(b + ylen),
                          reinterpret_cast<double*>(b + ylen + clen));
  }
  if (cur != h->dev) cudaSetDevice(cur);
  return s;
}
