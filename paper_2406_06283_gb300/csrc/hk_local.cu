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
#include <algorithm>

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

__global__ void k_block_lu(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                           const int* __restrict__ levptr, const int* __restrict__ lrow,
                           const int* __restrict__ lcntI, const int* __restrict__ lcol,
                           const double* __restrict__ lval, double* F, int s_in_smem, DevStatus* st) {
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
    // S = D_j - L_j G_{j-1}, in shared memory, or in place in the factor array for wide levels
    double* S = s_in_smem ? smem : F + bo;
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
    if (s_in_smem)
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
  if (n > 0) {
    k_to_f32<<<nblk(n, 256), 256, 0, st>>>(a, b, n);
    HK_COUNT_LAUNCH();
  }
}


// ====================================================================== apply
// Level records, streamed by the apply kernel one after another:
//   forward record j:  S_j^{-1} (b_j x b_j, T) | L_j values (nc_j, T) |
//                      L_j columns in level j-1 (nc_j, uint16) | L_j row pointers (b_j + 1, uint16)
//   backward record j: G_j (b_j x b_{j+1}, T)
// each padded to 16 bytes so that one 1-D TMA bulk copy moves it to shared memory.
// Level table entry (4 x int64 per level): fwd offset, bwd offset, fwd | bwd bytes << 32,
// nc | b << 20 | level start << 40.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false after ~2^22 polls (each poll may suspend the thread for a while).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (unsigned it = 0; it < (1u << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__host__ __device__ __forceinline__ long long pad16(long long x) { return (x + 15) & ~15LL; }
__host__ __device__ __forceinline__ int lv_nc(long long e3) { return (int)(e3 & 0xFFFFF); }
__host__ __device__ __forceinline__ int lv_b(long long e3) { return (int)((e3 >> 20) & 0xFFFFF); }
__host__ __device__ __forceinline__ int lv_start(long long e3) { return (int)(e3 >> 40); }

// Lower couplings per level (row in level j, column in level j-1).
__global__ void k_level_counts(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                               const int* __restrict__ levptr, const int* __restrict__ lrow,
                               const int* __restrict__ lcntI, const int* __restrict__ lcol, int* nc_out) {
  int s = blockIdx.x;
  const int* si = sub_info + 8 * s;
  int L = si[2], off = si[3], loff = si[5];
  long long coff = sub_off[3 * s + 1];
  const int* lp = levptr + loff;
  const int* lr = lrow + off + s;
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    int c = 0;
    if (j > 0)
      for (int a = lp[j]; a < lp[j + 1]; ++a)
        for (int q = 0; q < lcntI[off + a]; ++q) c += lcol[coff + lr[a] + q] < lp[j];
    nc_out[loff + j] = c;
  }
}

template <typename T>
__global__ void k_pack_levels(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                              const int* __restrict__ levptr, const int* __restrict__ lrow,
                              const int* __restrict__ lcntI, const int* __restrict__ lcol,
                              const double* __restrict__ lvalB, const double* __restrict__ F,
                              const long long* __restrict__ lvtab, unsigned char* pack) {
  int s = blockIdx.x, tid = threadIdx.x, T_ = blockDim.x;
  const int* si = sub_info + 8 * s;
  int L = si[2], off = si[3], loff = si[5];
  long long foff = sub_off[3 * s], coff = sub_off[3 * s + 1];
  const int* lp = levptr + loff;
  const int* lr = lrow + off + s;
  long long bo = foff;
  for (int j = 0; j < L; ++j) {
    int r0 = lp[j], b = lp[j + 1] - r0, bn = j + 1 < L ? lp[j + 2] - lp[j + 1] : 0;
    const long long* e = lvtab + 4 * (long long)(loff + j);
    int nc = lv_nc(e[3]);
    T* S = reinterpret_cast<T*>(pack + e[0]);
    T* Lv = S + (long long)b * b;
    uint16_t* Lc = reinterpret_cast<uint16_t*>(Lv + nc);
    uint16_t* Lp = Lc + nc;
    for (int q = tid; q < b * b; q += T_) S[q] = (T)F[bo + q];
    if (tid == 0 && j > 0) {
      int pr0 = lp[j - 1], c = 0;
      for (int a = r0; a < r0 + b; ++a) {
        Lp[a - r0] = (uint16_t)c;
        for (int q = 0; q < lcntI[off + a]; ++q) {
          int col = lcol[coff + lr[a] + q];
          if (col < r0) {
            Lv[c] = (T)lvalB[coff + lr[a] + q];
            Lc[c] = (uint16_t)(col - pr0);
            ++c;
          }
        }
      }
      Lp[b] = (uint16_t)c;
    }
    if (tid == 0 && j == 0) Lp[0] = 0, Lp[b] = 0;
    long long go = bo + pad4((long long)b * b);
    if (bn > 0) {
      T* G = reinterpret_cast<T*>(pack + e[1]);
      for (int q = tid; q < b * bn; q += T_) G[q] = (T)F[go + q];
    }
    bo = go + pad4((long long)b * bn);
  }
}

// One CTA per (subdomain, group of NR right-hand sides): gather r_i = v[dof(Omega_i)]
// (R_i of Eq. 2.22), coarse restriction c_i = Z_i^T r_i (R_0 = Z^T, Eq. 2.23), the
// forward and backward block sweeps of B_i^{-1}, and the local solution written to
// ybuf.  The level records stream through two shared-memory buffers by TMA bulk
// copies, the copy of record r+2 overlapping the work on record r.  Shared vectors
// are right-hand-side major (x[rr * nI + a]).  T: float (FP32 form) or double.
template <typename T, int NR>
__global__ void __launch_bounds__(256) k_local_apply(
    int n, int s_tot, const double* __restrict__ v, const int* __restrict__ active,
    const int* __restrict__ sub_info, const long long* __restrict__ sub_off, const int* __restrict__ Ilev,
    const long long* __restrict__ lvtab, const unsigned char* __restrict__ pack, const T* __restrict__ Zt,
    int do_local, int do_coarse, long long I_total, int n0, int stage_bytes, T* ybuf, T* cvec, DevStatus* st,
    const int* __restrict__ jp, long long jstride) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (jp) v += (long long)(*jp) * jstride;  // captured inner step: v = v_j with j read on the device
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int sh_fail;
  unsigned char* stage[2] = {smem_raw, smem_raw + stage_bytes};
  int s = blockIdx.x, r_base = blockIdx.y * NR;
  int tid = threadIdx.x, T_ = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T_ >> 5;
  const int* si = sub_info + 8 * s;
  int nI = si[0], L = si[2], off = si[3], loff = si[5], m = si[6], c_off = si[7];
  long long zoff = sub_off[3 * s + 2];
  T* x = reinterpret_cast<T*>(smem_raw + 2 * (long long)stage_bytes);  // NR x nI
  T* tmp = x + (long long)nI * NR;                                       // NR x HK_MAXB
  int nr = s_tot - r_base < NR ? s_tot - r_base : NR;
  bool act[NR];
  for (int r = 0; r < NR; ++r) act[r] = r < nr && (active == nullptr || active[8 * (r_base + r)]);
  const long long* lv = lvtab + 4 * (long long)loff;
  int nrec = do_local ? 2 * L - 1 : 0;
  auto rec_src = [&](int r, unsigned& bytes) -> const unsigned char* {
    const long long* e = lv + 4 * (r < L ? r : 2 * L - 2 - r);
    if (r < L) {
      bytes = (unsigned)(e[2] & 0xffffffffLL);
      return pack + e[0];
    }
    bytes = (unsigned)((unsigned long long)e[2] >> 32);
    return pack + e[1];
  };
  if (tid == 0) {
    sh_fail = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int r = 0; r < 2 && r < nrec; ++r) {
      unsigned bytes;
      const unsigned char* src = rec_src(r, bytes);
      mbar_expect_tx(&bar[r], bytes);
      tma_load_1d(stage[r], src, bytes, &bar[r]);
    }
  }
  // gather (overlaps the first two record copies)
  for (int e = tid; e < nI * NR; e += T_) {
    int rr = e / nI, a = e % nI;
    x[e] = act[rr] ? (T)v[(long long)(r_base + rr) * n + Ilev[off + a]] : (T)0;
  }
  __syncthreads();
  if (do_coarse) {
    for (int l = warp; l < m; l += nw) {
      const T* zc = Zt + zoff + (long long)l * nI;
      T acc[NR];
      for (int rr = 0; rr < NR; ++rr) acc[rr] = 0;
      for (int a = lane; a < nI; a += 32) {
        T zv = zc[a];
        for (int rr = 0; rr < NR; ++rr) acc[rr] += zv * x[rr * nI + a];
      }
      for (int rr = 0; rr < NR; ++rr) {
        T t = acc[rr];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0 && act[rr]) cvec[(long long)(r_base + rr) * n0 + c_off + l] = t;
      }
    }
  }
  if (!do_local) return;
  unsigned phase[2] = {0u, 0u};
  for (int r = 0; r < nrec; ++r) {
    int bi = r & 1;
    if (!mbar_wait_bounded(&bar[bi], phase[bi])) atomicExch(&sh_fail, 1);
    phase[bi] ^= 1u;
    __syncthreads();
    if (sh_fail) {
      if (tid == 0) dev_fail(st, HK_TIMEOUT, s, r);
      // let the other buffer's copy (if any) land before the CTA exits
      if (r + 1 < nrec) mbar_wait_bounded(&bar[bi ^ 1], phase[bi ^ 1]);
      return;
    }
    const unsigned char* buf = stage[bi];
    int j = r < L ? r : 2 * L - 2 - r;
    long long e3 = lv[4 * j + 3];
    int nc = lv_nc(e3), b = lv_b(e3), ls = lv_start(e3);
    // G threads per output row (a power of two with b * G <= blockDim)
    int G = 1;
    while (G < 32 && b * G * 2 <= T_) G <<= 1;
    int grp = tid / G, gl = tid % G, ngrp = T_ / G;
    if (r < L) {
      const T* S = reinterpret_cast<const T*>(buf);
      const T* Lv = S + (long long)b * b;
      const uint16_t* Lc = reinterpret_cast<const uint16_t*>(Lv + nc);
      const uint16_t* Lp = Lc + nc;
      // t_j = r_j - L_j y_{j-1}  into tmp
      int ps = j > 0 ? lv_start(lv[4 * (j - 1) + 3]) : 0;
      for (int q = tid; q < b * NR; q += T_) {
        int rr = q / b, a = q % b;
        T acc = x[rr * nI + ls + a];
        if (j > 0)
          for (int t = Lp[a]; t < Lp[a + 1]; ++t) acc -= Lv[t] * x[rr * nI + ps + Lc[t]];
        tmp[rr * HK_MAXB + a] = acc;
      }
      __syncthreads();
      // y_j = S_j^{-1} t_j, written in place
      // every thread runs the same trip count so that the group shuffles see full warps
      for (int q0 = 0; q0 < b; q0 += ngrp) {
        int q = q0 + grp;
        bool valid = q < b;
        T acc[NR];
        for (int rr = 0; rr < NR; ++rr) acc[rr] = 0;
        if (valid)
          for (int t = gl; t < b; t += G) {
            T sv = S[q * b + t];
            for (int rr = 0; rr < NR; ++rr) acc[rr] += sv * tmp[rr * HK_MAXB + t];
          }
        for (int rr = 0; rr < NR; ++rr) {
          T a2 = acc[rr];
          for (int o = G >> 1; o > 0; o >>= 1) a2 += __shfl_xor_sync(0xffffffffu, a2, o);
          if (valid && gl == 0) x[rr * nI + ls + q] = a2;
        }
      }
    } else {
      const T* Gm = reinterpret_cast<const T*>(buf);
      int bn = lv_b(lv[4 * (j + 1) + 3]);
      int ns = ls + b;
      for (int q0 = 0; q0 < b; q0 += ngrp) {
        int q = q0 + grp;
        bool valid = q < b;
        T acc[NR];
        for (int rr = 0; rr < NR; ++rr) acc[rr] = 0;
        if (valid)
          for (int t = gl; t < bn; t += G) {
            T gv = Gm[q * bn + t];
            for (int rr = 0; rr < NR; ++rr) acc[rr] += gv * x[rr * nI + ns + t];
          }
        for (int rr = 0; rr < NR; ++rr) {
          T a2 = acc[rr];
          for (int o = G >> 1; o > 0; o >>= 1) a2 += __shfl_xor_sync(0xffffffffu, a2, o);
          if (valid && gl == 0) x[rr * nI + ls + q] -= a2;
        }
      }
    }
    __syncthreads();  // every thread is done with this buffer
    if (tid == 0 && r + 2 < nrec) {
      unsigned bytes;
      const unsigned char* src = rec_src(r + 2, bytes);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bar[bi], bytes);
      tma_load_1d(stage[bi], src, bytes, &bar[bi]);
    }
  }
  for (int e2 = tid; e2 < nI * NR; e2 += T_) {
    int rr = e2 / nI, a = e2 % nI;
    if (act[rr]) ybuf[(long long)(r_base + rr) * I_total + off + a] = x[e2];
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
                          const int* __restrict__ active, const int* __restrict__ jp, long long jstride) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  if (jp) z += (long long)(*jp) * jstride;  // captured inner step: z = z_j
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
static hk_status launch_local(hk_handle* h, int s, const double* v, const int* active, const T* Zt, T* ybuf,
                              T* cvec, int do_local, int do_coarse) {
  size_t xbytes = sizeof(T) * ((size_t)h->max_dof * NR + (size_t)HK_MAXB * NR);
  size_t shm = 2 * (size_t)h->pack_stage + xbytes;
  HK_TRY(hk_allow_smem(k_local_apply<T, NR>));
  if (shm > 220 * 1024) {
    hk_set_error("subdomain too large for the shared-memory apply (%d dofs, record %lld bytes)", h->max_dof,
                 (long long)h->pack_stage);
    return HK_UNSUPPORTED;
  }
  dim3 grid(h->n_sub, (s + NR - 1) / NR);
  HK_TIMED(h, HK_T_LOCAL_APPLY,
           (k_local_apply<T, NR><<<grid, 256, shm, h->stream>>>(
               h->n, s, v, active, h->d_sub_info, h->d_sub_off, h->d_I, h->d_lvtab, h->d_pack, Zt, do_local,
               do_coarse, h->I_total, h->n0, (int)h->pack_stage, ybuf, cvec, h->d_status, h->g_jp,
               h->g_jstride))); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  return HK_OK;
}

template <typename T>
static hk_status apply_t(hk_handle* h, int s, const double* v, double* z, const int* active, T* ybuf, T* c,
                         T* cc) {
  const T* Zr = reinterpret_cast<const T*>(h->d_Zr);
  const T* Zt = reinterpret_cast<const T*>(h->d_Zt);
  const T* Einv = sizeof(T) == 4 ? reinterpret_cast<const T*>(h->d_Einv32) : reinterpret_cast<const T*>(h->d_Einv64);
  int do_local = h->p.levels != HK_COARSE_ONLY;
  int do_coarse = h->p.levels != HK_ONE_LEVEL && h->n0 > 0;
  size_t budget = 220 * 1024 - 2 * (size_t)h->pack_stage;
  int nr = 16;
  while (nr > 1 && (nr > s || sizeof(T) * ((size_t)h->max_dof + HK_MAXB) * nr > budget)) nr >>= 1;
  auto tuned = h->nr_tuned.find(s);
  if (tuned != h->nr_tuned.end() && tuned->second <= nr) nr = tuned->second;
  hk_status rc;
  switch (nr) {
    case 16: rc = launch_local<T, 16>(h, s, v, active, Zt, ybuf, c, do_local, do_coarse); break;
    case 8: rc = launch_local<T, 8>(h, s, v, active, Zt, ybuf, c, do_local, do_coarse); break;
    case 4: rc = launch_local<T, 4>(h, s, v, active, Zt, ybuf, c, do_local, do_coarse); break;
    case 2: rc = launch_local<T, 2>(h, s, v, active, Zt, ybuf, c, do_local, do_coarse); break;
    default: rc = launch_local<T, 1>(h, s, v, active, Zt, ybuf, c, do_local, do_coarse); break;
  }
  HK_TRY(rc);
  if (do_coarse) {
    int rows_per_block = 8;
    HK_TIMED(h, HK_T_COARSE_SOLVE,
             (k_coarse_solve<T><<<nblk(h->n0, rows_per_block), 32 * rows_per_block, 0, h->stream>>>(
                 h->n0, s, Einv, c, cc, active))); HK_COUNT_LAUNCH();
  }
  HK_TIMED(h, HK_T_SCATTER,
           (k_scatter<T><<<nblk(h->n, 128), 128, 0, h->stream>>>(
               h->n, s, h->d_pull_ptr, h->d_pull_row, h->d_pull_sub, h->d_sub_info, h->d_sub_off, ybuf, Zr, cc,
               h->I_total, h->n0, do_local, do_coarse, h->p.weighting == HK_RAS_POU, h->d_mu, z, active, h->g_jp,
               h->g_jstride))); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  return HK_OK;
}

hk_status apply_prepare(hk_handle*) {
  HK_TRY(hk_allow_smem(k_local_apply<float, 1>));
  HK_TRY(hk_allow_smem(k_local_apply<float, 2>));
  HK_TRY(hk_allow_smem(k_local_apply<float, 4>));
  HK_TRY(hk_allow_smem(k_local_apply<float, 8>));
  HK_TRY(hk_allow_smem(k_local_apply<float, 16>));
  HK_TRY(hk_allow_smem(k_local_apply<double, 1>));
  HK_TRY(hk_allow_smem(k_local_apply<double, 2>));
  HK_TRY(hk_allow_smem(k_local_apply<double, 4>));
  HK_TRY(hk_allow_smem(k_local_apply<double, 8>));
  HK_TRY(hk_allow_smem(k_local_apply<double, 16>));
  return HK_OK;
}

hk_status apply_autotune(hk_handle* h, int s) {
  if (s < 2) return HK_OK;
  bool timing = h->timing;
  h->timing = false;
  cudaEvent_t a, b;
  HK_CUDA(cudaEventCreate(&a));
  HK_CUDA(cudaEventCreate(&b));
  int best = 0;
  float best_ms = 1e30f;
  hk_status rc = HK_OK;
  for (int nr = 1; nr <= 16 && nr <= s && rc == HK_OK; nr *= 2) {
    h->nr_tuned[s] = nr;
    // inputs: the (zero-initialised) first Krylov block; output: the first flexible block
    rc = op_apply(h, s, h->d_V, h->d_Zk, nullptr);  // warm-up
    float t = 0;
    for (int rep = 0; rep < 3 && rc == HK_OK; ++rep) {
      cudaEventRecord(a, h->stream);
      rc = op_apply(h, s, h->d_V, h->d_Zk, nullptr);
      cudaEventRecord(b, h->stream);
      cudaEventSynchronize(b);
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      t += ms;
    }
    if (rc == HK_OK && t < best_ms) {
      best_ms = t;
      best = nr;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->timing = timing;
  if (best) h->nr_tuned[s] = best;
  else h->nr_tuned.erase(s);
  return rc;
}

hk_status op_apply(hk_handle* h, int s, const double* v, double* z, const int* active) {
  HK_TRY(ensure_workspace(h, s));
  if (h->p.precision == HK_FP32_PRECOND) return apply_t<float>(h, s, v, z, active, h->d_ybuf32, h->d_c32, h->d_cc32);
  return apply_t<double>(h, s, v, z, active, h->d_ybuf64, h->d_c64, h->d_cc64);
}

// Transposed (m x |dof|) copy of each Z_i in the apply's arithmetic type.
template <typename T>
__global__ void k_transpose_z(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                              const double* __restrict__ Z, T* Zt, T* Zr) {
  int s = blockIdx.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], m = si[6];
  long long zo = sub_off[3 * s + 2];
  for (long long e = threadIdx.x; e < (long long)nI * m; e += blockDim.x) {
    int a = (int)(e / m), l = (int)(e % m);
    Zt[zo + (long long)l * nI + a] = (T)Z[zo + e];
    if (Zr) Zr[zo + e] = (T)Z[zo + e];
  }
}

hk_status build_apply_z(hk_handle* h) {
  if (h->n0 == 0) return HK_OK;
  if (h->p.precision == HK_FP32_PRECOND) {
    float *zt = nullptr, *zr = nullptr;
    HK_TRY(dalloc(h, &zt, h->z_total));
    HK_TRY(dalloc(h, &zr, h->z_total));
    k_transpose_z<float><<<h->n_sub, 256, 0, h->stream>>>(h->d_sub_info, h->d_sub_off, h->d_Z64, zt, zr); HK_COUNT_LAUNCH();
    h->d_Zt = zt;
    h->d_Zr = zr;
  } else {
    double* zt = nullptr;
    HK_TRY(dalloc(h, &zt, h->z_total));
    k_transpose_z<double><<<h->n_sub, 256, 0, h->stream>>>(h->d_sub_info, h->d_sub_off, h->d_Z64, zt, nullptr); HK_COUNT_LAUNCH();
    h->d_Zt = zt;
    h->d_Zr = h->d_Z64;
  }
  HK_LAUNCH_CHECK();
  return HK_OK;
}

// Host work, sizes and allocations of the local factorisation on the setup stream; then the factor
// kernels (block LU, level records) on the handle's auxiliary stream, where they overlap the
// eigenproblems (which leave SMs and the FP64 pipes idle for most of their time).
// phase_local_factors_end joins them.
hk_status phase_local_factors_begin(hk_handle* h) {
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
  int* d_nc = nullptr;
  {
    unsigned long long* d_cnt = nullptr;
    HK_TRY(dalloc(h, &d_cnt, 1));
    HK_TRY(dalloc(h, &d_nc, h->I_total + ns));
    k_count_lower<<<ns, 128, 0, st>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI, h->d_lcol,
                                      d_cnt); HK_COUNT_LAUNCH();
    k_level_counts<<<ns, 128, 0, st>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI, h->d_lcol,
                                       d_nc); HK_COUNT_LAUNCH();
    unsigned long long c = 0;
    HK_CUDA(cudaMemcpyAsync(&c, d_cnt, sizeof(c), cudaMemcpyDeviceToHost, st));
    HK_CUDA(cudaStreamSynchronize(st));
    h->lower_nnz = (long long)c;
    dfree(h, d_cnt);
  }
  std::vector<int> nc(h->I_total + ns);
  HK_CUDA(cudaMemcpyAsync(nc.data(), d_nc, sizeof(int) * nc.size(), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  dfree(h, d_nc);
  // level records for the apply, in the arithmetic type of the precision form
  size_t esz = h->p.precision == HK_FP32_PRECOND ? 4 : 8;
  std::vector<long long> tab(4 * (h->I_total + ns), 0);
  long long cur = 0, stage = 16;
  for (int s = 0; s < ns; ++s) {
    const Sub& u = h->subs[s];
    const int* lp = &lev[u.lev_off];
    for (int j = 0; j < u.L; ++j) {
      long long b = lp[j + 1] - lp[j], bn = j + 1 < u.L ? lp[j + 2] - lp[j + 1] : 0, c = nc[u.lev_off + j];
      long long fb = pad16(b * b * esz + c * esz + c * 2 + (b + 1) * 2), bb = pad16(b * bn * esz);
      long long* e = &tab[4 * (size_t)(u.lev_off + j)];
      e[0] = cur;
      cur += fb;
      e[1] = cur;
      cur += bb;
      e[2] = fb | (bb << 32);
      e[3] = c | (b << 20) | ((long long)lp[j] << 40);
      stage = std::max(stage, std::max(fb, bb));
    }
  }
  h->pack_bytes = cur;
  h->pack_stage = stage;
  HK_TRY(dalloc(h, &h->d_F64, fo));
  HK_TRY(dalloc(h, &h->d_lvtab, tab.size()));
  HK_TRY(dalloc(h, &h->d_pack, cur));
  HK_CUDA(cudaMemcpyAsync(h->d_lvtab, tab.data(), sizeof(long long) * tab.size(), cudaMemcpyHostToDevice, st));
  size_t shm = sizeof(double) * (size_t)h->max_level * h->max_level;
  int s_in_smem = shm <= 200 * 1024;
  if (!s_in_smem) shm = 0;
  HK_TRY(hk_allow_smem(k_block_lu));
  // the auxiliary stream starts after everything above (allocations, memsets, table upload)
  if (!h->aux_stream) HK_CUDA(cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking));
  if (!h->ev_lf) HK_CUDA(cudaEventCreateWithFlags(&h->ev_lf, cudaEventDisableTiming));
  HK_CUDA(cudaEventRecord(h->ev_lf, st));
  HK_CUDA(cudaStreamWaitEvent(h->aux_stream, h->ev_lf, 0));
  cudaStream_t ax = h->aux_stream;
  k_block_lu<<<ns, 256, shm, ax>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI, h->d_lcol,
                                   h->d_lvalB, h->d_F64, s_in_smem, h->d_status); HK_COUNT_LAUNCH();
  if (esz == 4)
    k_pack_levels<float><<<ns, 256, 0, ax>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI,
                                             h->d_lcol, h->d_lvalB, h->d_F64, h->d_lvtab, h->d_pack);
  else
    k_pack_levels<double><<<ns, 256, 0, ax>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI,
                                              h->d_lcol, h->d_lvalB, h->d_F64, h->d_lvtab, h->d_pack);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_CUDA(cudaEventRecord(h->ev_lf, ax));
  h->lf_pending = true;
  return HK_OK;
}

// Joins the factor kernels into the setup stream, checks them, frees the FP64 factors.
hk_status phase_local_factors_end(hk_handle* h) {
  if (!h->lf_pending) return HK_OK;
  h->lf_pending = false;
  HK_CUDA(cudaStreamWaitEvent(h->stream, h->ev_lf, 0));
  HK_TRY(check_device_status(h, "local factors"));
  dfree(h, h->d_F64);
  h->d_F64 = nullptr;
  return HK_OK;
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
      s = apply_t<float>(h, n_rhs, v_dev, z_dev, nullptr, reinterpret_cast<float*>(b),
                         reinterpret_cast<float*>(b + ylen), reinterpret_cast<float*>(b + ylen + clen));
    else
      s = apply_t<double>(h, n_rhs, v_dev, z_dev, nullptr, reinterpret_cast<double*>(b),
                          reinterpret_cast<double*>(b + ylen), reinterpret_cast<double*>(b + ylen + clen));
  }
  if (cur != h->dev) cudaSetDevice(cur);
  return s;
}
