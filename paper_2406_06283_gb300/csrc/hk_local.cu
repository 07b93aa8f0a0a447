// Local Dirichlet factors of B_i = R_i B R_i^T (Eq. 2.22) and their use in
// the preconditioner apply (Eq. 2.22-2.23).
//
// In level order B_i is block tridiagonal: diagonal blocks D_j, couplings
// L_j = B[level j, level j-1] and U_j = B[level j, level j+1] = L_{j+1}^T.
// It is factored from both ends towards the middle level M = (L-1)/2 (a twisted
// block factorisation), with the Schur complements
//     top     S_0 = D_0,          S_j = D_j - L_j S_{j-1}^{-1} U_{j-1}      (j < M)
//     bottom  T_{L-1} = D_{L-1},  T_j = D_j - U_j T_{j+1}^{-1} L_{j+1}      (j > M)
//     middle  Sigma = D_M - L_M S_{M-1}^{-1} U_{M-1} - U_M T_{M+1}^{-1} L_{M+1},
// and a solve B_i x = r runs two half sweeps at once:
//     y_j = S_j^{-1} (r_j - L_j y_{j-1})          j = 0 .. M-1
//     z_j = T_j^{-1} (r_j - U_j z_{j+1})          j = L-1 .. M+1
//     x_M = Sigma^{-1} (r_M - L_M y_{M-1} - U_M z_{M+1})
//     x_j = y_j - G_j x_{j+1},  G_j = S_j^{-1} U_j    j = M-1 .. 0
//     x_j = z_j - H_j x_{j-1},  H_j = T_j^{-1} L_j    j = M+1 .. L-1
// so the dependent chain is about L steps instead of 2L - 1.  Setup stores, per
// level, the inverse block (b_j x b_j) and the coupling product (G_j, b_j x b_{j+1},
// above the middle; H_j, b_j x b_{j-1}, below it; none at the middle) densely,
// row-major, each starting on a 4-element boundary.  Inverses are formed in FP64 by
// Gauss-Jordan elimination with partial pivoting; a pivot below 1e-10 max|B_i|
// reports HK_SINGULAR_LOCAL.  For the apply, the first-sweep steps are rewritten as one
// dense product over consecutive levels of the level-ordered vector, e.g.
//     y_j = [-S_j^{-1} L_j | S_j^{-1}] [y_{j-1}; r_j].
#include <algorithm>

#include "hk_internal.cuh"

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }
__host__ __device__ __forceinline__ long long pad4(long long x) { return (x + 3) & ~3LL; }
__host__ __device__ __forceinline__ int twist_mid(int L) { return (L - 1) / 2; }

// Columns of the coupling product stored after the inverse block of level j (twist level M).
__host__ __device__ __forceinline__ long long coupling_cols(const int* lp, int L, int M, int j) {
  if (j < M) return lp[j + 2] - lp[j + 1];
  if (j > M) return lp[j] - lp[j - 1];
  return 0;
}

// Element count of the factor blocks of one subdomain factored towards level M.
long long factor_elems(const int* lp, int L, int M) {
  long long t = 0;
  for (int j = 0; j < L; ++j) {
    long long b = lp[j + 1] - lp[j];
    t += pad4(b * b) + pad4(b * coupling_cols(lp, L, M, j));
  }
  return t;
}

// One level of the twisted factorisation: the Schur complement of level j with the
// coupling products of its already eliminated neighbours (G_{j-1} above, H_{j+1} below),
// its inverse, and its own coupling product (G_j = X^{-1} U_j towards the middle from the
// top, H_j = X^{-1} L_j from the bottom).
// gout (or NULL) receives ||X^{-1}||_inf of the level, its largest absolute row sum (inf where the inverse
// is not finite or a pivot is at most `tiny`): the growth of the level's pivot block, from which the twist
// level is chosen.  *minpiv takes the smallest pivot met.
__device__ void twisted_level(int j, int L, int M, const int* lp, const long long* fo, const int* lr,
                              const int* lcntI, const int* lcol, const double* lval, int off, long long coff,
                              double* F, double* S, int s_in_smem, int* piv, double* red_v, int* red_i,
                              double* minpiv, double* gout, double tiny) {
  __shared__ double lvpiv;  // smallest pivot of this level's block
  int tid = threadIdx.x, T = blockDim.x;
  int r0 = lp[j], b = lp[j + 1] - r0;
  if (tid == 0) lvpiv = 1e300;
  bool up = j > 0 && j <= M;        // eliminated neighbour above (top part or middle)
  bool down = j < L - 1 && j >= M;  // eliminated neighbour below (bottom part or middle)
  int pr0 = j > 0 ? lp[j - 1] : r0, nr0 = lp[j + 1], nr1 = j + 1 < L ? lp[j + 2] : nr0;
  const double* Gp = up ? F + fo[j - 1] + pad4((long long)(r0 - pr0) * (r0 - pr0)) : nullptr;  // G_{j-1}: b_{j-1} x b
  const double* Hn = down ? F + fo[j + 1] + pad4((long long)(nr1 - nr0) * (nr1 - nr0)) : nullptr;  // H_{j+1}: b_{j+1} x b
  double* X = s_in_smem ? S : F + fo[j];
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
      else if (up && c >= pr0 && c < r0) v -= cv[q] * Gp[(long long)(c - pr0) * b + t];
      else if (down && c >= nr0 && c < nr1) v -= cv[q] * Hn[(long long)(c - nr0) * b + t];
    }
    X[e] = v;
  }
  __syncthreads();
  gauss_jordan_inverse(X, b, piv, red_v, red_i, &lvpiv);
  if (tid == 0) *minpiv = fmin(*minpiv, lvpiv);
  if (gout) {
    __syncthreads();
    double g = 0;
    for (int r = tid; r < b; r += T) {
      double a = 0;
      for (int c = 0; c < b; ++c) a += fabs(X[r * b + c]);
      g = a <= 1e300 ? fmax(g, a) : INFINITY;
    }
    for (int o = 16; o > 0; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
    if ((tid & 31) == 0) red_v[tid >> 5] = g;
    __syncthreads();
    if (tid == 0) {
      double m2 = 0;
      for (int w = 0; w < (T >> 5); ++w) m2 = fmax(m2, red_v[w]);
      gout[j] = lvpiv > tiny ? m2 : INFINITY;  // a pivot at the singularity floor: no usable inverse
    }
    __syncthreads();
  }
  if (s_in_smem)
    for (int e = tid; e < b * b; e += T) F[fo[j] + e] = X[e];
  if (j == M) {
    __syncthreads();
    return;
  }
  // coupling product: rows of the neighbour level towards the middle, whose entries in level j
  // are the coupling (B symmetric)
  int c0 = j < M ? nr0 : pr0, cb = j < M ? nr1 - nr0 : r0 - pr0;
  double* P = F + fo[j] + pad4((long long)b * b);
  for (int e = tid; e < b * cb; e += T) {
    int qt = e / cb, cc = e % cb;
    int c = c0 + cc;
    const int* cl = lcol + coff + lr[c];
    const double* cv = lval + coff + lr[c];
    int cnt = lcntI[off + c];
    double v = 0;
    for (int q = 0; q < cnt; ++q) {
      int a = cl[q];
      if (a >= r0 && a < r0 + b) v += X[qt * b + (a - r0)] * cv[q];
    }
    P[e] = v;
  }
  __syncthreads();
}

// max |B_i| entry of subdomain s (rows = 0: the scale of the singularity test), or ||B_i||_inf, its largest
// absolute row sum (rows = 1: the scale of the growth measure), over the CTA.
__device__ double block_scale(int nI, int off, long long coff, const int* lr, const int* lcntI, const double* lval,
                              double* red_v, int rows = 0) {
  int tid = threadIdx.x, T = blockDim.x;
  double mx = 0;
  for (int a = tid; a < nI; a += T) {
    double rs = 0;
    for (int q = 0; q < lcntI[off + a]; ++q) {
      double v = fabs(lval[coff + lr[a] + q]);
      mx = rows ? mx : fmax(mx, v);
      rs += v;
    }
    if (rows) mx = fmax(mx, rs);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) red_v[tid >> 5] = mx;
  __syncthreads();
  double m2 = 0;
  for (int w = 0; w < (T >> 5); ++w) m2 = fmax(m2, red_v[w]);
  __syncthreads();
  return m2;
}

// fo: per subdomain, L + 1 factor offsets (elements from the start of the factor array); twist: the
// level M each subdomain is factored towards.  Without gout a pivot below 1e-10 max|B_i| reports
// HK_SINGULAR_LOCAL.  With gout (the first factorisation, towards the middle levels) nothing is reported:
// gout receives ||pivot block inverse||_inf per level (indexed like the level pointers; inf for a block
// with a pivot at that floor), gscale[s] ||B_i||_inf and gscale[n_sub + s] the smallest pivot / max|B_i|,
// and the host refactors every subdomain whose growth or pivot is out of bounds (the refactorisation
// then reports a singular B_i).
__global__ void k_block_lu(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                           const int* __restrict__ levptr, const int* __restrict__ lrow,
                           const int* __restrict__ lcntI, const int* __restrict__ lcol,
                           const double* __restrict__ lval, const long long* __restrict__ lvfo,
                           const int* __restrict__ twist, double* F, int s_in_smem, DevStatus* st, double* gout,
                           double* gscale) {
  extern __shared__ double smem[];
  __shared__ int piv[HK_MAXB];
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ double minpiv;
  int s = blockIdx.x, tid = threadIdx.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], L = si[2], off = si[3], loff = si[5];
  long long coff = sub_off[3 * s + 1];
  const int* lp = levptr + loff;
  const int* lr = lrow + off + s;
  const long long* fo = lvfo + loff;
  double scale = block_scale(nI, off, coff, lr, lcntI, lval, red_v);
  double rscale = gscale ? block_scale(nI, off, coff, lr, lcntI, lval, red_v, 1) : 0.0;
  if (tid == 0) {
    minpiv = 1e300;
    if (gscale) gscale[s] = rscale;
  }
  __syncthreads();
  int M = twist[s];
  double* g = gout ? gout + loff : nullptr;
  double tiny = 1e-10 * scale;
  for (int j = 0; j < M; ++j)
    twisted_level(j, L, M, lp, fo, lr, lcntI, lcol, lval, off, coff, F, smem, s_in_smem, piv, red_v, red_i, &minpiv, g,
                  tiny);
  for (int j = L - 1; j > M; --j)
    twisted_level(j, L, M, lp, fo, lr, lcntI, lcol, lval, off, coff, F, smem, s_in_smem, piv, red_v, red_i, &minpiv, g,
                  tiny);
  twisted_level(M, L, M, lp, fo, lr, lcntI, lcol, lval, off, coff, F, smem, s_in_smem, piv, red_v, red_i, &minpiv, g,
                tiny);
  if (tid == 0) {
    if (gscale) gscale[gridDim.x + s] = minpiv / scale;
    else if (!(minpiv > tiny)) dev_fail(st, HK_SINGULAR_LOCAL, s, minpiv / scale);
  }
}

// Growth pass for the choice of the twist level.  Both one-sided block eliminations of B_i over all
// levels: from the top (the factorisation towards M = L - 1: S_0 = D_0, S_j = D_j - L_j S_{j-1}^{-1} U_{j-1})
// and from the bottom (towards M = 0: T_{L-1} = D_{L-1}, T_j = D_j - U_j T_{j+1}^{-1} L_{j+1}), each into its
// own scratch factor array, with ||S_j^{-1}||_inf into gtop and ||T_j^{-1}||_inf into gbot per level and
// ||B_i||_inf into gscale.  A twisted factorisation towards M uses S_j for j < M and T_j for j > M; its middle
// block Sigma_M has Sigma_M^{-1} = (B_i^{-1})_{MM}, bounded by B_i^{-1} whatever M is.
__global__ void k_chain_growth(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                               const int* __restrict__ levptr, const int* __restrict__ lrow,
                               const int* __restrict__ lcntI, const int* __restrict__ lcol,
                               const double* __restrict__ lval, const long long* __restrict__ fo_top,
                               const long long* __restrict__ fo_bot, double* Ftop, double* Fbot, int s_in_smem,
                               double* gtop, double* gbot, double* gscale) {
  extern __shared__ double smem[];
  __shared__ int piv[HK_MAXB];
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ double minpiv;
  int s = blockIdx.x, tid = threadIdx.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], L = si[2], off = si[3], loff = si[5];
  long long coff = sub_off[3 * s + 1];
  const int* lp = levptr + loff;
  const int* lr = lrow + off + s;
  double scale = block_scale(nI, off, coff, lr, lcntI, lval, red_v, 1);
  double tiny = 1e-10 * block_scale(nI, off, coff, lr, lcntI, lval, red_v);
  if (tid == 0) {
    minpiv = 1e300;
    gscale[s] = scale;
  }
  __syncthreads();
  const long long* ft = fo_top + loff;
  for (int j = 0; j < L; ++j)
    twisted_level(j, L, L - 1, lp, ft, lr, lcntI, lcol, lval, off, coff, Ftop, smem, s_in_smem, piv, red_v, red_i,
                  &minpiv, gtop + loff, tiny);
  const long long* fb = fo_bot + loff;
  for (int j = L - 1; j >= 0; --j)
    twisted_level(j, L, 0, lp, fb, lr, lcntI, lcol, lval, off, coff, Fbot, smem, s_in_smem, piv, red_v, red_i,
                  &minpiv, gbot + loff, tiny);
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
// Level records, streamed by the apply kernel, row-major with rows padded to a multiple
// of 4 entries (zeros), so that rows start on 16-byte boundaries (T = float or double):
//   first-sweep record j: above the middle [-S_j^{-1} L_j | S_j^{-1}] (b_j x pad4(b_{j-1}+b_j)),
//                         below it [T_j^{-1} | -T_j^{-1} U_j] (b_j x pad4(b_j+b_{j+1})),
//                         at the middle [-Sigma^{-1} L_M | Sigma^{-1} | -Sigma^{-1} U_M];
//   second-sweep record j: G_j (b_j x pad4(b_{j+1})) above the middle, H_j (b_j x pad4(b_{j-1}))
//                         below it, none at the middle.
// The top stream is: first sweep 0 .. M-1, middle, second sweep M-1 .. 0; the bottom stream:
// first sweep L-1 .. M+1, second sweep M+1 .. L-1.
// A record streams as chunks of consecutive rows, one 1-D TMA bulk copy each, of at most
// HK_CHUNK_BYTES (one chunk per record on 2D subdomains of up to 35^2 dofs; smaller chunks on
// subdomains so large that two ring stages would not fit beside the vectors).
// Level table entry (4 x int64 per level): fwd offset, bwd offset, fwd | bwd bytes << 32,
// fwd rows per chunk | bwd rows per chunk << 10 | b << 20 | level start << 40.
#define HK_CHUNK_BYTES (32 * 1024)
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
__host__ __device__ __forceinline__ int lv_rcf(long long e3) { return (int)(e3 & 0x3FF); }
__host__ __device__ __forceinline__ int lv_rcb(long long e3) { return (int)((e3 >> 10) & 0x3FF); }
__host__ __device__ __forceinline__ int lv_b(long long e3) { return (int)((e3 >> 20) & 0xFFFFF); }
__host__ __device__ __forceinline__ int lv_start(long long e3) { return (int)(e3 >> 40); }

template <typename T>
__global__ void k_pack_levels(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                              const int* __restrict__ levptr, const int* __restrict__ lrow,
                              const int* __restrict__ lcntI, const int* __restrict__ lcol,
                              const double* __restrict__ lvalB, const double* __restrict__ F,
                              const long long* __restrict__ lvfo, const long long* __restrict__ lvtab,
                              const int* __restrict__ twist, unsigned char* pack) {
  int s = blockIdx.x, tid = threadIdx.x, T_ = blockDim.x;
  const int* si = sub_info + 8 * s;
  int L = si[2], off = si[3], loff = si[5];
  long long coff = sub_off[3 * s + 1];
  const int* lp = levptr + loff;
  const int* lr = lrow + off + s;
  const long long* fo = lvfo + loff;
  int M = twist[s];
  // -X^{-1} B[level j, c] for a node c of a neighbour level: the couplings of row c inside level j
  auto coupled = [&](const double* Xi, int b, int r0, int row, int c) -> double {
    const int* cl = lcol + coff + lr[c];
    const double* cv = lvalB + coff + lr[c];
    double v = 0;
    for (int t = 0; t < lcntI[off + c]; ++t) {
      int a = cl[t];
      if (a >= r0 && a < r0 + b) v -= Xi[(long long)row * b + (a - r0)] * cv[t];
    }
    return v;
  };
  for (int j = 0; j < L; ++j) {
    int r0 = lp[j], b = lp[j + 1] - r0, bn = j + 1 < L ? lp[j + 2] - lp[j + 1] : 0;
    int pr0 = j > 0 ? lp[j - 1] : r0, bp = r0 - pr0, nr0 = lp[j + 1];
    int lb = (j > 0 && j <= M) ? bp : 0, rb = (j < L - 1 && j >= M) ? bn : 0;
    const long long* e = lvtab + 4 * (long long)(loff + j);
    int ldf = (int)pad4(lb + b + rb);
    const double* Xi = F + fo[j];
    // first-sweep record: [-X^{-1} L_j (top, middle) | X^{-1} | -X^{-1} U_j (bottom, middle)]
    T* Fr = reinterpret_cast<T*>(pack + e[0]);
    for (int q = tid; q < b * ldf; q += T_) {
      int row = q / ldf, col = q % ldf;
      double v = 0;
      if (col < lb) v = coupled(Xi, b, r0, row, pr0 + col);
      else if (col < lb + b) v = Xi[(long long)row * b + (col - lb)];
      else if (col < lb + b + rb) v = coupled(Xi, b, r0, row, nr0 + (col - lb - b));
      Fr[q] = (T)v;
    }
    if (j != M) {
      // second-sweep record: G_j (b x b_{j+1}) above the middle, H_j (b x b_{j-1}) below it
      int cb = j < M ? bn : bp, ldb = (int)pad4(cb);
      const double* P = Xi + pad4((long long)b * b);
      T* Gr = reinterpret_cast<T*>(pack + e[1]);
      for (int q = tid; q < b * ldb; q += T_) {
        int row = q / ldb, col = q % ldb;
        Gr[q] = col < cb ? (T)P[(long long)row * cb + col] : (T)0;
      }
    }
  }
}

// One CTA per (subdomain, group of NR right-hand sides): gather r_i = v[dof(Omega_i)]
// (R_i of Eq. 2.22), the two half sweeps of the twisted factorisation of B_i^{-1} at once,
// and the local solution written to ybuf.  T: float (FP32 form) or double.
//
// Warp roles.  The last two warps are producers, one per record stream (top: first sweep
// above the middle, the middle, second sweep above it; bottom: first and second sweep below
// the middle): one lane streams its records, chunk by chunk, into a ring of K shared-memory
// stages by 1-D TMA bulk copies, each stage guarded by a "full" mbarrier (transaction bytes)
// and an "empty" mbarrier (one arrival per consuming warp), so up to K chunks per stream are in
// flight while the sweeps run.  The other warps gather together, then split into
// right-hand-side groups: group g owns right-hand sides g*R .. g*R+R-1 (R = min(NR, 4)) and
// has two half groups of WG warps, one per stream.  A level's rows are spread over a half
// group's threads, G lanes per row on contiguous 4-column chunks (G as large as keeps every
// row in one pass), then a shuffle sum over the G lanes.  A level step is a few dependent
// shared-memory loads and FMAs and one or two barriers of the half group; the two halves of a
// group meet only around the middle level (the top half computes it once the bottom half's
// first sweep is done, the bottom half's second sweep starts from it).
// Shared vectors are level-row major within a group, x[(g * (nI + 4) + a) * R + i]; four
// zero rows after each group's rows keep the padded last columns of a record finite (padded
// columns are zero, so the values they meet never matter).
// Every wait is bounded; a wait that gives up reports HK_TIMEOUT, after which the warps keep
// only their barriers (so no barrier is left waiting), and a producer lets the copies it has in
// flight land before the CTA exits.
#define HK_APPLY_MAXK 12
#define HK_APPLY_MAXT 768  // threads of a CTA at most (24 warps)

// R-vector loads and stores of shared-memory rows, as 16- or 8-byte accesses where the
// row size allows (rows are aligned to their size).
template <typename T, int R>
__device__ __forceinline__ void ldv(T* o, const T* p) {
  if constexpr (sizeof(T) == 4 && R == 4) {
    float4 q = *reinterpret_cast<const float4*>(p);
    o[0] = q.x, o[1] = q.y, o[2] = q.z, o[3] = q.w;
  } else if constexpr (sizeof(T) == 4 && R == 2) {
    float2 q = *reinterpret_cast<const float2*>(p);
    o[0] = q.x, o[1] = q.y;
  } else if constexpr (sizeof(T) == 8 && R % 2 == 0) {
#pragma unroll
    for (int i = 0; i < R; i += 2) {
      double2 q = *reinterpret_cast<const double2*>(p + i);
      o[i] = q.x, o[i + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) o[i] = p[i];
  }
}

template <typename T, int R>
__device__ __forceinline__ void stv(T* p, const T* o) {
  if constexpr (sizeof(T) == 4 && R == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  } else if constexpr (sizeof(T) == 4 && R == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
  } else if constexpr (sizeof(T) == 8 && R % 2 == 0) {
#pragma unroll
    for (int i = 0; i < R; i += 2) *reinterpret_cast<double2*>(p + i) = make_double2(o[i], o[i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) p[i] = o[i];
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up once another warp of the CTA has flagged a failure.
__device__ __forceinline__ bool mbar_wait_or_fail(uint64_t* bar, unsigned parity, const volatile int* fail) {
  for (unsigned it = 0; it < (1u << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 63u && *fail) return false;
  }
  return false;
}

// Barrier over WG warps (a sweep half group, or both halves) that also ORs a flag across them.
__device__ __forceinline__ int group_any(int flag, int WG, int id) {
  if (WG == 1) {
    __syncwarp();
    return __any_sync(0xffffffffu, flag);
  }
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 q, %1, 0;\n bar.red.or.pred p, %2, %3, q;\n selp.s32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"(flag), "r"(id), "r"(WG * 32)
      : "memory");
  return r;
}

__device__ __forceinline__ void group_sync(int WG, int id) {
  if (WG == 1) __syncwarp();
  else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(WG * 32) : "memory");
}

// Four consecutive entries of a record row (16-byte aligned).
template <typename T>
__device__ __forceinline__ void ld4(T* m, const T* p) {
  if constexpr (sizeof(T) == 4) {
    float4 q = *reinterpret_cast<const float4*>(p);
    m[0] = q.x, m[1] = q.y, m[2] = q.z, m[3] = q.w;
  } else {
    double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    m[0] = a.x, m[1] = a.y, m[2] = b.x, m[3] = b.y;
  }
}

// acc += sum over the 4-column chunks v0 .. v1-1 of one record row of  row[t] * x[t]
// (x[t] an R-vector in shared memory).
template <typename T, int R>
__device__ __forceinline__ void row_chunk_dot(const T* __restrict__ row, const T* xin, int v0, int v1, T (&acc)[R]) {
#pragma unroll 2
  for (int v = v0; v < v1; ++v) {
    T m[4];
    ld4<T>(m, row + 4 * v);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      T w[R];
      ldv<T, R>(w, xin + (4 * v + u) * R);
#pragma unroll
      for (int i = 0; i < R; ++i) acc[i] += m[u] * w[i];
    }
  }
}

template <typename T, int NR>
__global__ void __launch_bounds__(HK_APPLY_MAXT, 1) k_local_apply(
    int n, int s_tot, const double* __restrict__ v, const int* __restrict__ active,
    const int* __restrict__ sub_info, const long long* __restrict__ sub_off, const int* __restrict__ Ilev,
    const long long* __restrict__ lvtab, const unsigned char* __restrict__ pack, long long I_total,
    int stage_bytes, int K, int WG, int max_L, int max_dof, T* ybuf, DevStatus* st, const int* __restrict__ jp,
    long long jstride, const int* __restrict__ twist) {
  constexpr int R = NR < 4 ? NR : 4;
  constexpr int WS = NR / R;  // right-hand-side groups, each two half groups of WG warps
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[2][HK_APPLY_MAXK], empty[2][HK_APPLY_MAXK], meta;
  __shared__ int sh_fail;
  if (jp) v += (long long)(*jp) * jstride;  // captured inner step: v = v_j with j read on the device
  int s = blockIdx.x, r_base = blockIdx.y * NR;
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int nwarps = blockDim.x >> 5, nwc = nwarps - 2;  // consumer warps; the last two warps produce
  int nct = nwc * 32;
  int prod = warp - nwc;  // 0: top stream, 1: bottom stream, < 0: consumer
  const int* si = sub_info + 8 * s;
  int nI = si[0], L = si[2], off = si[3], loff = si[5];
  int M = twist[s];
  int xs = nI + 4;  // rows per group slice of x
  int nst[2] = {2 * M + 1, 2 * (L - 1 - M)};  // steps of the top and bottom streams
  // shared memory: two record rings | level table (4 x int64 per level) | step parameters of both
  // streams (int4 each) | their record offsets | dof indices (16-byte aligned span) | x
  long long* tab = reinterpret_cast<long long*>(smem_raw + 2LL * K * stage_bytes);
  // a stream has at most 2L - 1 steps (the twist level may be any level)
  int SL = 2 * max_L;
  int4* sp = reinterpret_cast<int4*>(tab + 4 * (long long)max_L);  // [2][SL]
  long long* so = reinterpret_cast<long long*>(sp + 2 * (long long)SL);  // [2][SL]
  int* idx = reinterpret_cast<int*>(so + 2 * (long long)SL);
  int ioff = off & 3;  // position of the first index in the aligned span
  int ispan = (ioff + nI + 3) & ~3;
  T* x = reinterpret_cast<T*>(idx + ((max_dof + 7) & ~3));  // WS groups x (nI + 4) x R
  int nr = s_tot - r_base < NR ? s_tot - r_base : NR;
  if (tid == 0) {
    sh_fail = 0;
    for (int h = 0; h < 2; ++h)
      for (int k = 0; k < K; ++k) {
        mbar_init(&full[h][k], 1);
        mbar_init(&empty[h][k], WS * WG);
      }
    mbar_init(&meta, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the level table and the dof indices by two bulk copies
    mbar_expect_tx(&meta, 32u * L + 4u * ispan);
    tma_load_1d(tab, lvtab + 4 * (long long)loff, 32u * L, &meta);
    tma_load_1d(idx, Ilev + (off - ioff), 4u * ispan, &meta);
  }
  __syncthreads();
  bool meta_ok = mbar_wait_or_fail(&meta, 0u, &sh_fail);
  if (!meta_ok && tid == 0 && atomicExch(&sh_fail, 1) == 0) dev_fail(st, HK_TIMEOUT, s, -1);
  int nthr = 32 * WG;
  if (meta_ok) {
    // step parameters of both streams: b | lg << 16, ld | assign << 16, level start, first input
    // row | rows per chunk << 16; and the record's byte offset in the pack
    for (int e = tid; e < nst[0] + nst[1]; e += blockDim.x) {
      int h = e < nst[0] ? 0 : 1, k = h ? e - nst[0] : e;
      int j, kind;  // kind 0: first sweep (and middle), 1: second sweep
      if (h == 0) {
        j = k <= M ? k : 2 * M - k;
        kind = k <= M ? 0 : 1;
      } else {
        int nf = L - 1 - M;
        j = k < nf ? L - 1 - k : M + 1 + (k - nf);
        kind = k < nf ? 0 : 1;
      }
      const long long* en = tab + 4 * j;
      long long e3 = en[3];
      int b = lv_b(e3), ls = lv_start(e3);
      int bp = j > 0 ? ls - lv_start(tab[4 * (j - 1) + 3]) : 0;
      int bn = j + 1 < L ? lv_b(tab[4 * (j + 1) + 3]) : 0;
      int ld, in_row, rc;
      if (kind == 0) {
        int lb = (j > 0 && j <= M) ? bp : 0, rb = (j < L - 1 && j >= M) ? bn : 0;
        ld = (int)pad4(lb + b + rb);
        in_row = ls - lb;
        rc = lv_rcf(e3);
      } else {
        int cb = j < M ? bn : bp;
        ld = (int)pad4(cb);
        in_row = j < M ? ls + b : ls - bp;
        rc = lv_rcb(e3);
      }
      int lg = 0;  // G = 2^lg lanes per row, as many as keep b * G <= nthr (one pass)
      while (lg < 5 && (b << (lg + 1)) <= nthr) ++lg;
      sp[h * SL + k] = make_int4(b | (lg << 16), ld | ((kind == 0) << 16), ls, in_row | (rc << 16));
      so[h * SL + k] = kind == 0 ? en[0] : en[1];
    }
  }
  __syncthreads();
  // producer of stream h: position (step ps_k, chunk ps_c)
  int ps_k = 0, ps_c = 0;
  auto next_chunk = [&](int h, const unsigned char*& src, unsigned& bytes) -> bool {
    if (ps_k >= nst[h]) return false;
    int4 pv = sp[h * SL + ps_k];
    int b = pv.x & 0xFFFF, ld = pv.y & 0xFFFF, rc = pv.w >> 16;
    long long rowb = (long long)ld * sizeof(T);
    int row0 = ps_c * rc, nrows = b - row0 < rc ? b - row0 : rc;
    src = pack + so[h * SL + ps_k] + row0 * rowb;
    bytes = (unsigned)(nrows * rowb);
    if (row0 + nrows >= b) ++ps_k, ps_c = 0;
    else ++ps_c;
    return true;
  };
  int issued = 0;
  unsigned char* ring = prod >= 0 ? smem_raw + (long long)prod * K * stage_bytes : nullptr;
  if (prod >= 0 && lane == 0 && meta_ok) {
    const unsigned char* src;
    unsigned bytes;
    for (; issued < K && next_chunk(prod, src, bytes); ++issued) {
      mbar_expect_tx(&full[prod][issued], bytes);
      tma_load_1d(ring + (long long)issued * stage_bytes, src, bytes, &full[prod][issued]);
    }
  }
  if (prod < 0 && meta_ok) {
    // gather, eight values per thread in flight
    int tot = nI * NR;
    for (int e0 = tid; e0 < tot; e0 += 8 * nct) {
      T val[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        int e = e0 + u * nct;
        int rr = e / nI, a = e - rr * nI;
        bool on = e < tot && rr < nr && (active == nullptr || active[8 * (r_base + rr)]);
        val[u] = on ? (T)v[(long long)(r_base + rr) * n + idx[ioff + a]] : (T)0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        int e = e0 + u * nct;
        if (e < tot) {
          int rr = e / nI, a = e - rr * nI;
          x[((long long)(rr / R) * xs + a) * R + rr % R] = val[u];
        }
      }
    }
    for (int e = tid; e < WS * 4 * R; e += nct) {  // the zero rows after each group's slice
      int g = e / (4 * R), q = e % (4 * R);
      x[((long long)g * xs + nI) * R + q] = (T)0;
    }
  }
  __syncthreads();
  if (prod >= 0) {
    if (lane != 0 || !meta_ok) return;
    const unsigned char* src;
    unsigned bytes;
    bool failed = false;
    for (; next_chunk(prod, src, bytes); ++issued) {
      int k = issued % K;
      if (!mbar_wait_or_fail(&empty[prod][k], (unsigned)((issued / K) - 1) & 1u, &sh_fail)) {
        if (atomicExch(&sh_fail, 1) == 0) dev_fail(st, HK_TIMEOUT, s, issued);
        failed = true;
        break;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&full[prod][k], bytes);
      tma_load_1d(ring + (long long)k * stage_bytes, src, bytes, &full[prod][k]);
    }
    if (failed) {  // let the copies in flight land before the CTA exits
      for (int r = issued - K < 0 ? 0 : issued - K; r < issued; ++r)
        mbar_wait_bounded(&full[prod][r % K], (unsigned)(r / K) & 1u);
    }
    return;
  }
  if (!meta_ok) return;
  int g = warp / (2 * WG), h = (warp / WG) & 1, wr = warp % WG;
  int hid = 1 + 3 * g + h, jid = 3 + 3 * g;  // named barriers: this half, both halves
  int gt = wr * 32 + lane;
  T* xg = x + (long long)g * xs * R;
  const unsigned char* myring = smem_raw + (long long)h * K * stage_bytes;
  uint64_t* myfull = full[h];
  uint64_t* myempty = empty[h];
  bool dead = false;  // a wait gave up: from then on only the barriers are kept
  int ks = 0;          // stage of the next chunk
  unsigned kph = 0;    // its phase parity
  // joint point of the two halves: top, before and after the middle step; bottom, between its sweeps
  int n_first = h == 0 ? M : L - 1 - M;
  for (int k = 0; k <= nst[h]; ++k) {
    if (k == n_first) {
      dead = group_any(dead, 2 * WG, jid) != 0;  // the bottom sweep's z_{M+1} is ready
      if (h == 1) dead = group_any(dead, 2 * WG, jid) != 0;  // x_M is ready
    }
    if (h == 0 && k == n_first + 1) dead = group_any(dead, 2 * WG, jid) != 0;
    if (k == nst[h]) break;
    int4 pv = sp[h * SL + k];
    int b = pv.x & 0xFFFF, lg = pv.x >> 16, ld = pv.y & 0xFFFF, assign = pv.y >> 16, ls = pv.z,
        in_row = pv.w & 0xFFFF, rc = pv.w >> 16;
    const T* xin = xg + (long long)in_row * R;
    int G = 1 << lg;
    int q = gt >> lg, gl = gt & (G - 1);
    int nv = ld >> 2, cv = (nv + G - 1) >> lg;
    int v0 = gl * cv, v1 = min(nv, v0 + cv);
    T acc[R];
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = (T)0;
    bool okl = !dead;
    if (!dead)
      for (int row0 = 0; row0 < b; row0 += rc) {
        int kk = ks;
        bool ok = mbar_wait_or_fail(&myfull[kk], kph, &sh_fail);
        if (++ks == K) ks = 0, kph ^= 1u;
        if (!ok) {
          if (atomicExch(&sh_fail, 1) == 0) dev_fail(st, HK_TIMEOUT, s, k);
          okl = false;
          break;
        }
        const T* buf = reinterpret_cast<const T*>(myring + (long long)kk * stage_bytes);
        if (q >= row0 && q < b && q < row0 + rc) row_chunk_dot<T, R>(buf + (long long)(q - row0) * ld, xin, v0, v1, acc);
        __syncwarp();
        if (lane == 0) mbar_arrive(&myempty[kk]);
      }
#pragma unroll
    for (int i = 0; i < R; ++i)
      for (int o = G >> 1; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    bool own = q < b && gl == 0;
    if (assign) {
      // first sweep and middle: every read of r_j ends before the result overwrites it
      dead = group_any(!okl, WG, hid) != 0;
      if (!dead && own) stv<T, R>(xg + (long long)(ls + q) * R, acc);
      group_sync(WG, hid);
    } else {
      // second sweep: x_j = (first-sweep value) - coupling product x_neighbour
      if (okl && own) {
        T y[R];
        ldv<T, R>(y, xg + (long long)(ls + q) * R);
#pragma unroll
        for (int i = 0; i < R; ++i) y[i] -= acc[i];
        stv<T, R>(xg + (long long)(ls + q) * R, y);
      }
      dead = group_any(!okl, WG, hid) != 0;
    }
  }
  dead = group_any(dead, 2 * WG, jid) != 0;  // both halves done: x complete
  if (dead) return;
  for (int e = h * 32 * WG + gt; e < nI * R; e += 2 * nthr) {
    int a = e / R, i = e % R, rr = g * R + i;
    if (rr < nr && (active == nullptr || active[8 * (r_base + rr)]))
      ybuf[(long long)(r_base + rr) * I_total + off + a] = xg[e];
  }
}

// c_i = Z_i^T v[dof(Omega_i)]  (R_0 = Z^T applied to R_i v, Eq. 2.23) for RB right-hand sides
// per CTA: the gather of r_i into shared memory (right-hand sides fastest), then a warp per
// coarse vector l (lanes over dofs, then a fixed shuffle tree).  It runs beside the local
// sweeps, on the auxiliary stream, so the coarse path leaves the sweeps' critical path.
template <typename T, int RB>
__global__ void __launch_bounds__(256) k_restrict(int n, int s_tot, const double* __restrict__ v,
                                                  const int* __restrict__ active, const int* __restrict__ sub_info,
                                                  const long long* __restrict__ sub_off, const int* __restrict__ Ilev,
                                                  const T* __restrict__ Zt, int n0, T* cvec,
                                                  const int* __restrict__ jp, long long jstride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* r = reinterpret_cast<T*>(smem_raw);  // nI x RB
  if (jp) v += (long long)(*jp) * jstride;
  int sb = blockIdx.x, r_base = blockIdx.y * RB;
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int* si = sub_info + 8 * sb;
  int nI = si[0], off = si[3], m = si[6], c_off = si[7];
  long long zoff = sub_off[3 * sb + 2];
  int nr = s_tot - r_base < RB ? s_tot - r_base : RB;
  bool on[RB];
#pragma unroll
  for (int rr = 0; rr < RB; ++rr) on[rr] = rr < nr && (active == nullptr || active[8 * (r_base + rr)]);
  // gather: per dof its index, then the RB values, all in flight
#pragma unroll 4
  for (int a = tid; a < nI; a += blockDim.x) {
    int gi = Ilev[off + a];
    T val[RB];
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) val[rr] = on[rr] ? (T)v[(long long)(r_base + rr) * n + gi] : (T)0;
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) r[a * RB + rr] = val[rr];
  }
  __syncthreads();
  for (int l = warp; l < m; l += nw) {
    const T* zc = Zt + zoff + (long long)l * nI;
    T acc[RB];
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) acc[rr] = 0;
#pragma unroll 4
    for (int a = lane; a < nI; a += 32) {
      T zv = zc[a];
#pragma unroll
      for (int rr = 0; rr < RB; ++rr) acc[rr] += zv * r[a * RB + rr];
    }
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
      T t = acc[rr];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0 && rr < nr && (active == nullptr || active[8 * (r_base + rr)]))
        cvec[(long long)(r_base + rr) * n0 + c_off + l] = t;
    }
  }
}

// cc_r = E^{-1} c_r for s right-hand sides (E^{-1} dense n0 x n0 row-major), CR right-hand
// sides per pass.  A warp takes two rows of E^{-1} and streams them once per pass, sixteen
// loads in flight per lane; c is staged through shared memory in tiles of tc columns, stored
// column-major with a row pitch that makes the 16-byte reads of consecutive lanes hit
// distinct banks.  Each lane sums its columns lane, lane + 32, ... in order, then a fixed
// shuffle tree, so every run gives the same bits.
#define HK_CS_THREADS 256
#define HK_CS_RPW 2
template <typename T, int CR>
__host__ __device__ constexpr int cs_pitch() {
  constexpr int VW = 16 / (int)sizeof(T);  // elements per 16 bytes
  return CR <= VW ? CR : ((CR / VW) % 2 == 1 ? CR : CR + VW);
}

template <typename T, int CR>
__global__ void __launch_bounds__(HK_CS_THREADS) k_coarse_solve(int n0, int s, const T* __restrict__ Einv,
                                                                const T* __restrict__ c, T* cc,
                                                                const int* __restrict__ active, int tc) {
  constexpr int CS = cs_pitch<T, CR>();
  constexpr int RV = CR >= 4 ? 4 : CR;  // right-hand sides per shared-memory read
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* cs = reinterpret_cast<T*>(smem_raw);  // tc x CS
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int row0 = (blockIdx.x * nw + warp) * HK_CS_RPW;
  const T* e0p = Einv + (long long)min(row0, n0 - 1) * n0;
  const T* e1p = Einv + (long long)min(row0 + 1, n0 - 1) * n0;
  for (int r0 = 0; r0 < s; r0 += CR) {
    int nr = s - r0 < CR ? s - r0 : CR;
    T acc0[CR], acc1[CR];
#pragma unroll
    for (int r = 0; r < CR; ++r) acc0[r] = acc1[r] = 0;
    for (int t0 = 0; t0 < n0; t0 += tc) {
      int tn = n0 - t0 < tc ? n0 - t0 : tc;
      __syncthreads();
#pragma unroll 2
      for (int t = threadIdx.x; t < tn; t += blockDim.x) {
        T val[CR];
#pragma unroll
        for (int r = 0; r < CR; ++r) val[r] = r < nr ? c[(long long)(r0 + r) * n0 + t0 + t] : (T)0;
#pragma unroll
        for (int r = 0; r < CR; ++r) cs[t * CS + r] = val[r];
      }
      __syncthreads();
#pragma unroll 8
      for (int t = lane; t < tn; t += 32) {
        T ea = e0p[t0 + t], eb = e1p[t0 + t];
#pragma unroll
        for (int r4 = 0; r4 < CR; r4 += RV) {
          T w[RV];
          ldv<T, RV>(w, cs + t * CS + r4);
#pragma unroll
          for (int i = 0; i < RV; ++i) {
            acc0[r4 + i] += ea * w[i];
            acc1[r4 + i] += eb * w[i];
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < CR; ++r) {
      T a = acc0[r], b = acc1[r];
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
      if (lane == 0 && r < nr && (!active || active[8 * (r0 + r)])) {
        if (row0 < n0) cc[(long long)(r0 + r) * n0 + row0] = a;
        if (row0 + 1 < n0) cc[(long long)(r0 + r) * n0 + row0 + 1] = b;
      }
    }
  }
}

// zc_i = Z_i cc_i for CR right-hand sides per CTA (the coarse prolongation of Eq. 2.23 on each
// subdomain; the scatter adds it over the holders of every dof): cc_i in shared memory, a
// thread per dof of Omega_i summing over the coarse vectors in order.
template <typename T, int CR>
__global__ void __launch_bounds__(256) k_prolong(int s, const int* __restrict__ sub_info,
                                                 const long long* __restrict__ sub_off, const T* __restrict__ Zt,
                                                 const T* __restrict__ cc, int n0, long long I_total, T* zc,
                                                 const int* __restrict__ active) {
  __shared__ T ccs[HK_MAXM * CR];
  int sb = blockIdx.x, r0 = blockIdx.y * CR;
  const int* si = sub_info + 8 * sb;
  int nI = si[0], off = si[3], m = si[6], c_off = si[7];
  long long zoff = sub_off[3 * sb + 2];
  int nr = s - r0 < CR ? s - r0 : CR;
  for (int e = threadIdx.x; e < m * CR; e += blockDim.x) {
    int q = e / CR, r = e % CR;
    ccs[e] = r < nr ? cc[(long long)(r0 + r) * n0 + c_off + q] : (T)0;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < nI; a += blockDim.x) {
    T acc[CR];
#pragma unroll
    for (int r = 0; r < CR; ++r) acc[r] = 0;
    for (int q = 0; q < m; ++q) {
      T zv = Zt[zoff + (long long)q * nI + a];
#pragma unroll
      for (int r = 0; r < CR; ++r) acc[r] += zv * ccs[q * CR + r];
    }
#pragma unroll
    for (int r = 0; r < CR; ++r)
      if (r < nr && (!active || active[8 * (r0 + r)])) zc[(long long)(r0 + r) * I_total + off + a] = acc[r];
  }
}

// z_l = sum over (i, a) holding l of  w * y_i[a] + zc_i[a]   (pull form of the sums in
// Eq. 2.22-2.23; w = 1, or 1/mu_l for the RAS variant).  A thread per dof, right-hand sides
// innermost in chunks of SR; holders in a fixed order, so every run gives the same bits.
template <typename T, int SR>
__global__ void k_scatter(int n, int s, const int* __restrict__ pull_ptr, const int* __restrict__ pull_row,
                          const T* __restrict__ ybuf, const T* __restrict__ zc, long long I_total, int do_local,
                          int do_coarse, int ras, const int* __restrict__ mu, double* z,
                          const int* __restrict__ active, const int* __restrict__ jp, long long jstride, int accum) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  if (jp) z += (long long)(*jp) * jstride;  // captured inner step: z = z_j
  int p0 = pull_ptr[l], p1 = pull_ptr[l + 1];
  T wl = ras ? (T)1 / (T)mu[l] : (T)1;
  for (int r0 = 0; r0 < s; r0 += SR) {
    int nr = s - r0 < SR ? s - r0 : SR;
    T acc[SR];
#pragma unroll
    for (int r = 0; r < SR; ++r) acc[r] = 0;
    for (int p = p0; p < p1; ++p) {
      int row = pull_row[p];
#pragma unroll
      for (int r = 0; r < SR; ++r)
        if (r < nr) {
          long long o = (long long)(r0 + r) * I_total + row;
          if (do_local) acc[r] += wl * ybuf[o];
          if (do_coarse) acc[r] += zc[o];
        }
    }
#pragma unroll
    for (int r = 0; r < SR; ++r)
      if (r < nr && (!active || active[8 * (r0 + r)])) {
        long long o = (long long)(r0 + r) * n + l;
        z[o] = accum ? z[o] + (double)acc[r] : (double)acc[r];  // accum: added to the fine local part (nested)
      }
  }
}

// Launch shape of k_local_apply<T, NR> for this handle: warps per half group, ring depth,
// threads and dynamic shared memory.  Each of the two rings gets as many stages (up to
// HK_APPLY_MAXK) as fit: in the whole of an SM's shared memory when the grid is a single
// wave, in half of it otherwise (so that two CTAs can share an SM), and at least two.
struct ApplyShape {
  int WG = 1, K = 0, threads = 0;
  size_t shm = 0;
};

// Warps of a sweep group: a level is spread over at least max_level threads, four lanes per
// row where that fits in eight warps.
static int apply_wg(const hk_handle* h) {
  int wg = (4 * h->max_level + 31) / 32;
  int wmin = (h->max_level + 31) / 32;
  return std::max(1, std::max(wmin, std::min(wg, 8)));
}

template <typename T, int NR>
static ApplyShape apply_shape(hk_handle* h, int s) {
  constexpr int R = NR < 4 ? NR : 4, WS = NR / R;
  ApplyShape a;
  a.WG = apply_wg(h);
  a.threads = 32 * (WS * 2 * a.WG + 2);
  size_t vec = 128 * (size_t)h->max_L + 4 * (size_t)((h->max_dof + 7) & ~3) +
               sizeof(T) * (size_t)NR * ((size_t)h->max_dof + 4);
  size_t stage = (size_t)h->pack_stage;
  if (!h->n_sm) cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->dev);
  long long ctas = (long long)h->n_sub * ((s + NR - 1) / NR);
  // one wave: the whole shared memory for a deep ring; more: half of it, so two CTAs share an SM
  size_t budget = ctas <= h->n_sm ? 220 * 1024 : 112 * 1024;
  int K = HK_APPLY_MAXK;  // stages per ring (two rings)
  while (K > 4 && 2 * K * stage + vec > budget) --K;
  while (K > 2 && 2 * K * stage + vec > 220 * 1024) --K;
  a.K = K;
  a.shm = 2 * K * stage + vec;
  return a;
}

template <typename T, int NR>
static hk_status launch_local(hk_handle* h, int s, const double* v, const int* active, T* ybuf) {
  ApplyShape a = apply_shape<T, NR>(h, s);
  HK_TRY(hk_allow_smem(k_local_apply<T, NR>));
  if (a.shm > 220 * 1024 || h->max_level > HK_MAXB || a.threads > HK_APPLY_MAXT) {
    hk_set_error("subdomain too large for the shared-memory apply (%d dofs, level %d, record %lld bytes)",
                 h->max_dof, h->max_level, (long long)h->pack_stage);
    return HK_UNSUPPORTED;
  }
  dim3 grid(h->n_sub, (s + NR - 1) / NR);
  HK_TIMED(h, HK_T_LOCAL_APPLY,
           (k_local_apply<T, NR><<<grid, a.threads, a.shm, h->stream>>>(
               h->n, s, v, active, h->d_sub_info, h->d_sub_off, h->d_I, h->d_lvtab, h->d_pack, h->I_total,
               (int)h->pack_stage, a.K, a.WG, h->max_L, h->max_dof, ybuf, h->d_status, h->g_jp, h->g_jstride,
               h->d_twist))); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  return HK_OK;
}

template <typename T>
static hk_status apply_t(hk_handle* h, int s, const double* v, double* z, const int* active, T* ybuf, T* c,
                         T* cc) {
  const T* Zt = reinterpret_cast<const T*>(h->d_Zt);
  const T* Einv = sizeof(T) == 4 ? reinterpret_cast<const T*>(h->d_Einv32) : reinterpret_cast<const T*>(h->d_Einv64);
  int do_local = h->p.levels != HK_COARSE_ONLY;
  int do_coarse = h->p.levels != HK_ONE_LEVEL && h->n0 > 0;
  size_t budget = 220 * 1024 - 4 * (size_t)h->pack_stage;
  int nr = 16;
  budget -= 128 * (size_t)h->max_L + 4 * (size_t)((h->max_dof + 7) & ~3);
  int wg = apply_wg(h);
  while (nr > 1 && (nr > s || sizeof(T) * ((size_t)h->max_dof + 4) * nr > budget ||
                    32 * ((nr / std::min(nr, 4)) * 2 * wg + 2) > HK_APPLY_MAXT))
    nr >>= 1;
  auto tuned = h->nr_tuned.find(s);
  if (tuned != h->nr_tuned.end() && tuned->second <= nr) nr = tuned->second;
  // The coarse path (restriction, E^{-1}) and the local sweeps are independent until the
  // scatter: the coarse path runs on the auxiliary stream, forked from and joined back into
  // the handle's stream (in a captured solve graph these become parallel branches).
  int cr = s >= 8 ? 8 : s >= 4 ? 4 : s >= 2 ? 2 : 1;
  T* zc = ybuf + (size_t)s * h->I_total;  // coarse prolongation per subdomain row
  bool fork = do_local && do_coarse && h->co_stream && h->ev_fork && h->ev_join;
  cudaStream_t main_st = h->stream;
  // the restriction stages a subdomain's rows of rb right-hand sides in shared memory
  int rb = cr;
  while (rb > 1 && sizeof(T) * (size_t)h->max_dof * rb > 200 * 1024) rb >>= 1;
  if (do_coarse && sizeof(T) * (size_t)h->max_dof * rb > 200 * 1024) {
    hk_set_error("subdomain with %d dofs too large for the coarse restriction's shared memory", h->max_dof);
    return HK_UNSUPPORTED;
  }
  if (do_coarse) {
    if (fork) {
      HK_CUDA(cudaEventRecord(h->ev_fork, main_st));
      HK_CUDA(cudaStreamWaitEvent(h->co_stream, h->ev_fork, 0));
      h->stream = h->co_stream;
    }
    dim3 rg(h->n_sub, (s + rb - 1) / rb);
    size_t rshm = sizeof(T) * (size_t)h->max_dof * rb;
    // coarse solve: up to 16 right-hand sides per pass, c staged in column tiles
    int ccr = s >= 16 ? 16 : s >= 8 ? 8 : cr;
    int pitch = sizeof(T) == 4 ? (ccr == 16 ? cs_pitch<float, 16>() : ccr == 8 ? cs_pitch<float, 8>() : ccr == 4 ? cs_pitch<float, 4>() : ccr)
                               : (ccr == 16 ? cs_pitch<double, 16>() : ccr == 8 ? cs_pitch<double, 8>() : ccr == 4 ? cs_pitch<double, 4>() : ccr);
    int tc = (int)std::min<long long>(((long long)h->n0 + 31) / 32 * 32, (long long)(48 * 1024 / (sizeof(T) * pitch)) / 32 * 32);
    tc = std::max(tc, 32);
    size_t cshm = sizeof(T) * (size_t)tc * pitch;
    int cgrid = std::max(1, nblk(h->n0, (HK_CS_THREADS / 32) * HK_CS_RPW));
    bool cs_ok = cshm <= 200 * 1024;
#define HK_RESTRICT(RBV)                                                                                     \
  k_restrict<T, RBV><<<rg, 256, rshm, h->stream>>>(h->n, s, v, active, h->d_sub_info, h->d_sub_off, h->d_I, Zt, \
                                                   h->n0, c, h->g_jp, h->g_jstride)
#define HK_CSOLVE(CRV) k_coarse_solve<T, CRV><<<cgrid, HK_CS_THREADS, cshm, h->stream>>>(h->n0, s, Einv, c, cc, active, tc)
#define HK_PROLONG(CRV)                                                                                          \
  k_prolong<T, CRV><<<rg, 256, 0, h->stream>>>(s, h->d_sub_info, h->d_sub_off, Zt, cc, h->n0, h->I_total, zc, active)
    if (cs_ok) {
      HK_TIMED(h, HK_T_COARSE_SOLVE, {
        switch (rb) {
          case 8: HK_RESTRICT(8); break;
          case 4: HK_RESTRICT(4); break;
          case 2: HK_RESTRICT(2); break;
          default: HK_RESTRICT(1); break;
        }
        switch (ccr) {
          case 16: HK_CSOLVE(16); break;
          case 8: HK_CSOLVE(8); break;
          case 4: HK_CSOLVE(4); break;
          case 2: HK_CSOLVE(2); break;
          default: HK_CSOLVE(1); break;
        }
        switch (rb) {
          case 8: HK_PROLONG(8); break;
          case 4: HK_PROLONG(4); break;
          case 2: HK_PROLONG(2); break;
          default: HK_PROLONG(1); break;
        }
      });
    }
#undef HK_RESTRICT
#undef HK_CSOLVE
#undef HK_PROLONG
    HK_COUNT_LAUNCH();
    HK_COUNT_LAUNCH();
    HK_COUNT_LAUNCH();
    h->stream = main_st;
    if (fork) HK_CUDA(cudaEventRecord(h->ev_join, h->co_stream));
    if (!cs_ok) {
      hk_set_error("coarse space too large for the coarse solve (n0 = %d)", h->n0);
      return HK_UNSUPPORTED;
    }
    HK_LAUNCH_CHECK();
  }
  hk_status rc = HK_OK;
  bool use_tc = false;
  if constexpr (sizeof(T) == 4) {
    if (h->tc_ok && h->sweep_path != HK_SWEEPS_CUDA_CORE) {
      auto tt = h->tc_tuned.find(s);
      use_tc = h->sweep_path == HK_SWEEPS_TENSOR_CORE || tt == h->tc_tuned.end() || tt->second;
    }
    if (do_local && use_tc) rc = tc_launch(h, s, v, active, ybuf);
  }
  if (do_local) h->last_sweeps = use_tc ? HK_SWEEPS_TENSOR_CORE : HK_SWEEPS_CUDA_CORE;
  if (do_local && !use_tc) {
    switch (nr) {
      case 16: rc = launch_local<T, 16>(h, s, v, active, ybuf); break;
      case 8: rc = launch_local<T, 8>(h, s, v, active, ybuf); break;
      case 4: rc = launch_local<T, 4>(h, s, v, active, ybuf); break;
      case 2: rc = launch_local<T, 2>(h, s, v, active, ybuf); break;
      default: rc = launch_local<T, 1>(h, s, v, active, ybuf); break;
    }
  }
  if (fork) HK_CUDA(cudaStreamWaitEvent(main_st, h->ev_join, 0));
  HK_TRY(rc);
#define HK_SCATTER_LAUNCH(SRV)                                                                                \
  HK_TIMED(h, HK_T_SCATTER,                                                                                   \
           (k_scatter<T, SRV><<<nblk(h->n, 128), 128, 0, h->stream>>>(                                        \
               h->n, s, h->d_pull_ptr, h->d_pull_row, ybuf, zc, h->I_total, do_local, do_coarse,              \
               h->p.weighting == HK_RAS_POU, h->d_mu, z, active, h->g_jp, h->g_jstride, h->child != nullptr)))
  switch (cr) {
    case 8: HK_SCATTER_LAUNCH(8); break;
    case 4: HK_SCATTER_LAUNCH(4); break;
    case 2: HK_SCATTER_LAUNCH(2); break;
    default: HK_SCATTER_LAUNCH(1); break;
  }
#undef HK_SCATTER_LAUNCH
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  return HK_OK;
}

hk_status apply_prepare(hk_handle*) {
  HK_TRY(hk_allow_smem(k_coarse_solve<float, 1>));
  HK_TRY(hk_allow_smem(k_coarse_solve<float, 2>));
  HK_TRY(hk_allow_smem(k_coarse_solve<float, 4>));
  HK_TRY(hk_allow_smem(k_coarse_solve<float, 8>));
  HK_TRY(hk_allow_smem(k_coarse_solve<float, 16>));
  HK_TRY(hk_allow_smem(k_coarse_solve<double, 1>));
  HK_TRY(hk_allow_smem(k_coarse_solve<double, 2>));
  HK_TRY(hk_allow_smem(k_coarse_solve<double, 4>));
  HK_TRY(hk_allow_smem(k_coarse_solve<double, 8>));
  HK_TRY(hk_allow_smem(k_coarse_solve<double, 16>));
  HK_TRY(hk_allow_smem(k_restrict<float, 1>));
  HK_TRY(hk_allow_smem(k_restrict<float, 2>));
  HK_TRY(hk_allow_smem(k_restrict<float, 4>));
  HK_TRY(hk_allow_smem(k_restrict<float, 8>));
  HK_TRY(hk_allow_smem(k_restrict<double, 1>));
  HK_TRY(hk_allow_smem(k_restrict<double, 2>));
  HK_TRY(hk_allow_smem(k_restrict<double, 4>));
  HK_TRY(hk_allow_smem(k_restrict<double, 8>));
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
  HK_TRY(tc_prepare());
  return HK_OK;
}

bool apply_needs_tuning(const hk_handle* h, int s) {
  if (h->p.levels == HK_COARSE_ONLY) return false;  // no local sweeps to tune
  return (s > 1 && !h->nr_tuned.count(s)) || (h->tc_ok && h->sweep_path == HK_SWEEPS_AUTO && !h->tc_tuned.count(s));
}

hk_status apply_autotune(hk_handle* h, int s) {
  bool tune_tc = h->tc_ok && h->sweep_path == HK_SWEEPS_AUTO;
  if (s < 2 && !tune_tc) return HK_OK;
  bool timing = h->timing;
  int path = h->sweep_path;
  h->timing = false;
  cudaEvent_t a, b;
  HK_CUDA(cudaEventCreate(&a));
  HK_CUDA(cudaEventCreate(&b));
  // inputs: the (zero-initialised) first Krylov block; output: the first flexible block
  auto time_apply = [&](float& t) -> hk_status {
    hk_status r = op_apply(h, s, h->d_V, h->d_Zk, nullptr);  // warm-up
    t = 0;
    for (int rep = 0; rep < 3 && r == HK_OK; ++rep) {
      cudaEventRecord(a, h->stream);
      r = op_apply(h, s, h->d_V, h->d_Zk, nullptr);
      cudaEventRecord(b, h->stream);
      cudaEventSynchronize(b);
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      t += ms;
    }
    return r;
  };
  int best = 0;
  float best_ms = 1e30f;
  hk_status rc = HK_OK;
  h->sweep_path = HK_SWEEPS_CUDA_CORE;
  for (int nr = 1; nr <= 16 && nr <= s && rc == HK_OK; nr *= 2) {
    h->nr_tuned[s] = nr;
    float t = 0;
    rc = time_apply(t);
    if (rc == HK_OK && t < best_ms) {
      best_ms = t;
      best = nr;
    }
  }
  if (best) h->nr_tuned[s] = best;
  else h->nr_tuned.erase(s);
  if (tune_tc && rc == HK_OK) {
    h->sweep_path = HK_SWEEPS_TENSOR_CORE;
    float t = 0;
    rc = time_apply(t);
    if (rc == HK_OK) h->tc_tuned[s] = t < best_ms ? 1 : 0;
  }
  h->sweep_path = path;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->timing = timing;
  return rc;
}

hk_status op_apply(hk_handle* h, int s, const double* v, double* z, const int* active) {
  HK_TRY(ensure_workspace(h, s));
  if (h->child) {
    // nested decompositions: the local solves on the fine subdomains (the child writes z), then this
    // handle's coarse correction added to it (Eq. 2.23 with the one-level part of Eq. 2.22 on the fine ones)
    hk_handle* c = h->child;
    c->stream = h->stream;
    c->g_jp = h->g_jp;
    c->g_jstride = h->g_jstride;
    c->timing = h->timing;
    HK_TRY(op_apply(c, s, v, z, active));
  }
  if (precond_f32(h->p)) return apply_t<float>(h, s, v, z, active, h->d_ybuf32, h->d_c32, h->d_cc32);
  return apply_t<double>(h, s, v, z, active, h->d_ybuf64, h->d_c64, h->d_cc64);
}

// Transposed (m x |dof|) copy of each Z_i in the apply's arithmetic type (the restriction and
// the prolongation both read it, coalesced over the dofs).
template <typename T>
__global__ void k_transpose_z(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                              const double* __restrict__ Z, T* Zt) {
  int s = blockIdx.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], m = si[6];
  long long zo = sub_off[3 * s + 2];
  for (long long e = threadIdx.x; e < (long long)nI * m; e += blockDim.x) {
    int a = (int)(e / m), l = (int)(e % m);
    Zt[zo + (long long)l * nI + a] = (T)Z[zo + e];
  }
}

hk_status build_apply_z(hk_handle* h) {
  if (h->n0 == 0) return HK_OK;
  if (precond_f32(h->p)) {
    float* zt = nullptr;
    HK_TRY(dalloc(h, &zt, h->z_total));
    k_transpose_z<float><<<h->n_sub, 256, 0, h->stream>>>(h->d_sub_info, h->d_sub_off, h->d_Z64, zt); HK_COUNT_LAUNCH();
    h->d_Zt = zt;
  } else {
    double* zt = nullptr;
    HK_TRY(dalloc(h, &zt, h->z_total));
    k_transpose_z<double><<<h->n_sub, 256, 0, h->stream>>>(h->d_sub_info, h->d_sub_off, h->d_Z64, zt); HK_COUNT_LAUNCH();
    h->d_Zt = zt;
  }
  HK_LAUNCH_CHECK();
  return HK_OK;
}

// Host part of the local factorisation:
//   begin: the factor and record tables with every subdomain factored towards its middle level, then the
//     factor kernels (block LU, which also records ||pivot block inverse||_inf of every level, and the
//     level records) on the handle's auxiliary stream, where they overlap the eigenproblems;
//   mid: the growth of each factorisation (below; the middle block is never the problem: Sigma_M^{-1} is a
//     diagonal block of B_i^{-1}).  A subdomain whose growth is far above the others' has a nearly singular
//     leading (or trailing) level block and is factored towards another level:
//     both one-sided block eliminations over all levels (k_chain_growth) give the growth
//     G(M) = max(max_{j<M} g_top[j], max_{j>M} g_bot[j]) of every twist level, and the choice is the M
//     nearest the middle (the shortest dependent chain of the apply) with G(M) <= 2 min G.  The tables
//     and factors are then rebuilt (on the auxiliary stream again, beside the coarse phase);
//   end: joins them.
// Growth measure: max over the pivot blocks X of ||X^{-1}||_inf ||B_i||_inf.  The apply's own error is of
// the size of cond(B_i) u, so growth matters where it exceeds the conditioning of B_i, which an
// ill-conditioned (near-resonant) local problem can have as well; measured on the h = 1/256, k = 50
// checkerboard workload: median 82, largest 598 (never above 0.2 cond(B_i)); on the h = 1/512, k = 100
// layered one: median 22, and 9.5e3 = 3.65 cond(B_i) on the subdomains whose leading level block is nearly
// singular.  A factorisation is refactored when its growth exceeds both HK_GROWTH_OK and HK_GROWTH_REL
// times the median over the operator's subdomains, or when one of its pivots is at the singularity floor
// (1e-10 max|B_i|: a leading or trailing level block singular in floating point, while B_i may not be);
// the refactorisation reports HK_SINGULAR_LOCAL if a pivot is still at the floor (B_i itself singular).
// Where even the best twist level leaves a growth HK_MERGE_FACTOR times above that limit (a leading and a
// trailing level block both singular: on a constant-coefficient strip every band of the same rows is the
// same matrix), the first offending level of each one-sided elimination is merged with its successor in that
// elimination (one wider block, so the singular leading or trailing block is never formed) and the levels are
// scored again, up to HK_MERGE_ROUNDS times.
#define HK_GROWTH_OK 1000.0
#define HK_GROWTH_REL 50.0
#define HK_MERGE_ROUNDS 3    // rounds of level merging for subdomains that no twist level serves
#define HK_MERGE_FACTOR 20.0 // merge levels where the best twist level's growth is still this far above the limit

// Tables, allocations and factor kernels for the subdomains' current twist levels (Sub::M).
static hk_status factors_launch(hk_handle* h, bool growth) {
  cudaStream_t st = h->stream;
  int ns = h->n_sub;
  const std::vector<int>& lev = h->lev_host;
  std::vector<int> twist(ns);
  long long fo = 0;
  for (int s = 0; s < ns; ++s) {
    Sub& u = h->subs[s];
    twist[s] = u.M;
    u.f_off = fo;
    fo += factor_elems(&lev[u.lev_off], u.L, u.M);
  }
  h->f_total = fo;
  HK_TRY(upload_sub_info(h));
  if (!h->d_twist) HK_TRY(dalloc(h, &h->d_twist, (size_t)ns));
  HK_CUDA(cudaMemcpyAsync(h->d_twist, twist.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
  // level records for the apply, in the arithmetic type of the precision form
  size_t esz = precond_f32(h->p) ? 4 : 8;
  // record chunks of at most 32 KB, smaller where two stages per ring would not fit beside the vectors of
  // a one-right-hand-side apply of the largest subdomain
  long long chunk = HK_CHUNK_BYTES;
  {
    long long vec1 = 128LL * h->max_L + 4LL * ((h->max_dof + 7) & ~3) + (long long)esz * (h->max_dof + 4);
    while (chunk > 2048 && 4 * chunk + vec1 > 216 * 1024) chunk >>= 1;
  }
  std::vector<long long> tab(4 * (h->I_total + ns), 0);
  std::vector<long long> lvfo(h->I_total + ns, 0);  // per level: offset of its factor blocks
  long long cur = 0, stage = 16;
  for (int s = 0; s < ns; ++s) {
    const Sub& u = h->subs[s];
    const int* lp = &lev[u.lev_off];
    int M = u.M;
    long long fcur = u.f_off;
    for (int j = 0; j < u.L; ++j) {
      long long b = lp[j + 1] - lp[j], bn = j + 1 < u.L ? lp[j + 2] - lp[j + 1] : 0;
      long long bp = j > 0 ? lp[j] - lp[j - 1] : 0;
      lvfo[u.lev_off + j] = fcur;
      fcur += pad4(b * b) + pad4(b * coupling_cols(lp, u.L, M, j));
      long long lb = (j > 0 && j <= M) ? bp : 0, rb = (j < u.L - 1 && j >= M) ? bn : 0;
      long long cb = j < M ? bn : j > M ? bp : 0;
      long long rowf = pad4(lb + b + rb) * esz, rowb = pad4(cb) * esz;  // multiples of 16 bytes
      long long fb = b * rowf, bb = b * rowb;
      long long rcf = std::max(1LL, std::min(b, chunk / rowf));
      long long rcb = cb > 0 ? std::max(1LL, std::min(b, chunk / rowb)) : 1;
      long long* e = &tab[4 * (size_t)(u.lev_off + j)];
      e[0] = cur;
      cur += fb;
      e[1] = cur;
      cur += bb;
      e[2] = fb | (bb << 32);
      e[3] = rcf | (rcb << 10) | (b << 20) | ((long long)lp[j] << 40);
      stage = std::max(stage, std::max(rcf * rowf, rcb * rowb));
    }
  }
  h->pack_bytes = cur;
  h->pack_stage = stage;
  HK_TRY(tc_plan(h, lev));
  HK_TRY(dalloc(h, &h->d_F64, fo));
  HK_TRY(dalloc(h, &h->d_lvtab, tab.size()));
  HK_TRY(dalloc(h, &h->d_lvfo, lvfo.size()));
  HK_TRY(dalloc(h, &h->d_pack, cur));
  HK_CUDA(cudaMemcpyAsync(h->d_lvtab, tab.data(), sizeof(long long) * tab.size(), cudaMemcpyHostToDevice, st));
  HK_CUDA(cudaMemcpyAsync(h->d_lvfo, lvfo.data(), sizeof(long long) * lvfo.size(), cudaMemcpyHostToDevice, st));
  if (growth) HK_TRY(dalloc(h, &h->d_gval, lev.size() + 2 * (size_t)ns));
  size_t shm = sizeof(double) * (size_t)h->max_level * h->max_level;
  int s_in_smem = shm <= 200 * 1024;
  if (!s_in_smem) shm = 0;
  // the auxiliary stream starts after everything above (allocations, memsets, table upload)
  HK_CUDA(cudaEventRecord(h->ev_lf, st));
  HK_CUDA(cudaStreamWaitEvent(h->aux_stream, h->ev_lf, 0));
  cudaStream_t ax = h->aux_stream;
  k_block_lu<<<ns, 256, shm, ax>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI, h->d_lcol,
                                   h->d_lvalB, h->d_lvfo, h->d_twist, h->d_F64, s_in_smem, h->d_status,
                                   growth ? h->d_gval : nullptr, growth ? h->d_gval + lev.size() : nullptr);
  HK_COUNT_LAUNCH();
  if (esz == 4)
    k_pack_levels<float><<<ns, 256, 0, ax>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI,
                                             h->d_lcol, h->d_lvalB, h->d_F64, h->d_lvfo, h->d_lvtab, h->d_twist,
                                             h->d_pack);
  else
    k_pack_levels<double><<<ns, 256, 0, ax>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI,
                                              h->d_lcol, h->d_lvalB, h->d_F64, h->d_lvfo, h->d_lvtab, h->d_twist,
                                              h->d_pack);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_TRY(tc_pack(h, ax));
  HK_CUDA(cudaEventRecord(h->ev_lf, ax));
  h->lf_pending = true;
  return HK_OK;
}

// Frees what factors_launch allocated (after its kernels have finished).
static void factors_free(hk_handle* h) {
  void* fr[] = {h->d_F64, h->d_lvtab, h->d_lvfo, h->d_pack, h->d_pack_tc, h->d_lvtab_tc, h->d_tc_prow};
  for (void* p : fr)
    if (p) dfree(h, p);
  h->d_F64 = nullptr;
  h->d_lvtab = nullptr;
  h->d_lvfo = nullptr;
  h->d_pack = nullptr;
  h->d_pack_tc = nullptr;
  h->d_lvtab_tc = nullptr;
  h->d_tc_prow = nullptr;
  h->tc_ok = false;
}

hk_status phase_local_factors_begin(hk_handle* h) {
  cudaStream_t st = h->stream;
  int ns = h->n_sub;
  std::vector<int>& lev = h->lev_host;
  lev.assign(h->I_total + ns, 0);
  HK_CUDA(cudaMemcpyAsync(lev.data(), h->d_lev, sizeof(int) * lev.size(), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  h->max_L = 0;
  for (int s = 0; s < ns; ++s) {
    Sub& u = h->subs[s];
    h->max_L = std::max(h->max_L, u.L);
    u.M = twist_mid(u.L);
  }
  HK_TRY(upload_sub_info(h));
  if (h->p.levels == HK_COARSE_ONLY) return HK_OK;
  {
    unsigned long long* d_cnt = nullptr;
    HK_TRY(dalloc(h, &d_cnt, 1));
    k_count_lower<<<ns, 128, 0, st>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI, h->d_lcol,
                                      d_cnt); HK_COUNT_LAUNCH();
    unsigned long long c = 0;
    HK_CUDA(cudaMemcpyAsync(&c, d_cnt, sizeof(c), cudaMemcpyDeviceToHost, st));
    HK_CUDA(cudaStreamSynchronize(st));
    h->lower_nnz = (long long)c;
    dfree(h, d_cnt);
  }
  HK_TRY(hk_allow_smem(k_block_lu));
  HK_TRY(hk_allow_smem(k_chain_growth));
  HK_TRY(hk_max_carveout(k_block_lu));  // these run beside the eigensolver
  HK_TRY(hk_max_carveout(k_pack_levels<float>));
  HK_TRY(hk_max_carveout(k_pack_levels<double>));
  if (!h->aux_stream) HK_CUDA(cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking));
  if (!h->ev_lf) HK_CUDA(cudaEventCreateWithFlags(&h->ev_lf, cudaEventDisableTiming));
  if (!h->co_stream) {
    // the apply's coarse branch: short kernels that should not queue behind the local sweeps' CTAs
    int lo = 0, hi = 0;
    HK_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    HK_CUDA(cudaStreamCreateWithPriority(&h->co_stream, cudaStreamNonBlocking, hi));
  }
  if (!h->ev_fork) HK_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  if (!h->ev_join) HK_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  HK_TRY(factors_launch(h, true));
  h->lf_stage = 1;
  return HK_OK;
}

// Both one-sided block eliminations of every subdomain over its current levels (k_chain_growth), into scratch
// factors: gg = [||S_j^{-1}||_inf per level | ||T_j^{-1}||_inf per level | ||B_i||_inf per subdomain], the
// per-level parts indexed like the level pointers.
static hk_status chain_growth(hk_handle* h, std::vector<double>& gg) {
  cudaStream_t st = h->stream;
  int ns = h->n_sub;
  const std::vector<int>& lev = h->lev_host;
  std::vector<long long> fot(h->I_total + ns, 0), fob(h->I_total + ns, 0);
  long long tt = 0, tb = 0;
  for (int s = 0; s < ns; ++s) {
    const Sub& u = h->subs[s];
    const int* lp = &lev[u.lev_off];
    for (int j = 0; j < u.L; ++j) {
      long long b = lp[j + 1] - lp[j];
      fot[u.lev_off + j] = tt;
      fob[u.lev_off + j] = tb;
      tt += pad4(b * b) + pad4(b * coupling_cols(lp, u.L, u.L - 1, j));
      tb += pad4(b * b) + pad4(b * coupling_cols(lp, u.L, 0, j));
    }
  }
  HK_TRY(dalloc(h, &h->d_gF, (size_t)(tt + tb)));
  HK_TRY(dalloc(h, &h->d_gfo, fot.size() + fob.size()));
  HK_TRY(dalloc(h, &h->d_gval, 2 * lev.size() + (size_t)ns));
  HK_CUDA(cudaMemcpyAsync(h->d_gfo, fot.data(), sizeof(long long) * fot.size(), cudaMemcpyHostToDevice, st));
  HK_CUDA(cudaMemcpyAsync(h->d_gfo + fot.size(), fob.data(), sizeof(long long) * fob.size(), cudaMemcpyHostToDevice,
                          st));
  size_t shm = sizeof(double) * (size_t)h->max_level * h->max_level;
  int s_in_smem = shm <= 200 * 1024;
  if (!s_in_smem) shm = 0;
  double* gv = h->d_gval;
  k_chain_growth<<<ns, 256, shm, st>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI, h->d_lcol,
                                       h->d_lvalB, h->d_gfo, h->d_gfo + fot.size(), h->d_gF, h->d_gF + tt, s_in_smem,
                                       gv, gv + lev.size(), gv + 2 * lev.size());
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  gg.assign(2 * lev.size() + ns, 0.0);
  HK_CUDA(cudaMemcpyAsync(gg.data(), gv, sizeof(double) * gg.size(), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  dfree(h, h->d_gF);
  dfree(h, h->d_gfo);
  dfree(h, h->d_gval);
  h->d_gF = nullptr;
  h->d_gfo = nullptr;
  h->d_gval = nullptr;
  return HK_OK;
}

hk_status phase_local_factors_mid(hk_handle* h) {
  if (h->lf_stage != 1) return HK_OK;
  h->lf_stage = 2;
  cudaStream_t st = h->stream;
  int ns = h->n_sub;
  const std::vector<int>& lev = h->lev_host;
  // growth of the factorisations towards the middle levels
  std::vector<double> g(lev.size() + 2 * (size_t)ns);
  HK_CUDA(cudaEventSynchronize(h->ev_lf));
  HK_CUDA(cudaMemcpy(g.data(), h->d_gval, sizeof(double) * g.size(), cudaMemcpyDeviceToHost));
  dfree(h, h->d_gval);
  h->d_gval = nullptr;
  const double* gs = g.data() + lev.size();
  const double* gp = gs + ns;  // smallest pivot / max|B_i|
  std::vector<double> gmid(ns, 0.0);
  std::vector<int> bad;
  h->growth_mid = 0;
  for (int s = 0; s < ns; ++s) {
    const Sub& u = h->subs[s];
    double m = 0;
    for (int j = 0; j < u.L; ++j)
      if (j != u.M) m = std::max(m, g[u.lev_off + j] <= 1e300 ? g[u.lev_off + j] : INFINITY);
    gmid[s] = m * gs[s];
    h->growth_mid = std::max(h->growth_mid, gmid[s]);
  }
  // the median over the finite growths (a singular level block makes a growth infinite)
  std::vector<double> srt;
  for (double x : gmid)
    if (x <= 1e300) srt.push_back(x);
  double med = 0;
  if (!srt.empty()) {
    std::nth_element(srt.begin(), srt.begin() + srt.size() / 2, srt.end());
    med = srt[srt.size() / 2];
  }
  double limit = std::max(HK_GROWTH_OK, HK_GROWTH_REL * med);
  for (int s = 0; s < ns; ++s)
    if (!(gmid[s] <= limit) || !(gp[s] > 1e-10)) bad.push_back(s);
  h->growth_twist = h->growth_mid;
  h->twist_moved = 0;
  h->levels_merged = 0;
  if (bad.empty()) return HK_OK;  // the factors towards the middle levels stand
  factors_free(h);
  std::vector<int>& levm = h->lev_host;
  std::vector<char> pending(ns, 0);
  for (int s : bad) pending[s] = 1;
  h->growth_twist = 0;
  for (int s = 0; s < ns; ++s)
    if (!pending[s]) h->growth_twist = std::max(h->growth_twist, gmid[s]);
  for (int round = 0;; ++round) {
    std::vector<double> gg;
    HK_TRY(chain_growth(h, gg));
    const double* gt = gg.data();
    const double* gb = gg.data() + lev.size();
    const double* gsc = gg.data() + 2 * lev.size();
    bool merged = false;
    for (int s = 0; s < ns; ++s) {
      if (!pending[s]) continue;
      Sub& u = h->subs[s];
      int L = u.L, mid = twist_mid(L);
      const double* a = gt + u.lev_off;
      const double* b = gb + u.lev_off;
      auto fin = [](double x) { return x <= 1e300 ? x : INFINITY; };
      std::vector<double> pre(L + 1, 0), suf(L + 1, 0);  // pre[M] = max_{j<M} a_j, suf[M] = max_{j>M} b_j
      for (int j = 0; j < L; ++j) pre[j + 1] = std::max(pre[j], fin(a[j]));
      for (int j = L - 1; j > 0; --j) suf[j - 1] = std::max(suf[j], fin(b[j]));
      double best = INFINITY;
      for (int M = 0; M < L; ++M) best = std::min(best, std::max(pre[M], suf[M]));
      double tmerge = HK_MERGE_FACTOR * limit;
      if (!(best * gsc[s] <= tmerge) && round < HK_MERGE_ROUNDS) {
        // no twist level avoids a singular (or outlying) one-sided block: merge the first such level of
        // each chain with its successor in that chain, so that the offending leading block [0, j_t] and
        // trailing block [j_b, L - 1] are no longer formed, and score the new levels again
        int jt = -1, jb = -1;
        for (int j = 0; j < L && jt < 0; ++j)
          if (!(fin(a[j]) * gsc[s] <= tmerge)) jt = j;
        for (int j = L - 1; j >= 0 && jb < 0; --j)
          if (!(fin(b[j]) * gsc[s] <= tmerge)) jb = j;
        int* lp = &levm[u.lev_off];
        std::vector<char> drop(L + 1, 0);  // boundary q merges levels q - 1 and q
        if (jt >= 0 && jt + 1 < L) drop[jt + 1] = 1;
        if (jb >= 1) drop[jb] = 1;
        std::vector<int> nl;
        for (int q = 0; q <= L; ++q)
          if (!drop[q]) nl.push_back(lp[q]);
        int wmax = 0;
        for (size_t q = 0; q + 1 < nl.size(); ++q) wmax = std::max(wmax, nl[q + 1] - nl[q]);
        if ((int)nl.size() < L + 1 && wmax <= HK_MAXB) {
          for (size_t q = 0; q < nl.size(); ++q) lp[q] = nl[q];
          u.L = (int)nl.size() - 1;
          h->max_level = std::max(h->max_level, wmax);
          h->levels_merged += L - u.L;
          merged = true;
          continue;
        }
      }
      int choice = mid;
      for (int d = 0; d < L; ++d) {  // nearest the middle first
        int c0 = mid - d, c1 = mid + d;
        if (c0 >= 0 && std::max(pre[c0], suf[c0]) <= 2 * best) { choice = c0; break; }
        if (c1 < L && std::max(pre[c1], suf[c1]) <= 2 * best) { choice = c1; break; }
      }
      u.M = choice;
      pending[s] = 0;
      h->twist_moved += choice != mid;
      h->growth_twist = std::max(h->growth_twist, std::max(pre[choice], suf[choice]) * gsc[s]);
    }
    if (!merged) break;
    // the merged level pointers and level counts to the device, for the next scoring pass
    HK_CUDA(cudaMemcpyAsync(h->d_lev, levm.data(), sizeof(int) * levm.size(), cudaMemcpyHostToDevice, st));
    for (int s = 0; s < ns; ++s)
      if (pending[s]) h->subs[s].M = twist_mid(h->subs[s].L);
    HK_TRY(upload_sub_info(h));
  }
  return factors_launch(h, false);
}

// Joins the factor kernels into the setup stream, checks them, frees the FP64 factors.
hk_status phase_local_factors_end(hk_handle* h) {
  HK_TRY(phase_local_factors_mid(h));
  h->lev_host.clear();
  h->lev_host.shrink_to_fit();
  if (!h->lf_pending) return HK_OK;
  h->lf_pending = false;
  HK_CUDA(cudaStreamWaitEvent(h->stream, h->ev_lf, 0));
  HK_TRY(check_device_status(h, "local factors"));
  dfree(h, h->d_F64);
  h->d_F64 = nullptr;
  dfree(h, h->d_lvfo);
  h->d_lvfo = nullptr;
  return HK_OK;
}

// ======================================================= allocation-free apply
// Some callers cannot allocate device memory when they apply the
// preconditioner: code running while a stream is being captured into a CUDA
// graph (cudaMalloc is not allowed there), or a host framework that owns all
// device memory through its own allocator and forbids allocations on its hot
// path.  hk_apply_precond_noalloc serves them: it runs the same kernels as
// hk_apply_precond on caller-provided device vectors, and keeps its
// intermediate vectors (local solutions, coarse prolongation, coarse
// right-hand side and coarse solution) in the fixed device array below
// instead of allocating.
//
// The array is HK_NOALLOC_SCRATCH_BYTES per device and stays allocated on
// every device that loads the library until the process exits.  Its device
// address is looked up once per device (host code may not use the symbol
// itself as a pointer: it is only a host-side stand-in), on the first call
// made on that device, which also raises the apply kernels' shared-memory
// limits; that first call should happen before any stream capture.  Every call uses the same array, so calls whose kernels overlap on
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
  if (h->child) {
    hk_set_error("hk_apply_precond_noalloc: handles of nested decompositions are not supported (use hk_apply_precond)");
    return HK_UNSUPPORTED;
  }
  size_t esz = precond_f32(h->p) ? sizeof(float) : sizeof(double);
  size_t ylen = align256(esz * 2 * (size_t)n_rhs * (size_t)h->I_total);
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
  // raises the apply kernels' dynamic shared-memory limits (once per process and device; allocates
  // nothing), so that this call works when it is the first apply made on the device
  hk_status s = apply_prepare(h);
  if (s == HK_OK) s = noalloc_scratch(h->dev, &base);
  if (s == HK_OK) {
    unsigned char* b = static_cast<unsigned char*>(base);
    if (precond_f32(h->p))
      s = apply_t<float>(h, n_rhs, v_dev, z_dev, nullptr, reinterpret_cast<float*>(b),
                         reinterpret_cast<float*>(b + ylen), reinterpret_cast<float*>(b + ylen + clen));
    else
      s = apply_t<double>(h, n_rhs, v_dev, z_dev, nullptr, reinterpret_cast<double*>(b),
                          reinterpret_cast<double*>(b + ylen), reinterpret_cast<double*>(b + ylen + clen));
  }
  if (cur != h->dev) cudaSetDevice(cur);
  return s;
}
