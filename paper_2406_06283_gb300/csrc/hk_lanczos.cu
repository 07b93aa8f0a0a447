// Locating and counting the H_k-GenEO eigenvalues (Eq. 5.12, Def. 5.1) without dense reductions.
//
// The pencil lives on ovdof(Omega_i) (O = dof U Gamma): B^N p = lambda C p, with B^N the local Neumann
// Helmholtz matrix and C = Xi D^N Xi, which vanishes on Gamma.  Its finite eigenvalues are real (the
// paper's lemma on indefinite pencils), and B^N_GG is positive definite on the workloads (HK_EIG_FAIL
// otherwise, from the setup's Gamma block).  In the level-set order of O both matrices are block
// tridiagonal (levels couple only to their neighbours), so every factorisation below is a block
// elimination over the level sets with dense diagonal blocks.
//
// Two kernels:
//  * k_inertia (FP64): the number of eigenvalues below tau.  With B^N - tau C = L D L^T block-wise
//    (D_j the Schur complements of the levels), Sylvester's law and Haynsworth's inertia additivity give
//        #{lambda < tau} = #neg(B^N - tau C) - #neg(B^N_GG) = sum_j #neg(D_j)
//    (B^N_GG positive definite).  #neg(D_j) is read off a symmetric indefinite factorisation of D_j
//    with Bunch-Kaufman pivoting (1x1 and 2x2 pivots); D_j^{-1} for the next level comes from
//    Gauss-Jordan elimination with partial pivoting.  This count certifies the kept number m_i.
//  * k_lanczos (FP32): candidate eigenvalues.  A shift sigma below the smallest eigenvalue makes
//    M = B^N - sigma C positive definite (checked: its block elimination without pivoting must meet
//    only positive pivots, otherwise sigma is lowered, by 0.5, 0.5, 1, 2, 4, ... from -0.5, and the
//    factorisation repeated; two bisection steps between the last indefinite and the definite shift then
//    bring sigma within a quarter step of the smallest eigenvalue).  The operator
//    Op = M^{-1} C is self-adjoint in the C inner product with eigenvalues theta = 1 / (lambda - sigma),
//    so the wanted eigenvalues lambda < tau + delta are its largest ones.  A block Krylov basis
//    (block size 4, C-orthonormal, classical Gram-Schmidt twice against all earlier blocks, columns
//    that collapse replaced by fresh seeded vectors) spans Q; the Rayleigh quotient T = Q^T C (Op Q)
//    is formed from the stored products Op Q, reduced to tridiagonal form by Householder reflections in
//    FP64 and its eigenvalues above 1 / (tau + delta - sigma) found by bisection on Sturm counts.  The
//    candidates lambda = sigma + 1 / theta go to the FP64 refinement of hk_eigen.cu.
#include <algorithm>
#include <cmath>

#include "hk_internal.cuh"

#define LZ_P 4            // Krylov block size
#define LZ_THREADS 256
#define LZ_MAX_DIM 160    // largest Krylov basis (columns)
#define LZ_T_SMEM 128     // largest Rayleigh quotient kept in shared memory (columns)
#define LZ_SIGMA_TRIES 8  // shifts tried: sigma0, then 0.5, 0.5, 1, 2, 4, ... lower while the matrix is not definite
#define LZ_SIGMA_BISECT 2 // bisection steps between the last indefinite and the first definite shift

// Sparse rows of B^N and C over ovdof(Omega_i) of one subdomain, in level order.
struct OPen {
  int nO, L, maxrow;
  const int* lp;       // L + 1 level pointers
  const int* cnt;      // nO row lengths
  const int* col;      // nO x maxrow column (level-order index)
  const double* B;     // nO x maxrow values of B^N
  const double* C;     // nO x maxrow values of C
  const int* o2i;      // nO: position in the dof level order, -1 on Gamma
  const float* B32 = nullptr;  // FP32 copies of B and C (the Lanczos kernel's own, formed once per subdomain)
  const float* C32 = nullptr;
};

__device__ __forceinline__ OPen open_sub(int s, const int* o_off, const int* O_levptr, const int* O_L, int maxrow,
                                         const int* ocnt, const int* ocol, const double* oB, const double* oC,
                                         const int* o2i, const int* sub_info) {
  OPen p;
  int oo = o_off[s];
  p.nO = sub_info[8 * s] + sub_info[8 * s + 1];
  p.L = O_L[s];
  p.maxrow = maxrow;
  p.lp = O_levptr + oo + s;
  p.cnt = ocnt + oo;
  p.col = ocol + (long long)oo * maxrow;
  p.B = oB + (long long)oo * maxrow;
  p.C = oC + (long long)oo * maxrow;
  p.o2i = o2i + oo;
  return p;
}

// Seeded start and replacement vectors: SplitMix64 finaliser of a key, mapped to [-0.5, 0.5).
__device__ __forceinline__ float lz_hash_unit(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  x ^= x >> 31;
  return (float)((double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5);
}

// In-place inverse of the b x b row-major matrix A (shared or global memory) by Gauss-Jordan
// elimination without pivoting.  For a symmetric positive definite A the pivots are the diagonal of its
// LDL^T factorisation, all positive; the smallest one is returned through *minpiv (thread 0).  Two
// barriers per pivot: the other rows are eliminated with the unscaled pivot row, then the pivot row and
// column are scaled.
template <typename T>
__device__ void gj_inverse_nopiv(T* A, int b, T* sh_inv, double* minpiv) {
  int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, nw = NT >> 5;
  (void)sh_inv;
  __syncthreads();
  for (int k = 0; k < b; ++k) {
    T pv = A[k * b + k];
    T inv = pv > (T)0 ? (T)1 / pv : (T)0;
    if (tid == 0 && (double)pv < *minpiv) *minpiv = (double)pv;
    for (int i = tid >> 5; i < b; i += nw) {
      if (i == k) continue;
      T g = A[i * b + k] * inv;
      for (int c = lane; c < b; c += 32)
        if (c != k) A[i * b + c] -= g * A[k * b + c];
    }
    __syncthreads();
    for (int c = tid; c < b; c += NT) A[k * b + c] = c == k ? inv : A[k * b + c] * inv;
    for (int i = tid; i < b; i += NT)
      if (i != k) A[i * b + k] = -A[i * b + k] * inv;
    __syncthreads();
  }
}

// Block elimination of M = B^N - sigma C over the level sets without pivoting (T = float).  Per level j:
// the inverse of the Schur complement S_j = M_jj - M_{j,j-1} X_{j-1} (b_j x b_j), the forward record
// G_j = -S_j^{-1} M_{j,j-1} (b_j x b_{j-1}) and X_j = S_j^{-1} M_{j,j+1} (b_j x b_{j+1}), stored one after
// another in F, so that the forward sweep is y_j = S_j^{-1} r_j + G_j y_{j-1} (one dense product per level)
// and the backward sweep y_j -= X_j y_{j+1}.  S (max_b^2) is the working block (shared memory when it fits,
// else the level's place in F); Xsm (max_b^2, or null) keeps X_{j-1} in shared memory for the next level.
// Returns the smallest pivot (> 0 exactly when M is positive definite, up to rounding).
template <typename T>
__device__ double lz_factor(const OPen& P, double sigma, T* F, T* Ssm, T* Xsm, T* sh_inv, double* sh_min) {
  int tid = threadIdx.x, NT = blockDim.x;
  if (tid == 0) *sh_min = 1e300;
  __syncthreads();
  long long bo = 0, prev_x = -1;
  int prev_r0 = 0;
  T sg = (T)sigma;
  for (int j = 0; j < P.L; ++j) {
    int r0 = P.lp[j], r1 = P.lp[j + 1], b = r1 - r0;
    int bn = j + 1 < P.L ? P.lp[j + 2] - r1 : 0, bp = j > 0 ? r0 - prev_r0 : 0;
    T* S = Ssm ? Ssm : F + bo;
    const T* Xp = Xsm ? Xsm : F + prev_x;  // X_{j-1}: b_{j-1} x b
    for (int e = tid; e < b * b; e += NT) {
      int qa = e / b, t = e - qa * b;
      int a = r0 + qa;
      const int* cl = P.col + (long long)a * P.maxrow;
      const float* bv = P.B32 + (long long)a * P.maxrow;
      const float* cv = P.C32 + (long long)a * P.maxrow;
      int c_n = min(P.cnt[a], P.maxrow);
      T v = 0;
      for (int q = 0; q < c_n; ++q) {  // the entry of M formed only where it is used
        int c = cl[q];
        if (c == r0 + t) v += (T)bv[q] - sg * (T)cv[q];
        else if (j > 0 && c >= prev_r0 && c < r0) v -= ((T)bv[q] - sg * (T)cv[q]) * Xp[(long long)(c - prev_r0) * b + t];
      }
      S[e] = v;
    }
    __syncthreads();
    gj_inverse_nopiv<T>(S, b, sh_inv, sh_min);
    if (Ssm)
      for (int e = tid; e < b * b; e += NT) F[bo + e] = S[e];
    // G_j[q][c] = -sum_a S^{-1}[q][a] M[a][prev_r0 + c] and X_j[q][c] = sum_a S^{-1}[q][a] M[a][r1 + c]
    // (M symmetric: the entries of row prev_r0 + c, or r1 + c, that lie in level j)
    long long go = bo + (long long)b * b, xo = go + (long long)b * bp;
    for (int e = tid; e < b * (bp + bn); e += NT) {
      bool fwd = e < b * bp;
      int e2 = fwd ? e : e - b * bp, w = fwd ? bp : bn;
      int qt = e2 / w, cc = e2 - qt * w;
      int c = fwd ? prev_r0 + cc : r1 + cc;
      const int* cl = P.col + (long long)c * P.maxrow;
      const float* bv = P.B32 + (long long)c * P.maxrow;
      const float* cv = P.C32 + (long long)c * P.maxrow;
      int c_n = min(P.cnt[c], P.maxrow);
      T v = 0;
      for (int q = 0; q < c_n; ++q) {
        int a = cl[q];
        if (a >= r0 && a < r1) v += S[qt * b + (a - r0)] * ((T)bv[q] - sg * (T)cv[q]);
      }
      if (fwd) {
        F[go + e2] = -v;
      } else {
        F[xo + e2] = v;
        if (Xsm) Xsm[e2] = v;  // X_{j-1} is no longer read: the Schur complement above is complete
      }
    }
    __syncthreads();
    prev_x = xo;
    prev_r0 = r0;
    bo = xo + (long long)b * bn;
  }
  return *sh_min;
}

__device__ __forceinline__ unsigned lz_smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// Asynchronous 4-byte global -> shared copies (cp.async), one commit group per staged block.
__device__ __forceinline__ void lz_stage(float* dst, const float* src, int n) {
  for (int e = threadIdx.x; e < n; e += blockDim.x)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(lz_smem_u32(dst + e)), "l"(src + e) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void lz_stage_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Y = M^{-1} Y for LZ_P vectors (row-major nO x LZ_P, in shared memory) with the factors of lz_factor:
// forward  y_j = S_j^{-1} r_j + G_j y_{j-1};  backward  y_j -= X_j y_{j+1}.  One barrier per level step: the
// forward step writes y_j into one of two scratch blocks (tv: 2 x max_b x LZ_P) and the next step copies it
// into Y (whose level-j rows the step itself still reads as r_j); the backward step updates its own rows of
// Y in place from the finished rows of level j + 1.  Fb: two shared staging buffers of 2 max_b^2 floats (or
// null): each level's records are copied in by cp.async while the previous level computes.
__device__ void lz_solve(const OPen& P, const float* __restrict__ F, float* Y, float* tv, float* Fb, int max_b) {
  int tid = threadIdx.x, NT = blockDim.x, L = P.L;
  long long mb2 = 2LL * max_b * max_b, tvs = (long long)max_b * LZ_P;
  auto lvl = [&](int j, int& r0, int& b, int& bp, int& bn) {
    r0 = P.lp[j];
    b = P.lp[j + 1] - r0;
    bp = j > 0 ? r0 - P.lp[j - 1] : 0;
    bn = j + 1 < L ? P.lp[j + 2] - P.lp[j + 1] : 0;
  };
  long long fo = 0;
  int r0, b, bp, bn;
  lvl(0, r0, b, bp, bn);
  if (Fb) lz_stage(Fb, F, b * b);
  for (int j = 0; j < L; ++j) {
    lvl(j, r0, b, bp, bn);
    if (Fb) lz_stage_wait();
    __syncthreads();  // level j's records staged; y_{j-1} complete in tv[(j - 1) & 1]
    long long fn = fo + (long long)b * b + (long long)b * bp + (long long)b * bn;
    if (Fb && j + 1 < L) {
      int r0n, b1, bp1, bn1;
      lvl(j + 1, r0n, b1, bp1, bn1);
      lz_stage(Fb + ((j + 1) & 1) * mb2, F + fn, b1 * b1 + b1 * bp1);
    }
    const float* Sb = Fb ? Fb + (j & 1) * mb2 : F + fo;
    const float* Gb = Sb + (long long)b * b;
    const float* yp = tv + ((j + 1) & 1) * tvs;  // y_{j-1}
    float* yc = tv + (j & 1) * tvs;
    if (j > 0) {
      int pr0 = P.lp[j - 1];
      for (int e = tid; e < bp * LZ_P; e += NT) Y[pr0 * LZ_P + e] = yp[e];
    }
    for (int e = tid; e < b * LZ_P; e += NT) {
      int q = e / LZ_P, pc = e - q * LZ_P;
      const float* Sr = Sb + (long long)q * b;
      const float* Gr = Gb + (long long)q * bp;
      float acc0 = 0.f, acc1 = 0.f;
      int c = 0;
      for (; c + 1 < b; c += 2) {
        acc0 += Sr[c] * Y[(r0 + c) * LZ_P + pc];
        acc1 += Sr[c + 1] * Y[(r0 + c + 1) * LZ_P + pc];
      }
      if (c < b) acc0 += Sr[c] * Y[(r0 + c) * LZ_P + pc];
      for (c = 0; c + 1 < bp; c += 2) {
        acc0 += Gr[c] * yp[c * LZ_P + pc];
        acc1 += Gr[c + 1] * yp[(c + 1) * LZ_P + pc];
      }
      if (c < bp) acc0 += Gr[c] * yp[c * LZ_P + pc];
      yc[e] = acc0 + acc1;
    }
    fo = fn;
  }
  __syncthreads();
  for (int e = tid; e < b * LZ_P; e += NT) Y[r0 * LZ_P + e] = tv[((L - 1) & 1) * tvs + e];
  if (L < 2) {
    __syncthreads();
    return;
  }
  // backward, from level L - 2: fo walks back over the level sizes
  lvl(L - 1, r0, b, bp, bn);
  fo -= (long long)b * b + (long long)b * bp;  // start of level L - 1 (bn = 0)
  lvl(L - 2, r0, b, bp, bn);
  long long fj = fo - ((long long)b * b + (long long)b * bp + (long long)b * bn);
  if (Fb) lz_stage(Fb, F + fj + (long long)b * b + (long long)b * bp, b * bn);
  for (int j = L - 2, it = 0; j >= 0; --j, ++it) {
    lvl(j, r0, b, bp, bn);
    if (Fb) lz_stage_wait();
    __syncthreads();  // X_j staged; rows of level j + 1 final
    const float* Xm = Fb ? Fb + (it & 1) * mb2 : F + fj + (long long)b * b + (long long)b * bp;
    long long fp = 0;
    if (j > 0) {
      int r0p, b2, bp2, bn2;
      lvl(j - 1, r0p, b2, bp2, bn2);
      fp = fj - ((long long)b2 * b2 + (long long)b2 * bp2 + (long long)b2 * bn2);
      if (Fb) lz_stage(Fb + ((it + 1) & 1) * mb2, F + fp + (long long)b2 * b2 + (long long)b2 * bp2, b2 * bn2);
    }
    int r1 = r0 + b;
    for (int e = tid; e < b * LZ_P; e += NT) {
      int q = e / LZ_P, pc = e - q * LZ_P;
      const float* Xr = Xm + (long long)q * bn;
      float acc0 = 0.f, acc1 = 0.f;
      int c = 0;
      for (; c + 1 < bn; c += 2) {
        acc0 += Xr[c] * Y[(r1 + c) * LZ_P + pc];
        acc1 += Xr[c + 1] * Y[(r1 + c + 1) * LZ_P + pc];
      }
      if (c < bn) acc0 += Xr[c] * Y[(r1 + c) * LZ_P + pc];
      Y[(r0 + q) * LZ_P + pc] -= acc0 + acc1;
    }
    fj = fp;
  }
  __syncthreads();
}

// Y_out = C Y_in for LZ_P vectors (row-major nO x LZ_P); in and out distinct.
template <typename T>
__device__ void lz_cmul(const OPen& P, const T* Yin, T* Yout) {
  for (int e = threadIdx.x; e < P.nO * LZ_P; e += blockDim.x) {
    int a = e / LZ_P, pc = e - a * LZ_P;
    const int* cl = P.col + (long long)a * P.maxrow;
    const float* cv = P.C32 + (long long)a * P.maxrow;
    int c_n = min(P.cnt[a], P.maxrow);
    T acc = 0;
    for (int q = 0; q < c_n; ++q) acc += (T)cv[q] * Yin[cl[q] * LZ_P + pc];
    Yout[e] = acc;
  }
}

// Block-wide sums of NV floats (all threads get them); red: 32 * NV floats of shared memory.
template <int NV>
__device__ __forceinline__ void lz_block_sums(float (&v)[NV], float* red) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[w * NV + i] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    float t = 0;
    for (int q = 0; q < nw; ++q) t += red[q * NV + i];
    v[i] = t;
  }
  __syncthreads();
}

// One classical Gram-Schmidt pass of the block Y (nO x LZ_P, shared memory) against the C-orthonormal
// blocks Q_0 .. Q_{nb-1} (global, with their products C Q_i): Y -= Q_i (CQ_i^T Y).  A warp per block
// computes its LZ_P x LZ_P coefficients (coef, shared), then every thread updates its rows.
__device__ void lz_cgs_pass(int nO, int nb, const float* __restrict__ Qg, const float* __restrict__ CQg, float* Y,
                            float* coef) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long bs = (long long)nO * LZ_P;
  for (int i = warp; i < nb; i += nw) {
    const float4* cq = reinterpret_cast<const float4*>(CQg + i * bs);
    float acc[LZ_P][LZ_P];
#pragma unroll
    for (int p = 0; p < LZ_P; ++p)
#pragma unroll
      for (int q = 0; q < LZ_P; ++q) acc[p][q] = 0.f;
#pragma unroll 4
    for (int a = lane; a < nO; a += 32) {  // unrolled: several L2 loads in flight per lane
      float4 c4 = cq[a];
      float4 y4 = reinterpret_cast<const float4*>(Y)[a];
      float c[4] = {c4.x, c4.y, c4.z, c4.w}, y[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
      for (int p = 0; p < LZ_P; ++p)
#pragma unroll
        for (int q = 0; q < LZ_P; ++q) acc[p][q] += c[p] * y[q];
    }
#pragma unroll
    for (int p = 0; p < LZ_P; ++p)
#pragma unroll
      for (int q = 0; q < LZ_P; ++q) {
        float t = acc[p][q];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) coef[(i * LZ_P + p) * LZ_P + q] = t;
      }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < nO; a += blockDim.x) {
    float4 y4 = reinterpret_cast<float4*>(Y)[a];
    float y[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll 4
    for (int i = 0; i < nb; ++i) {
      float4 q4 = reinterpret_cast<const float4*>(Qg + i * bs)[a];
      float qv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
      for (int p = 0; p < LZ_P; ++p)
#pragma unroll
        for (int q = 0; q < LZ_P; ++q) y[q] -= qv[p] * coef[(i * LZ_P + p) * LZ_P + q];
    }
    reinterpret_cast<float4*>(Y)[a] = make_float4(y[0], y[1], y[2], y[3]);
  }
  __syncthreads();
}

// Seeded vector on the dof rows (zero on Gamma) into column pc of Y.
__device__ void lz_seed_column(const OPen& P, int s, int blk, int pc, int attempt, float* Y) {
  for (int a = threadIdx.x; a < P.nO; a += blockDim.x) {
    unsigned long long key = ((unsigned long long)s << 40) ^ ((unsigned long long)(blk * 16 + pc * 4 + attempt) << 24) ^
                             (unsigned long long)a;
    Y[a * LZ_P + pc] = P.o2i[a] >= 0 ? lz_hash_unit(key) : 0.f;
  }
}

// C-norm of column pc of Y (C Y written into column pc of CY).
__device__ float lz_cnorm_col(const OPen& P, const float* Y, float* CY, int pc, float* red) {
  float nv[1] = {0.f};
  for (int a = threadIdx.x; a < P.nO; a += blockDim.x) {
    const int* cl = P.col + (long long)a * P.maxrow;
    const float* cv = P.C32 + (long long)a * P.maxrow;
    int c_n = min(P.cnt[a], P.maxrow);
    float acc = 0;
    for (int q = 0; q < c_n; ++q) acc += cv[q] * Y[cl[q] * LZ_P + pc];
    CY[a * LZ_P + pc] = acc;
    nv[0] += acc * Y[a * LZ_P + pc];
  }
  lz_block_sums<1>(nv, red);
  return sqrtf(fmaxf(nv[0], 0.f));
}

// Projects column pc of Y (and of CY = C Y) against the C-orthonormal columns 0 .. pc-1 of the same block:
// one fused reduction gives their C inner products with Y_pc and Y_pc's own C-norm squared.  Returns the
// C-norm after the projection (all threads).
__device__ float lz_project_in_block(const OPen& P, float* Y, float* CY, int pc, float* red, float* before) {
  float v[LZ_P] = {0.f, 0.f, 0.f, 0.f};
  for (int a = threadIdx.x; a < P.nO; a += blockDim.x) {
    float y = Y[a * LZ_P + pc];
    for (int q = 0; q < pc; ++q) v[q] += CY[a * LZ_P + q] * y;
    v[LZ_P - 1] += CY[a * LZ_P + pc] * y;
  }
  lz_block_sums<LZ_P>(v, red);
  float n2 = v[LZ_P - 1];
  for (int q = 0; q < pc; ++q) n2 -= v[q] * v[q];
  if (before) *before = sqrtf(fmaxf(v[LZ_P - 1], 0.f));
  if (pc > 0) {
    for (int a = threadIdx.x; a < P.nO; a += blockDim.x) {
      float y = Y[a * LZ_P + pc], cy = CY[a * LZ_P + pc];
      for (int q = 0; q < pc; ++q) {
        y -= v[q] * Y[a * LZ_P + q];
        cy -= v[q] * CY[a * LZ_P + q];
      }
      Y[a * LZ_P + pc] = y;
      CY[a * LZ_P + pc] = cy;
    }
    __syncthreads();
  }
  return sqrtf(fmaxf(n2, 0.f));
}

// C-orthonormalises the columns of Y (after the block has been orthogonalised against the earlier
// blocks) and leaves C Y in CY.  C Y is formed once and then updated with Y.  Per column: a projection
// against the earlier columns of the block, repeated once when it removed more than half of the column
// (classical Gram-Schmidt twice), then a scaling.  ref[pc]: C-norm of column pc before any
// orthogonalisation.  A column whose C-norm falls below 1e-4 of it has collapsed into the span already
// built: it is replaced by a seeded vector, orthogonalised twice against every earlier block and column;
// if that keeps less than 1e-3 of its own norm, the column is set to zero (it then adds only a zero row
// and column to the Rayleigh quotient).
__device__ void lz_orthonormalise(const OPen& P, int s, int blk, int nb, const float* Qg, const float* CQg, float* Y,
                                  float* CY, const float* ref, float* coef, float* red) {
  lz_cmul(P, Y, CY);
  __syncthreads();
  for (int pc = 0; pc < LZ_P; ++pc) {
    float r0 = ref[pc];
    for (int attempt = 0; attempt < 2; ++attempt) {
      if (attempt == 1) {
        lz_seed_column(P, s, blk, pc, 1, Y);
        __syncthreads();
        r0 = lz_cnorm_col(P, Y, CY, pc, red);  // of the raw seed
        // the other columns are orthogonal to the earlier blocks already: the passes change them only by
        // rounding; column pc's C Y is formed again afterwards
        lz_cgs_pass(P.nO, nb, Qg, CQg, Y, coef);
        lz_cgs_pass(P.nO, nb, Qg, CQg, Y, coef);
        lz_cnorm_col(P, Y, CY, pc, red);
      }
      float before = 0.f;
      float nrm = lz_project_in_block(P, Y, CY, pc, red, &before);
      if (pc > 0 && nrm < 0.5f * before) nrm = lz_project_in_block(P, Y, CY, pc, red, nullptr);
      bool ok = nrm > (attempt == 0 ? 1e-4f : 1e-3f) * r0 && nrm > 0.f;
      if (ok || attempt == 1) {
        float inv = ok ? 1.f / nrm : 0.f;
        for (int a = threadIdx.x; a < P.nO; a += blockDim.x) {
          Y[a * LZ_P + pc] *= inv;
          CY[a * LZ_P + pc] *= inv;
        }
        __syncthreads();
        break;
      }
    }
  }
}

// Number of eigenvalues below x of the symmetric tridiagonal matrix with diagonal d and squared
// off-diagonal e2 (Sturm count, FP32).
__device__ int lz_sturm_below32(const float* d, const float* e2, int n, float x, float pivmin) {
  int c = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  c += q < 0.f;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// One CTA per subdomain.  Dynamic shared memory: Y (max_nO x 4) | C Y (max_nO x 4) | sweep scratch
// (2 max_b x 4) | the working block of the factorisation and X_{j-1} (2 max_b^2, when s_in_smem) | two
// staging buffers of the sweeps (2 x 2 max_b^2, when use_fb); once the Krylov steps are done the Rayleigh
// quotient (N x N
// doubles, N = 4 kdim[s]) reuses the same bytes.  When Yw is given, Y and C Y live there instead
// (2 nO x 4 floats at y_off[s]) and shared memory starts with the sweep scratch.
// CTA i works on subdomain sub_list[i].  Global workspace per subdomain: the factors (F + f_off[s]) and
// the basis Q, C Q and Op Q (3 kdim[s] blocks of nO x 4, Qw + q_off[s]), then FP32 copies of the rows of B^N
// and C (nO x maxrow each).
// Outputs: lam_hat[s * HK_MAXM + t] = the candidates below lam_cut in ascending order, cnt_out[s] their
// number, sigma_out[s] the shift used.
__global__ void __launch_bounds__(LZ_THREADS, 2) k_lanczos(
    const int* __restrict__ sub_info, const int* __restrict__ o_off, const int* __restrict__ O_levptr,
    const int* __restrict__ O_L, int maxrow, const int* __restrict__ ocnt, const int* __restrict__ ocol,
    const double* __restrict__ oB, const double* __restrict__ oC, const int* __restrict__ o2i,
    const int* __restrict__ sub_list, const int* __restrict__ kdim, const long long* __restrict__ f_off, float* F,
    const long long* __restrict__ q_off,
    float* Qw, float* Yw, const long long* __restrict__ y_off, int max_nO, int max_b, int s_in_smem, int use_fb,
    int nb0, double sigma0, double lam_cut, double* Tw, long long t_stride, int tcap,
    double* lam_hat, int* cnt_out, double* sigma_out, int* nb_out, DevStatus* st) {
  extern __shared__ __align__(16) unsigned char lz_smem[];
  __shared__ float coef[LZ_MAX_DIM * LZ_P];
  __shared__ float d32[LZ_MAX_DIM], e32[LZ_MAX_DIM];
  __shared__ float red[32 * LZ_P];
  __shared__ float ref[LZ_P];
  __shared__ float sh_inv;
  __shared__ double sh_min, sh_scal[4];
  __shared__ double hd[LZ_MAX_DIM], he[LZ_MAX_DIM], hv[LZ_MAX_DIM], hp[LZ_MAX_DIM];
  int s = sub_list[blockIdx.x], tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = NT >> 5;
  OPen P = open_sub(s, o_off, O_levptr, O_L, maxrow, ocnt, ocol, oB, oC, o2i, sub_info);
  // Y and C Y in shared memory, or (subdomains too large for it) in the global scratch Yw
  float* Ys = Yw ? Yw + y_off[s] : reinterpret_cast<float*>(lz_smem);
  float* CYs = Ys + (long long)(Yw ? P.nO : max_nO) * LZ_P;
  float* tv = Yw ? reinterpret_cast<float*>(lz_smem) : CYs + (long long)max_nO * LZ_P;  // 2 x max_b x LZ_P
  long long mb2 = (long long)max_b * max_b;
  float* Ssm = s_in_smem ? tv + 2LL * max_b * LZ_P : nullptr;
  float* Xsm = s_in_smem ? Ssm + mb2 : nullptr;
  float* Fb = use_fb ? tv + 2LL * max_b * LZ_P + (s_in_smem ? 2 * mb2 : 0) : nullptr;  // 2 x 2 max_b^2
  float* Fs = F + f_off[s];
  int nb_max = kdim[s], nb = min(nb0, nb_max);
  long long bs = (long long)P.nO * LZ_P;
  float* Qg = Qw + q_off[s];
  float* CQg = Qg + nb_max * bs;
  float* Wg = CQg + nb_max * bs;
  // FP32 copies of the pencil's rows (the sweeps, products with C and factorisations read them)
  {
    float* B32 = Wg + nb_max * bs;
    float* C32 = B32 + (long long)P.nO * maxrow;
    for (long long e = tid; e < (long long)P.nO * maxrow; e += NT) {
      int a = (int)(e / maxrow), q = (int)(e - (long long)a * maxrow);
      bool in = q < P.cnt[a];
      B32[e] = in ? (float)P.B[e] : 0.f;
      C32[e] = in ? (float)P.C[e] : 0.f;
    }
    P.B32 = B32;
    P.C32 = C32;
    __syncthreads();
  }

  // 1. a shift below the spectrum: M = B^N - sigma C positive definite
  double sigma = sigma0, step = 0.5, upper = 0.0;
  bool pd = false, bracket = false;
  for (int t = 0; t < LZ_SIGMA_TRIES && !pd; ++t) {
    double mp = lz_factor<float>(P, sigma, Fs, Ssm, Xsm, &sh_inv, &sh_min);
    __syncthreads();
    pd = mp > 0.0;
    if (!pd) {
      upper = sigma;
      bracket = true;
      sigma -= step;
      if (t >= 1) step *= 2.0;
    }
  }
  // closer to the spectrum (faster convergence): bisect between the definite and the indefinite shift,
  // then make sure the stored factors are those of the final shift
  bool factors_current = true;
  for (int t = 0; t < LZ_SIGMA_BISECT && pd && bracket; ++t) {
    double mid = 0.5 * (sigma + upper);
    double mp = lz_factor<float>(P, mid, Fs, Ssm, Xsm, &sh_inv, &sh_min);
    __syncthreads();
    if (mp > 0.0) {
      sigma = mid;
      factors_current = true;
    } else {
      upper = mid;
      factors_current = false;
    }
  }
  if (pd && !factors_current) {
    lz_factor<float>(P, sigma, Fs, Ssm, Xsm, &sh_inv, &sh_min);
    __syncthreads();
  }
  if (!pd) {
    if (tid == 0) {
      cnt_out[s] = 0;
      dev_fail(st, HK_EIG_FAIL, s, sigma);
    }
    return;
  }
  if (tid == 0) sigma_out[s] = sigma;

  // 2. seeded, C-orthonormal start block
  for (int pc = 0; pc < LZ_P; ++pc) lz_seed_column(P, s, 0, pc, 0, Ys);
  __syncthreads();
  for (int pc = 0; pc < LZ_P; ++pc) {
    float r = lz_cnorm_col(P, Ys, CYs, pc, red);
    if (tid == 0) ref[pc] = r;
  }
  __syncthreads();
  lz_orthonormalise(P, s, 0, 0, Qg, CQg, Ys, CYs, ref, coef, red);
  for (long long e = tid; e < bs; e += NT) {
    Qg[e] = Ys[e];
    CQg[e] = CYs[e];
  }
  __syncthreads();

  // 3. Krylov steps: W_k = Op Q_k, Q_{k+1} from W_k orthogonalised against Q_0 .. Q_k.  After nb blocks the
  // candidates below lam_cut are counted (steps 4 and 5); when a count c asks for more than the 4 nb
  // columns built (4 c + 48), the same sequence continues, up to nb_max blocks, and steps 4-5 repeat.
  int k_done = 0, N = 0;
  double th_hi_d = 0, pivmin_d = 0;
  while (true) {
  for (int k = k_done; k < nb; ++k) {
    for (long long e = tid; e < bs; e += NT) Ys[e] = CQg[k * bs + e];
    __syncthreads();
    lz_solve(P, Fs, Ys, tv, Fb, max_b);
    for (long long e = tid; e < bs; e += NT) Wg[k * bs + e] = Ys[e];
    __syncthreads();
    if (k == nb_max - 1) break;
    for (int pc = 0; pc < LZ_P; ++pc) {
      float r = lz_cnorm_col(P, Ys, CYs, pc, red);
      if (tid == 0) ref[pc] = r;
    }
    __syncthreads();
    lz_cgs_pass(P.nO, k + 1, Qg, CQg, Ys, coef);
    lz_cgs_pass(P.nO, k + 1, Qg, CQg, Ys, coef);
    lz_orthonormalise(P, s, k + 1, k + 1, Qg, CQg, Ys, CYs, ref, coef, red);
    for (long long e = tid; e < bs; e += NT) {
      Qg[(k + 1) * bs + e] = Ys[e];
      CQg[(k + 1) * bs + e] = CYs[e];
    }
    __syncthreads();
  }

  k_done = nb;
  // 4. Rayleigh quotient T = Q^T C (Op Q), a warp per pair of blocks; then symmetrised (FP64)
  N = nb * LZ_P;
  int ldT = N | 1;  // odd row stride (in doubles): row- and column-wise accesses of T hit distinct banks
  // T in the shared memory the vectors used (up to tcap columns), else in this block's global scratch
  double* Tm = N <= tcap ? reinterpret_cast<double*>(lz_smem) : Tw + (long long)blockIdx.x * t_stride;
  for (int pr = warp; pr < nb * nb; pr += nw) {
    int bi = pr / nb, bj = pr - bi * nb;
    const float4* cq = reinterpret_cast<const float4*>(CQg + bi * bs);
    const float4* wq = reinterpret_cast<const float4*>(Wg + bj * bs);
    float acc[LZ_P][LZ_P];
#pragma unroll
    for (int p = 0; p < LZ_P; ++p)
#pragma unroll
      for (int q = 0; q < LZ_P; ++q) acc[p][q] = 0.f;
#pragma unroll 4
    for (int a = lane; a < P.nO; a += 32) {
      float4 c4 = cq[a], w4 = wq[a];
      float c[4] = {c4.x, c4.y, c4.z, c4.w}, w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
      for (int p = 0; p < LZ_P; ++p)
#pragma unroll
        for (int q = 0; q < LZ_P; ++q) acc[p][q] += c[p] * w[q];
    }
#pragma unroll
    for (int p = 0; p < LZ_P; ++p)
#pragma unroll
      for (int q = 0; q < LZ_P; ++q) {
        float t = acc[p][q];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) Tm[(bi * LZ_P + p) * ldT + bj * LZ_P + q] = (double)t;
      }
  }
  __syncthreads();
  for (int e = tid; e < N * N; e += NT) {
    int i = e / N, j = e - i * N;
    if (i < j) {
      double v = 0.5 * (Tm[i * ldT + j] + Tm[j * ldT + i]);
      Tm[i * ldT + j] = v;
      Tm[j * ldT + i] = v;
    }
  }
  __syncthreads();

  // 5. Householder reduction of T to tridiagonal form (diagonal hd, off-diagonal he); warp 0 forms the
  // reflection's scalars by lane-parallel sums
  for (int k = 0; k + 2 < N; ++k) {
    if (warp == 0) {
      double ss = 0;
      for (int i = k + 2 + lane; i < N; i += 32) ss += Tm[i * ldT + k] * Tm[i * ldT + k];
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0) {
        double x0 = Tm[(k + 1) * ldT + k];
        hd[k] = Tm[k * ldT + k];
        if (ss == 0.0) {
          he[k] = x0;
          sh_scal[0] = 0.0;
        } else {
          double nrm = sqrt(x0 * x0 + ss), alpha = x0 > 0 ? -nrm : nrm, v0 = x0 - alpha;
          he[k] = alpha;
          sh_scal[0] = 2.0 / (v0 * v0 + ss);
          hv[k + 1] = v0;
        }
      }
    }
    __syncthreads();
    double beta = sh_scal[0];
    __syncthreads();  // every thread has read beta before warp 0 may overwrite it
    if (beta == 0.0) continue;
    for (int i = k + 2 + tid; i < N; i += NT) hv[i] = Tm[i * ldT + k];
    __syncthreads();
    // p = beta T v over rows k+1 .. N-1: two threads per row, each summing every other column
    for (int base = 0; base < 2 * (N - k - 1); base += NT) {
      int t2 = base + tid, i = k + 1 + (t2 >> 1);
      double acc = 0;
      if (i < N)
        for (int j = k + 1 + (t2 & 1); j < N; j += 2) acc += Tm[i * ldT + j] * hv[j];
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (i < N && !(t2 & 1)) hp[i] = beta * acc;
    }
    __syncthreads();
    if (warp == 0) {
      double kv = 0;
      for (int i = k + 1 + lane; i < N; i += 32) kv += hv[i] * hp[i];
      for (int o = 16; o > 0; o >>= 1) kv += __shfl_xor_sync(0xffffffffu, kv, o);
      if (lane == 0) sh_scal[1] = 0.5 * beta * kv;
    }
    __syncthreads();
    double kc = sh_scal[1];
    for (int i = k + 1 + tid; i < N; i += NT) hp[i] -= kc * hv[i];
    __syncthreads();
    // symmetric rank-2 update on the lower triangle, mirrored to the upper one
    int m = N - k - 1, tri = m * (m + 1) / 2;
    for (int e = tid; e < tri; e += NT) {
      int ii = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
      while (ii * (ii + 1) / 2 > e) --ii;
      while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
      int i = k + 1 + ii, j = k + 1 + (e - ii * (ii + 1) / 2);
      double v = Tm[i * ldT + j] - (hv[i] * hp[j] + hp[i] * hv[j]);
      Tm[i * ldT + j] = v;
      Tm[j * ldT + i] = v;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (N >= 2) {
      hd[N - 2] = Tm[(N - 2) * ldT + N - 2];
      he[N - 2] = Tm[(N - 1) * ldT + N - 2];
    }
    hd[N - 1] = Tm[(N - 1) * ldT + N - 1];
    he[N - 1] = 0.0;
    double hi = -1e300, me = 0;
    for (int i = 0; i < N; ++i) {
      double r = (i > 0 ? fabs(he[i - 1]) : 0.0) + (i < N - 1 ? fabs(he[i]) : 0.0);
      hi = fmax(hi, hd[i] + r);
      if (i < N - 1) me = fmax(me, he[i] * he[i]);
    }
    sh_scal[2] = hi + 1e-6 * fabs(hi) + 1e-30;
    sh_scal[3] = 1e-30 * fmax(1.0, me);
  }
  __syncthreads();
  th_hi_d = sh_scal[2];
  pivmin_d = sh_scal[3];
  // FP32 copy for the Sturm counts: diagonal and squared off-diagonal (the projected matrix is itself an
  // FP32 product)
  for (int i = tid; i < N; i += NT) {
    d32[i] = (float)hd[i];
    e32[i] = (float)(he[i] * he[i]);
  }
  __syncthreads();

  float th_cut = (float)(1.0 / (lam_cut - sigma)), th_hi = (float)th_hi_d, pivmin = (float)pivmin_d;
  int cnt = th_cut >= th_hi ? 0 : N - lz_sturm_below32(d32, e32, N, th_cut, pivmin);
  int need = (4 * cnt + 48 + LZ_P - 1) / LZ_P;
  __syncthreads();  // every thread has its count before the buffers are reused
  if (need <= nb || nb >= nb_max) break;
  nb = min(nb_max, need);
  }  // extension loop

  // 6. candidates: eigenvalues theta > 1 / (lam_cut - sigma) of T, lambda = sigma + 1 / theta, each found by
  // a warp by 32-way multisection on FP32 Sturm counts down to 2e-7 of the spectral scale
  float th_cut = (float)(1.0 / (lam_cut - sigma)), th_hi = (float)th_hi_d, pivmin = (float)pivmin_d;
  int cnt = th_cut >= th_hi ? 0 : N - lz_sturm_below32(d32, e32, N, th_cut, pivmin);
  if (tid == 0) {
    cnt_out[s] = cnt;
    nb_out[s] = nb;
    if (cnt > HK_MAXM) dev_fail(st, HK_UNSUPPORTED, s, cnt);
  }
  float tol = 2e-7f * fmaxf(fabsf(th_hi), fabsf(th_cut));
  for (int t = warp; t < cnt && t < HK_MAXM; t += nw) {
    int kidx = N - 1 - t;  // ascending index of the t-th largest theta
    float lo = th_cut, hi = th_hi;
    for (int it = 0; it < 12 && hi - lo > tol; ++it) {
      float x = lo + (hi - lo) * (float)(lane + 1) / 33.f;
      int below = lz_sturm_below32(d32, e32, N, x, pivmin) > kidx;  // eigenvalue kidx lies below x
      unsigned mask = __ballot_sync(0xffffffffu, below);
      int first = mask ? __ffs(mask) - 1 : 32;
      float nlo = first == 0 ? lo : lo + (hi - lo) * (float)first / 33.f;
      float nhi = first == 32 ? hi : lo + (hi - lo) * (float)(first + 1) / 33.f;
      lo = nlo;
      hi = nhi;
    }
    if (lane == 0) lam_hat[(long long)s * HK_MAXM + t] = sigma + 1.0 / (0.5 * ((double)lo + (double)hi));
  }
}

// ====================================================================== inertia (FP64)
// Block-wide (max |value|, its index) over the candidates each thread offers; ties go to the smaller
// index.  rv/ri: 32 entries of shared memory; the result is returned to every thread.
__device__ void bk_argmax(double v, int i, double* rv, int* ri, double* out_v, int* out_i) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) v = ov, i = oi;
  }
  __syncthreads();
  if (lane == 0) rv[w] = v, ri[w] = i;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bv = rv[0];
    int bi = ri[0];
    for (int q = 1; q < nw; ++q)
      if (rv[q] > bv || (rv[q] == bv && ri[q] < bi)) bv = rv[q], bi = ri[q];
    *out_v = bv;
    *out_i = bi;
  }
  __syncthreads();
}

// Swaps index i and j of the symmetric b x b matrix A (rows, then columns).
__device__ void bk_sym_swap(double* A, int b, int i, int j) {
  if (i == j) return;
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    double t = A[i * b + c];
    A[i * b + c] = A[j * b + c];
    A[j * b + c] = t;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < b; r += blockDim.x) {
    double t = A[r * b + i];
    A[r * b + i] = A[r * b + j];
    A[r * b + j] = t;
  }
  __syncthreads();
}

// Number of negative eigenvalues of the symmetric b x b matrix A (row-major, full storage; destroyed),
// from the Bunch-Kaufman factorisation P A P^T = L D L^T with 1x1 and 2x2 diagonal blocks (partial
// pivoting, alpha = (1 + sqrt 17) / 8): by Sylvester's law A and D have the same inertia, and a 2x2
// block [a b; b c] has one negative eigenvalue when ac - b^2 < 0, two when ac - b^2 > 0 and a + c < 0.
// A zero column is a zero eigenvalue (not counted).  Returns the count to every thread.
__device__ int bk_neg_count(double* A, int b, double* rv, int* ri, double* shd, int* shi) {
  const double alpha = 0.6403882032022076;  // (1 + sqrt(17)) / 8
  int tid = threadIdx.x, NT = blockDim.x;
  if (tid == 0) shi[2] = 0;  // negative count
  int k = 0;
  while (k < b) {
    // column k below the diagonal: largest entry and its row
    double cv = 0.0;
    int ci = b;
    for (int i = k + 1 + tid; i < b; i += NT) {
      double a = fabs(A[i * b + k]);
      if (a > cv || (a == cv && i < ci)) cv = a, ci = i;
    }
    bk_argmax(cv, ci, rv, ri, &shd[0], &shi[0]);
    double colmax = shd[0], akk = fabs(A[k * b + k]);
    int r = shi[0];
    bool need_row = fmax(akk, colmax) > 0.0 && akk < alpha * colmax;
    double rowmax = 0.0;
    if (need_row) {
      double rvv = 0.0;
      int rii = b;
      for (int j = k + tid; j < b; j += NT) {
        if (j == r) continue;
        double a = fabs(A[r * b + j]);
        if (a > rvv || (a == rvv && j < rii)) rvv = a, rii = j;
      }
      bk_argmax(rvv, rii, rv, ri, &shd[1], &shi[1]);
      rowmax = shd[1];
    }
    int kind, swap_from = -1, swap_to = -1;
    if (fmax(akk, colmax) == 0.0) kind = 0;
    else if (!need_row || akk * rowmax >= alpha * colmax * colmax) kind = 1;
    else if (fabs(A[r * b + r]) >= alpha * rowmax) kind = 1, swap_from = r, swap_to = k;
    else kind = 2, swap_from = r, swap_to = k + 1;
    // every thread has taken its decision (read A[r][r]) before the swap or the elimination writes
    __syncthreads();
    if (swap_from >= 0) bk_sym_swap(A, b, swap_to, swap_from);
    if (kind == 0) {
      k += 1;
      continue;
    }
    if (kind == 1) {
      double d = A[k * b + k];
      if (tid == 0 && d < 0.0) shi[2] += 1;
      double inv = 1.0 / d;
      int m = b - k - 1;
      for (int e = tid; e < m * m; e += NT) {
        int i = k + 1 + e / m, j = k + 1 + e % m;
        A[i * b + j] -= A[i * b + k] * inv * A[k * b + j];
      }
      __syncthreads();
      k += 1;
    } else {
      double a = A[k * b + k], bb = A[(k + 1) * b + k], c = A[(k + 1) * b + k + 1];
      double det = a * c - bb * bb;
      if (tid == 0) shi[2] += det < 0.0 ? 1 : (a + c < 0.0 ? (det > 0.0 ? 2 : 1) : 0);
      double i00 = c / det, i01 = -bb / det, i11 = a / det;
      int m = b - k - 2;
      for (int e = tid; e < m * m; e += NT) {
        int i = k + 2 + e / m, j = k + 2 + e % m;
        double x0 = A[i * b + k], x1 = A[i * b + k + 1];
        double y0 = A[k * b + j], y1 = A[(k + 1) * b + j];
        A[i * b + j] -= x0 * (i00 * y0 + i01 * y1) + x1 * (i01 * y0 + i11 * y1);
      }
      __syncthreads();
      k += 2;
    }
  }
  __syncthreads();
  int neg = shi[2];
  __syncthreads();
  return neg;
}

// #{lambda < tau} of subdomain s (one CTA each): block LDL^T of B^N - tau C over the ovdof level sets,
// #neg of every Schur complement D_j by bk_neg_count, D_j^{-1} by Gauss-Jordan with partial pivoting
// (a pivot below 1e-14 max|M| is replaced by +-1e-14 max|M|: the count is then that of a matrix within
// rounding of it).  Work blocks (D_j, its copy, X_{j-1} = D_{j-1}^{-1} M_{j-1,j} and X_j, max_b^2 each)
// sit in shared memory when in_smem, else in the subdomain's part of ws (ws_off).
__global__ void __launch_bounds__(256) k_inertia(
    const int* __restrict__ sub_info, const int* __restrict__ o_off, const int* __restrict__ O_levptr,
    const int* __restrict__ O_L, int maxrow, const int* __restrict__ ocnt, const int* __restrict__ ocol,
    const double* __restrict__ oB, const double* __restrict__ oC, const int* __restrict__ o2i, double tau,
    int max_b, int in_smem, const long long* __restrict__ ws_off, double* ws, int* neg_out) {
  extern __shared__ __align__(16) double in_smem_buf[];
  __shared__ int piv[HK_MAXB];
  __shared__ double rv[32], shd[4], minpiv;
  __shared__ int ri[32], shi[4];
  int s = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
  OPen P = open_sub(s, o_off, O_levptr, O_L, maxrow, ocnt, ocol, oB, oC, o2i, sub_info);
  long long mb2 = (long long)max_b * max_b;
  double* base = in_smem ? in_smem_buf : ws + ws_off[s];
  double* S = base;
  double* Sc = base + mb2;
  double* Xp = base + 2 * mb2;
  double* Xn = base + 3 * mb2;
  // scale for the pivot floor
  double mx = 0;
  for (long long e = tid; e < (long long)P.nO * P.maxrow; e += NT) {
    int a = (int)(e / P.maxrow), q = (int)(e % P.maxrow);
    if (q < P.cnt[a]) mx = fmax(mx, fabs(P.B[e] - tau * P.C[e]));
  }
  bk_argmax(mx, 0, rv, ri, &shd[3], &shi[3]);
  double floor_piv = 1e-14 * shd[3];
  int neg = 0, prev_r0 = 0;
  for (int j = 0; j < P.L; ++j) {
    int r0 = P.lp[j], r1 = P.lp[j + 1], b = r1 - r0;
    int bn = j + 1 < P.L ? P.lp[j + 2] - r1 : 0;
    for (int e = tid; e < b * b; e += NT) {
      int qa = e / b, t = e - qa * b;
      int a = r0 + qa;
      const int* cl = P.col + (long long)a * P.maxrow;
      const double* bv = P.B + (long long)a * P.maxrow;
      const double* cv = P.C + (long long)a * P.maxrow;
      int c_n = min(P.cnt[a], P.maxrow);
      double v = 0;
      for (int q = 0; q < c_n; ++q) {  // the entry of M = B^N - tau C formed only where it is used
        int c = cl[q];
        if (c == r0 + t) v += bv[q] - tau * cv[q];
        else if (j > 0 && c >= prev_r0 && c < r0) v -= (bv[q] - tau * cv[q]) * Xp[(long long)(c - prev_r0) * b + t];
      }
      S[e] = v;
      Sc[e] = v;
    }
    __syncthreads();
    // D_j is symmetric up to rounding: count on its symmetric part
    for (int e = tid; e < b * b; e += NT) {
      int i = e / b, t = e - i * b;
      if (i < t) {
        double v = 0.5 * (Sc[i * b + t] + Sc[t * b + i]);
        Sc[i * b + t] = v;
        Sc[t * b + i] = v;
      }
    }
    __syncthreads();
    neg += bk_neg_count(Sc, b, rv, ri, shd, shi);
    if (bn > 0) {
      if (tid == 0) minpiv = 1e300;
      __syncthreads();
      gauss_jordan_inverse(S, b, piv, rv, ri, &minpiv, floor_piv);
      for (int e = tid; e < b * bn; e += NT) {
        int qt = e / bn, cc = e - qt * bn;
        int c = r1 + cc;
        const int* cl = P.col + (long long)c * P.maxrow;
        const double* bv = P.B + (long long)c * P.maxrow;
        const double* cv = P.C + (long long)c * P.maxrow;
        int c_n = min(P.cnt[c], P.maxrow);
        double v = 0;
        for (int q = 0; q < c_n; ++q) {
          int a = cl[q];
          if (a >= r0 && a < r1) v += S[qt * b + (a - r0)] * (bv[q] - tau * cv[q]);
        }
        Xn[e] = v;
      }
      __syncthreads();
      double* t = Xp;
      Xp = Xn;
      Xn = t;
    }
    prev_r0 = r0;
  }
  if (tid == 0) neg_out[s] = neg;
}

// ====================================================================== host
hk_status eigen_inertia(hk_handle* h, const OvdofPencil& op, double tau, int* d_neg, cudaStream_t st) {
  int ns = h->n_sub;
  size_t need = sizeof(double) * 4 * (size_t)op.max_b * op.max_b;
  int in_smem = need <= 200 * 1024;
  double* d_ws = nullptr;
  long long* d_wo = nullptr;
  if (!in_smem) {
    std::vector<long long> wo(ns);
    for (int s = 0; s < ns; ++s) wo[s] = 4LL * op.max_b * op.max_b * s;
    // allocated on the setup stream, which the caller has forked the inertia stream from afterwards
    HK_TRY(dalloc(h, &d_ws, 4ULL * op.max_b * op.max_b * ns));
    HK_TRY(dalloc(h, &d_wo, ns));
    HK_CUDA(cudaMemcpyAsync(d_wo, wo.data(), 8 * ns, cudaMemcpyHostToDevice, h->stream));
    if (st != h->stream) {
      HK_CUDA(cudaEventRecord(h->ev_fork, h->stream));
      HK_CUDA(cudaStreamWaitEvent(st, h->ev_fork, 0));
    }
  }
  HK_TRY(hk_allow_smem(k_inertia));
  HK_TRY(hk_max_carveout(k_inertia));  // runs beside the Lanczos blocks
  {
    // algorithmic FMAs: per level Gauss-Jordan (b^3) and Bunch-Kaufman (b^3 / 3)
    double fma = 0;
    for (int s = 0; s < ns; ++s) {
      const int* lp = &op.h_levptr[op.h_off[s] + s];
      for (int j = 0; j < op.h_L[s]; ++j) {
        double b = lp[j + 1] - lp[j];
        fma += b * b * b * (4.0 / 3.0);
      }
    }
    h->eigen_gflop[0] = 2.0 * fma * 1e-9;
  }
  k_inertia<<<ns, 256, in_smem ? need : 0, st>>>(h->d_sub_info, op.o_off, op.levptr, op.L, op.maxrow, op.cnt, op.col,
                                                  op.B, op.C, op.o2i, tau, op.max_b, in_smem, d_wo, d_ws, d_neg);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  if (!in_smem) {
    // freed on the inertia stream once the kernel is done (stream-ordered)
    h->allocs.erase(std::remove_if(h->allocs.begin(), h->allocs.end(),
                                   [&](const std::pair<void*, size_t>& a) {
                                     if (a.first == d_ws || a.first == d_wo) {
                                       h->bytes -= a.second;
                                       return true;
                                     }
                                     return false;
                                   }),
                    h->allocs.end());
    cudaFreeAsync(d_ws, st);
    cudaFreeAsync(d_wo, st);
  }
  return HK_OK;
}

hk_status eigen_lanczos(hk_handle* h, const OvdofPencil& op, const std::vector<int>& cols, int cols0,
                        double lam_cut, double* d_lamhat, int* d_cnt, float* ms) {
  cudaStream_t st = h->stream;
  int ns = h->n_sub;
  std::vector<int> kd(ns, 0), list;
  std::vector<long long> fo(ns, 0), qo(ns, 0);
  long long ftot = 0, qtot = 0;
  int kmax = 1;
  for (int s = 0; s < ns; ++s) {
    if (cols[s] <= 0) continue;
    list.push_back(s);
    // no more columns than the dof space holds (plus a block for the collapsed ones)
    int c = std::min(std::min(LZ_MAX_DIM, cols[s]), 4 * ((h->subs[s].nI + 3) / 4) + 4);
    kd[s] = std::max(2, (c + LZ_P - 1) / LZ_P);
    kmax = std::max(kmax, kd[s]);
    const int* lp = &op.h_levptr[op.h_off[s] + s];
    long long f = 0;
    for (int j = 0; j < op.h_L[s]; ++j) {
      long long b = lp[j + 1] - lp[j], bn = j + 1 < op.h_L[s] ? lp[j + 2] - lp[j + 1] : 0;
      long long bp = j > 0 ? lp[j] - lp[j - 1] : 0;
      f += b * b + b * bp + b * bn;  // S_j^{-1}, G_j, X_j
    }
    fo[s] = ftot;
    ftot += (f + 3) & ~3LL;
    qo[s] = qtot;
    qtot += 3LL * kd[s] * op.h_nO[s] * LZ_P + ((2LL * op.h_nO[s] * op.maxrow + 3) & ~3LL);  // 16-byte aligned
  }
  *ms = 0;
  if (list.empty()) return HK_OK;
  int nl = (int)list.size();
  int *d_kd = nullptr, *d_list = nullptr;
  long long *d_fo = nullptr, *d_qo = nullptr;
  float *d_F = nullptr, *d_Q = nullptr;
  double* d_sig = nullptr;
  HK_TRY(dalloc(h, &d_kd, ns));
  HK_TRY(dalloc(h, &d_list, nl));
  HK_TRY(dalloc(h, &d_fo, ns));
  HK_TRY(dalloc(h, &d_qo, ns));
  HK_TRY(dalloc(h, &d_F, ftot));
  HK_TRY(dalloc(h, &d_Q, qtot));
  HK_TRY(dalloc(h, &d_sig, ns));
  int* d_nb = nullptr;
  HK_TRY(dalloc(h, &d_nb, ns));
  HK_CUDA(cudaMemcpyAsync(d_kd, kd.data(), 4 * ns, cudaMemcpyHostToDevice, st));
  HK_CUDA(cudaMemcpyAsync(d_list, list.data(), 4 * nl, cudaMemcpyHostToDevice, st));
  HK_CUDA(cudaMemcpyAsync(d_fo, fo.data(), 8 * ns, cudaMemcpyHostToDevice, st));
  HK_CUDA(cudaMemcpyAsync(d_qo, qo.data(), 8 * ns, cudaMemcpyHostToDevice, st));
  size_t vec = sizeof(float) * LZ_P * (2 * (size_t)op.max_nO + 2 * (size_t)op.max_b);
  size_t sblk = sizeof(float) * (size_t)op.max_b * op.max_b;
  float* d_Y = nullptr;
  long long* d_yo = nullptr;
  if (vec > 120 * 1024) {
    // the vectors of large subdomains go to global memory
    std::vector<long long> yo(ns, 0);
    long long ytot = 0;
    for (int s : list) {
      yo[s] = ytot;
      ytot += 2LL * op.h_nO[s] * LZ_P;
    }
    HK_TRY(dalloc(h, &d_Y, ytot));
    HK_TRY(dalloc(h, &d_yo, ns));
    HK_CUDA(cudaMemcpyAsync(d_yo, yo.data(), 8 * ns, cudaMemcpyHostToDevice, st));
    vec = sizeof(float) * LZ_P * 2 * (size_t)op.max_b;
  }
  // the Rayleigh quotient (N x (N | 1) doubles) in shared memory up to LZ_T_SMEM columns, beyond in a global
  // scratch: a block that needs the whole shared memory waits for an empty SM, and the setup kernels beside
  // this one occupy most of them
  int tcap = std::min(kmax * LZ_P, LZ_T_SMEM);
  size_t tmat = sizeof(double) * (size_t)tcap * (tcap | 1);
  double* d_T = nullptr;
  long long t_stride = 0;
  if (kmax * LZ_P > tcap) {
    t_stride = (long long)(kmax * LZ_P) * ((kmax * LZ_P) | 1);
    HK_TRY(dalloc(h, &d_T, (size_t)t_stride * nl));
  }
  int s_in_smem = vec + 2 * sblk <= 200 * 1024;  // S and X_{j-1} of the factorisation
  int use_fb = vec + (s_in_smem ? 2 * sblk : 0) + 4 * sblk <= 200 * 1024;  // two record stages of 2 max_b^2
  size_t shm = std::max(vec + (s_in_smem ? 2 * sblk : 0) + (use_fb ? 4 * sblk : 0), tmat);
  if (shm > 220 * 1024) {
    hk_set_error("subdomain with %d ovdof rows too large for the Lanczos kernel's shared memory", op.max_nO);
    return HK_UNSUPPORTED;
  }
  HK_TRY(hk_allow_smem(k_lanczos));
  HK_TRY(hk_max_carveout(k_lanczos));
  cudaEvent_t e0, e1;
  HK_CUDA(cudaEventCreate(&e0));
  HK_CUDA(cudaEventCreate(&e1));
  cudaEventRecord(e0, st);
  k_lanczos<<<nl, LZ_THREADS, shm, st>>>(h->d_sub_info, op.o_off, op.levptr, op.L, op.maxrow, op.cnt, op.col, op.B,
                                         op.C, op.o2i, d_list, d_kd, d_fo, d_F, d_qo, d_Q, d_Y, d_yo, op.max_nO, op.max_b,
                                         s_in_smem,
                                         use_fb, (cols0 + LZ_P - 1) / LZ_P, -0.5, lam_cut, d_T, t_stride, tcap,
                                         d_lamhat, d_cnt, d_sig, d_nb, h->d_status);
  HK_COUNT_LAUNCH();
  cudaEventRecord(e1, st);
  HK_LAUNCH_CHECK();
  HK_CUDA(cudaEventSynchronize(e1));
  cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // algorithmic FMAs of the launch (dense level operations; the sparse products are small beside them):
  // the factorisation at the final shift (Gauss-Jordan, b^3 per level), every Krylov step (a sweep with 4
  // right-hand sides, C Q, two Gram-Schmidt passes over the earlier blocks), the projection (N^2 nO) and the
  // FP64 Householder reduction (4 N^3 / 3)
  std::vector<int> nbv(ns);
  HK_CUDA(cudaMemcpy(nbv.data(), d_nb, 4 * ns, cudaMemcpyDeviceToHost));
  double fma = 0;
  for (int s : list) {
    const int* lp = &op.h_levptr[op.h_off[s] + s];
    double fac = 0, sweep = 0;
    for (int j = 0; j < op.h_L[s]; ++j) {
      double b = lp[j + 1] - lp[j], bn = j + 1 < op.h_L[s] ? lp[j + 2] - lp[j + 1] : 0;
      double bp = j > 0 ? lp[j] - lp[j - 1] : 0;
      fac += b * b * b + b * b * (bp + bn);
      sweep += (b * b + b * bp + b * bn) * LZ_P;
    }
    double nO = op.h_nO[s], nbs = nbv[s], N = nbs * LZ_P;
    fma += fac + nbs * (sweep + 28.0 * nO) + 2.0 * 32.0 * nO * nbs * (nbs + 1) / 2.0 + N * N * nO +
           4.0 * N * N * N / 3.0;
  }
  h->eigen_gflop[1] += 2.0 * fma * 1e-9;
  void* tmp[] = {d_kd, d_list, d_fo, d_qo, d_F, d_Q, d_sig, d_nb, d_Y, d_yo, d_T};
  for (void* p : tmp) dfree(h, p);
  return HK_OK;
}
