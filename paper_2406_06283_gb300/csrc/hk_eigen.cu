// H_k-GenEO local eigenproblems (Eq. 5.12) and the coarse basis (Def. 5.1).
//
// On ovdof(Omega_i) the problem is B^N p = lambda C p with B^N the local
// Neumann Helmholtz matrix (element sums over Omega_i) and C = Xi D^N Xi,
// Xi = diag(1/mu on dof, 0 on Gamma = ovdof \ dof).  For dof rows and
// columns B^N and D^N equal the global B and D_k (the star of a dof lies in
// Omega_i); only the Gamma-Gamma block of B^N is local.  Eliminating the
// Gamma unknowns (C vanishes there) gives the symmetric-definite pencil
//     S p = lambda C_II p,   S = B_II - B_IG (B^N_GG)^{-1} B_GI,  C_II = X D_II X,  X = diag(1/mu),
// whose eigenvalues are real (the paper's lemma on indefinite pencils).
//
// The pencil is never formed densely.  Three steps, all on the sparse rows of (B^N, C) over ovdof in
// its level-set order (block tridiagonal), FP64 wherever the result is kept:
//  1. FP64 count m_tau = #{lambda < tau} by inertia (hk_lanczos.cu, k_inertia).
//  2. FP32 candidates below tau + delta (delta = 0.05) by shift-invert block Lanczos at a shift below the
//     spectrum (hk_lanczos.cu, k_lanczos); the basis is sized from m_tau.
//  3. FP64 refinement on the sparse pencil.  Candidates closer than 1e-3 max(1,|lambda|) form a
//     cluster; for each cluster the block-tridiagonal LU of B^N - sigma C over level sets of
//     ovdof(Omega_i) is formed in FP64 (sigma = the cluster's mean candidate), a seeded block of
//     cluster size + 2 guard vectors takes block inverse iteration (3 steps for a single candidate, 6 for
//     a cluster)
//     ((B^N - sigma C)^{-1} C, C-orthonormalised after each step; the contraction per step is
//     |lambda - sigma| over the distance to the next eigenvalue outside the block), and a Rayleigh-Ritz
//     step on B^N gives FP64 eigenpairs; the window of Ritz values closest to the cluster's candidates
//     is kept.  The Gamma part of each iterate satisfies the Gamma rows of the pencil exactly, so
//     x^T B^N x = x_I^T S x_I.
// The number of refined values below tau must equal m_tau (HK_EIG_FAIL otherwise).
// Selection then keeps lambda < tau on the FP64 values, extending across ties (gap <= 1e-8 max(1,|tau|)),
// and the coarse vectors are Xi p = p / mu on dof(Omega_i), c-normalised (Def. 5.1).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "hk_internal.cuh"

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

#define HK_EIG_DELTA 0.05
#define LZ_BASIS_MAX 160  // largest Krylov basis of the Lanczos candidates (hk_lanczos.cu)
#define HK_CLUSTER_GAP 1e-3
#define HK_MAX_CLUSTER 32
#define HK_REFINE_STEPS 6          // block inverse-iteration steps of a cluster of candidates
#define HK_REFINE_STEPS_SINGLE 3   // ... of a single candidate
#define HK_GUARD 2
#define HK_MAX_BLOCK (HK_MAX_CLUSTER + HK_GUARD)

// ---- 1. B^N on Gamma x Gamma: element sums over the subdomain's elements.
__global__ void k_gamma_block(int dim, int ne, const double* __restrict__ xyz, const int* __restrict__ elems,
                              const double* __restrict__ coeff, double k2, const int* __restrict__ node_of_dof,
                              const int* __restrict__ dof_of_node, const int* __restrict__ ne_ptr,
                              const int* __restrict__ ne_idx, const uint8_t* __restrict__ elem_in,
                              const int* __restrict__ sub_info, const int* __restrict__ G,
                              const long long* __restrict__ ws_G, double* ws) {
  int s = blockIdx.x;
  const int* si = sub_info + 8 * s;
  int nG = si[1], goff = si[4];
  const int* Gs = G + goff;
  double* BG = ws + ws_G[s];
  int nv = dim + 1;
  double mdiag = 2.0 / (nv * (nv + 1)), moff = 1.0 / (nv * (nv + 1));
  const uint8_t* ein = elem_in + (long long)s * ne;
  for (int e = threadIdx.x; e < nG * nG; e += blockDim.x) BG[e] = 0.0;
  __syncthreads();
  for (int gi = threadIdx.x; gi < nG; gi += blockDim.x) {
    int v = node_of_dof[Gs[gi]];
    for (int q = ne_ptr[v]; q < ne_ptr[v + 1]; ++q) {
      int e = ne_idx[q];
      if (!ein[e]) continue;
      int vid[4], iv = 0;
      for (int j = 0; j < nv; ++j) {
        vid[j] = elems[e * nv + j];
        if (vid[j] == v) iv = j;
      }
      double g[4][3];
      double vol = simplex_geometry(dim, xyz, vid, g);
      double a = coeff[e];
      for (int j = 0; j < nv; ++j) {
        int d = dof_of_node[vid[j]];
        if (d < 0) continue;
        int gj = bsearch_int(Gs, nG, d);
        if (gj < 0) continue;
        double dot = 0;
        for (int c = 0; c < dim; ++c) dot += g[iv][c] * g[j][c];
        BG[(long long)gi * nG + gj] += a * vol * dot - k2 * vol * (j == iv ? mdiag : moff);
      }
    }
  }
}

// Deterministic start vectors for the refinement: SplitMix64 finaliser of a key, mapped to [-0.5, 0.5).
__device__ float hash_unitf(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  x ^= x >> 31;
  return (float)((double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5);
}

// ---- 8. ovdof(Omega_i) = dof U Gamma: merged sorted list, membership and index in dof / Gamma.
__global__ void k_o_merge(const int* __restrict__ sub_info, const int* __restrict__ Isorted,
                          const int* __restrict__ G, const int* __restrict__ o_off, int* O, int* o_kind) {
  int s = blockIdx.x;
  if (threadIdx.x != 0) return;
  const int* si = sub_info + 8 * s;
  int nI = si[0], nG = si[1], ioff = si[3], goff = si[4], oo = o_off[s];
  int a = 0, b = 0, k = 0;
  while (a < nI || b < nG) {
    bool takeI = b >= nG || (a < nI && Isorted[ioff + a] < G[goff + b]);
    if (takeI) {
      O[oo + k] = Isorted[ioff + a];
      o_kind[oo + k] = a;  // >= 0: index in the sorted dof list
      ++a;
    } else {
      O[oo + k] = G[goff + b];
      o_kind[oo + k] = -1 - b;  // < 0: -(1 + index in the Gamma list)
      ++b;
    }
    ++k;
  }
}

// Local CSR of B^N and C over ovdof in its level order (capacity maxrow per row).  B^N: global B
// where a dof is involved, the element sums over the subdomain (BG, dense) on Gamma x Gamma.
// C = X D X on dof x dof, 0 elsewhere.  o2i: level position of each ovdof row in the dof level order
// (-1 on Gamma).
__global__ void k_o_csr(const int* __restrict__ sub_info, const int* __restrict__ o_off,
                        const int* __restrict__ O, const int* __restrict__ o_kind, const int* __restrict__ O_perm,
                        const int* __restrict__ O_lev, const int* __restrict__ perm_I,
                        const int* __restrict__ rowptr, const int* __restrict__ col, const double* __restrict__ valB,
                        const double* __restrict__ valD, const int* __restrict__ mu,
                        const long long* __restrict__ wsG, const double* __restrict__ ws, int maxrow, int* ocnt,
                        int* ocol, double* oB, double* oC, int* o2i) {
  int s = blockIdx.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], nG = si[1], ioff = si[3];
  int oo = o_off[s], nO = nI + nG;
  const double* BG = ws + wsG[s];
  for (int a = threadIdx.x; a < nO; a += blockDim.x) {
    int g = O_lev[oo + a];
    int gi = bsearch_int(O + oo, nO, g);
    int kg = o_kind[oo + gi];
    o2i[oo + a] = kg >= 0 ? perm_I[ioff + kg] : -1;
    long long base = (long long)(oo + a) * maxrow;
    int c = 0;
    for (int q = rowptr[g]; q < rowptr[g + 1]; ++q) {
      int h = col[q];
      int hi = bsearch_int(O + oo, nO, h);
      if (hi < 0) continue;
      int kh = o_kind[oo + hi];
      double b;
      if (kg >= 0 || kh >= 0) b = valB[q];
      else b = BG[(long long)(-1 - kg) * nG + (-1 - kh)];
      double cval = (kg >= 0 && kh >= 0) ? valD[q] / ((double)mu[g] * (double)mu[h]) : 0.0;
      if (c < maxrow) {
        ocol[base + c] = O_perm[oo + hi];
        oB[base + c] = b;
        oC[base + c] = cval;
      }
      ++c;
    }
    ocnt[oo + a] = c;
  }
}

// Small symmetric eigenproblem by cyclic Jacobi (one thread): A (p x p, row-major, destroyed),
// eigenvalues ascending in w, eigenvectors as columns of U.
__device__ void jacobi_eig(double* A, double* U, double* w, int p) {
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) U[i * p + j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0, dia = 0;
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) (i == j ? dia : off) += A[i * p + j] * A[i * p + j];
    if (off <= 1e-30 * dia || off == 0.0) break;
    for (int i = 0; i < p; ++i)
      for (int j = i + 1; j < p; ++j) {
        double aij = A[i * p + j];
        if (aij == 0.0) continue;
        double th = (A[j * p + j] - A[i * p + i]) / (2 * aij);
        double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < p; ++k) {
          double aki = A[k * p + i], akj = A[k * p + j];
          A[k * p + i] = c * aki - sn * akj;
          A[k * p + j] = sn * aki + c * akj;
        }
        for (int k = 0; k < p; ++k) {
          double aik = A[i * p + k], ajk = A[j * p + k];
          A[i * p + k] = c * aik - sn * ajk;
          A[j * p + k] = sn * aik + c * ajk;
        }
        for (int k = 0; k < p; ++k) {
          double uki = U[k * p + i], ukj = U[k * p + j];
          U[k * p + i] = c * uki - sn * ukj;
          U[k * p + j] = sn * uki + c * ukj;
        }
      }
  }
  for (int i = 0; i < p; ++i) w[i] = A[i * p + i];
  // sort ascending (selection sort on columns)
  for (int i = 0; i < p; ++i) {
    int b = i;
    for (int j = i + 1; j < p; ++j)
      if (w[j] < w[b]) b = j;
    if (b != i) {
      double t = w[i]; w[i] = w[b]; w[b] = t;
      for (int k = 0; k < p; ++k) {
        double u = U[k * p + i]; U[k * p + i] = U[k * p + b]; U[k * p + b] = u;
      }
    }
  }
}

// Deterministic block-wide dot product of two device vectors.
__device__ double block_dot(const double* x, const double* y, int n, double* red) {
  double acc = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += x[i] * y[i];
  return block_sum(acc, red);
}

// y = M x for the sparse ovdof matrix M = (which ? C : B^N) - shift C, p vectors (rows in level order).
__device__ void o_matvec(int nO, int oo, int maxrow, const int* ocnt, const int* ocol, const double* oB,
                         const double* oC, double shift, int use_B, const double* X, double* Y, int p) {
  for (int e = threadIdx.x; e < nO * p; e += blockDim.x) {
    int t = e / nO, a = e % nO;
    long long base = (long long)(oo + a) * maxrow;
    int c = min(ocnt[oo + a], maxrow);
    double acc = 0;
    for (int q = 0; q < c; ++q) {
      double v = (use_B ? oB[base + q] : 0.0) + shift * oC[base + q];
      acc += v * X[(long long)t * nO + ocol[base + q]];
    }
    Y[(long long)t * nO + a] = acc;
  }
}

// ---- 9. FP64 refinement of one cluster of candidates (one CTA per cluster).
// Work item: subdomain s, first candidate t0, count p; shift sigma.
__global__ void k_refine(const int* __restrict__ items, const double* __restrict__ sigmas,
                         const int* __restrict__ sub_info, const int* __restrict__ o_off,
                         const int* __restrict__ O_levptr, const int* __restrict__ O_L, int maxrow,
                         const int* __restrict__ ocnt, const int* __restrict__ ocol, const double* __restrict__ oB,
                         const double* __restrict__ oC, const int* __restrict__ o2i,
                         const long long* __restrict__ f_off, const long long* __restrict__ x_off, double* F,
                         double* Xw, const long long* __restrict__ poff, double* P, const double* __restrict__ lam_hat,
                         double* lam_ref, int max_b, int s_in_smem, DevStatus* st) {
  extern __shared__ double smem[];
  __shared__ int piv[HK_MAXB];
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ double minpiv, sh_val;
  __shared__ double Hs[HK_MAX_BLOCK * HK_MAX_BLOCK], Us[HK_MAX_BLOCK * HK_MAX_BLOCK], ws_[HK_MAX_BLOCK];
  __shared__ int win_s;
  int it = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  int s = items[4 * it], t0 = items[4 * it + 1], pc = items[4 * it + 2];
  int p = pc + HK_GUARD;  // block: cluster + guard vectors
  double sigma = sigmas[it];
  const int* si = sub_info + 8 * s;
  int nI = si[0], nG = si[1];
  int oo = o_off[s], nO = nI + nG, L = O_L[s];
  const int* lp = O_levptr + oo + s;
  double* tv = smem;                          // max_b x p
  double* Ssm = smem + (long long)max_b * p;  // max_b x max_b when the level blocks fit in shared memory
  double* Fw = F + f_off[it];
  double* X = Xw + x_off[it];                 // p x nO
  double* R = X + (long long)p * nO;          // p x nO
  double* Mv = R + (long long)p * nO;         // nO x maxrow: the entries of M = B^N - sigma C, formed once
  double* Ps = P + poff[s];
  // the entries of M and the scale for the pivot floor
  double mx = 0;
  for (long long e = tid; e < (long long)nO * maxrow; e += T) {
    int a = (int)(e / maxrow), q = (int)(e % maxrow);
    if (q < ocnt[oo + a]) {
      double v = oB[(long long)oo * maxrow + e] - sigma * oC[(long long)oo * maxrow + e];
      Mv[e] = v;
      mx = fmax(mx, fabs(v));
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) red_v[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    double m2 = 0;
    for (int w = 0; w < (T >> 5); ++w) m2 = fmax(m2, red_v[w]);
    sh_val = m2;
    minpiv = 1e300;
  }
  __syncthreads();
  double floor_piv = 1e-14 * sh_val;
  // 1. block LU of M = B^N - sigma C over the ovdof level sets
  long long bo = 0, prev_go = -1;
  int prev_r0 = 0;
  for (int j = 0; j < L; ++j) {
    int r0 = lp[j], b = lp[j + 1] - r0, r1 = lp[j + 1];
    int bn = j + 1 < L ? lp[j + 2] - r1 : 0;
    double* S = s_in_smem ? Ssm : Fw + bo;  // wide levels: in place in the factor array
    for (int e = tid; e < b * b; e += T) {
      int qa = e / b, t = e % b;
      int a = r0 + qa;
      long long base = (long long)(oo + a) * maxrow;
      const double* mr = Mv + (long long)a * maxrow;
      int cnt = min(ocnt[oo + a], maxrow);
      double v = 0;
      for (int q = 0; q < cnt; ++q) {
        int c = ocol[base + q];
        if (c == r0 + t) v += mr[q];
        else if (j > 0 && c >= prev_r0 && c < r0) v -= mr[q] * Fw[prev_go + (long long)(c - prev_r0) * b + t];
      }
      S[e] = v;
    }
    __syncthreads();
    gauss_jordan_inverse(S, b, piv, red_v, red_i, &minpiv, floor_piv);
    if (s_in_smem)
      for (int e = tid; e < b * b; e += T) Fw[bo + e] = S[e];
    long long go = bo + (long long)b * b;
    for (int e = tid; e < b * bn; e += T) {
      int qt = e / bn, cc = e % bn;
      int c = r1 + cc;
      long long base = (long long)(oo + c) * maxrow;
      const double* mr = Mv + (long long)c * maxrow;
      int cnt = min(ocnt[oo + c], maxrow);
      double v = 0;
      for (int q = 0; q < cnt; ++q) {
        int a = ocol[base + q];
        if (a >= r0 && a < r1) v += S[qt * b + (a - r0)] * mr[q];
      }
      Fw[go + e] = v;
    }
    __syncthreads();
    prev_go = go;
    prev_r0 = r0;
    bo = go + (long long)b * bn;
  }
  // 2. seeded start block on dof, zero on Gamma
  for (int t = 0; t < p; ++t)
    for (int a = tid; a < nO; a += T) {
      int ia = o2i[oo + a];
      unsigned long long key = ((unsigned long long)s << 40) ^ ((unsigned long long)(t0 * 64 + t) << 20) ^ a;
      X[(long long)t * nO + a] = ia >= 0 ? (double)hash_unitf(key) : 0.0;
    }
  __syncthreads();
  // candidates are accurate to about 1e-7: a single eigenvalue converges at |lambda - sigma| / gap <= 1e-3
  // per step; a cluster's members converge at their spread over the distance to the block's next value
  int steps = pc == 1 ? HK_REFINE_STEPS_SINGLE : HK_REFINE_STEPS;
  for (int step = 0; step < steps; ++step) {
    // R = C X, then X = M^{-1} R by the two block sweeps
    o_matvec(nO, oo, maxrow, ocnt, ocol, oB, oC, 1.0, 0, X, R, p);
    __syncthreads();
    long long fo = 0;
    for (int j = 0; j < L; ++j) {
      int r0 = lp[j], b = lp[j + 1] - r0, bn = j + 1 < L ? lp[j + 2] - lp[j + 1] : 0;
      for (int e = tid; e < b * p; e += T) {
        int t = e / b, a = r0 + e % b;
        long long base = (long long)(oo + a) * maxrow;
        const double* mr = Mv + (long long)a * maxrow;
        int cnt = min(ocnt[oo + a], maxrow);
        double acc = R[(long long)t * nO + a];
        for (int q = 0; q < cnt; ++q) {
          int c = ocol[base + q];
          if (c < r0) acc -= mr[q] * R[(long long)t * nO + c];
        }
        tv[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < b * p; e += T) {
        int t = e / b, q = e % b;
        const double* Sr = Fw + fo + (long long)q * b;
        double acc = 0;
        for (int c = 0; c < b; ++c) acc += Sr[c] * tv[t * b + c];
        R[(long long)t * nO + r0 + q] = acc;
      }
      __syncthreads();
      fo += (long long)b * b + (long long)b * bn;
    }
    // backward: x_j -= G_j x_{j+1}
    {
      int bl = lp[L] - lp[L - 1];
      fo -= (long long)bl * bl;
    }
    for (int j = L - 2; j >= 0; --j) {
      int r0 = lp[j], b = lp[j + 1] - r0, r1 = lp[j + 1], bn = lp[j + 2] - r1;
      fo -= (long long)b * b + (long long)b * bn;
      const double* Gm = Fw + fo + (long long)b * b;
      for (int e = tid; e < b * p; e += T) {
        int t = e / b, q = e % b;
        double acc = 0;
        for (int c = 0; c < bn; ++c) acc += Gm[(long long)q * bn + c] * R[(long long)t * nO + r1 + c];
        tv[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < b * p; e += T) {
        int t = e / b, q = e % b;
        R[(long long)t * nO + r0 + q] -= tv[e];
      }
      __syncthreads();
    }
    // X = R, C-orthonormalised (modified Gram-Schmidt twice; CX kept alongside in R)
    for (long long e = tid; e < (long long)p * nO; e += T) X[e] = R[e];
    __syncthreads();
    o_matvec(nO, oo, maxrow, ocnt, ocol, oB, oC, 1.0, 0, X, R, p);  // R = C X
    __syncthreads();
    for (int rep = 0; rep < 2; ++rep)
      for (int t = 0; t < p; ++t) {
        double* xt = X + (long long)t * nO;
        double* cxt = R + (long long)t * nO;
        for (int u = 0; u < t; ++u) {
          double dcu = block_dot(xt, R + (long long)u * nO, nO, red_v);
          for (int a = tid; a < nO; a += T) {
            xt[a] -= dcu * X[(long long)u * nO + a];
            cxt[a] -= dcu * R[(long long)u * nO + a];
          }
          __syncthreads();
        }
        double nrm = block_dot(xt, cxt, nO, red_v);
        double inv = nrm > 0 ? 1.0 / sqrt(nrm) : 0.0;
        for (int a = tid; a < nO; a += T) {
          xt[a] *= inv;
          cxt[a] *= inv;
        }
        __syncthreads();
      }
  }
  // 3. Rayleigh-Ritz on B^N: H = X^T B^N X (X is C-orthonormal)
  o_matvec(nO, oo, maxrow, ocnt, ocol, oB, oC, 0.0, 1, X, R, p);  // R = B^N X
  __syncthreads();
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) {
      double h = block_dot(X + (long long)i * nO, R + (long long)j * nO, nO, red_v);
      if (tid == 0) Hs[i * p + j] = h;
    }
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < p; ++i)
      for (int j = i + 1; j < p; ++j) {
        double a = 0.5 * (Hs[i * p + j] + Hs[j * p + i]);
        Hs[i * p + j] = Hs[j * p + i] = a;
      }
    jacobi_eig(Hs, Us, ws_, p);
    // the window of pc consecutive Ritz values closest to the cluster's candidates
    int best = 0;
    double bestd = 1e300;
    for (int w0 = 0; w0 + pc <= p; ++w0) {
      double dsum = 0;
      for (int i = 0; i < pc; ++i) dsum += fabs(ws_[w0 + i] - lam_hat[(long long)s * HK_MAXM + t0 + i]);
      if (dsum < bestd) {
        bestd = dsum;
        best = w0;
      }
    }
    win_s = best;
    for (int i = 0; i < pc; ++i) lam_ref[(long long)s * HK_MAXM + t0 + i] = ws_[best + i];
    if (!(minpiv > 0)) dev_fail(st, HK_EIG_FAIL, s, minpiv);
  }
  __syncthreads();
  // refined vectors X U (the selected window), written (dof part, level order) over the candidates
  int w0 = win_s;
  for (int i = 0; i < pc; ++i)
    for (int a = tid; a < nO; a += T) {
      int ia = o2i[oo + a];
      if (ia < 0) continue;
      double acc = 0;
      for (int k = 0; k < p; ++k) acc += X[(long long)k * nO + a] * Us[k * p + w0 + i];
      Ps[(long long)(t0 + i) * nI + ia] = acc;
    }
}

// ---- 10. selection on the FP64 values: keep lambda < tau, extended across ties; order ascending.
// Certification: the number of refined values below tau must equal neg[s], the FP64 inertia count of
// B^N - tau C (every eigenvalue below tau found once); a difference is accepted only where the value at
// the boundary lies within 1e-9 max(1, |tau|) of tau (the count then depends on rounding).  Otherwise
// fail[s] = 1 (the setup redoes the subdomain once with a larger Krylov basis, then reports HK_EIG_FAIL).
// lam_next[s]: the smallest refined value not kept (lambda_{m_i+1} when the candidates below tau + delta
// are complete), or +inf when every candidate was kept.
__global__ void k_select(const int* __restrict__ cnt, const double* __restrict__ lam_ref, double tau,
                         const int* __restrict__ neg, int* sel, int* m_out, double* lam_out, int* fail,
                         double* lam_next, DevStatus* st) {
  int s = blockIdx.x;
  if (threadIdx.x != 0) return;
  int c = min(cnt[s], HK_MAXM);
  const double* lr = lam_ref + (long long)s * HK_MAXM;
  int* ord = sel + (long long)s * HK_MAXM;
  for (int i = 0; i < c; ++i) ord[i] = i;
  for (int i = 1; i < c; ++i) {
    int k = ord[i], j = i - 1;
    while (j >= 0 && lr[ord[j]] > lr[k]) {
      ord[j + 1] = ord[j];
      --j;
    }
    ord[j + 1] = k;
  }
  int m = 0;
  while (m < c && lr[ord[m]] < tau) ++m;
  double near = 1e-9 * fmax(1.0, fabs(tau));
  fail[s] = 0;
  if (m != neg[s]) {
    bool boundary = (m > 0 && tau - lr[ord[m - 1]] <= near) || (m < c && lr[ord[m]] - tau <= near);
    if (!boundary) fail[s] = 1;
  }
  double thr = 1e-8 * fmax(1.0, fabs(tau));
  while (m > 0 && m < c && lr[ord[m]] - lr[ord[m - 1]] <= thr) ++m;
  if (m == c && c == cnt[s] && m > 0 && lr[ord[m - 1]] >= tau) dev_fail(st, HK_EIG_FAIL, s, m);
  m_out[s] = m;
  lam_next[s] = m < c ? lr[ord[m]] : INFINITY;
  for (int i = 0; i < m; ++i) lam_out[(long long)s * HK_MAXM + i] = lr[ord[i]];
}

// Z_i columns = Xi p = p / mu on dof(Omega_i) (row-major |dof| x m, level order).
__global__ void k_write_z(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                          const int* __restrict__ Ilev, const int* __restrict__ mu, const int* __restrict__ sel,
                          const long long* __restrict__ poff, const double* __restrict__ P, double* Z) {
  int s = blockIdx.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], off = si[3], m = si[6];
  long long zo = sub_off[3 * s + 2];
  const int* ord = sel + (long long)s * HK_MAXM;
  const double* Ps = P + poff[s];
  for (long long e = threadIdx.x; e < (long long)nI * m; e += blockDim.x) {
    int a = (int)(e / m), l = (int)(e % m);
    Z[zo + e] = Ps[(long long)ord[l] * nI + a] / (double)mu[Ilev[off + a]];
  }
}

hk_status phase_eigen(hk_handle* h, const uint8_t* d_elem_in) {
  cudaStream_t st = h->stream;
  int ns = h->n_sub;
  // ---- sizes: B^N on Gamma x Gamma (dense, per subdomain) and the ovdof rows
  std::vector<long long> Gw(ns);
  std::vector<int> o_off(ns), oc(ns);
  long long tot = 0;
  int O_total = 0;
  for (int s = 0; s < ns; ++s) {
    const Sub& u = h->subs[s];
    Gw[s] = tot;
    tot += (long long)u.nG * u.nG;
    o_off[s] = O_total;
    oc[s] = u.nI + u.nG;
    O_total += oc[s];
  }
  double* d_ws = nullptr;
  long long* d_Gw = nullptr;
  int *d_cnt = nullptr, *d_o_off = nullptr, *d_neg = nullptr;
  double *d_lamhat = nullptr, *d_lamref = nullptr;
  HK_TRY(dalloc(h, &d_ws, tot));
  HK_TRY(dalloc(h, &d_Gw, ns));
  HK_TRY(dalloc(h, &d_cnt, ns));
  HK_TRY(dalloc(h, &d_o_off, ns));
  HK_TRY(dalloc(h, &d_neg, ns));
  HK_TRY(dalloc(h, &d_lamhat, (size_t)ns * HK_MAXM));
  HK_TRY(dalloc(h, &d_lamref, (size_t)ns * HK_MAXM));
  HK_TRY(dalloc(h, &h->d_lam, (size_t)ns * HK_MAXM));
  auto up = [&](void* d, const void* hsrc, size_t bytes) {
    return cudaMemcpyAsync(d, hsrc, bytes, cudaMemcpyHostToDevice, st);
  };
  HK_CUDA(up(d_Gw, Gw.data(), 8 * ns));
  HK_CUDA(up(d_o_off, o_off.data(), 4 * ns));

  // ---- B^N on Gamma x Gamma, then the ovdof structure and the sparse pencil over it
  k_gamma_block<<<ns, 128, 0, st>>>(h->dim, h->n_elems, h->d_xyz, h->d_elems, h->d_coeff, h->k * h->k,
                                    h->d_node_of_dof, h->d_dof_of_node, h->d_ne_ptr, h->d_ne_idx, d_elem_in,
                                    h->d_sub_info, h->d_G, d_Gw, d_ws);
  HK_COUNT_LAUNCH();
  int *d_O = nullptr, *d_okind = nullptr, *d_Operm = nullptr, *d_Olev = nullptr, *d_Olevptr = nullptr;
  HK_TRY(dalloc(h, &d_O, O_total));
  HK_TRY(dalloc(h, &d_okind, O_total));
  HK_TRY(dalloc(h, &d_Operm, O_total));
  HK_TRY(dalloc(h, &d_Olev, O_total));
  HK_TRY(dalloc(h, &d_Olevptr, O_total + ns));
  k_o_merge<<<ns, 32, 0, st>>>(h->d_sub_info, h->d_Isorted, h->d_G, d_o_off, d_O, d_okind);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  std::vector<int> OL;
  int maxbO = 0;
  HK_TRY(build_levels(h, oc, o_off, d_O, d_Olevptr, d_Operm, d_Olev, OL, &maxbO));
  int* d_OL = nullptr;
  HK_TRY(dalloc(h, &d_OL, ns));
  HK_CUDA(up(d_OL, OL.data(), 4 * ns));
  std::vector<int> rp(h->n + 1);
  HK_CUDA(cudaMemcpyAsync(rp.data(), h->d_rowptr, sizeof(int) * (h->n + 1), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  int maxrow = 1;
  for (int i = 0; i < h->n; ++i) maxrow = std::max(maxrow, rp[i + 1] - rp[i]);
  int *d_ocnt = nullptr, *d_ocol = nullptr, *d_o2i = nullptr;
  double *d_oB = nullptr, *d_oC = nullptr;
  HK_TRY(dalloc(h, &d_ocnt, O_total));
  HK_TRY(dalloc(h, &d_o2i, O_total));
  HK_TRY(dalloc(h, &d_ocol, (size_t)O_total * maxrow));
  HK_TRY(dalloc(h, &d_oB, (size_t)O_total * maxrow));
  HK_TRY(dalloc(h, &d_oC, (size_t)O_total * maxrow));
  k_o_csr<<<ns, 128, 0, st>>>(h->d_sub_info, d_o_off, d_O, d_okind, d_Operm, d_Olev, h->d_perm, h->d_rowptr,
                              h->d_col, h->d_valB, h->d_valD, h->d_mu, d_Gw, d_ws, maxrow, d_ocnt, d_ocol, d_oB, d_oC,
                              d_o2i);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  std::vector<int> levO(O_total + ns);
  HK_CUDA(cudaMemcpyAsync(levO.data(), d_Olevptr, sizeof(int) * levO.size(), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  OvdofPencil op;
  op.o_off = d_o_off;
  op.levptr = d_Olevptr;
  op.L = d_OL;
  op.cnt = d_ocnt;
  op.col = d_ocol;
  op.B = d_oB;
  op.C = d_oC;
  op.o2i = d_o2i;
  op.maxrow = maxrow;
  op.max_b = maxbO;
  op.max_nO = *std::max_element(oc.begin(), oc.end());
  op.h_off = o_off;
  op.h_nO = oc;
  op.h_L = OL;
  op.h_levptr = levO;

  // ---- FP64 count below tau (certifies m_i) on the second stream, joined at the selection; meanwhile the
  //      FP32 Lanczos candidates below tau + delta and their FP64 refinement on the setup stream
  cudaStream_t ist = h->co_stream ? h->co_stream : st;
  cudaEvent_t e0, e1;
  HK_CUDA(cudaEventCreate(&e0));
  HK_CUDA(cudaEventCreate(&e1));
  if (ist != st) {
    HK_CUDA(cudaEventRecord(h->ev_fork, st));
    HK_CUDA(cudaStreamWaitEvent(ist, h->ev_fork, 0));
  }
  cudaEventRecord(e0, ist);
  HK_TRY(eigen_inertia(h, op, h->p.tau, d_neg, ist));
  cudaEventRecord(e1, ist);
  cudaEvent_t inertia_done = nullptr;
  HK_CUDA(cudaEventCreateWithFlags(&inertia_done, cudaEventDisableTiming));
  HK_CUDA(cudaEventRecord(inertia_done, ist));
  h->eigen_gflop[1] = 0;
  // a basis of 96 columns, grown inside the kernel to 4 c + 48 where c candidates ask for more
  std::vector<int> cols(ns, LZ_BASIS_MAX), cnt(ns);
  std::vector<double> lamhat((size_t)ns * HK_MAXM);
  float lz_ms = 0;
  HK_TRY(eigen_lanczos(h, op, cols, 96, h->p.tau + HK_EIG_DELTA, d_lamhat, d_cnt, &lz_ms));
  HK_TRY(check_device_status(h, "eigen: Lanczos candidates"));
  h->eigen_ms[1] = lz_ms;
  int *d_sel = nullptr, *d_m = nullptr, *d_fail = nullptr;
  HK_TRY(dalloc(h, &d_sel, (size_t)ns * HK_MAXM));
  HK_TRY(dalloc(h, &d_m, ns));
  HK_TRY(dalloc(h, &d_fail, ns));
  double* d_lamnext = nullptr;
  HK_TRY(dalloc(h, &d_lamnext, ns));
  double* d_P = nullptr;
  long long* d_poff = nullptr;
  HK_TRY(dalloc(h, &d_poff, ns));
  std::vector<long long> poff(ns);
  std::vector<long long> fsize(ns, 0);
  for (int s = 0; s < ns; ++s) {
    const int* lp = &levO[o_off[s] + s];
    for (int j = 0; j < OL[s]; ++j) {
      long long b = lp[j + 1] - lp[j], bn = j + 1 < OL[s] ? lp[j + 2] - lp[j + 1] : 0;
      fsize[s] += b * b + b * bn;
    }
  }
  h->eigen_ms[2] = 0;
  h->eigen_gflop[2] = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    HK_CUDA(cudaMemcpyAsync(cnt.data(), d_cnt, 4 * ns, cudaMemcpyDeviceToHost, st));
    HK_CUDA(cudaMemcpyAsync(lamhat.data(), d_lamhat, sizeof(double) * lamhat.size(), cudaMemcpyDeviceToHost, st));
    HK_CUDA(cudaStreamSynchronize(st));
    long long ptot = 0;
    for (int s = 0; s < ns; ++s) {
      poff[s] = ptot;
      ptot += (long long)h->subs[s].nI * cnt[s];
    }
    if (d_P) dfree(h, d_P);
    HK_TRY(dalloc(h, &d_P, ptot));
    HK_CUDA(up(d_poff, poff.data(), 8 * ns));
    // ---- FP64 refinement: clusters of candidates, one CTA each
    std::vector<int> items;
    std::vector<double> sig;
    std::vector<long long> foff, xoff;
    long long ftot = 0, xtot = 0;
    int pmax = 1;
    for (int s = 0; s < ns; ++s) {
      const double* lh = &lamhat[(size_t)s * HK_MAXM];
      int c = std::min(cnt[s], HK_MAXM);
      int t = 0;
      while (t < c) {
        int t1 = t + 1;
        while (t1 < c && t1 - t < HK_MAX_CLUSTER &&
               lh[t1] - lh[t1 - 1] <= HK_CLUSTER_GAP * std::max(1.0, std::fabs(lh[t1]))) ++t1;
        double sm = 0;
        for (int q = t; q < t1; ++q) sm += lh[q];
        items.push_back(s); items.push_back(t); items.push_back(t1 - t); items.push_back(0);
        sig.push_back(sm / (t1 - t));
        foff.push_back(ftot);
        ftot += fsize[s];
        xoff.push_back(xtot);
        xtot += 2LL * (t1 - t + HK_GUARD) * oc[s] + (long long)oc[s] * maxrow;
        pmax = std::max(pmax, t1 - t + HK_GUARD);
        t = t1;
      }
    }
    int nit = (int)sig.size();
    // items run in batches whose factor and iterate storage stays below 1 GiB (each item holds the block
    // LU of its own shifted pencil)
    const long long batch_bytes = 1LL << 30;
    for (int i0 = 0; i0 < nit;) {
      int i1 = i0;
      long long fb = 0, xb = 0;
      while (i1 < nit) {
        long long fi = (i1 + 1 < nit ? foff[i1 + 1] : ftot) - foff[i1];
        long long xi = (i1 + 1 < nit ? xoff[i1 + 1] : xtot) - xoff[i1];
        if (i1 > i0 && 8 * (fb + fi + xb + xi) > batch_bytes) break;
        fb += fi;
        xb += xi;
        ++i1;
      }
      int nb_it = i1 - i0;
      std::vector<long long> fo2(nb_it), xo2(nb_it);
      for (int i = 0; i < nb_it; ++i) {
        fo2[i] = foff[i0 + i] - foff[i0];
        xo2[i] = xoff[i0 + i] - xoff[i0];
      }
      int* d_items = nullptr;
      double *d_sig = nullptr, *d_F = nullptr, *d_X = nullptr;
      long long *d_foff = nullptr, *d_xoff = nullptr;
      HK_TRY(dalloc(h, &d_items, 4 * (size_t)nb_it));
      HK_TRY(dalloc(h, &d_sig, nb_it));
      HK_TRY(dalloc(h, &d_foff, nb_it));
      HK_TRY(dalloc(h, &d_xoff, nb_it));
      HK_TRY(dalloc(h, &d_F, fb));
      HK_TRY(dalloc(h, &d_X, xb));
      HK_CUDA(up(d_items, items.data() + 4 * (size_t)i0, 16 * (size_t)nb_it));
      HK_CUDA(up(d_sig, sig.data() + i0, 8 * nb_it));
      HK_CUDA(up(d_foff, fo2.data(), 8 * nb_it));
      HK_CUDA(up(d_xoff, xo2.data(), 8 * nb_it));
      int pmax_b = 1;
      for (int i = i0; i < i1; ++i) pmax_b = std::max(pmax_b, items[4 * i + 2] + HK_GUARD);
      size_t rshm = sizeof(double) * ((size_t)maxbO * maxbO + (size_t)maxbO * pmax_b);
      int s_in_smem = rshm <= 190 * 1024;
      if (!s_in_smem) rshm = sizeof(double) * (size_t)maxbO * pmax_b;
      HK_TRY(hk_allow_smem(k_refine));
      {
        // algorithmic FMAs per item: the block LU of B^N - sigma C (Gauss-Jordan, b^3 per level), every
        // inverse-iteration step (a sweep with p vectors, C X, C-orthonormalisation twice: 4 p^2 nO) and the
        // Rayleigh-Ritz products (p^2 nO)
        double fma = 0;
        for (int it = i0; it < i1; ++it) {
          int s = items[4 * it], pc = items[4 * it + 2], p = pc + HK_GUARD;
          int steps = pc == 1 ? HK_REFINE_STEPS_SINGLE : HK_REFINE_STEPS;
          const int* lp = &levO[o_off[s] + s];
          double fac = 0, sweep = 0;
          for (int j = 0; j < OL[s]; ++j) {
            double b = lp[j + 1] - lp[j], bn = j + 1 < OL[s] ? lp[j + 2] - lp[j + 1] : 0;
            fac += b * b * b;
            sweep += (b * b + b * bn) * p;
          }
          double nO = oc[s];
          fma += fac + steps * (sweep + 14.0 * nO * p + 4.0 * p * p * nO) + p * p * nO;
        }
        h->eigen_gflop[2] += 2.0 * fma * 1e-9;
      }
      cudaEvent_t r0, r1;
      HK_CUDA(cudaEventCreate(&r0));
      HK_CUDA(cudaEventCreate(&r1));
      cudaEventRecord(r0, st);
      k_refine<<<nb_it, 128, rshm, st>>>(d_items, d_sig, h->d_sub_info, d_o_off, d_Olevptr, d_OL, maxrow, d_ocnt,
                                         d_ocol, d_oB, d_oC, d_o2i, d_foff, d_xoff, d_F, d_X, d_poff, d_P, d_lamhat,
                                         d_lamref, maxbO, s_in_smem, h->d_status);
      HK_COUNT_LAUNCH();
      cudaEventRecord(r1, st);
      HK_LAUNCH_CHECK();
      HK_CUDA(cudaStreamSynchronize(st));
      {
        float ms = 0;
        cudaEventElapsedTime(&ms, r0, r1);
        h->eigen_ms[2] += ms;
        cudaEventDestroy(r0);
        cudaEventDestroy(r1);
      }
      HK_TRY(check_device_status(h, "eigen: refinement"));
      void* tmpf[] = {d_items, d_sig, d_foff, d_xoff, d_F, d_X};
      for (void* q : tmpf) dfree(h, q);
      i0 = i1;
    }
    // selection and certification against the FP64 count (joined here)
    HK_CUDA(cudaStreamWaitEvent(st, inertia_done, 0));
    k_select<<<ns, 32, 0, st>>>(d_cnt, d_lamref, h->p.tau, d_neg, d_sel, d_m, h->d_lam, d_fail, d_lamnext,
                                h->d_status);
    HK_COUNT_LAUNCH();
    HK_LAUNCH_CHECK();
    std::vector<int> fail(ns);
    HK_CUDA(cudaMemcpyAsync(fail.data(), d_fail, 4 * ns, cudaMemcpyDeviceToHost, st));
    HK_CUDA(cudaStreamSynchronize(st));
    int nfail = 0, first = -1;
    for (int s = 0; s < ns; ++s)
      if (fail[s]) {
        ++nfail;
        if (first < 0) first = s;
      }
    if (nfail == 0) {
      // tau of Thm. 3.1: min over subdomains of lambda_{m_i+1}; subdomains without a candidate above the
      // kept ones only bound it below by tau + delta
      std::vector<double> nx(ns);
      HK_CUDA(cudaMemcpy(nx.data(), d_lamnext, sizeof(double) * ns, cudaMemcpyDeviceToHost));
      double lo = INFINITY;
      bool unknown = false;
      for (int s = 0; s < ns; ++s) {
        if (std::isfinite(nx[s])) lo = std::min(lo, nx[s]);
        else unknown = true;
      }
      h->tau_next = lo;
      h->tau_next_lb = unknown && !(lo < h->p.tau + HK_EIG_DELTA);
      if (h->tau_next_lb) h->tau_next = h->p.tau + HK_EIG_DELTA;
      break;
    }
    if (attempt == 1) {
      std::vector<int> negv(ns);
      HK_CUDA(cudaMemcpy(negv.data(), d_neg, 4 * ns, cudaMemcpyDeviceToHost));
      int most = 0;
      for (int s = 0; s < ns; ++s)
        if (fail[s]) most = std::max(most, negv[s]);
      if (4 * most + 48 > LZ_BASIS_MAX) {
        // more eigenvalues below tau than a Krylov basis of LZ_BASIS_MAX columns resolves
        hk_set_error("eigen: subdomain %d has %d eigenvalues below tau; the Lanczos candidates resolve at most %d "
                     "per subdomain (use more subdomains or a smaller tau)", first, negv[first],
                     (LZ_BASIS_MAX - 48) / 4);
        return HK_UNSUPPORTED;
      }
      hk_set_error("eigen: %d subdomain(s), first %d: the refined eigenvalues below tau do not match the FP64 "
                   "inertia count (even with a %d-column Krylov basis)", nfail, first, LZ_BASIS_MAX);
      return HK_EIG_FAIL;
    }
    // the failed subdomains again with the largest basis; every subdomain is then refined again (the
    // others reproduce their results: the refinement is deterministic)
    for (int s = 0; s < ns; ++s) cols[s] = fail[s] ? LZ_BASIS_MAX : 0;
    float ms = 0;
    HK_TRY(eigen_lanczos(h, op, cols, LZ_BASIS_MAX, h->p.tau + HK_EIG_DELTA, d_lamhat, d_cnt, &ms));
    HK_TRY(check_device_status(h, "eigen: Lanczos candidates"));
    h->eigen_ms[1] += ms;
  }
  {
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    h->eigen_ms[0] = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(inertia_done);
  }
  HK_TRY(check_device_status(h, "eigen: selection"));
  std::vector<int> m(ns);
  HK_CUDA(cudaMemcpyAsync(m.data(), d_m, 4 * ns, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  int c0 = 0;
  long long zo = 0;
  for (int s = 0; s < ns; ++s) {
    Sub& u = h->subs[s];
    u.m = m[s];
    u.c_off = c0;
    u.z_off = zo;
    c0 += u.m;
    zo += (long long)u.nI * u.m;
  }
  h->n0 = c0;
  h->z_total = zo;
  HK_TRY(upload_sub_info(h));
  if (c0 > 0) {
    HK_TRY(dalloc(h, &h->d_Z64, zo));
    k_write_z<<<ns, 256, 0, st>>>(h->d_sub_info, h->d_sub_off, h->d_I, h->d_mu, d_sel, d_poff, d_P, h->d_Z64);
    HK_COUNT_LAUNCH();
    HK_LAUNCH_CHECK();
  }
  HK_CUDA(cudaStreamSynchronize(st));
  void* tmp[] = {d_ws, d_Gw, d_cnt, d_o_off, d_neg, d_lamhat, d_lamref, d_O, d_okind, d_Operm, d_Olev, d_Olevptr,
                 d_OL, d_ocnt, d_o2i, d_ocol, d_oB, d_oC, d_P, d_poff, d_sel, d_m, d_fail, d_lamnext};
  for (void* p : tmp) dfree(h, p);
  return HK_OK;
}
