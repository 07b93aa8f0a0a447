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
// Two stages, because FP64 arithmetic on this GPU runs at 1/58 of FP32:
//  1. FP32 dense stage (eigenvalue candidates).  With D_II = L L^T (banded, level order) the standard
//     form is A q = lambda q, A = L^{-1} (mu S mu) L^{-T}.  A is reduced to tridiagonal form by
//     Householder reflections in FP32, and 32-way multisection on Sturm counts finds every eigenvalue
//     below tau + delta (delta = 0.05, far above the FP32 error of these eigenvalues).
//  2. FP64 refinement on the sparse pencil.  Candidates closer than 1e-3 max(1,|lambda|) form a
//     cluster; for each cluster the block-tridiagonal LU of B^N - sigma C over level sets of
//     ovdof(Omega_i) is formed in FP64 (sigma = the cluster's mean candidate), a seeded block of
//     cluster size + 2 guard vectors takes five steps of block inverse iteration
//     ((B^N - sigma C)^{-1} C, C-orthonormalised after each step; the contraction per step is
//     |lambda - sigma| over the distance to the next eigenvalue outside the block), and a Rayleigh-Ritz
//     step on B^N gives FP64 eigenpairs; the window of Ritz values closest to the cluster's candidates
//     is kept.  The Gamma part of each iterate satisfies the Gamma rows of the pencil exactly, so
//     x^T B^N x = x_I^T S x_I.
// Selection then keeps lambda < tau on the FP64 values, extending across ties (gap <= 1e-8 max(1,|tau|)),
// and the coarse vectors are Xi p = p / mu on dof(Omega_i), c-normalised (Def. 5.1).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "hk_internal.cuh"

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

#define HK_EIG_DELTA 0.05
#define HK_CLUSTER_GAP 1e-3
#define HK_MAX_CLUSTER 32
#define HK_REFINE_STEPS 5
#define HK_GUARD 2
#define HK_MAX_BLOCK (HK_MAX_CLUSTER + HK_GUARD)
#define HK_SCHUR_DINV 1024

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

// ---- 2. S = B_II - B_IG (B^N_GG)^{-1} B_GI (dense, level order) in W.
// Ring = dofs with a Gamma neighbour.  R holds B_GR (nG x nR), then X = BGG^{-1} B_GR.
__global__ void k_schur(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                        const int* __restrict__ lrow, const int* __restrict__ lcntI, const int* __restrict__ lcntG,
                        const int* __restrict__ lcol, const double* __restrict__ lvalB,
                        const long long* __restrict__ wsW, const long long* __restrict__ wsG,
                        const long long* __restrict__ wsR, int* ring_ws, double* ws, DevStatus* st) {
  __shared__ double sh_piv[2];
  __shared__ double dinv[HK_SCHUR_DINV];  // reciprocal Cholesky diagonal of B^N_GG
  __shared__ int shi[32];
  __shared__ int nR_sh;
  int s = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], nG = si[1], off = si[3];
  long long coff = sub_off[3 * s + 1];
  const int* lr = lrow + off + s;
  double* W = ws + wsW[s];
  double* BG = ws + wsG[s];
  double* R = ws + wsR[s];
  int* ring = ring_ws + off;  // up to nI entries
  // dense B_II
  for (long long e = tid; e < (long long)nI * nI; e += T) W[e] = 0.0;  // no division: flat fill
  __syncthreads();
  for (int a = tid; a < nI; a += T) {
    long long b0 = coff + lr[a];
    for (int q = 0; q < lcntI[off + a]; ++q) W[(long long)a * nI + lcol[b0 + q]] = lvalB[b0 + q];
  }
  // ring list (ordered)
  if (tid == 0) {
    int c = 0;
    for (int a = 0; a < nI; ++a)
      if (lcntG[off + a] > 0) ring[c++] = a;
    nR_sh = c;
  }
  __syncthreads();
  int nR = nR_sh;
  if (nG == 0 || nR == 0) return;
  // Cholesky of BGG in place (lower), right-looking.  The pivot's square root and reciprocal are
  // computed once, by thread 0 (FP64 division and square root are slow: per thread they would fill
  // the FP64 pipe), and kept for the triangular solves below.
  for (int k = 0; k < nG; ++k) {
    if (tid == 0) {
      double piv = BG[(long long)k * nG + k];
      sh_piv[0] = piv;
      if (piv > 0.0) {
        double lkk = sqrt(piv), il = 1.0 / lkk;
        BG[(long long)k * nG + k] = lkk;
        sh_piv[1] = il;
        if (k < HK_SCHUR_DINV) dinv[k] = il;
      }
    }
    __syncthreads();
    if (!(sh_piv[0] > 0.0)) {
      if (tid == 0) dev_fail(st, HK_EIG_FAIL, s, sh_piv[0]);
      return;
    }
    double il = sh_piv[1];
    for (int i = k + 1 + tid; i < nG; i += T) BG[(long long)i * nG + k] *= il;
    __syncthreads();
    for (int i = k + 1 + (tid >> 5); i < nG; i += T >> 5) {
      double lik = BG[(long long)i * nG + k];
      for (int j = k + 1 + (tid & 31); j <= i; j += 32) BG[(long long)i * nG + j] -= lik * BG[(long long)j * nG + k];
    }
    __syncthreads();
  }
  // R = B_GR (nG x nR): B[g][ring r] = B[ring r][g] from the ring rows' Gamma entries
  for (long long e = tid; e < (long long)nG * nR; e += T) R[e] = 0.0;
  __syncthreads();
  for (int r = tid; r < nR; r += T) {
    int a = ring[r];
    long long b0 = coff + lr[a] + lcntI[off + a];
    for (int q = 0; q < lcntG[off + a]; ++q) R[(long long)lcol[b0 + q] * nR + r] = lvalB[b0 + q];
  }
  __syncthreads();
  // X = BGG^{-1} R in place, column per thread (forward with L, back with L^T)
  for (int r = tid; r < nR; r += T) {
    for (int i = 0; i < nG; ++i) {
      double v = R[(long long)i * nR + r];
      for (int k = 0; k < i; ++k) v -= BG[(long long)i * nG + k] * R[(long long)k * nR + r];
      R[(long long)i * nR + r] = i < HK_SCHUR_DINV ? v * dinv[i] : v / BG[(long long)i * nG + i];
    }
    for (int i = nG - 1; i >= 0; --i) {
      double v = R[(long long)i * nR + r];
      for (int k = i + 1; k < nG; ++k) v -= BG[(long long)k * nG + i] * R[(long long)k * nR + r];
      R[(long long)i * nR + r] = i < HK_SCHUR_DINV ? v * dinv[i] : v / BG[(long long)i * nG + i];
    }
  }
  __syncthreads();
  // W[ring a][ring b] -= sum_g B[a][g] X[g][b]
  for (int ra = tid >> 5; ra < nR; ra += T >> 5) {
    int a = ring[ra];
    long long b0 = coff + lr[a] + lcntI[off + a];
    int cg = lcntG[off + a];
    for (int rb = tid & 31; rb < nR; rb += 32) {
      double v = 0;
      for (int q = 0; q < cg; ++q) v += lvalB[b0 + q] * R[(long long)lcol[b0 + q] * nR + rb];
      W[(long long)a * nI + ring[rb]] -= v;
    }
  }
}

// ---- 3. FP32 standard form A = L^{-1} (mu S mu) L^{-T} with D_II = L L^T.
// (a) banded Cholesky of D_II in FP64 (one CTA per subdomain): Lb[a][t] = L[a][a - bw + t], and its
//     FP32 copy L32;
// (b) Y = L^{-1} (mu S mu) column by column (S read in FP64 and scaled on the fly);
// (c) A = L^{-1} Y^T, where column c of Y^T is row c of Y, read through shared-memory tiles.
// In (b) and (c) each CTA owns a tile of columns and each thread one column; the last bw solved
// entries of a column sit in a shared-memory ring, and the next 8 input rows are loaded ahead.
// A is symmetric up to rounding and is used as computed.
__global__ void k_dchol(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                        const int* __restrict__ bw_arr, const int* __restrict__ lrow, const int* __restrict__ lcntI,
                        const int* __restrict__ lcol, const double* __restrict__ lvalD,
                        const long long* __restrict__ wsL, const long long* __restrict__ wsL32, double* ws,
                        float* ws32, DevStatus* st) {
  int s = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], off = si[3];
  int bw = bw_arr[s], ld = bw + 1;
  long long coff = sub_off[3 * s + 1];
  const int* lr = lrow + off + s;
  // the factor is only used in FP32 (the standard form of the candidate stage): factor in FP32
  float* Lb = ws32 + wsL32[s];
  for (long long e = tid; e < (long long)nI * ld; e += T) Lb[e] = 0.f;
  __syncthreads();
  for (int a = tid; a < nI; a += T) {
    long long b0 = coff + lr[a];
    for (int q = 0; q < lcntI[off + a]; ++q) {
      int c = lcol[b0 + q];
      if (c <= a) Lb[(long long)a * ld + (c - a + bw)] = (float)lvalD[b0 + q];
    }
  }
  __syncthreads();
  __shared__ float sh_piv[2];
  for (int k = 0; k < nI; ++k) {
    // pivot square root and reciprocal once, by thread 0 (see k_schur)
    if (tid == 0) {
      float piv = Lb[(long long)k * ld + bw];
      sh_piv[0] = piv;
      if (piv > 0.f) {
        float lkk = sqrtf(piv);
        Lb[(long long)k * ld + bw] = lkk;
        sh_piv[1] = 1.f / lkk;
      }
    }
    __syncthreads();
    if (!(sh_piv[0] > 0.f)) {
      if (tid == 0) dev_fail(st, HK_EIG_FAIL, s, sh_piv[0]);
      return;
    }
    float il = sh_piv[1];
    int iend = min(nI - 1, k + bw);
    for (int i = k + 1 + tid; i <= iend; i += T) Lb[(long long)i * ld + (k - i + bw)] *= il;
    __syncthreads();
    for (int i = k + 1 + (tid >> 5); i <= iend; i += T >> 5) {
      float lik = Lb[(long long)i * ld + (k - i + bw)];
      for (int j = k + 1 + (tid & 31); j <= i; j += 32)
        Lb[(long long)i * ld + (j - i + bw)] -= lik * Lb[(long long)j * ld + (k - j + bw)];
    }
    __syncthreads();
  }
}

// One forward substitution step for row a of a thread's column: v = (x - sum L[a][k] y[k]) / L[a][a]
// with the previous solved entries y[k], k in [a - bw, a), in the ring.
// x_a = (x - sum_{k in band, k < a} L[a][k] x_k) / L[a][a] for one column (this thread's), the previous
// band of solutions in the ring (slot-major, T columns).  Lrow: row a of L in band storage (ld = bw + 1,
// column k at Lrow[k - a + bw]) staged in shared memory, with 1 / L[a][a] at Lrow[bw].
__device__ __forceinline__ float ring_solve_row(float x, int a, int bw, int R, int wslot, const float* Lrow,
                                                const float* ring, int T, int tid) {
  int k0 = max(0, a - bw);
  const float* la = Lrow + (k0 - a + bw);
  int slot = wslot - (a - k0);
  if (slot < 0) slot += R;
  int len = a - k0, seg = min(len, R - slot);
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
  const float* r1 = ring + (long long)slot * T + tid;
  int q = 0;
  for (; q + 4 <= seg; q += 4) {
    acc0 += la[q] * r1[(long long)q * T];
    acc1 += la[q + 1] * r1[(long long)(q + 1) * T];
    acc2 += la[q + 2] * r1[(long long)(q + 2) * T];
    acc3 += la[q + 3] * r1[(long long)(q + 3) * T];
  }
  for (; q < seg; ++q) acc0 += la[q] * r1[(long long)q * T];
  const float* la2 = la + seg;
  const float* r2 = ring + tid;
  int rest = len - seg;
  q = 0;
  for (; q + 4 <= rest; q += 4) {
    acc0 += la2[q] * r2[(long long)q * T];
    acc1 += la2[q + 1] * r2[(long long)(q + 1) * T];
    acc2 += la2[q + 2] * r2[(long long)(q + 2) * T];
    acc3 += la2[q + 3] * r2[(long long)(q + 3) * T];
  }
  for (; q < rest; ++q) acc0 += la2[q] * r2[(long long)q * T];
  return (x - ((acc0 + acc1) + (acc2 + acc3))) * Lrow[bw];
}

#define HK_SF_TILE 128   // columns per CTA in the standard-form solves (= threads)
#define HK_SF_AHEAD 8    // rows loaded ahead
#define HK_SF_CHUNK 32   // rows of L staged in shared memory at a time

// Rows a0 .. a0 + HK_SF_CHUNK - 1 of the banded L (ld = bw + 1 per row) into shared memory, diagonal
// entries replaced by their reciprocals.  All threads of the CTA take part; barriers on both sides.
__device__ __forceinline__ void stage_band_rows(float* Lsh, const float* L32, int a0, int nI, int bw, int T,
                                                int tid) {
  int ld = bw + 1, rows = min(HK_SF_CHUNK, nI - a0);
  __syncthreads();
  for (int e = tid; e < rows * ld; e += T) {
    float v = L32[(long long)a0 * ld + e];
    Lsh[e] = (e % ld == bw) ? 1.f / v : v;
  }
  __syncthreads();
}

// (b): Y[:, tile] = L^{-1} (mu S mu)[:, tile].  grid = (subdomain, column tile).
__global__ void __launch_bounds__(HK_SF_TILE) k_sf_solve1(const int* __restrict__ sub_info,
                                                          const int* __restrict__ bw_arr,
                                                          const int* __restrict__ Ilev, const int* __restrict__ mu,
                                                          const long long* __restrict__ wsW,
                                                          const long long* __restrict__ wsA,
                                                          const long long* __restrict__ wsL32,
                                                          const double* __restrict__ ws, float* ws32) {
  extern __shared__ float ring[];
  int s = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], off = si[3];
  int c = blockIdx.y * T + tid;
  if (blockIdx.y * T >= nI) return;
  int bw = bw_arr[s], ld = bw + 1, R = bw + 1, lda = (nI + 3) & ~3;
  const double* W = ws + wsW[s];
  float* Y = ws32 + wsA[s];  // output slot (the caller passes the Y workspace offsets)
  const float* L32 = ws32 + wsL32[s];
  bool act = c < nI;
  double mc = act ? (double)mu[Ilev[off + c]] : 0.0;
  float* Lsh = ring + (long long)R * T;  // HK_SF_CHUNK x ld
  int wslot = 0;
  for (int a0 = 0; a0 < nI; a0 += HK_SF_AHEAD) {
    if (a0 % HK_SF_CHUNK == 0) stage_band_rows(Lsh, L32, a0, nI, bw, T, tid);
    float xin[HK_SF_AHEAD];
#pragma unroll
    for (int u = 0; u < HK_SF_AHEAD; ++u) {
      int a = a0 + u;
      xin[u] = (act && a < nI) ? (float)(W[(long long)a * nI + c] * mc * (double)mu[Ilev[off + a]]) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < HK_SF_AHEAD; ++u) {
      int a = a0 + u;
      if (a >= nI) break;
      float v = ring_solve_row(xin[u], a, bw, R, wslot, Lsh + (a % HK_SF_CHUNK) * ld, ring, T, tid);
      ring[(long long)wslot * T + tid] = v;
      if (act) Y[(long long)a * lda + c] = v;
      if (++wslot == R) wslot = 0;
    }
  }
}

// (c): A[:, tile] = L^{-1} (Y^T)[:, tile]; the tile's columns are rows of Y, staged 32 entries at a
// time through shared memory so that global reads stay coalesced.
__global__ void __launch_bounds__(HK_SF_TILE) k_sf_solve2(const int* __restrict__ sub_info,
                                                          const int* __restrict__ bw_arr,
                                                          const long long* __restrict__ wsY,
                                                          const long long* __restrict__ wsA,
                                                          const long long* __restrict__ wsL32, float* ws32) {
  extern __shared__ float ring[];
  __shared__ float stage[32][HK_SF_TILE + 1];
  int s = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  int nI = sub_info[8 * s];
  int c0 = blockIdx.y * T, c = c0 + tid;
  if (c0 >= nI) return;
  int bw = bw_arr[s], ld = bw + 1, R = bw + 1, lda = (nI + 3) & ~3;
  const float* Y = reinterpret_cast<const float*>(ws32 + wsY[s]);
  float* A = ws32 + wsA[s];
  const float* L32 = ws32 + wsL32[s];
  bool act = c < nI;
  float* Lsh = ring + (long long)R * T;  // HK_SF_CHUNK x ld
  int wslot = 0;
  for (int a0 = 0; a0 < nI; a0 += 32) {
    // stage Y[c0 + i][a0 + j] -> stage[j][i]: a warp reads 32 consecutive entries of one row
    __syncthreads();
    int lane = tid & 31, wp = tid >> 5, nwp = T >> 5;
    for (int i = wp; i < T; i += nwp) {
      int row = c0 + i, col = a0 + lane;
      stage[lane][i] = (row < nI && col < nI) ? Y[(long long)row * lda + col] : 0.f;
    }
    __syncthreads();
    stage_band_rows(Lsh, L32, a0, nI, bw, T, tid);
    for (int u = 0; u < 32 && a0 + u < nI; ++u) {
      int a = a0 + u;
      float v = ring_solve_row(stage[u][tid], a, bw, R, wslot, Lsh + u * ld, ring, T, tid);
      ring[(long long)wslot * T + tid] = v;
      if (act) A[(long long)a * lda + c] = v;
      if (++wslot == R) wslot = 0;
    }
  }
}

// ---- 4. Householder tridiagonalisation of the dense symmetric A in FP32 (O(n) reductions in FP64),
// reading and writing only the lower triangle (row stride lda = n rounded up to 4); only the
// tridiagonal (d, e) is kept.
// Step k forms the reflector H_k = I - tau v v^T (v[k+1] = 1) from column k below the diagonal, then
// needs p = tau A22 v and w = p - (tau/2)(p.v) v for the rank-2 update A22 -= v w^T + w v^T.  The
// update of step k-1 and the product of step k share one pass over the lower triangle: row i is read
// once, the pending update (v', w') is applied and written back, its dot with v gives the row part of
// p_i, and a_ij v_i (j < i) is the column part of p_j, summed in a per-warp shared-memory slice.
// The CS CTAs of a thread-block cluster share one matrix (CTA r owns rows i = r mod CS); each CTA
// rebuilds column k and the reflector redundantly, and the partial p vectors of the CTAs are added in
// rank order through distributed shared memory after one cluster barrier per step.  Shared vectors are
// zero below the active column and in the padding so that row loops start on a 16-byte boundary.
#define HK_TRI_WARPS 16
template <int CS>
__global__ void __launch_bounds__(HK_TRI_WARPS * 32) k_tridiag32(const int* __restrict__ sub_info,
                                                                 const long long* __restrict__ wsA, float* ws,
                                                                 double* dvec, double* evec,
                                                                 const int* __restrict__ vec_off) {
  extern __shared__ __align__(16) float smf[];
  __shared__ double red[32];
  __shared__ float sc[5];  // ||x||^2, beta, tau, scale, K of the current step
  int s = blockIdx.x / CS, r = blockIdx.x % CS;
  int tid = threadIdx.x, Tn = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = Tn >> 5;
  int n = sub_info[8 * s];
  int lda = (n + 3) & ~3;
  float* A = ws + wsA[s];
  double* d = dvec + vec_off[s];
  double* e = evec + vec_off[s];
  float* vo = smf;             // v of the pending update
  float* wo = vo + lda;        // w of the pending update
  float* vn = wo + lda;        // v of the current step
  float* pp = vn + lda;        // this CTA's partial p, double buffered (2 * lda)
  float* pf = pp + 2 * lda;    // full p
  float* colk = pf + lda;      // column k with the pending update applied
  float* cacc = colk + lda;    // per-warp column sums (nw * lda)
  const float4* vo4 = reinterpret_cast<const float4*>(vo);
  const float4* wo4 = reinterpret_cast<const float4*>(wo);
  const float4* vn4 = reinterpret_cast<const float4*>(vn);
  for (int j = tid; j < (7 + nw) * lda; j += Tn) smf[j] = 0.f;
  if (CS > 1) cooperative_groups::this_cluster().sync(); else __syncthreads();
  for (int k = 0; k < n - 2; ++k) {
    float vk = vo[k], wk = wo[k];
    for (int j = k + tid; j < n; j += Tn) colk[j] = A[(long long)j * lda + k] - (vo[j] * wk + wo[j] * vk);
    __syncthreads();
    float xs = 0.f;
    for (int j = k + 2 + tid; j < n; j += Tn) xs += colk[j] * colk[j];
    // ||x||^2, then the Householder scalars once, by thread 0 (FP32 like the matrix; computed by every
    // thread they would cost the whole block the latency of the square root and divisions)
    for (int o = 16; o > 0; o >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, o);
    if (lane == 0) red[warp] = xs;
    __syncthreads();
    if (warp == 0) {
      float t = lane < nw ? (float)red[lane] : 0.f;
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) {
        float alpha = colk[k + 1], beta = alpha, tau_ = 0.f, scale = 0.f;
        if (t > 0.f) {
          beta = -copysignf(sqrtf(alpha * alpha + t), alpha);
          tau_ = (beta - alpha) / beta;
          scale = 1.f / (alpha - beta);
        }
        sc[0] = t;
        sc[1] = beta;
        sc[2] = tau_;
        sc[3] = scale;
      }
    }
    __syncthreads();
    xs = sc[0];
    float beta = sc[1], tau = sc[2], scale = sc[3];
    for (int j = k + 2 + tid; j < n; j += Tn) vn[j] = colk[j] * scale;
    if (tid == 0) {
      vn[k] = 0.f;
      vn[k + 1] = xs > 0.0 ? 1.f : 0.f;
      if (r == 0) {
        d[k] = (double)colk[k];
        e[k] = beta;
      }
    }
    // clear this step's column sums
    for (int j = k + 1 + lane; j < n; j += 32) cacc[warp * lda + j] = 0.f;
    __syncthreads();
    // fused pass over the owned rows i > k, columns [k+1, i].  Column k (being read by every CTA of
    // the cluster during this step) is never written: the head chunk holding column k+1 and the
    // chunk holding the diagonal are done element by element, the chunks between them as float4.
    float* pc = pp + (k & 1) * lda;
    float* my = cacc + warp * lda;
    int i0 = k + 1 + (((r - (k + 1)) % CS) + CS) % CS;
    int hc = (k + 1) >> 2;
    float4* my4 = reinterpret_cast<float4*>(my);
    // Each warp takes its rows four at a time (rows CS*nw apart): the four rows' loads of a chunk are
    // issued together, so a lane has four independent loads in flight instead of one per row.
    const int RG = 4;
    for (int ib = i0 + CS * warp; ib < n; ib += RG * CS * nw) {
      float4* A4 = reinterpret_cast<float4*>(A);
      int ro[RG];  // row offsets in float4 units (n <= 1440: fits in int)
      float vi[RG], wi[RG], vni[RG], acc[RG];
      int cl[RG], clmax = 0;
#pragma unroll
      for (int q = 0; q < RG; ++q) {
        int i = ib + q * CS * nw;
        bool ok = i < n;
        int ii = ok ? i : ib;
        ro[q] = ii * (lda >> 2);
        vi[q] = ok ? vo[i] : 0.f;
        wi[q] = ok ? wo[i] : 0.f;
        vni[q] = ok ? vn[i] : 0.f;
        cl[q] = ok ? (i >> 2) : 0;  // chunk holding the diagonal (0: row absent)
        clmax = max(clmax, cl[q]);
        acc[q] = 0.f;
      }
      for (int c = hc + 1 + lane; c < clmax; c += 32) {
        float4 a[RG];
#pragma unroll
        for (int q = 0; q < RG; ++q)
          if (c < cl[q]) a[q] = A4[ro[q] + c];
        float4 vv = vo4[c], ww = wo4[c], nv = vn4[c];
        float4 cs = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < RG; ++q) {
          if (c >= cl[q]) continue;
          float4 t = a[q];
          t.x -= vi[q] * ww.x + wi[q] * vv.x;
          t.y -= vi[q] * ww.y + wi[q] * vv.y;
          t.z -= vi[q] * ww.z + wi[q] * vv.z;
          t.w -= vi[q] * ww.w + wi[q] * vv.w;
          A4[ro[q] + c] = t;
          acc[q] += t.x * nv.x + t.y * nv.y + t.z * nv.z + t.w * nv.w;
          cs.x += t.x * vni[q];
          cs.y += t.y * vni[q];
          cs.z += t.z * vni[q];
          cs.w += t.w * vni[q];
        }
        float4 mm = my4[c];
        mm.x += cs.x;
        mm.y += cs.y;
        mm.z += cs.z;
        mm.w += cs.w;
        my4[c] = mm;
      }
      __syncwarp();
      // head chunk (columns k+1 .. 4 hc + 3) and diagonal chunk (4 cl .. i), one element per lane:
      // lanes 8q .. 8q+7 serve row q (0-3 head, 4-7 diagonal chunk), all four rows at once.  The
      // head chunk's columns are shared by the four rows: their column sums are added across the
      // row groups by shuffles and written once; the diagonal chunks of the rows are disjoint.
      {
        int q = lane >> 3, l8 = lane & 7;
        int i = ib + q * CS * nw;
        float vq = q == 0 ? vi[0] : q == 1 ? vi[1] : q == 2 ? vi[2] : vi[3];
        float wq = q == 0 ? wi[0] : q == 1 ? wi[1] : q == 2 ? wi[2] : wi[3];
        float nq = q == 0 ? vni[0] : q == 1 ? vni[1] : q == 2 ? vni[2] : vni[3];
        int clq = q == 0 ? cl[0] : q == 1 ? cl[1] : q == 2 ? cl[2] : cl[3];
        int j = l8 < 4 ? 4 * hc + l8 : (clq > hc ? 4 * clq + l8 - 4 : -1);
        bool ok = i < n && j >= k + 1 && j <= i;
        float ex = 0.f, cv = 0.f;
        if (ok) {
          float* rowp = A + (long long)i * lda;
          float a = rowp[j] - (vq * wo[j] + wq * vo[j]);
          rowp[j] = a;
          ex = a * vn[j];
          if (j < i) cv = a * nq;
        }
        float hs = cv + __shfl_xor_sync(0xffffffffu, cv, 8);
        hs += __shfl_xor_sync(0xffffffffu, hs, 16);
        if (l8 < 4) {
          if (q == 0 && j >= k + 1 && j < n) my[j] += hs;  // 4 hc + 3 may pass the last row
        } else if (ok && j < i) {
          my[j] += cv;
        }
#pragma unroll
        for (int t = 0; t < RG; ++t) acc[t] += (q == t) ? ex : 0.f;
      }
      // the four row sums at once: butterfly over lanes keeping two, then one value per lane
      {
        bool b4 = lane & 16, b3 = lane & 8;
        float x0 = b4 ? acc[2] : acc[0], x1 = b4 ? acc[3] : acc[1];
        float y0 = b4 ? acc[0] : acc[2], y1 = b4 ? acc[1] : acc[3];
        x0 += __shfl_xor_sync(0xffffffffu, y0, 16);
        x1 += __shfl_xor_sync(0xffffffffu, y1, 16);
        float z = b3 ? x1 : x0, zo = b3 ? x0 : x1;
        z += __shfl_xor_sync(0xffffffffu, zo, 8);
        z += __shfl_xor_sync(0xffffffffu, z, 4);
        z += __shfl_xor_sync(0xffffffffu, z, 2);
        z += __shfl_xor_sync(0xffffffffu, z, 1);
        int q = (b4 ? 2 : 0) + (b3 ? 1 : 0);
        int i = ib + q * CS * nw;
        if ((lane & 7) == 0 && i < n) pc[i] = z;  // row part (owned rows only)
      }
      __syncwarp();
    }
    __syncthreads();
    // partial p of this CTA: row parts of its rows + column sums of all its warps
    for (int j = k + 1 + tid; j < n; j += Tn) {
      float t0 = (j % CS == r) ? pc[j] : 0.f, t1 = 0.f;
#pragma unroll
      for (int w = 0; w < HK_TRI_WARPS; w += 2) {
        t0 += cacc[w * lda + j];
        t1 += cacc[(w + 1) * lda + j];
      }
      pc[j] = t0 + t1;
    }
    if (CS > 1) {
      cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
      cl.sync();
      for (int j = k + 1 + tid; j < n; j += Tn) {
        float t = 0.f;
        for (int q = 0; q < CS; ++q) t += q == r ? pc[j] : *cl.map_shared_rank(pc + j, q);
        pf[j] = (float)tau * t;
      }
    } else {
      __syncthreads();
      for (int j = k + 1 + tid; j < n; j += Tn) pf[j] = (float)tau * pc[j];
    }
    __syncthreads();
    float pv = 0.f;
    for (int j = k + 1 + tid; j < n; j += Tn) pv += pf[j] * vn[j];
    for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
    if (lane == 0) red[warp] = pv;
    __syncthreads();
    if (warp == 0) {
      float t = lane < nw ? (float)red[lane] : 0.f;
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) sc[4] = 0.5f * tau * t;
    }
    __syncthreads();
    float K = sc[4];
    for (int j = tid; j < lda; j += Tn) {
      float vj = j > k ? vn[j] : 0.f;
      vo[j] = vj;
      wo[j] = j > k ? pf[j] - K * vj : 0.f;
    }
    __syncthreads();
  }
  if (CS > 1) cooperative_groups::this_cluster().sync(); else __syncthreads();
  if (r == 0 && tid == 0) {
    if (n >= 2) {
      int a2 = n - 2, a3 = n - 1;
      float x22 = A[(long long)a2 * lda + a2] - 2.f * vo[a2] * wo[a2];
      float x32 = A[(long long)a3 * lda + a2] - (vo[a3] * wo[a2] + wo[a3] * vo[a2]);
      float x33 = A[(long long)a3 * lda + a3] - 2.f * vo[a3] * wo[a3];
      d[a2] = (double)x22;
      e[a2] = (double)x32;
      d[a3] = (double)x33;
    } else {
      d[0] = (double)A[0];
    }
  }
}

// Sturm count (number of eigenvalues below x) of the symmetric tridiagonal matrix (d, e), FP32.
__device__ __forceinline__ int sturm_count32(const float* d, const float* e2, int n, float x, float pivmin) {
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

// ---- 5. candidates: every eigenvalue of the tridiagonal matrix below tau + delta.  The FP32
// tridiagonal matrix sits in shared memory; each warp refines one eigenvalue by 32-way multisection
// (its lanes count at 32 points of the current bracket) down to 1e-6 of the spectral scale.
__global__ void k_candidates(const int* __restrict__ sub_info, const double* __restrict__ dvec,
                             const double* __restrict__ evec, const int* __restrict__ vec_off, double tau,
                             double* lam_hat, int* cnt_out, DevStatus* st) {
  extern __shared__ float smc[];
  __shared__ float lo_s, hi_s, pm_s;
  __shared__ int cnt_s;
  int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int n = sub_info[8 * s];
  float* d = smc;
  float* e2 = smc + n;
  const double* dg = dvec + vec_off[s];
  const double* eg = evec + vec_off[s];
  for (int i = tid; i < n; i += blockDim.x) {
    d[i] = (float)dg[i];
    e2[i] = i < n - 1 ? (float)(eg[i] * eg[i]) : 0.f;
  }
  __syncthreads();
  if (tid == 0) {
    double lo = 1e300, hi = -1e300, me = 0;
    for (int i = 0; i < n; ++i) {
      double r = (i > 0 ? fabs(eg[i - 1]) : 0.0) + (i < n - 1 ? fabs(eg[i]) : 0.0);
      lo = fmin(lo, dg[i] - r);
      hi = fmax(hi, dg[i] + r);
      if (i < n - 1) me = fmax(me, eg[i] * eg[i]);
    }
    double span = fmax(fabs(lo), fabs(hi));
    lo -= 1e-6 * span + 1e-30;
    hi += 1e-6 * span + 1e-30;
    lo_s = (float)lo;
    hi_s = (float)hi;
    pm_s = (float)(1e-30 * fmax(1.0, me));
    float x = (float)(tau + HK_EIG_DELTA);
    int c = x >= hi_s ? n : (x <= lo_s ? 0 : sturm_count32(d, e2, n, x, pm_s));
    cnt_s = c;
    cnt_out[s] = c;
    if (c > HK_MAXM) dev_fail(st, HK_UNSUPPORTED, s, c);
  }
  __syncthreads();
  int c = min(cnt_s, HK_MAXM);
  float tol = 1e-6f * fmaxf(fabsf(lo_s), fabsf(hi_s));
  for (int t = warp; t < c; t += nw) {
    float lo = lo_s, hi = hi_s;
    for (int it = 0; it < 12 && hi - lo > tol; ++it) {
      float x = lo + (hi - lo) * (float)(lane + 1) / 33.f;
      int below = sturm_count32(d, e2, n, x, pm_s) > t;  // eigenvalue t lies below x
      unsigned mask = __ballot_sync(0xffffffffu, below);
      int first = mask ? __ffs(mask) - 1 : 32;          // lowest point above eigenvalue t
      float nlo = first == 0 ? lo : lo + (hi - lo) * (float)first / 33.f;
      float nhi = first == 32 ? hi : lo + (hi - lo) * (float)(first + 1) / 33.f;
      lo = nlo;
      hi = nhi;
    }
    if (lane == 0) lam_hat[(long long)s * HK_MAXM + t] = 0.5 * ((double)lo + (double)hi);
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
  double* Ps = P + poff[s];
  // scale for the pivot floor
  double mx = 0;
  for (long long e = tid; e < (long long)nO * maxrow; e += T) {
    int a = (int)(e / maxrow), q = (int)(e % maxrow);
    if (q < ocnt[oo + a]) mx = fmax(mx, fabs(oB[(long long)oo * maxrow + e] - sigma * oC[(long long)oo * maxrow + e]));
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
      int cnt = min(ocnt[oo + a], maxrow);
      double v = 0;
      for (int q = 0; q < cnt; ++q) {
        int c = ocol[base + q];
        double mv = oB[base + q] - sigma * oC[base + q];
        if (c == r0 + t) v += mv;
        else if (j > 0 && c >= prev_r0 && c < r0) v -= mv * Fw[prev_go + (long long)(c - prev_r0) * b + t];
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
      int cnt = min(ocnt[oo + c], maxrow);
      double v = 0;
      for (int q = 0; q < cnt; ++q) {
        int a = ocol[base + q];
        if (a >= r0 && a < r1) v += S[qt * b + (a - r0)] * (oB[base + q] - sigma * oC[base + q]);
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
  for (int step = 0; step < HK_REFINE_STEPS; ++step) {
    // R = C X, then X = M^{-1} R by the two block sweeps
    o_matvec(nO, oo, maxrow, ocnt, ocol, oB, oC, 1.0, 0, X, R, p);
    __syncthreads();
    long long fo = 0;
    for (int j = 0; j < L; ++j) {
      int r0 = lp[j], b = lp[j + 1] - r0, bn = j + 1 < L ? lp[j + 2] - lp[j + 1] : 0;
      for (int e = tid; e < b * p; e += T) {
        int t = e / b, a = r0 + e % b;
        long long base = (long long)(oo + a) * maxrow;
        int cnt = min(ocnt[oo + a], maxrow);
        double acc = R[(long long)t * nO + a];
        for (int q = 0; q < cnt; ++q) {
          int c = ocol[base + q];
          if (c < r0) acc -= (oB[base + q] - sigma * oC[base + q]) * R[(long long)t * nO + c];
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
__global__ void k_select(const int* __restrict__ cnt, const double* __restrict__ lam_ref, double tau, int* sel,
                         int* m_out, double* lam_out, DevStatus* st) {
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
  double thr = 1e-8 * fmax(1.0, fabs(tau));
  while (m > 0 && m < c && lr[ord[m]] - lr[ord[m - 1]] <= thr) ++m;
  if (m == c && c == cnt[s] && m > 0 && lr[ord[m - 1]] >= tau) dev_fail(st, HK_EIG_FAIL, s, m);
  m_out[s] = m;
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
  // ---- workspace layout (FP64 part and FP32 part)
  std::vector<long long> W(ns), Lw(ns), Gw(ns), Rw(ns), Aw(ns), L32w(ns), Yw(ns);
  std::vector<int> voff(ns), bw(ns), o_off(ns), oc(ns);
  long long tot = 0, tot32 = 0;
  int vo = 0, maxn = 0, O_total = 0;
  for (int s = 0; s < ns; ++s) {
    const Sub& u = h->subs[s];
    long long nI = u.nI, nG = u.nG;
    W[s] = tot; tot += nI * nI;
    Lw[s] = tot; tot += nI * (u.bw + 1);
    Gw[s] = tot; tot += nG * nG;
    Rw[s] = tot; tot += nG * nI;
    tot = (tot + 3) & ~3LL;
    Aw[s] = tot32; tot32 += nI * ((nI + 3) & ~3LL);
    Yw[s] = tot32; tot32 += nI * ((nI + 3) & ~3LL);
    L32w[s] = tot32; tot32 += nI * (u.bw + 1);
    tot32 = (tot32 + 3) & ~3LL;
    voff[s] = vo;
    vo += u.nI;
    bw[s] = u.bw;
    maxn = std::max(maxn, u.nI);
    o_off[s] = O_total;
    oc[s] = u.nI + u.nG;
    O_total += oc[s];
  }
  double* d_ws = nullptr;
  float* d_ws32 = nullptr;
  long long *d_W = nullptr, *d_L = nullptr, *d_Gw = nullptr, *d_Rw = nullptr, *d_A = nullptr, *d_L32 = nullptr,
            *d_Y = nullptr;
  int *d_voff = nullptr, *d_bw = nullptr, *d_ring = nullptr, *d_cnt = nullptr, *d_o_off = nullptr;
  double *d_d = nullptr, *d_e = nullptr, *d_lamhat = nullptr, *d_lamref = nullptr;
  float* d_tau = nullptr;
  HK_TRY(dalloc(h, &d_ws, tot));
  HK_TRY(dalloc(h, &d_ws32, tot32));
  HK_TRY(dalloc(h, &d_W, ns));
  HK_TRY(dalloc(h, &d_L, ns));
  HK_TRY(dalloc(h, &d_Gw, ns));
  HK_TRY(dalloc(h, &d_Rw, ns));
  HK_TRY(dalloc(h, &d_A, ns));
  HK_TRY(dalloc(h, &d_L32, ns));
  HK_TRY(dalloc(h, &d_Y, ns));
  HK_TRY(dalloc(h, &d_voff, ns));
  HK_TRY(dalloc(h, &d_bw, ns));
  HK_TRY(dalloc(h, &d_ring, h->I_total));
  HK_TRY(dalloc(h, &d_cnt, ns));
  HK_TRY(dalloc(h, &d_o_off, ns));
  HK_TRY(dalloc(h, &d_d, vo));
  HK_TRY(dalloc(h, &d_e, vo));
  HK_TRY(dalloc(h, &d_tau, vo));
  HK_TRY(dalloc(h, &d_lamhat, (size_t)ns * HK_MAXM));
  HK_TRY(dalloc(h, &d_lamref, (size_t)ns * HK_MAXM));
  HK_TRY(dalloc(h, &h->d_lam, (size_t)ns * HK_MAXM));
  auto up = [&](void* d, const void* hsrc, size_t bytes) {
    return cudaMemcpyAsync(d, hsrc, bytes, cudaMemcpyHostToDevice, st);
  };
  HK_CUDA(up(d_W, W.data(), 8 * ns));
  HK_CUDA(up(d_L, Lw.data(), 8 * ns));
  HK_CUDA(up(d_Gw, Gw.data(), 8 * ns));
  HK_CUDA(up(d_Rw, Rw.data(), 8 * ns));
  HK_CUDA(up(d_A, Aw.data(), 8 * ns));
  HK_CUDA(up(d_L32, L32w.data(), 8 * ns));
  HK_CUDA(up(d_Y, Yw.data(), 8 * ns));
  HK_CUDA(up(d_voff, voff.data(), 4 * ns));
  HK_CUDA(up(d_bw, bw.data(), 4 * ns));
  HK_CUDA(up(d_o_off, o_off.data(), 4 * ns));
  // The banded Cholesky of D_II needs only D_k and the band widths: it runs on the handle's second
  // stream beside the Gamma-block, ovdof and Gamma-elimination kernels (disjoint workspace regions)
  // and joins before the standard form.
  bool side = h->co_stream && h->ev_fork && h->ev_join;
  if (side) {
    HK_CUDA(cudaEventRecord(h->ev_fork, st));
    HK_CUDA(cudaStreamWaitEvent(h->co_stream, h->ev_fork, 0));
    k_dchol<<<ns, 512, 0, h->co_stream>>>(h->d_sub_info, h->d_sub_off, d_bw, h->d_lrow, h->d_lcntI, h->d_lcol,
                                          h->d_lvalD, d_L, d_L32, d_ws, d_ws32, h->d_status);
    HK_COUNT_LAUNCH();
    HK_LAUNCH_CHECK();
    HK_CUDA(cudaEventRecord(h->ev_join, h->co_stream));
  }

  // ---- B^N on Gamma x Gamma, then the ovdof structure (before the Cholesky of BG overwrites it)
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

  // ---- FP32 dense stage
  k_schur<<<ns, 256, 0, st>>>(h->d_sub_info, h->d_sub_off, h->d_lrow, h->d_lcntI, h->d_lcntG, h->d_lcol,
                              h->d_lvalB, d_W, d_Gw, d_Rw, d_ring, d_ws, h->d_status);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  int maxbw = 0;
  for (int s = 0; s < ns; ++s) maxbw = std::max(maxbw, bw[s]);
  size_t sf_shm = sizeof(float) * (size_t)(maxbw + 1) * (HK_SF_TILE + HK_SF_CHUNK);
  if (sf_shm > 180 * 1024) {
    hk_set_error("local band width %d too large for the standard-form kernels", maxbw);
    return HK_UNSUPPORTED;
  }
  if (side) {
    HK_CUDA(cudaStreamWaitEvent(st, h->ev_join, 0));
  } else {
    k_dchol<<<ns, 512, 0, st>>>(h->d_sub_info, h->d_sub_off, d_bw, h->d_lrow, h->d_lcntI, h->d_lcol, h->d_lvalD,
                                d_L, d_L32, d_ws, d_ws32, h->d_status);
    HK_COUNT_LAUNCH();
    HK_LAUNCH_CHECK();
  }
  HK_TRY(check_device_status(h, "eigen: Gamma elimination and Cholesky of D_II"));
  dim3 sfgrid(ns, (maxn + HK_SF_TILE - 1) / HK_SF_TILE);
  HK_TRY(hk_allow_smem(k_sf_solve1));
  HK_TRY(hk_allow_smem(k_sf_solve2));
  k_sf_solve1<<<sfgrid, HK_SF_TILE, sf_shm, st>>>(h->d_sub_info, d_bw, h->d_I, h->d_mu, d_W, d_Y, d_L32, d_ws,
                                                  d_ws32);
  HK_COUNT_LAUNCH();
  k_sf_solve2<<<sfgrid, HK_SF_TILE, sf_shm, st>>>(h->d_sub_info, d_bw, d_Y, d_A, d_L32, d_ws32);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_TRY(check_device_status(h, "eigen: standard form"));
  size_t shm = sizeof(float) * (7 + HK_TRI_WARPS) * (size_t)((maxn + 3) & ~3);
  if (shm > 225 * 1024) {
    hk_set_error("subdomain with %d dofs too large for the shared-memory tridiagonalisation", maxn);
    return HK_UNSUPPORTED;
  }
  int CS = 1;
  {
    // spread the subdomains over the SMs: a cluster of CS CTAs per subdomain, as many CTAs as fit at
    // once (two per SM when their shared memory allows)
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev);
    int per_sm = 2 * (shm + 2048) <= 228 * 1024 ? 2 : 1;
    while (CS < 4 && (long long)ns * CS * 2 <= (long long)nsm * per_sm) CS *= 2;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ns * CS);
    cfg.blockDim = dim3(HK_TRI_WARPS * 32);
    cfg.dynamicSmemBytes = shm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (CS == 4) {
      HK_TRY(hk_allow_smem(k_tridiag32<4>));
      HK_CUDA(cudaLaunchKernelEx(&cfg, k_tridiag32<4>, (const int*)h->d_sub_info, (const long long*)d_A, d_ws32, d_d,
                                 d_e, (const int*)d_voff));
    } else if (CS == 2) {
      HK_TRY(hk_allow_smem(k_tridiag32<2>));
      HK_CUDA(cudaLaunchKernelEx(&cfg, k_tridiag32<2>, (const int*)h->d_sub_info, (const long long*)d_A, d_ws32, d_d,
                                 d_e, (const int*)d_voff));
    } else {
      HK_TRY(hk_allow_smem(k_tridiag32<1>));
      HK_CUDA(cudaLaunchKernelEx(&cfg, k_tridiag32<1>, (const int*)h->d_sub_info, (const long long*)d_A, d_ws32, d_d,
                                 d_e, (const int*)d_voff));
    }
    HK_COUNT_LAUNCH();
  }
  cudaEventRecord(e1, st);
  HK_LAUNCH_CHECK();
  size_t cshm = sizeof(float) * 2 * (size_t)maxn;
  HK_TRY(hk_allow_smem(k_candidates));
  k_candidates<<<ns, 512, cshm, st>>>(h->d_sub_info, d_d, d_e, d_voff, h->p.tau, d_lamhat, d_cnt, h->d_status);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_TRY(check_device_status(h, "eigen: candidates"));
  std::vector<int> cnt(ns);
  std::vector<double> lamhat((size_t)ns * HK_MAXM);
  HK_CUDA(cudaMemcpyAsync(cnt.data(), d_cnt, 4 * ns, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaMemcpyAsync(lamhat.data(), d_lamhat, sizeof(double) * lamhat.size(), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  {
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    h->setup_ms[6] = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  std::vector<long long> poff(ns);
  long long ptot = 0;
  for (int s = 0; s < ns; ++s) {
    poff[s] = ptot;
    ptot += (long long)h->subs[s].nI * cnt[s];
  }
  double* d_P = nullptr;
  long long* d_poff = nullptr;
  HK_TRY(dalloc(h, &d_P, ptot));
  HK_TRY(dalloc(h, &d_poff, ns));
  HK_CUDA(up(d_poff, poff.data(), 8 * ns));

  // ---- FP64 refinement: clusters of candidates, one CTA each
  std::vector<int> levO(O_total + ns);
  HK_CUDA(cudaMemcpyAsync(levO.data(), d_Olevptr, sizeof(int) * levO.size(), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  std::vector<long long> fsize(ns, 0);
  for (int s = 0; s < ns; ++s) {
    const int* lp = &levO[o_off[s] + s];
    for (int j = 0; j < OL[s]; ++j) {
      long long b = lp[j + 1] - lp[j], bn = j + 1 < OL[s] ? lp[j + 2] - lp[j + 1] : 0;
      fsize[s] += b * b + b * bn;
    }
  }
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
      xtot += 2LL * (t1 - t + HK_GUARD) * oc[s];
      pmax = std::max(pmax, t1 - t + HK_GUARD);
      t = t1;
    }
  }
  int nit = (int)sig.size();
  if (nit > 0) {
    int* d_items = nullptr;
    double *d_sig = nullptr, *d_F = nullptr, *d_X = nullptr;
    long long *d_foff = nullptr, *d_xoff = nullptr;
    HK_TRY(dalloc(h, &d_items, items.size()));
    HK_TRY(dalloc(h, &d_sig, nit));
    HK_TRY(dalloc(h, &d_foff, nit));
    HK_TRY(dalloc(h, &d_xoff, nit));
    HK_TRY(dalloc(h, &d_F, ftot));
    HK_TRY(dalloc(h, &d_X, xtot));
    HK_CUDA(up(d_items, items.data(), 4 * items.size()));
    HK_CUDA(up(d_sig, sig.data(), 8 * nit));
    HK_CUDA(up(d_foff, foff.data(), 8 * nit));
    HK_CUDA(up(d_xoff, xoff.data(), 8 * nit));
    size_t rshm = sizeof(double) * ((size_t)maxbO * maxbO + (size_t)maxbO * pmax);
    int s_in_smem = rshm <= 190 * 1024;
    if (!s_in_smem) rshm = sizeof(double) * (size_t)maxbO * pmax;
    HK_TRY(hk_allow_smem(k_refine));
    k_refine<<<nit, 128, rshm, st>>>(d_items, d_sig, h->d_sub_info, d_o_off, d_Olevptr, d_OL, maxrow, d_ocnt, d_ocol,
                                     d_oB, d_oC, d_o2i, d_foff, d_xoff, d_F, d_X, d_poff, d_P, d_lamhat, d_lamref,
                                     maxbO, s_in_smem, h->d_status);
    HK_COUNT_LAUNCH();
    HK_LAUNCH_CHECK();
    HK_CUDA(cudaStreamSynchronize(st));
    HK_TRY(check_device_status(h, "eigen: refinement"));
    void* tmpf[] = {d_items, d_sig, d_foff, d_xoff, d_F, d_X};
    for (void* p : tmpf) dfree(h, p);
  }
  int *d_sel = nullptr, *d_m = nullptr;
  HK_TRY(dalloc(h, &d_sel, (size_t)ns * HK_MAXM));
  HK_TRY(dalloc(h, &d_m, ns));
  k_select<<<ns, 32, 0, st>>>(d_cnt, d_lamref, h->p.tau, d_sel, d_m, h->d_lam, h->d_status);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
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
  void* tmp[] = {d_ws, d_ws32, d_W, d_L, d_Gw, d_Rw, d_A, d_L32, d_Y, d_voff, d_bw, d_ring, d_cnt, d_o_off, d_d, d_e,
                 d_tau, d_lamhat, d_lamref, d_O, d_okind, d_Operm, d_Olev, d_Olevptr, d_OL, d_ocnt, d_o2i, d_ocol,
                 d_oB, d_oC, d_P, d_poff, d_sel, d_m};
  for (void* p : tmp) dfree(h, p);
  return HK_OK;
}
