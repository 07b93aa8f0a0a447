// H_k-GenEO local eigenproblems (Eq. 5.12) and the coarse basis (Def. 5.1),
// one CTA per subdomain, FP64 throughout.
//
// On ovdof(Omega_i) the problem is B^N p = lambda C p with B^N the local
// Neumann Helmholtz matrix (element sums over Omega_i) and C = Xi D^N Xi,
// Xi = diag(1/mu on dof, 0 on Gamma = ovdof \ dof).  For dof rows and
// columns B^N and D^N equal the global B and D_k (the star of a dof lies in
// Omega_i); only the Gamma-Gamma block of B^N is local.  Eliminating the
// Gamma unknowns (C vanishes there) gives the symmetric-definite pencil
//     S p = lambda C_II p,   S = B_II - B_IG (B^N_GG)^{-1} B_GI,
//     C_II = X D_II X,  X = diag(1/mu),
// whose eigenvalues are real (the paper's lemma on indefinite pencils).
// With the Cholesky factor D_II = L L^T (banded in level order) the standard
// form is  A q = lambda q,  A = L^{-1} (mu S mu) L^{-T},  p = X^{-1} L^{-T} q,
// and the coarse vector is Xi p = L^{-T} q, already c-normalised.
// A is reduced to tridiagonal form by Householder reflections; eigenvalues
// below tau come from Sturm-count bisection, eigenvectors from inverse
// iteration on the tridiagonal matrix, then the reflections and L^{-T} are
// applied.  Ties across tau (gap <= 1e-8 max(1,|tau|)) are kept together.
#include "hk_internal.cuh"

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

struct EigWs {
  long long W_off, T_off, L_off, G_off, R_off;  // per-subdomain offsets in the workspace
};

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
  for (long long e = tid; e < (long long)nI * nI; e += T) W[e] = 0.0;
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
  // Cholesky of BGG in place (lower), right-looking
  for (int k = 0; k < nG; ++k) {
    double piv = BG[(long long)k * nG + k];
    if (piv <= 0.0) {
      if (tid == 0) dev_fail(st, HK_EIG_FAIL, s, piv);
      return;
    }
    double lkk = sqrt(piv);
    __syncthreads();
    for (int i = k + 1 + tid; i < nG; i += T) BG[(long long)i * nG + k] /= lkk;
    __syncthreads();
    if (tid == 0) BG[(long long)k * nG + k] = lkk;
    for (long long e = tid; e < (long long)(nG - k - 1) * (nG - k - 1); e += T) {
      int i = k + 1 + (int)(e / (nG - k - 1)), j = k + 1 + (int)(e % (nG - k - 1));
      if (j <= i) BG[(long long)i * nG + j] -= BG[(long long)i * nG + k] * BG[(long long)j * nG + k];
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
      R[(long long)i * nR + r] = v / BG[(long long)i * nG + i];
    }
    for (int i = nG - 1; i >= 0; --i) {
      double v = R[(long long)i * nR + r];
      for (int k = i + 1; k < nG; ++k) v -= BG[(long long)k * nG + i] * R[(long long)k * nR + r];
      R[(long long)i * nR + r] = v / BG[(long long)i * nG + i];
    }
  }
  __syncthreads();
  // W[ring a][ring b] -= sum_g B[a][g] X[g][b]
  for (long long e = tid; e < (long long)nR * nR; e += T) {
    int ra = (int)(e / nR), rb = (int)(e % nR);
    int a = ring[ra];
    long long b0 = coff + lr[a] + lcntI[off + a];
    double v = 0;
    for (int q = 0; q < lcntG[off + a]; ++q) v += lvalB[b0 + q] * R[(long long)lcol[b0 + q] * nR + rb];
    W[(long long)a * nI + ring[rb]] -= v;
  }
}

// ---- 3. banded Cholesky of D_II (level order) into Lb (nI x (bw+1)):
// Lb[a][t] = L[a][a - bw + t].  Then A = L^{-1} (mu S mu) L^{-T}.
__global__ void k_stdform(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                          const int* __restrict__ bw_arr, const int* __restrict__ Ilev, const int* __restrict__ mu,
                          const int* __restrict__ lrow, const int* __restrict__ lcntI, const int* __restrict__ lcol,
                          const double* __restrict__ lvalD, const long long* __restrict__ wsW,
                          const long long* __restrict__ wsT, const long long* __restrict__ wsL, double* ws,
                          DevStatus* st) {
  int s = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], off = si[3];
  int bw = bw_arr[s];
  int ld = bw + 1;
  long long coff = sub_off[3 * s + 1];
  const int* lr = lrow + off + s;
  double* W = ws + wsW[s];
  double* Tm = ws + wsT[s];
  double* Lb = ws + wsL[s];
  for (long long e = tid; e < (long long)nI * ld; e += T) Lb[e] = 0.0;
  __syncthreads();
  for (int a = tid; a < nI; a += T) {
    long long b0 = coff + lr[a];
    for (int q = 0; q < lcntI[off + a]; ++q) {
      int c = lcol[b0 + q];
      if (c <= a) Lb[(long long)a * ld + (c - a + bw)] = lvalD[b0 + q];
    }
  }
  __syncthreads();
  // right-looking banded Cholesky
  for (int k = 0; k < nI; ++k) {
    double piv = Lb[(long long)k * ld + bw];
    if (!(piv > 0.0)) {
      if (tid == 0) dev_fail(st, HK_EIG_FAIL, s, piv);
      return;
    }
    double lkk = sqrt(piv);
    int iend = min(nI - 1, k + bw);
    __syncthreads();
    for (int i = k + 1 + tid; i <= iend; i += T) Lb[(long long)i * ld + (k - i + bw)] /= lkk;
    __syncthreads();
    if (tid == 0) Lb[(long long)k * ld + bw] = lkk;
    int w = iend - k;
    for (int e = tid; e < w * w; e += T) {
      int i = k + 1 + e / w, j = k + 1 + e % w;
      if (j <= i) Lb[(long long)i * ld + (j - i + bw)] -= Lb[(long long)i * ld + (k - i + bw)] * Lb[(long long)j * ld + (k - j + bw)];
    }
    __syncthreads();
  }
  // W <- mu S mu, then column-wise forward substitution W <- L^{-1} W
  for (long long e = tid; e < (long long)nI * nI; e += T) {
    int a = (int)(e / nI), c = (int)(e % nI);
    W[e] *= (double)mu[Ilev[off + a]] * (double)mu[Ilev[off + c]];
  }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    double* M = pass == 0 ? W : Tm;
    for (int c = tid; c < nI; c += T) {
      for (int a = 0; a < nI; ++a) {
        double v = M[(long long)a * nI + c];
        int k0 = max(0, a - bw);
        const double* la = Lb + (long long)a * ld + (k0 - a + bw);
        for (int k = k0; k < a; ++k) v -= la[k - k0] * M[(long long)k * nI + c];
        M[(long long)a * nI + c] = v / Lb[(long long)a * ld + bw];
      }
    }
    __syncthreads();
    if (pass == 0) {
      for (long long e = tid; e < (long long)nI * nI; e += T) {
        int a = (int)(e / nI), c = (int)(e % nI);
        Tm[(long long)c * nI + a] = W[e];
      }
      __syncthreads();
    }
  }
  // symmetrise into W
  for (long long e = tid; e < (long long)nI * nI; e += T) {
    int a = (int)(e / nI), c = (int)(e % nI);
    W[e] = 0.5 * (Tm[e] + Tm[(long long)c * nI + a]);
  }
}

// ---- 4. Householder tridiagonalisation of the dense symmetric A (full storage).
// Reflector k: H_k = I - tau_k v v^T, v[k+1] = 1, v[j] stored in A[k][j] (j >= k+2).
// d = diagonal, e = off-diagonal of the tridiagonal matrix.
__global__ void k_tridiag(const int* __restrict__ sub_info, const long long* __restrict__ wsW, double* ws,
                          double* dvec, double* evec, double* tauv, const int* __restrict__ vec_off) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  int s = blockIdx.x, tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  const int* si = sub_info + 8 * s;
  int n = si[0];
  double* A = ws + wsW[s];
  double* d = dvec + vec_off[s];
  double* e = evec + vec_off[s];
  double* tv = tauv + vec_off[s];
  double* v = sm;       // n
  double* p = sm + n;   // n
  for (int k = 0; k < n - 2; ++k) {
    double* rk = A + (long long)k * n;
    double alpha = rk[k + 1];
    double xs = 0;
    for (int j = k + 2 + tid; j < n; j += T) xs += rk[j] * rk[j];
    xs = block_sum(xs, red);
    double tau = 0, beta = alpha;
    if (xs > 0.0) {
      beta = -copysign(sqrt(alpha * alpha + xs), alpha);
      tau = (beta - alpha) / beta;
      double scale = 1.0 / (alpha - beta);
      for (int j = k + 2 + tid; j < n; j += T) {
        double vj = rk[j] * scale;
        rk[j] = vj;
        v[j] = vj;
      }
    } else {
      for (int j = k + 2 + tid; j < n; j += T) v[j] = rk[j];
    }
    if (tid == 0) {
      v[k + 1] = 1.0;
      d[k] = rk[k];
      e[k] = beta;
      tv[k] = tau;
    }
    __syncthreads();
    if (tau == 0.0) continue;
    // p = tau * A22 v  (warp per row)
    for (int i = k + 1 + warp; i < n; i += nw) {
      const double* ri = A + (long long)i * n;
      double acc = 0;
      for (int j = k + 1 + lane; j < n; j += 32) acc += ri[j] * v[j];
      acc = warp_sum(acc);
      if (lane == 0) p[i] = tau * acc;
    }
    __syncthreads();
    double pv = 0;
    for (int j = k + 1 + tid; j < n; j += T) pv += p[j] * v[j];
    pv = block_sum(pv, red);
    double K = 0.5 * tau * pv;
    for (int j = k + 1 + tid; j < n; j += T) p[j] -= K * v[j];  // p becomes w
    __syncthreads();
    int m = n - k - 1;
    for (long long q = tid; q < (long long)m * m; q += T) {
      int i = k + 1 + (int)(q / m), j = k + 1 + (int)(q % m);
      A[(long long)i * n + j] -= v[i] * p[j] + p[i] * v[j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(long long)(n - 2) * n + n - 2];
      e[n - 2] = A[(long long)(n - 1) * n + n - 2];
      tv[n - 2] = 0.0;
    }
    d[n - 1] = A[(long long)(n - 1) * n + n - 1];
  }
}

__device__ int sturm_count(const double* d, const double* e, int n, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++c;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++c;
  }
  return c;
}

// ---- 5. bisection: eigenvalues 0 .. (count below tau) + extra, selection rule.
#define HK_EXTRA 8
__global__ void k_bisect(const int* __restrict__ sub_info, const double* __restrict__ dvec,
                         const double* __restrict__ evec, const int* __restrict__ vec_off, double tau,
                         double* lam_all, int* m_out, DevStatus* st) {
  __shared__ double lo_s, hi_s, pm_s;
  __shared__ int cnt_s, nc_s;
  __shared__ double lamsh[HK_MAXM + HK_EXTRA];
  int s = blockIdx.x, tid = threadIdx.x;
  int n = sub_info[8 * s];
  const double* d = dvec + vec_off[s];
  const double* e = evec + vec_off[s];
  if (tid == 0) {
    double lo = 1e300, hi = -1e300, me = 0;
    for (int i = 0; i < n; ++i) {
      double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
      lo = fmin(lo, d[i] - r);
      hi = fmax(hi, d[i] + r);
      if (i < n - 1) me = fmax(me, e[i] * e[i]);
    }
    double span = fmax(fabs(lo), fabs(hi));
    lo -= 1e-14 * span + 1e-300;
    hi += 1e-14 * span + 1e-300;
    lo_s = lo;
    hi_s = hi;
    pm_s = 1e-290 * fmax(1.0, me);
    int c = tau >= hi ? n : (tau <= lo ? 0 : sturm_count(d, e, n, tau, pm_s));
    cnt_s = c;
    nc_s = min(n, c + HK_EXTRA);
  }
  __syncthreads();
  int c = cnt_s, nc = nc_s;
  if (nc > HK_MAXM + HK_EXTRA) {
    if (tid == 0) dev_fail(st, HK_UNSUPPORTED, s, c);
    return;
  }
  for (int t = tid; t < nc; t += blockDim.x) {
    double lo = lo_s, hi = hi_s;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (hi - lo <= 2.2e-16 * fmax(fabs(lo), fabs(hi))) break;
      if (sturm_count(d, e, n, mid, pm_s) > t) hi = mid; else lo = mid;
    }
    lamsh[t] = 0.5 * (lo + hi);
  }
  __syncthreads();
  if (tid == 0) {
    double thr = 1e-8 * fmax(1.0, fabs(tau));
    int m = c;
    while (m > 0 && m < nc && lamsh[m] - lamsh[m - 1] <= thr) ++m;
    if (m == nc && nc < n && m > 0 && lamsh[m - 1] - lamsh[m - 2 >= 0 ? m - 2 : 0] <= thr && m > c)
      dev_fail(st, HK_EIG_FAIL, s, m);
    if (m > HK_MAXM) dev_fail(st, HK_UNSUPPORTED, s, m);
    m_out[s] = m;
    for (int t = 0; t < m && t < HK_MAXM; ++t) lam_all[(long long)s * HK_MAXM + t] = lamsh[t];
  }
}

// ---- 6. inverse iteration on T for the kept eigenvalues, with
// reorthogonalisation inside groups of close eigenvalues.  One thread per
// group; tridiagonal LU with partial pivoting (as in LAPACK's gttrf).
__device__ double hash_unit(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  x ^= x >> 31;
  return (double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

__global__ void k_inviter(const int* __restrict__ sub_info, const double* __restrict__ dvec,
                          const double* __restrict__ evec, const int* __restrict__ vec_off,
                          const double* __restrict__ lam_all, const long long* __restrict__ qoff, double* Q,
                          const long long* __restrict__ woff, double* wk) {
  int s = blockIdx.x;
  const int* si = sub_info + 8 * s;
  int n = si[0], m = si[6];
  const double* d = dvec + vec_off[s];
  const double* e = evec + vec_off[s];
  const double* lam = lam_all + (long long)s * HK_MAXM;
  double* Qs = Q + qoff[s];                 // m vectors of length n (vector-major)
  double tnorm = 0;
  for (int i = 0; i < n; ++i)
    tnorm = fmax(tnorm, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0));
  double ortol = 1e-3 * tnorm, eps = 2.2e-16;
  // group starts: thread t handles the t-th group
  int gcount = 0;
  for (int l = 0; l < m; ++l) {
    bool start = l == 0 || lam[l] - lam[l - 1] > ortol;
    if (!start) continue;
    if (gcount++ % blockDim.x != threadIdx.x) continue;
    int l1 = l + 1;
    while (l1 < m && lam[l1] - lam[l1 - 1] <= ortol) ++l1;
    double* dd = wk + woff[s] + (long long)threadIdx.x * 5 * n;
    double* du = dd + n;
    double* du2 = du + n;
    double* dl = du2 + n;
    double* x = dl + n;
    double prev = -1e300;
    for (int t = l; t < l1; ++t) {
      double lt = lam[t];
      if (lt - prev < 10 * eps * fmax(1.0, fabs(lt))) lt = prev + 10 * eps * fmax(1.0, fabs(prev));
      prev = lt;
      // factor T - lt I
      for (int i = 0; i < n; ++i) {
        dd[i] = d[i] - lt;
        du[i] = i < n - 1 ? e[i] : 0.0;
        dl[i] = i < n - 1 ? e[i] : 0.0;
        du2[i] = 0.0;
      }
      unsigned long long pivbits = 0;  // not enough for n > 64; store pivots as sign of du2 marker
      for (int i = 0; i < n - 1; ++i) {
        if (fabs(dd[i]) >= fabs(dl[i])) {
          if (dd[i] == 0.0) dd[i] = eps * tnorm;
          double f = dl[i] / dd[i];
          dl[i] = f;
          dd[i + 1] -= f * du[i];
          du2[i] = 0.0;
          x[i] = 0.0;  // no interchange
        } else {
          double f = dd[i] / dl[i];
          dd[i] = dl[i];
          dl[i] = f;
          double tmp = du[i];
          du[i] = dd[i + 1];
          dd[i + 1] = tmp - f * dd[i + 1];
          if (i < n - 2) {
            du2[i] = du[i + 1];
            du[i + 1] = -f * du[i + 1];
          }
          x[i] = 1.0;  // interchange marker
        }
      }
      if (dd[n - 1] == 0.0) dd[n - 1] = eps * tnorm;
      (void)pivbits;
      // pivot markers live in x[0..n-2]; move them into dl's sign-free spare: use Qs vector as rhs
      double* y = Qs + (long long)t * n;
      for (int i = 0; i < n; ++i) y[i] = hash_unit(((unsigned long long)s << 32) ^ ((unsigned long long)t << 20) ^ i);
      for (int it = 0; it < 3; ++it) {
        // forward: apply L with interchanges
        for (int i = 0; i < n - 1; ++i) {
          if (x[i] == 0.0) {
            y[i + 1] -= dl[i] * y[i];
          } else {
            double tmp = y[i];
            y[i] = y[i + 1];
            y[i + 1] = tmp - dl[i] * y[i];
          }
        }
        // back substitution with U (dd, du, du2)
        y[n - 1] /= dd[n - 1];
        if (n > 1) y[n - 2] = (y[n - 2] - du[n - 2] * y[n - 1]) / dd[n - 2];
        for (int i = n - 3; i >= 0; --i) y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) / dd[i];
        // orthogonalise against the group's earlier vectors (twice)
        for (int rep = 0; rep < 2; ++rep)
          for (int u = l; u < t; ++u) {
            const double* yu = Qs + (long long)u * n;
            double dot = 0;
            for (int i = 0; i < n; ++i) dot += yu[i] * y[i];
            for (int i = 0; i < n; ++i) y[i] -= dot * yu[i];
          }
        double nrm = 0;
        for (int i = 0; i < n; ++i) nrm += y[i] * y[i];
        nrm = 1.0 / sqrt(nrm);
        for (int i = 0; i < n; ++i) y[i] *= nrm;
      }
    }
  }
}

// ---- 7. back-transform q = H_0 ... H_{n-3} y, then Z = L^{-T} q (row-major nI x m).
__global__ void k_backtransform(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                                const int* __restrict__ bw_arr, const long long* __restrict__ wsW,
                                const long long* __restrict__ wsL, const double* __restrict__ ws,
                                const double* __restrict__ tauv, const int* __restrict__ vec_off,
                                const long long* __restrict__ qoff, double* Q, double* Z) {
  int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int* si = sub_info + 8 * s;
  int n = si[0], m = si[6];
  int bw = bw_arr[s], ld = bw + 1;
  const double* A = ws + wsW[s];
  const double* Lb = ws + wsL[s];
  const double* tv = tauv + vec_off[s];
  double* Qs = Q + qoff[s];
  double* Zs = Z + sub_off[3 * s + 2];
  for (int k = n - 3; k >= 0; --k) {
    double tau = tv[k];
    if (tau == 0.0) continue;
    const double* rk = A + (long long)k * n;
    for (int l = warp; l < m; l += nw) {
      double* q = Qs + (long long)l * n;
      double acc = lane == 0 ? q[k + 1] : 0.0;
      for (int j = k + 2 + lane; j < n; j += 32) acc += rk[j] * q[j];
      acc = warp_sum(acc) * tau;
      if (lane == 0) q[k + 1] -= acc;
      for (int j = k + 2 + lane; j < n; j += 32) q[j] -= acc * rk[j];
    }
    __syncthreads();
  }
  // Z[:, l] = L^{-T} q_l (thread per vector)
  for (int l = tid; l < m; l += blockDim.x) {
    double* q = Qs + (long long)l * n;
    for (int a = n - 1; a >= 0; --a) {
      double v = q[a];
      int cend = min(n - 1, a + bw);
      for (int c = a + 1; c <= cend; ++c) v -= Lb[(long long)c * ld + (a - c + bw)] * q[c];
      q[a] = v / Lb[(long long)a * ld + bw];
    }
    for (int a = 0; a < n; ++a) Zs[(long long)a * m + l] = q[a];
  }
}

hk_status phase_eigen(hk_handle* h, const uint8_t* d_elem_in) {
  cudaStream_t st = h->stream;
  int ns = h->n_sub;
  // workspace layout
  std::vector<long long> W(ns), Tt(ns), Lw(ns), Gw(ns), Rw(ns);
  std::vector<int> voff(ns), bw(ns);
  long long tot = 0;
  int vo = 0, maxn = 0;
  for (int s = 0; s < ns; ++s) {
    const Sub& u = h->subs[s];
    long long nI = u.nI, nG = u.nG;
    W[s] = tot; tot += nI * nI;
    Tt[s] = tot; tot += nI * nI;
    Lw[s] = tot; tot += nI * (u.bw + 1);
    Gw[s] = tot; tot += nG * nG;
    Rw[s] = tot; tot += nG * nI;
    tot = (tot + 3) & ~3LL;
    voff[s] = vo;
    vo += u.nI;
    bw[s] = u.bw;
    if (u.nI > maxn) maxn = u.nI;
  }
  double* d_ws = nullptr;
  long long *d_W = nullptr, *d_T = nullptr, *d_L = nullptr, *d_Gw = nullptr, *d_Rw = nullptr;
  int *d_voff = nullptr, *d_bw = nullptr, *d_ring = nullptr, *d_m = nullptr;
  double *d_d = nullptr, *d_e = nullptr, *d_tau = nullptr;
  HK_TRY(dalloc(h, &d_ws, tot));
  HK_TRY(dalloc(h, &d_W, ns));
  HK_TRY(dalloc(h, &d_T, ns));
  HK_TRY(dalloc(h, &d_L, ns));
  HK_TRY(dalloc(h, &d_Gw, ns));
  HK_TRY(dalloc(h, &d_Rw, ns));
  HK_TRY(dalloc(h, &d_voff, ns));
  HK_TRY(dalloc(h, &d_bw, ns));
  HK_TRY(dalloc(h, &d_ring, h->I_total));
  HK_TRY(dalloc(h, &d_m, ns));
  HK_TRY(dalloc(h, &d_d, vo));
  HK_TRY(dalloc(h, &d_e, vo));
  HK_TRY(dalloc(h, &d_tau, vo));
  HK_TRY(dalloc(h, &h->d_lam, (size_t)ns * HK_MAXM));
  HK_CUDA(cudaMemcpyAsync(d_W, W.data(), 8 * ns, cudaMemcpyHostToDevice, st));
  HK_CUDA(cudaMemcpyAsync(d_T, Tt.data(), 8 * ns, cudaMemcpyHostToDevice, st));
  HK_CUDA(cudaMemcpyAsync(d_L, Lw.data(), 8 * ns, cudaMemcpyHostToDevice, st));
  HK_CUDA(cudaMemcpyAsync(d_Gw, Gw.data(), 8 * ns, cudaMemcpyHostToDevice, st));
  HK_CUDA(cudaMemcpyAsync(d_Rw, Rw.data(), 8 * ns, cudaMemcpyHostToDevice, st));
  HK_CUDA(cudaMemcpyAsync(d_voff, voff.data(), 4 * ns, cudaMemcpyHostToDevice, st));
  HK_CUDA(cudaMemcpyAsync(d_bw, bw.data(), 4 * ns, cudaMemcpyHostToDevice, st));

  k_gamma_block<<<ns, 128, 0, st>>>(h->dim, h->n_elems, h->d_xyz, h->d_elems, h->d_coeff, h->k * h->k,
                                    h->d_node_of_dof, h->d_dof_of_node, h->d_ne_ptr, h->d_ne_idx, d_elem_in,
                                    h->d_sub_info, h->d_G, d_Gw, d_ws); HK_COUNT_LAUNCH();
  k_schur<<<ns, 256, 0, st>>>(h->d_sub_info, h->d_sub_off, h->d_lrow, h->d_lcntI, h->d_lcntG, h->d_lcol,
                              h->d_lvalB, d_W, d_Gw, d_Rw, d_ring, d_ws, h->d_status); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_TRY(check_device_status(h, "eigen: Gamma elimination"));
  k_stdform<<<ns, 512, 0, st>>>(h->d_sub_info, h->d_sub_off, d_bw, h->d_I, h->d_mu, h->d_lrow, h->d_lcntI,
                                h->d_lcol, h->d_lvalD, d_W, d_T, d_L, d_ws, h->d_status); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_TRY(check_device_status(h, "eigen: standard form"));
  size_t shm = sizeof(double) * 2 * (size_t)maxn;
  HK_CUDA(cudaFuncSetAttribute(k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  k_tridiag<<<ns, 1024, shm, st>>>(h->d_sub_info, d_W, d_ws, d_d, d_e, d_tau, d_voff); HK_COUNT_LAUNCH();
  cudaEventRecord(e1, st);
  HK_LAUNCH_CHECK();
  k_bisect<<<ns, 64, 0, st>>>(h->d_sub_info, d_d, d_e, d_voff, h->p.tau, h->d_lam, d_m, h->d_status); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_TRY(check_device_status(h, "eigen: bisection"));
  std::vector<int> m(ns);
  HK_CUDA(cudaMemcpyAsync(m.data(), d_m, 4 * ns, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  {
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    h->setup_ms[6] = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  int c0 = 0;
  long long zo = 0;
  std::vector<long long> qoff(ns), woff(ns);
  long long wtot = 0;
  for (int s = 0; s < ns; ++s) {
    Sub& u = h->subs[s];
    u.m = m[s];
    u.c_off = c0;
    u.z_off = zo;
    qoff[s] = zo;
    c0 += u.m;
    zo += (long long)u.nI * u.m;
    woff[s] = wtot;
    wtot += 5LL * u.nI * (u.m < 32 ? (u.m > 0 ? u.m : 1) : 32);
  }
  h->n0 = c0;
  h->z_total = zo;
  HK_TRY(upload_sub_info(h));
  if (c0 > 0) {
    double *d_Q = nullptr, *d_wk = nullptr;
    long long *d_qoff = nullptr, *d_woff = nullptr;
    HK_TRY(dalloc(h, &d_Q, zo));
    HK_TRY(dalloc(h, &d_wk, wtot));
    HK_TRY(dalloc(h, &d_qoff, ns));
    HK_TRY(dalloc(h, &d_woff, ns));
    HK_TRY(dalloc(h, &h->d_Z64, zo));
    HK_CUDA(cudaMemcpyAsync(d_qoff, qoff.data(), 8 * ns, cudaMemcpyHostToDevice, st));
    HK_CUDA(cudaMemcpyAsync(d_woff, woff.data(), 8 * ns, cudaMemcpyHostToDevice, st));
    k_inviter<<<ns, 32, 0, st>>>(h->d_sub_info, d_d, d_e, d_voff, h->d_lam, d_qoff, d_Q, d_woff, d_wk); HK_COUNT_LAUNCH();
    HK_LAUNCH_CHECK();
    k_backtransform<<<ns, 256, 0, st>>>(h->d_sub_info, h->d_sub_off, d_bw, d_W, d_L, d_ws, d_tau, d_voff, d_qoff,
                                        d_Q, h->d_Z64); HK_COUNT_LAUNCH();
    HK_LAUNCH_CHECK();
    HK_CUDA(cudaStreamSynchronize(st));
    dfree(h, d_Q);
    dfree(h, d_wk);
    dfree(h, d_qoff);
    dfree(h, d_woff);
  }
  HK_CUDA(cudaStreamSynchronize(st));
  void* tmp[] = {d_ws, d_W, d_T, d_L, d_Gw, d_Rw, d_voff, d_bw, d_ring, d_m, d_d, d_e, d_tau};
  for (void* p : tmp) dfree(h, p);
  return HK_OK;
}
