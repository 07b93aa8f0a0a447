// Overlapping decomposition on the device.
//  * Def. 2.3: one layer adds the stars (supports) of every interior vertex
//    (basis function of V^h) of the current element set; applied
//    overlap_layers times.  The starting elements are kept.
//  * Def. 3.2: ovdof = interior vertices of the set; dof = interior nodes
//    whose whole star lies in the set.
//  * Def. 2.7: mu_l = number of subdomains with l in dof.
// Each subdomain's dofs are then ordered by breadth-first level sets of the
// local matrix graph, so that B_i is block tridiagonal (a level couples only
// to its neighbours) - the structure the local factors and solves use.
#include "hk_internal.cuh"

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

__global__ void k_init_elem_in(const int* __restrict__ e2s, int ne, int n_sub, uint8_t* elem_in, DevStatus* st) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)ne * n_sub) return;
  int s = (int)(i / ne), e = (int)(i % ne);
  int t = e2s[e];
  if (s == 0 && (t < 0 || t >= n_sub)) dev_fail(st, HK_BAD_ARG, e, t);
  elem_in[i] = (t == s) ? 1 : 0;
}

__global__ void k_mark_nodes(int nn, int n_sub, int ne, const int* __restrict__ dof_of_node,
                             const int* __restrict__ ne_ptr, const int* __restrict__ ne_idx,
                             const uint8_t* __restrict__ elem_in, uint8_t* node_in) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nn * n_sub) return;
  int s = (int)(i / nn), v = (int)(i % nn);
  uint8_t m = 0;
  if (dof_of_node[v] >= 0) {
    const uint8_t* ein = elem_in + (long long)s * ne;
    for (int q = ne_ptr[v]; q < ne_ptr[v + 1]; ++q)
      if (ein[ne_idx[q]]) { m = 1; break; }
  }
  node_in[i] = m;
}

__global__ void k_grow(int ne, int n_sub, int nn, int nv, const int* __restrict__ elems,
                       const uint8_t* __restrict__ node_in, uint8_t* elem_in) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)ne * n_sub) return;
  int s = (int)(i / ne), e = (int)(i % ne);
  if (elem_in[i]) return;
  const uint8_t* nin = node_in + (long long)s * nn;
  for (int j = 0; j < nv; ++j)
    if (nin[elems[e * nv + j]]) { elem_in[i] = 1; return; }
}

// cls = 2 for dof(Omega_s), 1 for ovdof \ dof, 0 otherwise.
__global__ void k_classify(int n, int n_sub, int ne, const int* __restrict__ node_of_dof,
                           const int* __restrict__ ne_ptr, const int* __restrict__ ne_idx,
                           const uint8_t* __restrict__ elem_in, uint8_t* cls) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * n_sub) return;
  int s = (int)(i / n), l = (int)(i % n);
  int v = node_of_dof[l];
  const uint8_t* ein = elem_in + (long long)s * ne;
  int lo = ne_ptr[v], hi = ne_ptr[v + 1], c = 0;
  for (int q = lo; q < hi; ++q) c += ein[ne_idx[q]];
  cls[i] = c == 0 ? 0 : (c == hi - lo ? 2 : 1);
}

__global__ void k_mu(int n, int n_sub, const uint8_t* __restrict__ cls, int* mu, int* maxmu, DevStatus* st) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  int m = 0;
  for (int s = 0; s < n_sub; ++s) m += cls[(long long)s * n + l] == 2;
  mu[l] = m;
  if (m == 0) dev_fail(st, HK_BAD_ARG, l, 0);
  atomicMax(maxmu, m);
}

__global__ void k_elem_mult(int ne, int n_sub, const uint8_t* __restrict__ elem_in, int* lam) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  int c = 0;
  for (int s = 0; s < n_sub; ++s) c += elem_in[(long long)s * ne + e];
  atomicMax(lam, c);
}

__global__ void k_count_cls(int n, const uint8_t* __restrict__ cls, int* nI, int* nG) {
  __shared__ int sh[32];
  int s = blockIdx.x;
  const uint8_t* c = cls + (long long)s * n;
  int a = 0, b = 0;
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    a += c[l] == 2;
    b += c[l] == 1;
  }
  a = block_sumi(a, sh);
  b = block_sumi(b, sh);
  if (threadIdx.x == 0) {
    nI[s] = a;
    nG[s] = b;
  }
}

// Ordered compaction of cls == 2 (dof) and cls == 1 (Gamma) positions.
__global__ void k_compact(int n, const uint8_t* __restrict__ cls, const int* __restrict__ sub_info, int* Isorted,
                          int* G) {
  __shared__ int shA[1024], shB[1024];
  int s = blockIdx.x;
  const int* si = sub_info + 8 * s;
  int* Io = Isorted + si[3];
  int* Go = G + si[4];
  const uint8_t* c = cls + (long long)s * n;
  int carryA = 0, carryB = 0;
  for (int base = 0; base < n; base += blockDim.x) {
    int l = base + threadIdx.x;
    int fa = (l < n && c[l] == 2), fb = (l < n && c[l] == 1);
    shA[threadIdx.x] = fa;
    shB[threadIdx.x] = fb;
    __syncthreads();
    for (int off = 1; off < blockDim.x; off <<= 1) {
      int va = threadIdx.x >= off ? shA[threadIdx.x - off] : 0;
      int vb = threadIdx.x >= off ? shB[threadIdx.x - off] : 0;
      __syncthreads();
      shA[threadIdx.x] += va;
      shB[threadIdx.x] += vb;
      __syncthreads();
    }
    if (fa) Io[carryA + shA[threadIdx.x] - 1] = l;
    if (fb) Go[carryB + shB[threadIdx.x] - 1] = l;
    int ta = shA[blockDim.x - 1], tb = shB[blockDim.x - 1];
    __syncthreads();
    carryA += ta;
    carryB += tb;
  }
}

// Breadth-first level sets of the graph of B restricted to dof(Omega_s),
// seeded with the dofs of smallest last coordinate (a new seed set for each
// further connected component).  Outputs the level of each dof (in Isorted
// order), the number of levels and the local CSR capacity.
__global__ void k_levels(int dim, const double* __restrict__ xyz, const int* __restrict__ node_of_dof,
                         const int* __restrict__ rowptr, const int* __restrict__ col,
                         const int* __restrict__ sub_info, const int* __restrict__ Isorted, int* level,
                         int* Lout, int* capout, DevStatus* st) {
  __shared__ double shd[32];
  __shared__ int shi[32];
  int s = blockIdx.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], off = si[3];
  const int* Is = Isorted + off;
  int* lev = level + off;
  auto coord = [&](int a) { return xyz[(long long)node_of_dof[Is[a]] * dim + dim - 1]; };
  int cap = 0;
  for (int a = threadIdx.x; a < nI; a += blockDim.x) {
    lev[a] = -1;
    cap += rowptr[Is[a] + 1] - rowptr[Is[a]];
  }
  cap = block_sumi(cap, shi);
  __syncthreads();
  int visited = 0, cur = -1;
  while (visited < nI) {
    // seed the next level with the unvisited dofs of smallest last coordinate
    double cm = 1e300;
    for (int a = threadIdx.x; a < nI; a += blockDim.x)
      if (lev[a] < 0) cm = fmin(cm, coord(a));
    for (int o = 16; o > 0; o >>= 1) cm = fmin(cm, __shfl_xor_sync(0xffffffffu, cm, o));
    if ((threadIdx.x & 31) == 0) shd[threadIdx.x >> 5] = cm;
    __syncthreads();
    if (threadIdx.x < 32) {
      double t = threadIdx.x < (blockDim.x >> 5) ? shd[threadIdx.x] : 1e300;
      for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_xor_sync(0xffffffffu, t, o));
      if (threadIdx.x == 0) shd[0] = t;
    }
    __syncthreads();
    cm = shd[0];
    __syncthreads();
    ++cur;
    int c = 0;
    for (int a = threadIdx.x; a < nI; a += blockDim.x)
      if (lev[a] < 0 && coord(a) <= cm + 1e-9) {
        lev[a] = cur;
        ++c;
      }
    __syncthreads();
    c = block_sumi(c, shi);
    visited += c;
    // breadth-first growth from level cur
    while (true) {
      int nc = 0;
      for (int a = threadIdx.x; a < nI; a += blockDim.x) {
        if (lev[a] != cur) continue;
        int g = Is[a];
        for (int q = rowptr[g]; q < rowptr[g + 1]; ++q) {
          int idx = bsearch_int(Is, nI, col[q]);
          if (idx >= 0 && lev[idx] < 0) lev[idx] = cur + 1;
        }
      }
      __syncthreads();
      for (int a = threadIdx.x; a < nI; a += blockDim.x) nc += lev[a] == cur + 1;
      nc = block_sumi(nc, shi);
      if (nc == 0) break;
      visited += nc;
      ++cur;
    }
  }
  if (threadIdx.x == 0) {
    Lout[s] = cur + 1;
    capout[s] = cap;
  }
}

// Level pointers, level-order permutation and level widths.
__global__ void k_order(const int* __restrict__ sub_info, const int* __restrict__ Isorted,
                        const int* __restrict__ level, int* levptr, int* perm, int* Ilev, int* maxb,
                        DevStatus* st) {
  int s = blockIdx.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], L = si[2], off = si[3], loff = si[5];
  const int* lev = level + off;
  int* lp = levptr + loff;
  for (int j = threadIdx.x; j <= L; j += blockDim.x) lp[j] = 0;
  __syncthreads();
  for (int a = threadIdx.x; a < nI; a += blockDim.x) atomicAdd(&lp[lev[a] + 1], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int mb = 0;
    for (int j = 0; j < L; ++j) {
      int w = lp[j + 1];
      if (w > mb) mb = w;
      lp[j + 1] += lp[j];
    }
    atomicMax(maxb, mb);
    if (mb > HK_MAXB) dev_fail(st, HK_UNSUPPORTED, s, mb);
  }
  __syncthreads();
  for (int a = threadIdx.x; a < nI; a += blockDim.x) {
    int la = lev[a], r = 0;
    for (int b = 0; b < a; ++b) r += lev[b] == la;
    int pos = lp[la] + r;
    perm[off + a] = pos;
    Ilev[off + pos] = Isorted[off + a];
  }
}

// Local CSR of B_i (and D_k) in level order; each row holds its entries
// inside dof (local column = level position) followed by its entries on
// Gamma (column = index in the sorted Gamma list, B values only).
__global__ void k_local_csr(const int* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ valB, const double* __restrict__ valD,
                            const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                            const int* __restrict__ Isorted, const int* __restrict__ perm,
                            const int* __restrict__ Ilev, const int* __restrict__ G, int* lrow, int* lcntI,
                            int* lcntG, int* lcol, double* lvalB, double* lvalD, int* bw_out, DevStatus* st) {
  __shared__ int shi[32];
  int s = blockIdx.x;
  const int* si = sub_info + 8 * s;
  int nI = si[0], nG = si[1], off = si[3], goff = si[4];
  long long coff = sub_off[3 * s + 1];
  int* lr = lrow + off + s;
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int a = 0; a < nI; ++a) {
      lr[a] = acc;
      int g = Ilev[off + a];
      acc += rowptr[g + 1] - rowptr[g];
    }
    lr[nI] = acc;
  }
  __syncthreads();
  const int* Is = Isorted + off;
  const int* Gs = G + goff;
  int bw = 0;
  for (int a = threadIdx.x; a < nI; a += blockDim.x) {
    int g = Ilev[off + a];
    long long base = coff + lr[a];
    int ci = 0, cg = 0;
    int minc = a;
    for (int q = rowptr[g]; q < rowptr[g + 1]; ++q) {
      int idx = bsearch_int(Is, nI, col[q]);
      if (idx >= 0) {
        int lc = perm[off + idx];
        lcol[base + ci] = lc;
        lvalB[base + ci] = valB[q];
        lvalD[base + ci] = valD[q];
        ++ci;
        if (lc < minc) minc = lc;
      }
    }
    for (int q = rowptr[g]; q < rowptr[g + 1]; ++q) {
      if (bsearch_int(Is, nI, col[q]) >= 0) continue;
      int gi = bsearch_int(Gs, nG, col[q]);
      if (gi < 0) {
        dev_fail(st, HK_CUDA_ERROR, s, col[q]);  // a neighbour of a dof outside ovdof: inconsistent maps
        continue;
      }
      lcol[base + ci + cg] = gi;
      lvalB[base + ci + cg] = valB[q];
      lvalD[base + ci + cg] = valD[q];
      ++cg;
    }
    lcntI[off + a] = ci;
    lcntG[off + a] = cg;
    if (a - minc > bw) bw = a - minc;
  }
  // block max of bw
  for (int o = 16; o > 0; o >>= 1) bw = max(bw, __shfl_xor_sync(0xffffffffu, bw, o));
  if ((threadIdx.x & 31) == 0) shi[threadIdx.x >> 5] = bw;
  __syncthreads();
  if (threadIdx.x == 0) {
    int b = 0;
    for (int w = 0; w < (blockDim.x >> 5); ++w) b = max(b, shi[w]);
    bw_out[s] = b;
  }
}

__global__ void k_pull_fill(int n, int n_sub, const uint8_t* __restrict__ cls, const int* __restrict__ sub_info,
                            const int* __restrict__ Isorted, const int* __restrict__ perm,
                            const int* __restrict__ pull_ptr, int* pull_row, int* pull_sub) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  int slot = pull_ptr[l];
  for (int s = 0; s < n_sub; ++s) {
    if (cls[(long long)s * n + l] != 2) continue;
    const int* si = sub_info + 8 * s;
    int idx = bsearch_int(Isorted + si[3], si[0], l);
    pull_row[slot] = si[3] + perm[si[3] + idx];
    pull_sub[slot] = s;
    ++slot;
  }
}

// Level sets and level order of arbitrary per-subdomain node sets (global dof ids, increasing):
// counts[s] nodes at offsets[s] in d_nodes.  Writes the level order (d_nodes_lev), the position of
// each sorted node in it (d_perm), and level pointers at offsets[s] + s (capacity counts[s] + 1).
hk_status build_levels(hk_handle* h, const std::vector<int>& counts, const std::vector<int>& offsets,
                       const int* d_nodes, int* d_levptr, int* d_perm, int* d_nodes_lev, std::vector<int>& L_out,
                       int* max_width) {
  cudaStream_t st = h->stream;
  int ns = (int)counts.size();
  long long tot = 0;
  for (int c : counts) tot += c;
  std::vector<int> info(8 * ns, 0);
  for (int s = 0; s < ns; ++s) {
    info[8 * s + 0] = counts[s];
    info[8 * s + 3] = offsets[s];
    info[8 * s + 5] = offsets[s] + s;
  }
  int *d_info = nullptr, *d_level = nullptr, *d_L = nullptr, *d_cap = nullptr, *d_mw = nullptr;
  HK_TRY(dalloc(h, &d_info, info.size()));
  HK_TRY(dalloc(h, &d_level, tot));
  HK_TRY(dalloc(h, &d_L, ns));
  HK_TRY(dalloc(h, &d_cap, ns));
  HK_TRY(dalloc(h, &d_mw, 1));
  HK_CUDA(cudaMemcpyAsync(d_info, info.data(), sizeof(int) * info.size(), cudaMemcpyHostToDevice, st));
  k_levels<<<ns, 512, 0, st>>>(h->dim, h->d_xyz, h->d_node_of_dof, h->d_rowptr, h->d_col, d_info, d_nodes, d_level,
                               d_L, d_cap, h->d_status);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  L_out.assign(ns, 0);
  HK_CUDA(cudaMemcpyAsync(L_out.data(), d_L, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  HK_TRY(check_device_status(h, "level sets"));
  for (int s = 0; s < ns; ++s) info[8 * s + 2] = L_out[s];
  HK_CUDA(cudaMemcpyAsync(d_info, info.data(), sizeof(int) * info.size(), cudaMemcpyHostToDevice, st));
  k_order<<<ns, 512, 0, st>>>(d_info, d_nodes, d_level, d_levptr, d_perm, d_nodes_lev, d_mw, h->d_status);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_CUDA(cudaMemcpyAsync(max_width, d_mw, sizeof(int), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  HK_TRY(check_device_status(h, "level order"));
  dfree(h, d_info);
  dfree(h, d_level);
  dfree(h, d_L);
  dfree(h, d_cap);
  dfree(h, d_mw);
  return HK_OK;
}

hk_status upload_sub_info(hk_handle* h) {
  std::vector<int> info(8 * h->n_sub);
  std::vector<long long> off(3 * h->n_sub);
  for (int s = 0; s < h->n_sub; ++s) {
    const Sub& u = h->subs[s];
    int* q = &info[8 * s];
    q[0] = u.nI; q[1] = u.nG; q[2] = u.L; q[3] = u.I_off; q[4] = u.G_off; q[5] = u.lev_off; q[6] = u.m; q[7] = u.c_off;
    off[3 * s] = u.f_off;
    off[3 * s + 1] = u.csr_off;
    off[3 * s + 2] = u.z_off;
  }
  HK_CUDA(cudaMemcpyAsync(h->d_sub_info, info.data(), sizeof(int) * info.size(), cudaMemcpyHostToDevice, h->stream));
  HK_CUDA(cudaMemcpyAsync(h->d_sub_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice,
                          h->stream));
  HK_CUDA(cudaStreamSynchronize(h->stream));
  return HK_OK;
}

hk_status phase_decomposition(hk_handle* h, const int32_t* elem_to_sub, uint8_t** d_elem_in_out) {
  cudaStream_t st = h->stream;
  int ns = h->n_sub, ne = h->n_elems, nn = h->n_nodes, nv = h->nv;
  int* d_e2s = nullptr;
  HK_TRY(dalloc(h, &d_e2s, ne));
  HK_CUDA(cudaMemcpyAsync(d_e2s, elem_to_sub, sizeof(int) * ne,
                          h->dev_inputs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  uint8_t *d_elem_in = nullptr, *d_node_in = nullptr;
  HK_TRY(dalloc(h, &d_elem_in, (size_t)ne * ns));
  HK_TRY(dalloc(h, &d_node_in, (size_t)nn * ns));
  long long NE = (long long)ne * ns, NN = (long long)nn * ns;
  k_init_elem_in<<<nblk(NE, 256), 256, 0, st>>>(d_e2s, ne, ns, d_elem_in, h->d_status); HK_COUNT_LAUNCH();
  for (int layer = 0; layer < h->p.overlap_layers; ++layer) {
    k_mark_nodes<<<nblk(NN, 256), 256, 0, st>>>(nn, ns, ne, h->d_dof_of_node, h->d_ne_ptr, h->d_ne_idx, d_elem_in,
                                                d_node_in); HK_COUNT_LAUNCH();
    k_grow<<<nblk(NE, 256), 256, 0, st>>>(ne, ns, nn, nv, h->d_elems, d_node_in, d_elem_in); HK_COUNT_LAUNCH();
  }
  HK_LAUNCH_CHECK();
  HK_TRY(check_device_status(h, "partition"));
  dfree(h, d_node_in);
  dfree(h, d_e2s);
  *d_elem_in_out = d_elem_in;
  return decomposition_from_membership(h, d_elem_in);
}

// Everything after the element membership of the overlapping subdomains (elem_in[s * n_elems + e]): dof
// and ovdof (Def. 3.2), mu (Def. 2.7), Lambda, the level order of every dof(Omega_s), the local matrices
// and the pull map of the scatter.  The membership stays owned by the caller.
hk_status decomposition_from_membership(hk_handle* h, const uint8_t* d_elem_in) {
  cudaStream_t st = h->stream;
  int ns = h->n_sub, ne = h->n_elems, n = h->n;
  long long ND = (long long)n * ns;
  uint8_t* d_cls = nullptr;
  HK_TRY(dalloc(h, &d_cls, (size_t)n * ns));
  k_classify<<<nblk(ND, 256), 256, 0, st>>>(n, ns, ne, h->d_node_of_dof, h->d_ne_ptr, h->d_ne_idx, d_elem_in,
                                            d_cls); HK_COUNT_LAUNCH();
  int* d_scal = nullptr;  // [0] max mu, [1] Lambda, [2] max level width
  HK_TRY(dalloc(h, &d_scal, 4));
  HK_TRY(dalloc(h, &h->d_mu, n));
  k_mu<<<nblk(n, 256), 256, 0, st>>>(n, ns, d_cls, h->d_mu, d_scal, h->d_status); HK_COUNT_LAUNCH();
  k_elem_mult<<<nblk(ne, 256), 256, 0, st>>>(ne, ns, d_elem_in, d_scal + 1); HK_COUNT_LAUNCH();
  int *d_nI = nullptr, *d_nG = nullptr;
  HK_TRY(dalloc(h, &d_nI, ns));
  HK_TRY(dalloc(h, &d_nG, ns));
  k_count_cls<<<ns, 512, 0, st>>>(n, d_cls, d_nI, d_nG); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_TRY(check_device_status(h, "partition of unity"));
  std::vector<int> nI(ns), nG(ns), scal(4);
  HK_CUDA(cudaMemcpyAsync(nI.data(), d_nI, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaMemcpyAsync(nG.data(), d_nG, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaMemcpyAsync(scal.data(), d_scal, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  h->max_mu = scal[0];
  h->lambda_elems = scal[1];
  h->subs.assign(ns, Sub{});
  long long Ioff = 0, Goff = 0;
  for (int s = 0; s < ns; ++s) {
    Sub& u = h->subs[s];
    u.nI = nI[s];
    u.nG = nG[s];
    if (u.nI == 0) {
      hk_set_error("subdomain %d has no interior dof", s);
      return HK_BAD_ARG;
    }
    u.I_off = (int)Ioff;
    u.G_off = (int)Goff;
    u.lev_off = (int)(Ioff + s);
    Ioff += u.nI;
    Goff += u.nG;
    if (u.nI > h->max_dof) h->max_dof = u.nI;
  }
  h->I_total = Ioff;
  h->G_total = Goff;
  HK_TRY(dalloc(h, &h->d_sub_info, 8 * ns));
  HK_TRY(dalloc(h, &h->d_sub_off, 3 * ns));
  HK_TRY(upload_sub_info(h));
  HK_TRY(dalloc(h, &h->d_Isorted, Ioff));
  HK_TRY(dalloc(h, &h->d_I, Ioff + 4));  // + 4: the apply copies 16-byte aligned spans of it
  HK_TRY(dalloc(h, &h->d_perm, Ioff));
  HK_TRY(dalloc(h, &h->d_G, Goff));
  HK_TRY(dalloc(h, &h->d_lev, Ioff + ns));
  k_compact<<<ns, 1024, 0, st>>>(n, d_cls, h->d_sub_info, h->d_Isorted, h->d_G); HK_COUNT_LAUNCH();
  int *d_level = nullptr, *d_L = nullptr, *d_cap = nullptr;
  HK_TRY(dalloc(h, &d_level, Ioff));
  HK_TRY(dalloc(h, &d_L, ns));
  HK_TRY(dalloc(h, &d_cap, ns));
  k_levels<<<ns, 512, 0, st>>>(h->dim, h->d_xyz, h->d_node_of_dof, h->d_rowptr, h->d_col, h->d_sub_info,
                               h->d_Isorted, d_level, d_L, d_cap, h->d_status); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  std::vector<int> L(ns), cap(ns);
  HK_CUDA(cudaMemcpyAsync(L.data(), d_L, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaMemcpyAsync(cap.data(), d_cap, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  HK_TRY(check_device_status(h, "level sets"));
  long long coff = 0;
  for (int s = 0; s < ns; ++s) {
    h->subs[s].L = L[s];
    h->subs[s].csr_off = coff;
    coff += cap[s];
  }
  h->csr_total = coff;
  HK_TRY(upload_sub_info(h));
  k_order<<<ns, 512, 0, st>>>(h->d_sub_info, h->d_Isorted, d_level, h->d_lev, h->d_perm, h->d_I, d_scal + 2,
                              h->d_status); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_TRY(check_device_status(h, "level order"));
  HK_CUDA(cudaMemcpyAsync(&h->max_level, d_scal + 2, sizeof(int), cudaMemcpyDeviceToHost, st));

  HK_TRY(dalloc(h, &h->d_lrow, Ioff + ns));
  HK_TRY(dalloc(h, &h->d_lcntI, Ioff));
  HK_TRY(dalloc(h, &h->d_lcntG, Ioff));
  HK_TRY(dalloc(h, &h->d_lcol, coff));
  HK_TRY(dalloc(h, &h->d_lvalB, coff));
  HK_TRY(dalloc(h, &h->d_lvalD, coff));
  int* d_bw = d_L;
  k_local_csr<<<ns, 256, 0, st>>>(h->d_rowptr, h->d_col, h->d_valB, h->d_valD, h->d_sub_info, h->d_sub_off,
                                  h->d_Isorted, h->d_perm, h->d_I, h->d_G, h->d_lrow, h->d_lcntI, h->d_lcntG,
                                  h->d_lcol, h->d_lvalB, h->d_lvalD, d_bw, h->d_status); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  std::vector<int> bw(ns);
  HK_CUDA(cudaMemcpyAsync(bw.data(), d_bw, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  HK_TRY(check_device_status(h, "local matrices"));
  for (int s = 0; s < ns; ++s) h->subs[s].bw = bw[s];

  // pull map: for every dof, the (subdomain, local row) pairs holding it
  HK_TRY(dalloc(h, &h->d_pull_ptr, n + 1));
  launch_scan_exclusive(h->d_mu, h->d_pull_ptr, n, h->d_pull_ptr + n, st);
  HK_TRY(dalloc(h, &h->d_pull_row, Ioff));
  HK_TRY(dalloc(h, &h->d_pull_sub, Ioff));
  k_pull_fill<<<nblk(n, 256), 256, 0, st>>>(n, ns, d_cls, h->d_sub_info, h->d_Isorted, h->d_perm, h->d_pull_ptr,
                                            h->d_pull_row, h->d_pull_sub); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_CUDA(cudaStreamSynchronize(st));
  dfree(h, d_cls);
  dfree(h, d_level);
  dfree(h, d_L);
  dfree(h, d_cap);
  dfree(h, d_nI);
  dfree(h, d_nG);
  dfree(h, d_scal);
  return HK_OK;
}


// ================================================================ nested decompositions (Sec. 2.3)
// The fine subdomains Omega^f_{i,j} inside each coarse subdomain Omega_i^c: its elements grouped by their
// fine label, each group extended fine_overlap times by Def. 2.3 in the mesh of Omega_i^c (a layer adds
// only elements of Omega_i^c), so that the union of the fine subdomains of Omega_i^c is Omega_i^c.

// present[s * nlab + t] = 1 when coarse subdomain s has an element of fine label t.
__global__ void k_fine_labels(int ne, int n_sub, int nlab, const int* __restrict__ e2f,
                              const uint8_t* __restrict__ cin, uint8_t* present, DevStatus* st) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)ne * n_sub) return;
  int s = (int)(i / ne), e = (int)(i % ne);
  int t = e2f[e];
  if (s == 0 && (t < 0 || t >= nlab)) dev_fail(st, HK_BAD_ARG, e, t);
  if (cin[i] && t >= 0 && t < nlab) present[(long long)s * nlab + t] = 1;
}

// Fine subdomain f: the elements of coarse subdomain par[f] whose label is lab[f].
__global__ void k_init_fine(int ne, int nf, const int* __restrict__ par, const int* __restrict__ lab,
                            const int* __restrict__ e2f, const uint8_t* __restrict__ cin, uint8_t* fin) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)ne * nf) return;
  int f = (int)(i / ne), e = (int)(i % ne);
  fin[i] = (cin[(long long)par[f] * ne + e] && e2f[e] == lab[f]) ? 1 : 0;
}

// One growth layer (as k_grow) kept inside the parent coarse subdomain.
__global__ void k_grow_within(int ne, int nf, int nn, int nv, const int* __restrict__ elems,
                              const uint8_t* __restrict__ node_in, const int* __restrict__ par,
                              const uint8_t* __restrict__ cin, uint8_t* fin) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)ne * nf) return;
  int f = (int)(i / ne), e = (int)(i % ne);
  if (fin[i] || !cin[(long long)par[f] * ne + e]) return;
  const uint8_t* nin = node_in + (long long)f * nn;
  for (int j = 0; j < nv; ++j)
    if (nin[elems[e * nv + j]]) { fin[i] = 1; return; }
}

// dst row r = src row keep[r] (rows of ne bytes).
__global__ void k_gather_rows(int ne, int nk, const int* __restrict__ keep, const uint8_t* __restrict__ src,
                              uint8_t* dst) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)ne * nk) return;
  int r = (int)(i / ne), e = (int)(i % ne);
  dst[i] = src[(long long)keep[r] * ne + e];
}

hk_status nested_fine_membership(hk_handle* h, const uint8_t* d_cin, int nlab, const int32_t* elem_to_fine,
                                 int fine_overlap, uint8_t** d_fin_out, int* nf_out, std::vector<int>* parent_out) {
  cudaStream_t st = h->stream;
  int N = h->n_sub, ne = h->n_elems, nn = h->n_nodes, n = h->n, nv = h->nv;
  int* d_e2f = nullptr;
  uint8_t* d_present = nullptr;
  HK_TRY(dalloc(h, &d_e2f, ne));
  HK_CUDA(cudaMemcpyAsync(d_e2f, elem_to_fine, sizeof(int) * ne,
                          h->dev_inputs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  HK_TRY(dalloc(h, &d_present, (size_t)N * nlab));
  HK_CUDA(cudaMemsetAsync(d_present, 0, (size_t)N * nlab, st));
  k_fine_labels<<<nblk((long long)ne * N, 256), 256, 0, st>>>(ne, N, nlab, d_e2f, d_cin, d_present, h->d_status);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  std::vector<uint8_t> present((size_t)N * nlab);
  HK_CUDA(cudaMemcpyAsync(present.data(), d_present, present.size(), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  HK_TRY(check_device_status(h, "fine labels"));
  dfree(h, d_present);
  std::vector<int> par, lab;
  for (int s = 0; s < N; ++s)
    for (int t = 0; t < nlab; ++t)
      if (present[(size_t)s * nlab + t]) par.push_back(s), lab.push_back(t);
  int nf = (int)par.size();
  int *d_par = nullptr, *d_lab = nullptr;
  uint8_t *d_fin = nullptr, *d_node = nullptr, *d_cls = nullptr;
  HK_TRY(dalloc(h, &d_par, nf));
  HK_TRY(dalloc(h, &d_lab, nf));
  HK_TRY(dalloc(h, &d_fin, (size_t)ne * nf));
  HK_TRY(dalloc(h, &d_node, (size_t)nn * nf));
  HK_CUDA(cudaMemcpyAsync(d_par, par.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, st));
  HK_CUDA(cudaMemcpyAsync(d_lab, lab.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, st));
  long long NE = (long long)ne * nf, NN = (long long)nn * nf, ND = (long long)n * nf;
  k_init_fine<<<nblk(NE, 256), 256, 0, st>>>(ne, nf, d_par, d_lab, d_e2f, d_cin, d_fin);
  HK_COUNT_LAUNCH();
  for (int layer = 0; layer < fine_overlap; ++layer) {
    k_mark_nodes<<<nblk(NN, 256), 256, 0, st>>>(nn, nf, ne, h->d_dof_of_node, h->d_ne_ptr, h->d_ne_idx, d_fin,
                                                d_node);
    HK_COUNT_LAUNCH();
    k_grow_within<<<nblk(NE, 256), 256, 0, st>>>(ne, nf, nn, nv, h->d_elems, d_node, d_par, d_cin, d_fin);
    HK_COUNT_LAUNCH();
  }
  // leave out the fine subdomains without a dof (slivers of Omega_i^c: they span the zero space)
  HK_TRY(dalloc(h, &d_cls, (size_t)ND));
  int *d_nI = nullptr, *d_nG = nullptr;
  HK_TRY(dalloc(h, &d_nI, nf));
  HK_TRY(dalloc(h, &d_nG, nf));
  k_classify<<<nblk(ND, 256), 256, 0, st>>>(n, nf, ne, h->d_node_of_dof, h->d_ne_ptr, h->d_ne_idx, d_fin, d_cls);
  HK_COUNT_LAUNCH();
  k_count_cls<<<nf, 512, 0, st>>>(n, d_cls, d_nI, d_nG);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  std::vector<int> nI(nf);
  HK_CUDA(cudaMemcpyAsync(nI.data(), d_nI, sizeof(int) * nf, cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  std::vector<int> keep;
  parent_out->clear();
  for (int f = 0; f < nf; ++f)
    if (nI[f] > 0) keep.push_back(f), parent_out->push_back(par[f]);
  int nk = (int)keep.size();
  int* d_keep = nullptr;
  uint8_t* d_out = nullptr;
  HK_TRY(dalloc(h, &d_keep, nk));
  HK_TRY(dalloc(h, &d_out, (size_t)ne * nk));
  HK_CUDA(cudaMemcpyAsync(d_keep, keep.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
  k_gather_rows<<<nblk((long long)ne * nk, 256), 256, 0, st>>>(ne, nk, d_keep, d_fin, d_out);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_CUDA(cudaStreamSynchronize(st));
  void* fr[] = {d_e2f, d_par, d_lab, d_fin, d_node, d_cls, d_nI, d_nG, d_keep};
  for (void* p : fr) dfree(h, p);
  *d_fin_out = d_out;
  *nf_out = nk;
  return HK_OK;
}
