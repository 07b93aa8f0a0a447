// Device assembly of the P1 Helmholtz matrices (Sec. 2.1, Eq. 2.11-2.12;
// D_k = A + k^2 S from Prop. 2.6).  Row-parallel and atomic-free in the
// values, so the sums run in a fixed order (sorted element stars) and every
// run gives the same bits.
#include <cstdarg>
#include <cstdio>

#include "hk_internal.cuh"

// ---------------------------------------------------------------- scan
// Exclusive scan of n ints by one CTA of 1024 threads: each thread scans a
// contiguous chunk, then the chunk totals are scanned in shared memory.
__global__ void k_scan_exclusive(const int* __restrict__ in, int* __restrict__ out, int n, int* total) {
  __shared__ int sh[1024];
  int t = threadIdx.x, T = blockDim.x;
  long long chunk = ((long long)n + T - 1) / T;
  long long lo = t * chunk, hi = lo + chunk < n ? lo + chunk : n;
  int s = 0;
  for (long long i = lo; i < hi; ++i) s += in[i];
  sh[t] = s;
  __syncthreads();
  for (int off = 1; off < T; off <<= 1) {
    int v = t >= off ? sh[t - off] : 0;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  int run = sh[t] - s;
  for (long long i = lo; i < hi; ++i) {
    int v = in[i];
    out[i] = run;
    run += v;
  }
  if (t == T - 1 && total) *total = sh[T - 1];
}

void launch_scan_exclusive(const int* in, int* out, int n, int* total, cudaStream_t st) {
  k_scan_exclusive<<<1, 1024, 0, st>>>(in, out, n, total); HK_COUNT_LAUNCH();
}

// ---------------------------------------------------------------- kernels
__global__ void k_interior_flags(const uint8_t* __restrict__ bnd, int* __restrict__ flag, int n_nodes) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n_nodes) flag[v] = bnd[v] ? 0 : 1;
}

__global__ void k_dof_maps(const uint8_t* __restrict__ bnd, const int* __restrict__ scan, int* dof_of_node,
                           int* node_of_dof, int n_nodes) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_nodes) return;
  if (bnd[v]) {
    dof_of_node[v] = -1;
  } else {
    dof_of_node[v] = scan[v];
    node_of_dof[scan[v]] = v;
  }
}

__global__ void k_check_elems(const int* __restrict__ elems, int n_elems, int nv, int n_nodes, DevStatus* st) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_elems) return;
  for (int j = 0; j < nv; ++j) {
    int v = elems[e * nv + j];
    if (v < 0 || v >= n_nodes) dev_fail(st, HK_BAD_ARG, e, v);
  }
}

__global__ void k_count_star(const int* __restrict__ elems, int n_elems, int nv, int* cnt) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_elems) return;
  for (int j = 0; j < nv; ++j) atomicAdd(&cnt[elems[e * nv + j]], 1);
}

__global__ void k_fill_star(const int* __restrict__ elems, int n_elems, int nv, const int* __restrict__ ptr,
                            int* cursor, int* idx) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_elems) return;
  for (int j = 0; j < nv; ++j) {
    int v = elems[e * nv + j];
    int slot = atomicAdd(&cursor[v], 1);
    idx[ptr[v] + slot] = e;
  }
}

// Sort each node's star (insertion sort; stars are short) so that sums over
// the star run in increasing element order.
__global__ void k_sort_star(const int* __restrict__ ptr, int* idx, int n_nodes, DevStatus* st) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_nodes) return;
  int lo = ptr[v], hi = ptr[v + 1];
  if (hi - lo > HK_MAXSTAR) dev_fail(st, HK_UNSUPPORTED, v, hi - lo);
  for (int i = lo + 1; i < hi; ++i) {
    int key = idx[i], j = i - 1;
    while (j >= lo && idx[j] > key) {
      idx[j + 1] = idx[j];
      --j;
    }
    idx[j + 1] = key;
  }
}

// Collects the sorted, distinct dof neighbours of dof row l (including l).
__device__ int row_pattern(int l, const int* __restrict__ node_of_dof, const int* __restrict__ dof_of_node,
                           const int* __restrict__ ne_ptr, const int* __restrict__ ne_idx,
                           const int* __restrict__ elems, int nv, int* cols) {
  int v = node_of_dof[l];
  int cnt = 0;
  for (int s = ne_ptr[v]; s < ne_ptr[v + 1]; ++s) {
    int e = ne_idx[s];
    for (int j = 0; j < nv; ++j) {
      int d = dof_of_node[elems[e * nv + j]];
      if (d < 0) continue;
      int q = 0;
      while (q < cnt && cols[q] != d) ++q;
      if (q == cnt) {
        if (cnt >= HK_MAXROW) return -1;
        cols[cnt++] = d;
      }
    }
  }
  for (int i = 1; i < cnt; ++i) {
    int key = cols[i], j = i - 1;
    while (j >= 0 && cols[j] > key) {
      cols[j + 1] = cols[j];
      --j;
    }
    cols[j + 1] = key;
  }
  return cnt;
}

__global__ void k_row_count(int n, const int* __restrict__ node_of_dof, const int* __restrict__ dof_of_node,
                            const int* __restrict__ ne_ptr, const int* __restrict__ ne_idx,
                            const int* __restrict__ elems, int nv, int* rowcnt, DevStatus* st) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  int cols[HK_MAXROW];
  int c = row_pattern(l, node_of_dof, dof_of_node, ne_ptr, ne_idx, elems, nv, cols);
  if (c < 0) {
    dev_fail(st, HK_UNSUPPORTED, l, HK_MAXROW);
    c = 0;
  }
  rowcnt[l] = c;
}

// Row l of K (stiffness with a_T) and M (mass): element contributions summed
// in increasing element order (Sec. 2.1 element matrices).
__global__ void k_row_fill(int n, int dim, const double* __restrict__ xyz, const int* __restrict__ elems,
                           const double* __restrict__ coeff, const int* __restrict__ node_of_dof,
                           const int* __restrict__ dof_of_node, const int* __restrict__ ne_ptr,
                           const int* __restrict__ ne_idx, const int* __restrict__ rowptr, int* col,
                           double* valK, double* valM) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  int nv = dim + 1;
  int cols[HK_MAXROW];
  double k_acc[HK_MAXROW], m_acc[HK_MAXROW];
  int cnt = row_pattern(l, node_of_dof, dof_of_node, ne_ptr, ne_idx, elems, nv, cols);
  if (cnt < 0) return;
  for (int q = 0; q < cnt; ++q) k_acc[q] = m_acc[q] = 0.0;
  int v = node_of_dof[l];
  double mdiag = 2.0 / ((nv) * (nv + 1)), moff = 1.0 / ((nv) * (nv + 1));
  for (int s = ne_ptr[v]; s < ne_ptr[v + 1]; ++s) {
    int e = ne_idx[s];
    int vid[4];
    int iv = 0;
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
      double dot = 0;
      for (int c = 0; c < dim; ++c) dot += g[iv][c] * g[j][c];
      int q = 0;
      while (cols[q] != d) ++q;
      k_acc[q] += a * vol * dot;
      m_acc[q] += vol * (j == iv ? mdiag : moff);
    }
  }
  int base = rowptr[l];
  for (int q = 0; q < cnt; ++q) {
    col[base + q] = cols[q];
    valK[base + q] = k_acc[q];
    valM[base + q] = m_acc[q];
  }
}

__global__ void k_combine(int nnz, double k2, const double* __restrict__ K, const double* __restrict__ M,
                          double* B, double* D) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnz) return;
  double kk = K[i], mm = M[i];
  B[i] = kk - k2 * mm;
  D[i] = kk + k2 * mm;
}

__global__ void k_check_coeff(const double* __restrict__ c, int n, DevStatus* st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(c[i] > 0.0)) dev_fail(st, HK_BAD_ARG, i, c[i]);
}

// Load vector of the P1 interpolant: rhs_l = sum_T sum_j M_T[l, j] f_j.
__global__ void k_load(int n, int dim, const double* __restrict__ xyz, const int* __restrict__ elems,
                       const int* __restrict__ node_of_dof, const int* __restrict__ ne_ptr,
                       const int* __restrict__ ne_idx, const double* __restrict__ f, double* rhs) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  int nv = dim + 1;
  int v = node_of_dof[l];
  double mdiag = 2.0 / (nv * (nv + 1)), moff = 1.0 / (nv * (nv + 1));
  double acc = 0;
  for (int s = ne_ptr[v]; s < ne_ptr[v + 1]; ++s) {
    int e = ne_idx[s];
    int vid[4];
    for (int j = 0; j < nv; ++j) vid[j] = elems[e * nv + j];
    double g[4][3];
    double vol = simplex_geometry(dim, xyz, vid, g);
    for (int j = 0; j < nv; ++j) acc += vol * (vid[j] == v ? mdiag : moff) * f[vid[j]];
  }
  rhs[l] = acc;
}

// ---------------------------------------------------------------- host
static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

hk_status phase_assembly(hk_handle* h, const hk_mesh* mesh, const double* coeff) {
  cudaStream_t st = h->stream;
  int nv = h->nv, nn = h->n_nodes, ne = h->n_elems;
  HK_TRY(dalloc(h, &h->d_xyz, (size_t)nn * h->dim));
  HK_TRY(dalloc(h, &h->d_elems, (size_t)ne * nv));
  HK_TRY(dalloc(h, &h->d_coeff, (size_t)ne));
  uint8_t* d_bnd = nullptr;
  HK_TRY(dalloc(h, &d_bnd, (size_t)nn));
  cudaMemcpyKind kind = h->dev_inputs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  HK_CUDA(cudaMemcpyAsync(h->d_xyz, mesh->xyz, sizeof(double) * nn * h->dim, kind, st));
  HK_CUDA(cudaMemcpyAsync(h->d_elems, mesh->elems, sizeof(int) * ne * nv, kind, st));
  HK_CUDA(cudaMemcpyAsync(h->d_coeff, coeff, sizeof(double) * ne, kind, st));
  HK_CUDA(cudaMemcpyAsync(d_bnd, mesh->is_boundary, nn, kind, st));
  k_check_elems<<<nblk(ne, 256), 256, 0, st>>>(h->d_elems, ne, nv, nn, h->d_status); HK_COUNT_LAUNCH();
  k_check_coeff<<<nblk(ne, 256), 256, 0, st>>>(h->d_coeff, ne, h->d_status); HK_COUNT_LAUNCH();
  HK_TRY(check_device_status(h, "mesh input"));

  // dof numbering: interior nodes in increasing node order
  int *d_flag = nullptr, *d_scan = nullptr, *d_tot = nullptr;
  HK_TRY(dalloc(h, &d_flag, nn));
  HK_TRY(dalloc(h, &d_scan, nn));
  HK_TRY(dalloc(h, &d_tot, 1));
  k_interior_flags<<<nblk(nn, 256), 256, 0, st>>>(d_bnd, d_flag, nn); HK_COUNT_LAUNCH();
  launch_scan_exclusive(d_flag, d_scan, nn, d_tot, st);
  int n = 0;
  HK_CUDA(cudaMemcpyAsync(&n, d_tot, sizeof(int), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  if (n <= 0) {
    hk_set_error("mesh has no interior node");
    return HK_BAD_ARG;
  }
  h->n = n;
  HK_TRY(dalloc(h, &h->d_dof_of_node, nn));
  HK_TRY(dalloc(h, &h->d_node_of_dof, n));
  k_dof_maps<<<nblk(nn, 256), 256, 0, st>>>(d_bnd, d_scan, h->d_dof_of_node, h->d_node_of_dof, nn); HK_COUNT_LAUNCH();

  // node -> element stars
  int* d_cnt = d_flag;  // reuse
  HK_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(int) * nn, st));
  k_count_star<<<nblk(ne, 256), 256, 0, st>>>(h->d_elems, ne, nv, d_cnt); HK_COUNT_LAUNCH();
  HK_TRY(dalloc(h, &h->d_ne_ptr, nn + 1));
  launch_scan_exclusive(d_cnt, h->d_ne_ptr, nn, h->d_ne_ptr + nn, st);
  HK_TRY(dalloc(h, &h->d_ne_idx, (size_t)ne * nv));
  HK_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(int) * nn, st));
  k_fill_star<<<nblk(ne, 256), 256, 0, st>>>(h->d_elems, ne, nv, h->d_ne_ptr, d_cnt, h->d_ne_idx); HK_COUNT_LAUNCH();
  k_sort_star<<<nblk(nn, 256), 256, 0, st>>>(h->d_ne_ptr, h->d_ne_idx, nn, h->d_status); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_TRY(check_device_status(h, "element stars"));

  // CSR pattern and values
  int* d_rowcnt = nullptr;
  HK_TRY(dalloc(h, &d_rowcnt, n));
  k_row_count<<<nblk(n, 128), 128, 0, st>>>(n, h->d_node_of_dof, h->d_dof_of_node, h->d_ne_ptr, h->d_ne_idx,
                                            h->d_elems, nv, d_rowcnt, h->d_status); HK_COUNT_LAUNCH();
  HK_TRY(dalloc(h, &h->d_rowptr, n + 1));
  launch_scan_exclusive(d_rowcnt, h->d_rowptr, n, h->d_rowptr + n, st);
  HK_TRY(check_device_status(h, "matrix pattern"));
  HK_CUDA(cudaMemcpyAsync(&h->nnz, h->d_rowptr + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  HK_CUDA(cudaStreamSynchronize(st));
  int nnz = h->nnz;
  double *d_K = nullptr, *d_M = nullptr;
  HK_TRY(dalloc(h, &h->d_col, nnz));
  HK_TRY(dalloc(h, &h->d_valB, nnz));
  HK_TRY(dalloc(h, &h->d_valD, nnz));
  HK_TRY(dalloc(h, &d_K, nnz));
  HK_TRY(dalloc(h, &d_M, nnz));
  k_row_fill<<<nblk(n, 128), 128, 0, st>>>(n, h->dim, h->d_xyz, h->d_elems, h->d_coeff, h->d_node_of_dof,
                                           h->d_dof_of_node, h->d_ne_ptr, h->d_ne_idx, h->d_rowptr, h->d_col,
                                           d_K, d_M); HK_COUNT_LAUNCH();
  k_combine<<<nblk(nnz, 256), 256, 0, st>>>(nnz, h->k * h->k, d_K, d_M, h->d_valB, h->d_valD); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  HK_CUDA(cudaStreamSynchronize(st));
  dfree(h, d_K);
  dfree(h, d_M);
  dfree(h, d_rowcnt);
  dfree(h, d_flag);
  dfree(h, d_scan);
  dfree(h, d_tot);
  dfree(h, d_bnd);
  return HK_OK;
}

hk_status op_load(hk_handle* h, const double* f_nodal_dev, double* rhs_dev) {
  k_load<<<nblk(h->n, 128), 128, 0, h->stream>>>(h->n, h->dim, h->d_xyz, h->d_elems, h->d_node_of_dof,
                                                 h->d_ne_ptr, h->d_ne_idx, f_nodal_dev, rhs_dev); HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  return HK_OK;
}
