// Tensor-core local sweeps of the split-BF16 preconditioner form (Eq. 2.22).
//
// The sweeps are those of the twisted block factorisation of hk_local.cu: per level step a dense
// product of a level record (b_j rows, the columns of one to three consecutive levels) with the same
// levels' rows of the level-ordered vectors of up to 16 right-hand sides.  Here one product is a chain
// of tcgen05.mma instructions (kind::f16, BF16 operands, FP32 accumulator in tensor memory) on
// D[b x 16] = A[b x K] B[16 x K]^T: A is the record, B holds the 16 right-hand sides' rows of the
// window (one row per right-hand side, K along the dofs).  Each operand is a BF16 pair, A = A_hi + A_lo
// and B = B_hi + B_lo, and D accumulates A_hi B_hi + A_hi B_lo + A_lo B_hi (the A_lo B_lo term is below
// the pair's resolution).
//
// Padded level order.  Every level starts on an 8-row boundary of the padded vector (P_j = sum of
// pad8(b_i) over i < j, zero rows in between, 16 zero rows after the last level), so that a window of
// consecutive levels starts on a core-matrix boundary of B.  Record columns follow the same padding
// (zero columns where the vector has zero rows) and are padded to a multiple of 16 (one MMA's K).
//
// Operand layouts (no swizzle; a core matrix is 8 rows x 16 bytes, i.e. 8 rows x 8 BF16):
//   record: K-slices of 16 columns, one after another; a slice holds, for pb = pad8(b) rows, the
//     BF16 high parts (two core-matrix columns of pb rows: row group g at 128 g bytes, the second
//     8 columns pb*16 bytes further) and then the low parts in the same layout, pb*64 bytes per slice;
//     descriptor LBO (K direction) = pb*16, SBO (row direction) = 128.  A record streams as chunks of
//     whole slices, so its MMAs start as soon as the first chunk has landed.
//   vector (B, MN-major: the right-hand sides contiguous): 8-dof blocks of 256 bytes; in a block, per
//     dof, the 16-byte row of right-hand sides 0..7, and 128 bytes further that of 8..15; high and low
//     parts in two such arrays.  Descriptor LBO (dof direction) = 256, SBO (right-hand sides) = 128.
//     A thread that owns a level row writes its 16 right-hand sides as four 16-byte stores.
// The MMA reads M = 64 (or 128) rows of A whatever b is; the rows past b read whatever follows in
// shared memory (the next slice, the next stage, the guard after the rings), only ever to produce
// accumulator rows that are discarded.  M = 64 puts row r of D in tensor-memory lane
// 32 (r >> 4) + (r & 15); M = 128 puts it in lane r.  Levels up to 128 dofs wide are taken (one tile;
// a wider level needs a box whose vectors do not fit shared memory: a breadth-first level of an n^3
// box holds at most about 0.75 n^2 dofs).
//
// Kernel.  One CTA per (subdomain, group of 16 right-hand sides); two warpgroups run the top and
// bottom half sweeps (the top one also the middle level), each with one elected thread issuing its
// MMAs into its own accumulator columns; two producer warps stream the records by 1-D TMA bulk copies
// into two rings of shared-memory stages (full mbarrier: transaction bytes; empty mbarrier: a
// tcgen05.commit after the MMAs that read the stage).  A step: wait for the record's chunks and issue
// their MMAs, commit to the step's mbarrier; every thread of the warpgroup waits on it, loads its
// accumulator row (tcgen05.ld), forms the level's new values (first sweep and middle: the product;
// second sweep: the stored first-sweep value minus the product), splits them into BF16 pairs and
// stores them into the vector; then a proxy fence and a warpgroup barrier before the next MMAs read
// them.  Every wait is bounded; a wait that gives up reports HK_TIMEOUT (the warps then keep only
// their barriers, the issuing threads wait for their MMAs, the producers for their copies, and the
// tensor memory is released).
#include <cuda_bf16.h>

#include <algorithm>

#include "hk_internal.cuh"

#define TC_THREADS 320   // two warpgroups of sweeps + two producer warps
#define TC_MAXK 16       // ring stages per stream at most
#define TC_GUARD 2048    // bytes after the rings that an MMA's rows past a record may read
#define TC_NRHS 16       // right-hand sides per CTA (the MMA's N)
#define TC_TMEM_COLS 32  // two streams x 16 columns
#define TC_MAXB 128      // widest level the sweeps take (one M = 128 tile)

__host__ __device__ __forceinline__ int tc_pad8(int x) { return (x + 7) & ~7; }
__host__ __device__ __forceinline__ int tc_pad16(int x) { return (x + 15) & ~15; }
__host__ __device__ __forceinline__ long long tc_align128(long long x) { return (x + 127) & ~127LL; }

// Level table entry (4 x int64 per level): [0] first-sweep record offset (bytes), [1] second-sweep
// record offset, [2] level start | P_j << 32, [3] b | Kf << 16 | Kb << 32 (record columns, multiples
// of 16).  Entry L of a subdomain: [2] = |dof| | Apad << 32.
__host__ __device__ __forceinline__ int tce_b(long long e3) { return (int)(e3 & 0xFFFF); }
__host__ __device__ __forceinline__ int tce_kf(long long e3) { return (int)((e3 >> 16) & 0xFFFF); }
__host__ __device__ __forceinline__ int tce_kb(long long e3) { return (int)((e3 >> 32) & 0xFFFF); }

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ unsigned tc_su32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tc_mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void tc_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_su32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tc_bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc_su32(dst)),
               "l"(src), "r"(bytes), "r"(tc_su32(bar))
               : "memory");
}

__device__ __forceinline__ bool tc_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(tc_su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait that also gives up once another thread of the CTA has flagged a failure.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, unsigned parity, const volatile int* fail) {
  for (unsigned it = 0; it < (1u << 22); ++it) {
    if (tc_try_wait(bar, parity)) return true;
    if ((it & 63u) == 63u && *fail) return false;
  }
  return false;
}

__device__ __forceinline__ bool tc_wait_bounded(uint64_t* bar, unsigned parity) {
  for (unsigned it = 0; it < (1u << 22); ++it)
    if (tc_try_wait(bar, parity)) return true;
  return false;
}

// Barrier over `count` threads (named barrier id) that also ORs a flag across them.
__device__ __forceinline__ int tc_bar_any(int flag, int id, int count) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 q, %1, 0;\n bar.red.or.pred p, %2, %3, q;\n selp.s32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"(flag), "r"(id), "r"(count)
      : "memory");
  return r;
}

// Shared-memory matrix descriptor: start address, leading (K direction) and stride (row direction)
// byte offsets, descriptor version 1 (tcgen05), no swizzle.
__device__ __forceinline__ uint64_t tc_sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, A K-major, B MN-major (the
// right-hand sides contiguous), N = 16, M.
__device__ __forceinline__ uint32_t tc_idesc(int M) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(TC_NRHS >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// The same with the accumulate flag fixed: D = A B^T (first product of a step), D += A B^T.
__device__ __forceinline__ void tc_mma0(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc) {
  asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 0;" ::"r"(d_tmem), "l"(da), "l"(db), "r"(idesc)
               : "memory");
}
__device__ __forceinline__ void tc_mma1(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc) {
  asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;" ::"r"(d_tmem), "l"(da), "l"(db), "r"(idesc)
               : "memory");
}

// Arrives on `bar` once every MMA this thread issued so far has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_su32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive accumulator columns of this thread's lane (lane quarter of its warp).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}


// Byte offset of (right-hand side n, padded row a) in a vector array: 8-row blocks of 256 bytes, in a
// block the 16-byte row of right-hand sides 0..7 of each dof, then that of right-hand sides 8..15.
__device__ __forceinline__ int tc_xoff(int n, int a) { return (a >> 3) * 256 + (n >> 3) * 128 + (a & 7) * 16 + (n & 7) * 2; }

// Eight floats as eight BF16 high parts and eight low parts (two 16-byte words).
__device__ __forceinline__ void tc_split8(const float* y, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat162 p = __floats2bfloat162_rn(y[2 * i], y[2 * i + 1]);
    float2 pf = __bfloat1622float2(p);
    __nv_bfloat162 q = __floats2bfloat162_rn(y[2 * i] - pf.x, y[2 * i + 1] - pf.y);
    h[i] = *reinterpret_cast<uint32_t*>(&p);
    l[i] = *reinterpret_cast<uint32_t*>(&q);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Eight values from their high and low parts.
__device__ __forceinline__ void tc_join8(uint4 hi, uint4 lo, float* y) {
  const uint32_t h[4] = {hi.x, hi.y, hi.z, hi.w}, l[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h[i]));
    float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&l[i]));
    y[2 * i] = a.x + b.x;
    y[2 * i + 1] = a.y + b.y;
  }
}

// Byte offset of (row m, column c) in the high part of a record of pb rows.
__host__ __device__ __forceinline__ long long tc_roff(int m, int c, int pb) {
  return (long long)(c >> 4) * pb * 64 + (m >> 3) * 128 + ((c >> 3) & 1) * pb * 16 + (m & 7) * 16 + (c & 7) * 2;
}

// ------------------------------------------------------------------ records
// One CTA per subdomain: both records of every level from the FP64 factors (the inverse block X_j of
// the level's Schur complement and its coupling product, see hk_local.cu), as BF16 pairs.
//   first sweep, columns over the levels [j-1 | j | j+1] present in the step (j-1 for the top part and
//     the middle, j+1 for the bottom part and the middle): -X_j B[j, j-1], X_j, -X_j B[j, j+1];
//   second sweep: G_j (b_j x b_{j+1}) above the middle, H_j (b_j x b_{j-1}) below it.
__global__ void k_pack_tc(const int* __restrict__ sub_info, const long long* __restrict__ sub_off,
                          const int* __restrict__ levptr, const int* __restrict__ lrow,
                          const int* __restrict__ lcntI, const int* __restrict__ lcol,
                          const double* __restrict__ lvalB, const double* __restrict__ F,
                          const long long* __restrict__ lvfo, const long long* __restrict__ tab,
                          const int* __restrict__ twist, unsigned char* pack) {
  int s = blockIdx.x, tid = threadIdx.x, T_ = blockDim.x;
  const int* si = sub_info + 8 * s;
  int L = si[2], off = si[3], loff = si[5];
  long long coff = sub_off[3 * s + 1];
  const int* lp = levptr + loff;
  const int* lr = lrow + off + s;
  const long long* fo = lvfo + loff;
  const long long* tb = tab + 4 * (long long)loff;
  int M = twist[s];
  for (int j = 0; j < L; ++j) {
    int r0 = lp[j], b = lp[j + 1] - r0, pb = tc_pad8(b);
    int bn = j + 1 < L ? lp[j + 2] - lp[j + 1] : 0, bp = j > 0 ? r0 - lp[j - 1] : 0;
    int lb = (j > 0 && j <= M) ? bp : 0, rb = (j < L - 1 && j >= M) ? bn : 0;
    long long e3 = tb[4 * j + 3];
    int Kf = tce_kf(e3), Kb = tce_kb(e3);
    const double* Xi = F + fo[j];
    // first-sweep record: window levels in padded order [j-1 if lb] [j] [j+1 if rb]
    int wl = lb ? j - 1 : j, wn = (lb ? 1 : 0) + 1 + (rb ? 1 : 0);
    unsigned char* Fr = pack + tb[4 * j + 0];
    for (int q = tid; q < pb * Kf; q += T_) {
      int m = q / Kf, c = q % Kf;
      double v = 0;
      if (m < b) {
        // padded column c -> level of the window and the position in it
        int pc = 0;
        for (int t = 0; t < wn; ++t) {
          int lv = wl + t, bw = lp[lv + 1] - lp[lv], pw = tc_pad8(bw);
          if (c < pc + pw) {
            int o = c - pc;
            if (o < bw) {
              int node = lp[lv] + o;  // local row of the column
              if (lv == j) {
                v = Xi[(long long)m * b + o];
              } else {
                // -X_j B[level j, node]: the couplings of row `node` inside level j (B symmetric)
                const int* cl = lcol + coff + lr[node];
                const double* cv = lvalB + coff + lr[node];
                for (int t2 = 0; t2 < lcntI[off + node]; ++t2) {
                  int a = cl[t2];
                  if (a >= r0 && a < r0 + b) v -= Xi[(long long)m * b + (a - r0)] * cv[t2];
                }
              }
            }
            break;
          }
          pc += pw;
        }
      }
      __nv_bfloat16 hi = __double2bfloat16(v);
      __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
      long long o = tc_roff(m, c, pb);
      *reinterpret_cast<__nv_bfloat16*>(Fr + o) = hi;
      *reinterpret_cast<__nv_bfloat16*>(Fr + o + pb * 32) = lo;
    }
    if (j != M) {
      int cb = j < M ? bn : bp;
      const double* P = Xi + ((long long)b * b + 3) / 4 * 4;
      unsigned char* Gr = pack + tb[4 * j + 1];
      for (int q = tid; q < pb * Kb; q += T_) {
        int m = q / Kb, c = q % Kb;
        double v = (m < b && c < cb) ? P[(long long)m * cb + c] : 0.0;
        __nv_bfloat16 hi = __double2bfloat16(v);
        __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
        long long o = tc_roff(m, c, pb);
        *reinterpret_cast<__nv_bfloat16*>(Gr + o) = hi;
        *reinterpret_cast<__nv_bfloat16*>(Gr + o + pb * 32) = lo;
      }
    }
  }
}

// ------------------------------------------------------------------ sweeps
// Shared memory: two record rings (2 x K x stage_bytes) | guard | vector high parts | low parts
// (32 x max_apad bytes each) | level table (4 x int64 per level, L + 1 entries) | step parameters of
// both streams (int4) | their record offsets | dof indices | padded rows of the dofs.
__global__ void __launch_bounds__(TC_THREADS, 1) k_local_apply_tc(
    int n, int s_tot, const double* __restrict__ v, const int* __restrict__ active,
    const int* __restrict__ sub_info, const int* __restrict__ Ilev, const int* __restrict__ Iprow,
    const long long* __restrict__ tabg, const unsigned char* __restrict__ pack, long long I_total,
    int stage_bytes, int K, int max_L, int max_dof, int max_apad, float* ybuf, DevStatus* st,
    const int* __restrict__ jp, long long jstride, const int* __restrict__ twist) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[2][TC_MAXK], empty[2][TC_MAXK], mbar[2], meta;
  __shared__ int sh_fail, sh_act;
  __shared__ uint32_t sh_tmem;
  const int* si = sub_info + 8 * blockIdx.x;
  int nI = si[0], L = si[2], off = si[3], loff = si[5];
  if (L <= 0) return;
  if (jp) v += (long long)(*jp) * jstride;  // captured inner step: v = v_j with j read on the device
  int s = blockIdx.x, r_base = blockIdx.y * TC_NRHS;
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int prod = warp - 8;  // 0: top stream, 1: bottom stream, < 0: sweeps
  int M = twist[s];
  int nst[2] = {2 * M + 1, 2 * (L - 1 - M)};
  unsigned char* rings = smem_raw;
  unsigned char* xh = smem_raw + 2LL * K * stage_bytes + TC_GUARD;
  unsigned char* xl = xh + 32LL * max_apad;
  long long* tab = reinterpret_cast<long long*>(xl + 32LL * max_apad);
  // a stream has at most 2L - 1 steps (the twist level may be any level)
  int SL = 2 * max_L;
  int4* sp = reinterpret_cast<int4*>(tab + 4LL * (max_L + 1));  // [2][SL]
  long long* so = reinterpret_cast<long long*>(sp + 2LL * SL);  // [2][SL]
  int* idx = reinterpret_cast<int*>(so + 2LL * SL);
  int* prow = idx + ((max_dof + 7) & ~3);
  int ioff = off & 3;  // position of the subdomain's first dof in the aligned spans
  int ispan = (ioff + nI + 3) & ~3;
  int nr = s_tot - r_base < TC_NRHS ? s_tot - r_base : TC_NRHS;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_su32(&sh_tmem)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    sh_fail = 0;
    for (int h = 0; h < 2; ++h) {
      for (int k = 0; k < K; ++k) {
        tc_mbar_init(&full[h][k], 1);
        tc_mbar_init(&empty[h][k], 1);
      }
      tc_mbar_init(&mbar[h], 1);
    }
    tc_mbar_init(&meta, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tc_expect_tx(&meta, 32u * (L + 1) + 8u * ispan);
    tc_bulk_load(tab, tabg + 4LL * loff, 32u * (L + 1), &meta);
    tc_bulk_load(idx, Ilev + (off - ioff), 4u * ispan, &meta);
    tc_bulk_load(prow, Iprow + (off - ioff), 4u * ispan, &meta);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  uint32_t tmem = sh_tmem;
  bool meta_ok = tc_wait(&meta, 0u, &sh_fail);
  if (!meta_ok && atomicExch(&sh_fail, 1) == 0) dev_fail(st, HK_TIMEOUT, s, -1);
  int apad = 0;
  if (meta_ok) {
    apad = (int)(tab[4 * L + 2] >> 32);
    // step parameters: b | kind << 16, K-slices | slices per ring stage << 16, first window row, P_j
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
      long long e3 = tab[4 * j + 3];
      int b = tce_b(e3);
      int Pj = (int)(tab[4 * j + 2] >> 32);
      int kc, w;
      if (kind == 0) {
        kc = tce_kf(e3);
        w = (j > 0 && j <= M) ? (int)(tab[4 * (j - 1) + 2] >> 32) : Pj;
      } else {
        kc = tce_kb(e3);
        w = j < M ? (int)(tab[4 * (j + 1) + 2] >> 32) : (int)(tab[4 * (j - 1) + 2] >> 32);
      }
      int spc = stage_bytes / (tc_pad8(b) * 64);
      sp[h * SL + k] = make_int4(b | (kind << 16), (kc >> 4) | (spc << 16), w, Pj);
      so[h * SL + k] = tab[4 * j + kind];
    }
  }
  __syncthreads();
  // the producer of stream h walks its records chunk by chunk (whole K-slices, as many as fill a
  // stage), in the order in which the issuing thread consumes them
  int issued = 0, ps_k = 0, ps_c = 0;
  auto next_chunk = [&](int h, const unsigned char*& src, unsigned& bytes) -> bool {
    if (ps_k >= nst[h]) return false;
    int4 pv = sp[h * SL + ps_k];
    int sb = tc_pad8(pv.x & 0xFFFF) * 64, ns = pv.y & 0xFFFF, spc = pv.y >> 16;
    int c0 = ps_c * spc, cnt = ns - c0 < spc ? ns - c0 : spc;
    src = pack + so[h * SL + ps_k] + (long long)c0 * sb;
    bytes = (unsigned)(cnt * sb);
    if (c0 + cnt >= ns) ++ps_k, ps_c = 0;
    else ++ps_c;
    return true;
  };
  unsigned char* ring = prod >= 0 ? rings + (long long)prod * K * stage_bytes : nullptr;
  if (prod >= 0 && lane == 0 && meta_ok) {
    const unsigned char* src;
    unsigned bytes;
    for (; issued < K && next_chunk(prod, src, bytes); ++issued) {
      tc_expect_tx(&full[prod][issued], bytes);
      tc_bulk_load(ring + (long long)issued * stage_bytes, src, bytes, &full[prod][issued]);
    }
  }
  if (prod < 0 && meta_ok) {
    // gather r_i = v[dof(Omega_i)] into the padded vectors as BF16 pairs: zeros first (padding rows stay
    // zero), then per dof its 16 right-hand sides (16 loads in flight, four 16-byte stores)
    uint4* xh4 = reinterpret_cast<uint4*>(xh);
    uint4* xl4 = reinterpret_cast<uint4*>(xl);
    for (int e = tid; e < 2 * apad; e += 256) xh4[e] = xl4[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
      int m = 0;
      for (int rr = 0; rr < nr; ++rr)
        if (active == nullptr || active[8 * (r_base + rr)]) m |= 1 << rr;
      sh_act = m;
    }
    tc_bar_any(0, 4, 256);
    int act = sh_act;
    const double* vb = v + (long long)r_base * n;
    for (int a = tid; a < nI; a += 256) {
      int g = idx[ioff + a];
      float y[16];
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) y[rr] = (act >> rr) & 1 ? (float)vb[(long long)rr * n + g] : 0.f;
      uint4 h0, l0, h1, l1;
      tc_split8(y, h0, l0);
      tc_split8(y + 8, h1, l1);
      int o = tc_xoff(0, prow[ioff + a]) >> 4;
      xh4[o] = h0;
      xh4[o + 8] = h1;
      xl4[o] = l0;
      xl4[o + 8] = l1;
    }
    tc_fence_proxy();
  }
  __syncthreads();
  if (prod >= 0) {
    if (lane != 0 || !meta_ok) return;
    const unsigned char* src;
    unsigned bytes;
    bool failed = false;
    for (; next_chunk(prod, src, bytes); ++issued) {
      int k = issued % K;
      if (!tc_wait(&empty[prod][k], (unsigned)((issued / K) - 1) & 1u, &sh_fail)) {
        if (atomicExch(&sh_fail, 1) == 0) dev_fail(st, HK_TIMEOUT, s, issued);
        failed = true;
        break;
      }
      tc_expect_tx(&full[prod][k], bytes);
      tc_bulk_load(ring + (long long)k * stage_bytes, src, bytes, &full[prod][k]);
    }
    if (failed) {  // let the copies in flight land before the CTA exits
      for (int r = issued - K < 0 ? 0 : issued - K; r < issued; ++r)
        tc_wait_bounded(&full[prod][r % K], (unsigned)(r / K) & 1u);
    }
    return;
  }
  // ---- sweeps: warpgroup h (warps 4h .. 4h+3) runs stream h; lane 0 of its warp 4h + 2 + h issues
  // the MMAs (the two issuing warps and the two producer warps sit on four different SM
  // sub-partitions: warp w issues from sub-partition w % 4)
  int h = warp >> 2, wq = warp & 3;
  bool iwarp = wq == 2 + h;
  bool issuer = iwarp && lane == 0;
  bool dead = !meta_ok;  // a wait gave up: from then on only the barriers are kept
  bool pend = false;     // the issuer's last commit has not been waited for
  int ks = 0;            // ring stage of the next chunk, and its phase parity
  unsigned kph = 0, mph = 0;
  unsigned ring_a = tc_su32(rings + (long long)h * K * stage_bytes);
  unsigned xh_a = tc_su32(xh), xl_a = tc_su32(xl);
  uint32_t tcol = tmem + 16u * h;  // this stream's accumulator columns
  uint32_t tlane = (uint32_t)(32 * wq) << 16;
  int n_first = h == 0 ? M : L - 1 - M;
  for (int k = 0; k <= nst[h]; ++k) {
    // the two halves meet around the middle level: the bottom's z_{M+1} is ready for the middle
    // step, then x_M for the bottom's second sweep
    if (k == n_first) {
      dead = tc_bar_any(dead, 3, 256) != 0;
      if (h == 1) dead = tc_bar_any(dead, 3, 256) != 0;
    }
    if (h == 0 && k == n_first + 1) dead = tc_bar_any(dead, 3, 256) != 0;
    if (k == nst[h]) break;
    int4 pv = sp[h * SL + k];
    int b = pv.x & 0xFFFF, kind = pv.x >> 16, w = pv.z, Pj = pv.w;
    int pb = tc_pad8(b), sb = pb * 64, ns = pv.y & 0xFFFF, spc = pv.y >> 16;
    bool m128 = b > 64;
    if (iwarp) {
     if (issuer && !dead) {
      tc_fence_after();
      // Issue is the cost here (tens of cycles per instruction from one thread), so the descriptors
      // are formed once per step and advanced by constant adds to their address field: a slice
      // further is sb bytes on in the record and 512 bytes (16 dofs) on in the vectors.
      const uint32_t idesc = tc_idesc(m128 ? 128 : 64);
      const uint64_t a_first = tc_sdesc(ring_a, (unsigned)pb * 16u, 128u);
      const uint64_t a_lo = (uint64_t)(pb * 32) >> 4, a_slice = (uint64_t)sb >> 4;
      uint64_t bh = tc_sdesc(xh_a + (unsigned)(w >> 3) * 256u, 256u, 128u);
      uint64_t bl = tc_sdesc(xl_a + (unsigned)(w >> 3) * 256u, 256u, 128u);
      bool okc = true, first = true;
      for (int c0 = 0; c0 < ns; c0 += spc) {
        if (!tc_wait(&full[h][ks], kph, &sh_fail)) {
          okc = false;
          break;
        }
        uint64_t ah = a_first + (((uint64_t)ks * (uint64_t)stage_bytes) >> 4);
        int cnt = ns - c0 < spc ? ns - c0 : spc;
        for (int i = 0; i < cnt; ++i) {
          if (first) tc_mma0(tcol, ah, bh, idesc);
          else tc_mma1(tcol, ah, bh, idesc);
          tc_mma1(tcol, ah, bl, idesc);
          tc_mma1(tcol, ah + a_lo, bh, idesc);
          first = false;
          ah += a_slice;
          bh += 32;
          bl += 32;
        }
        tc_commit(&empty[h][ks]);  // the stage is free once these MMAs have read it
        if (++ks == K) ks = 0, kph ^= 1u;
      }
      tc_commit(&mbar[h]);
      pend = true;
      if (!okc && atomicExch(&sh_fail, 1) == 0) dev_fail(st, HK_TIMEOUT, s, k);
     }
      __syncwarp();  // the issuing warp's other lanes wait here, not in a spin beside the issuer
    }
    bool okl = false;
    if (!dead) {
      bool got = tc_wait(&mbar[h], mph, &sh_fail);
      if (got) {
        mph ^= 1u;
        if (issuer) pend = false;
      }
      okl = got && !sh_fail;
    }
    okl = __all_sync(0xffffffffu, okl);  // tcgen05.ld is warp-collective
    tc_fence_after();
    if (okl) {
      {
        float acc[16];
        tc_ld16(tcol + tlane, acc);
        int q = m128 ? 32 * wq + lane : 16 * wq + lane;
        bool mine = q < b && (m128 || lane < 16);
        if (mine) {
          // this row's 16 right-hand sides: two 16-byte words in each of the two vector arrays
          int o = tc_xoff(0, Pj + q);
          uint4* ph = reinterpret_cast<uint4*>(xh + o);
          uint4* pl = reinterpret_cast<uint4*>(xl + o);
          if (kind) {
            // second sweep: x_j = (first-sweep value) - coupling product x_neighbour
            float y[16];
            tc_join8(ph[0], pl[0], y);
            tc_join8(ph[8], pl[8], y + 8);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = y[i] - acc[i];
          }
          uint4 h0, l0, h1, l1;
          tc_split8(acc, h0, l0);
          tc_split8(acc + 8, h1, l1);
          ph[0] = h0;
          ph[8] = h1;
          pl[0] = l0;
          pl[8] = l1;
        }
      }
    }
    tc_fence_proxy();
    tc_fence_before();
    dead = tc_bar_any(!okl, 1 + h, 128) != 0;
  }
  if (issuer && pend) tc_wait_bounded(&mbar[h], mph);  // no MMA of this CTA may outlive it
  tc_fence_before();
  dead = tc_bar_any(dead, 3, 256) != 0;  // both halves done: x complete
  if (!dead) {
    // local solutions: per dof its 16 right-hand sides from four 16-byte words
    const uint4* xh4 = reinterpret_cast<const uint4*>(xh);
    const uint4* xl4 = reinterpret_cast<const uint4*>(xl);
    int act = sh_act;
    float* yb = ybuf + (long long)r_base * I_total + off;
    for (int a = tid; a < nI; a += 256) {
      int o = tc_xoff(0, prow[ioff + a]) >> 4;
      float y[16];
      tc_join8(xh4[o], xl4[o], y);
      tc_join8(xh4[o + 8], xl4[o + 8], y + 8);
#pragma unroll
      for (int rr = 0; rr < 16; ++rr)
        if ((act >> rr) & 1) yb[(long long)rr * I_total + a] = y[rr];
    }
  }
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------------ host
// Shared memory of the sweeps apart from the rings.
static size_t tc_fixed_smem(const hk_handle* h) {
  return TC_GUARD + 64 * (size_t)h->tc_max_apad + 32 * (size_t)(h->max_L + 1) + 96 * (size_t)h->max_L +
         8 * (size_t)((h->max_dof + 7) & ~3);
}

hk_status tc_plan(hk_handle* h, const std::vector<int>& lev) {
  h->tc_ok = false;
  if (h->p.precision != HK_SPLIT_BF16_PRECOND || h->p.levels == HK_COARSE_ONLY) return HK_OK;
  int ns = h->n_sub;
  std::vector<long long> tab(4 * (size_t)(h->I_total + ns), 0);
  std::vector<int> prow((size_t)h->I_total + 4, 0);  // padded row of every local dof
  long long cur = 0;
  int max_pb = 8, max_apad = 0;
  for (int s = 0; s < ns; ++s) {
    const Sub& u = h->subs[s];
    const int* lp = &lev[u.lev_off];
    int L = u.L, M = u.M;
    std::vector<int> P(L + 1, 0);
    for (int j = 0; j < L; ++j) {
      P[j + 1] = P[j] + tc_pad8(lp[j + 1] - lp[j]);
      for (int a = lp[j]; a < lp[j + 1]; ++a) prow[(size_t)u.I_off + a] = P[j] + (a - lp[j]);
    }
    max_apad = std::max(max_apad, P[L] + 16);
    for (int j = 0; j < L; ++j) {
      int b = lp[j + 1] - lp[j], bn = j + 1 < L ? lp[j + 2] - lp[j + 1] : 0, bp = j > 0 ? lp[j] - lp[j - 1] : 0;
      int lb = (j > 0 && j <= M) ? bp : 0, rb = (j < L - 1 && j >= M) ? bn : 0;
      int pb = tc_pad8(b);
      max_pb = std::max(max_pb, pb);
      int kf = tc_pad16(pb + (lb ? tc_pad8(bp) : 0) + (rb ? tc_pad8(bn) : 0));
      int cb = j < M ? bn : j > M ? bp : 0;
      int kb = cb ? tc_pad16(tc_pad8(cb)) : 0;
      long long* e = &tab[4 * (size_t)(u.lev_off + j)];
      e[0] = cur;
      cur += tc_align128(4LL * pb * kf);
      e[1] = cur;
      cur += tc_align128(4LL * pb * kb);
      e[2] = (long long)lp[j] | ((long long)P[j] << 32);
      e[3] = (long long)b | ((long long)kf << 16) | ((long long)kb << 32);
    }
    tab[4 * (size_t)(u.lev_off + L) + 2] = (long long)u.nI | ((long long)(P[L] + 16) << 32);
  }
  h->tc_max_apad = max_apad;
  h->tc_stage = (int)tc_align128(std::max(8192, 64 * max_pb));
  h->tc_bytes = cur;
  bool fits = h->max_level <= TC_MAXB && tc_fixed_smem(h) + 4 * (size_t)h->tc_stage <= 220 * 1024;
  if (!fits) return HK_OK;  // the FP32 sweeps serve this handle
  HK_TRY(dalloc(h, &h->d_pack_tc, (size_t)cur));
  HK_TRY(dalloc(h, &h->d_lvtab_tc, tab.size()));
  HK_TRY(dalloc(h, &h->d_tc_prow, prow.size()));
  HK_CUDA(cudaMemcpyAsync(h->d_tc_prow, prow.data(), sizeof(int) * prow.size(), cudaMemcpyHostToDevice, h->stream));
  HK_CUDA(cudaMemcpyAsync(h->d_lvtab_tc, tab.data(), sizeof(long long) * tab.size(), cudaMemcpyHostToDevice,
                          h->stream));
  h->tc_ok = true;
  return HK_OK;
}

hk_status tc_pack(hk_handle* h, cudaStream_t st) {
  if (!h->tc_ok) return HK_OK;
  HK_TRY(hk_max_carveout(k_pack_tc));  // runs beside the eigensolver
  k_pack_tc<<<h->n_sub, 256, 0, st>>>(h->d_sub_info, h->d_sub_off, h->d_lev, h->d_lrow, h->d_lcntI, h->d_lcol,
                                      h->d_lvalB, h->d_F64, h->d_lvfo, h->d_lvtab_tc, h->d_twist, h->d_pack_tc);
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  return HK_OK;
}

hk_status tc_prepare() { return hk_allow_smem(k_local_apply_tc); }

hk_status tc_launch(hk_handle* h, int s, const double* v, const int* active, float* ybuf) {
  if (!h->tc_ok) {
    hk_set_error("tensor-core sweeps unavailable for this handle");
    return HK_UNSUPPORTED;
  }
  if (!h->n_sm) cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->dev);
  int groups = (s + TC_NRHS - 1) / TC_NRHS;
  long long ctas = (long long)h->n_sub * groups;
  size_t fixed = tc_fixed_smem(h), stage = (size_t)h->tc_stage;
  // one wave, or vectors too large for two CTAs per SM: deep rings in the whole shared memory; else
  // half of it, so that two CTAs share an SM
  size_t budget = (ctas <= h->n_sm || fixed + 4 * stage > 112 * 1024) ? 220 * 1024 : 112 * 1024;
  int K = TC_MAXK;
  while (K > 2 && fixed + 2 * K * stage > budget) --K;
  size_t shm = fixed + 2 * (size_t)K * stage;
  HK_TRY(tc_prepare());
  dim3 grid(h->n_sub, groups);
  HK_TIMED(h, HK_T_LOCAL_APPLY,
           (k_local_apply_tc<<<grid, TC_THREADS, shm, h->stream>>>(
               h->n, s, v, active, h->d_sub_info, h->d_I, h->d_tc_prow, h->d_lvtab_tc, h->d_pack_tc, h->I_total, (int)stage, K,
               h->max_L, h->max_dof, h->tc_max_apad, ybuf, h->d_status, h->g_jp, h->g_jstride, h->d_twist)));
  HK_COUNT_LAUNCH();
  HK_LAUNCH_CHECK();
  return HK_OK;
}
