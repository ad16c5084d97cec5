// Tensor-core user pass (A4, with A8's batched score): S = U . Q^T over every user tile and
// the distinct query vectors of a sub-batch, on tcgen05, consumed in the epilogue by the A4
// tests and never written out.
//
// Columns.  The rows of a sub-batch are (q, k) requests; rows asking for the same vector q
// (with k <= k_max) share one GEMM column, so a batch that asks each item at several k
// costs one column per item.  The distinct vectors are found by a hash table on a 64-bit
// hash of each row's bits, the columns put in descending order of ||q|| and each column's
// rows listed; every row is then checked bitwise against its column's first row, and should
// two different vectors share a hash, one CTA builds the table again comparing whole
// vectors.  Up to kSmallTable rows one CTA builds the table in shared memory; past that five
// grid-wide kernels do (a single CTA's sort and probes would take longer than the rest of
// the table).
//
// Operands.  The users' rows and the column vectors are BF16 (8 significant bits), one
// product per score, accumulated in FP32 over K = dk:
//   |s_tc - <u,q>| <= c_bf ||u|| ||q||,   c_bf = 1.01 (2^-7 + 2^-16 + (2 dk + 16) 2^-23),
// the two roundings to BF16, the FP32 rounding of the inputs and an accumulation in which
// every addition may lose up to two units in the last place (no rounding mode is assumed).
// The kernel also takes split operands (x_hi = bf16(x), x_lo = bf16(x - x_hi), three
// products u_hi q_hi + u_hi q_lo + u_lo q_hi, a band near 1e-4): measured, the lo stream
// doubled the traffic and cost more MMA time than the narrower band saved in re-scores.
// With tc_user_pass = 2 the operands are E4M3 with a scale per row (kind::f8f6f4) and the
// band c_8 = 0.130.
//
// Tests per (user, row) whose leaf the node-level bound (Lemma 2) kept, with L = L_u^k,
// E the error of L, and the band e = c ||u|| ||q||:
//   s + e <  L - E                                            -> "no" (k items beat <u,q>)
//   s - e >= L + E, when L is the exact k-th score (|P'| = n)  -> "yes"
//   s - e >= ||u|| ||p_k|| (1 + 2 gamma)                       -> "yes" (Alg. 5)
//   otherwise the pair is re-scored in FP32 (and in FP64 against the exact threshold) by
//   pair_rescore_kernel, which lists what stays open for the kMIPS decision.
// Since L_u^k falls as k grows, a column is tested first against the lower bound of its
// largest k: a user below it is "no" for every row of the column.  Lemma 3 (the
// vector-level bound) is not applied: with the score from the tensor cores it would cost
// more than it saves.
//
// Column prefixes.  The columns are sorted by descending ||q||, and every 128-user tile has
// a bound tile_lb^k = min over its users of (L_u^k - E_u) / ||u||.  A column can pass a
// user's fast test only if (1 + 2c) ||u|| ||q|| >= L_u^k - E_u, so a tile needs only the
// prefix of a column set whose norms reach tile_lb^K times a rounding margin (K the set's
// largest k); every other pair is "no" by Cauchy-Schwarz.  A tile with an empty prefix is
// not loaded, and a set that no tile of the CTA needs is skipped.
//
// Kernel shape: one persistent launch per sub-batch, one CTA per SM, 352 threads.  Warp 0
// streams the CTA's needed user tiles by TMA through a ring of stages; warp 1 issues the
// MMAs (M = 128 users, N = the tile's prefix within a TMEM slot of up to 256 columns); warps
// 2-9 are the epilogue, two groups of four that take the slots alternately, one user per
// lane; warp 10 copies the next tiles' bounds into a shared-memory ring with cp.async.  A
// column set of up to 512 columns stays in shared memory as the B operand.  The epilogue
// reads its TMEM lanes 64 columns at a time and runs the fast test per group of 32 columns
// (the group's largest score against the bound of the group's largest k, less the group's
// band); with exact thresholds it only marks the groups some user passes, and a rare loop
// reads those again and writes candidate blocks for cand_resolve_kernel; with the paper's
// |P'| the candidates are resolved in the epilogue itself.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cmath>

#include "sah_internal.cuh"
#include "tc.cuh"

namespace sah {
namespace {

constexpr int kUM = 128;             // users per tile (UMMA M)
constexpr int kUThreads = 352;       // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue, warp 10 bounds loader
constexpr int kLoaderWarp = 10;
constexpr int kRingMax = 8;          // tiles of user bounds staged ahead by the loader warp (at most)
constexpr int kEpiWarps = 8;
constexpr int kMaxTileList = 1024;   // needed tiles per CTA and launch (the host splits longer ranges)
constexpr int kMaxRows = kTcMaxRows;   // rows of a sub-batch the column table takes

// The columns of a sub-batch and their rows.
struct ColTable {
  int32_t* ncol;      // [2]: the number of columns; a flag raised when two rows share a hash but not their bits
  int32_t* rep;       // [nq]: a row holding the column's vector
  int32_t* kq;        // [nq]: largest k <= k_max among the column's rows (0: none)
  int32_t* start;     // [nq + 1]: the column's rows in rows[start[c], start[c + 1])
  int4* rows;         // [nq]: {j | sa << 30, k, bits of ||p_k|| (-inf past n), 0}
  float* qnc;         // [nq]: ||q|| of each column
  float4* qt;         // [dp / 4][nq]: the columns' vectors, transposed (16-byte words)
  uint8_t* q8;        // [nq][128]: every row in E4M3 (FP8 user pass), scaled by 448 / max|q_i|
  float* qsc;         // [nq]: max|q_i| / 448, the row's scale back
  int32_t* colof;     // [nq]: the column of each row (-1: none)
  int32_t* scratch;   // the column table kernel's work arrays when they exceed shared memory
};

// The hash table's slots (a power of two >= 2 nq, at least 64) and the sort's width (a
// power of two >= nq).
inline void col_table_dims(int nq, int* ht, int* npow) {
  *ht = 64;
  while (*ht < 2 * nq) *ht <<= 1;
  *npow = 1;
  while (*npow < nq) *npow <<= 1;
}

// The grid-wide table build's work arrays (int32), in the table's scratch: the hash table,
// then the parts that start zero, then the rest.
struct ColWork {
  int32_t* owner;    // [ht] a row of the slot's vector, -1 empty
  int32_t* minrow;   // [ht] the first row of the slot's vector
  int32_t* kqr;      // [nq] per first row: the column's largest k <= k_max (0: none)
  int32_t* cntr;     // [nq] per first row: the column's rows
  int32_t* rank;     // [nq] per listed column: columns ahead of it in the order
  int32_t* before;   // [nq] per listed column: rows of the columns ahead of it
  int32_t* ctr;      // [8] columns listed, rows with a column
  int32_t* slot;     // [nq] per row: its slot (-1: no column)
  int32_t* reps;     // [nq] the columns' first rows, in no particular order
  int32_t* posr;     // [nq] per first row: the column's place in the order
  int32_t* cursor;   // [nq] per place: the next free entry of its rows
};

__host__ __device__ inline ColWork col_work_at(int32_t* s, int nq, int ht) {
  ColWork W;
  W.owner = s;
  W.minrow = W.owner + ht;
  W.kqr = W.minrow + ht;
  W.cntr = W.kqr + nq;
  W.rank = W.cntr + nq;
  W.before = W.rank + nq;
  W.ctr = W.before + nq;
  W.slot = W.ctr + 8;
  W.reps = W.slot + nq;
  W.posr = W.reps + nq;
  W.cursor = W.posr + nq;
  return W;
}

// int32 entries of the table's scratch: the grid-wide build's arrays (2 ht + 9 nq + 8),
// which also hold the single-CTA rebuild's (2 ht + 5 nq + 2 npow, npow < 2 nq)
inline size_t col_scratch_ints(int nq) {
  int ht = 0, npow = 0;
  col_table_dims(nq, &ht, &npow);
  return 2 * (size_t)ht + 9 * (size_t)nq + 8;
}

size_t col_table_bytes(int nq, int dp) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return up(sizeof(int32_t)) + 3 * up(sizeof(int32_t) * (nq + 1)) + up(sizeof(int4) * (nq + 1)) +
         up(sizeof(float) * nq) + up(sizeof(float4) * (size_t)(dp / 4) * nq) + up((size_t)128 * nq) +
         up(sizeof(float) * nq) + up(sizeof(int32_t) * nq) + up(sizeof(int32_t) * col_scratch_ints(nq));
}

ColTable col_table_at(void* base, int nq, int dp) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* p = (char*)base;
  ColTable T;
  T.ncol = (int32_t*)p;
  p += up(sizeof(int32_t));
  T.rep = (int32_t*)p;
  p += up(sizeof(int32_t) * (nq + 1));
  T.kq = (int32_t*)p;
  p += up(sizeof(int32_t) * (nq + 1));
  T.start = (int32_t*)p;
  p += up(sizeof(int32_t) * (nq + 1));
  T.rows = (int4*)p;
  p += up(sizeof(int4) * (nq + 1));
  T.qnc = (float*)p;
  p += up(sizeof(float) * nq);
  T.qt = (float4*)p;
  p += up(sizeof(float4) * (size_t)(dp / 4) * nq);
  T.q8 = (uint8_t*)p;
  p += up((size_t)128 * nq);
  T.qsc = (float*)p;
  p += up(sizeof(float) * nq);
  T.colof = (int32_t*)p;
  p += up(sizeof(int32_t) * nq);
  T.scratch = (int32_t*)p;
  return T;
}

// A candidate block of the user pass: one user's 32 tensor scores of a 32-column group
// whose fast test it passed (144 bytes).
struct __align__(16) CandBlock {
  int32_t upos;       // user position (leaf order)
  int32_t col0;       // sub-batch column of s[0]
  int32_t pad[2];
  float s[32];        // tensor scores of columns col0 .. col0 + 31
};
static_assert(sizeof(CandBlock) == 144, "candidate blocks are 144 bytes");

// Exclusive prefix of v over the block (blockDim.x a multiple of 32, at most 1024); the
// block's total goes to *total.  Every thread must call it.
__device__ int block_exclusive_scan(int v, int* wsum, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = lane < nw ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) wsum[lane] = s;   // inclusive over warps
    if (lane == 31) *total = s;
  }
  __syncthreads();
  const int before = wid > 0 ? wsum[wid - 1] : 0;
  const int r = before + x - v;
  __syncthreads();
  return r;
}

// The table built by one CTA of 1024 threads.  mode 0: the hash table probed on (hash of the
// padded row's bits, k <= k_max), for sub-batches of up to kSmallTable rows, whose rows
// column_check_kernel then checks bitwise.  mode 1: nothing unless a check raised the
// table's flag (two different vectors with one hash); then every probe compares the rows
// bitwise.  The same table as the grid-wide build's: rows with k > n get no column; a column
// per (vector, k <= k_max); columns in descending order of the key (+inf for columns whose
// rows all have k > k_max, ||q|| otherwise), equal keys by first row.
constexpr int kSmallTable = 2048;
__global__ void __launch_bounds__(1024, 1)
column_table_cta_kernel(const float* __restrict__ Qd, const float* __restrict__ qn, const uint64_t* __restrict__ qh,
                        int nq, int dp, const int32_t* __restrict__ kk, const int32_t* __restrict__ modes, int kmax,
                        int64_t n, const float* __restrict__ pnorm, int ht, int npow, ColTable T, int mode,
                        int in_global) {
  extern __shared__ int32_t sm_dyn[];
  // the work arrays: in shared memory, or (a sub-batch too large for it) in the table's
  // global scratch, which the CTA's barriers order just as well; the sort's keys and
  // indices stay in shared memory either way
  int32_t* sm = in_global ? T.scratch : sm_dyn;
  __shared__ int wsum[32];
  __shared__ int total_sh;
  if (mode == 1 && *(volatile int32_t*)(T.ncol + 1) == 0) return;
  int32_t* owner = sm;             // [ht] a row of the slot's vector, -1 empty
  int32_t* minrow = owner + ht;    // [ht] the first row of the slot's vector
  int32_t* colof = minrow + ht;    // [nq] slot, then column, of each row (-1: none)
  int32_t* cid = colof + nq;       // [nq] column of each first row
  int32_t* cnt = cid + nq;         // [nq] rows per column, then the scatter cursor
  int32_t* kq = cnt + nq;          // [nq] largest k <= k_max per column
  int32_t* crep = kq + nq;         // [nq] the first row of each column
  // [npow] sort keys and column indices (npow: a power of two >= nq)
  float* skey = in_global ? reinterpret_cast<float*>(sm_dyn) : reinterpret_cast<float*>(crep + nq);
  int32_t* sidx = reinterpret_cast<int32_t*>(skey + npow);
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < ht; i += nt) {
    owner[i] = -1;
    minrow[i] = INT_MAX;
  }
  for (int i = tid; i < nq; i += nt) {
    cnt[i] = 0;
    kq[i] = 0;
  }
  __syncthreads();
  // a thread per row: linear probing on (hash of the padded row's bits, k <= k_max); a
  // slot's owner is a row of its vector (mode 1: of its bits)
  const int dp4 = dp / 4;
  const int pass = mode;
  {
    for (int j = tid; j < nq; j += nt) {
      const int k = kk[j];
      colof[j] = -1;
      if (k < 1 || k > n) continue;
      const int cls = k <= kmax ? 0 : 1;
      const uint64_t key = qh[j];
      int slot = (int)(splitmix64(key + (uint64_t)cls) & (uint64_t)(ht - 1));
      for (int probe = 0; probe < ht; ++probe) {
        int cur = owner[slot];
        if (cur == -1) {
          const int prev = atomicCAS(&owner[slot], -1, j);
          if (prev == -1) break;
          cur = prev;
        }
        bool same = qh[cur] == key && (kk[cur] <= kmax ? 0 : 1) == cls;
        if (same && pass == 1) {
          const uint4* a4 = reinterpret_cast<const uint4*>(Qd + (int64_t)j * dp);
          const uint4* c4 = reinterpret_cast<const uint4*>(Qd + (int64_t)cur * dp);
          for (int i = 0; same && i < dp4; ++i) {
            const uint4 x = a4[i], y = c4[i];
            same = x.x == y.x && x.y == y.y && x.z == y.z && x.w == y.w;
          }
        }
        if (same) break;
        slot = (slot + 1) & (ht - 1);
      }
      colof[j] = slot;
      atomicMin(&minrow[slot], j);
    }
    __syncthreads();
  }
  // columns numbered by their first rows, in row order
  const int per = (nq + nt - 1) / nt;
  const int j0 = tid * per, j1 = min(nq, j0 + per);
  int nrep = 0;
  for (int j = j0; j < j1; ++j) nrep += (colof[j] >= 0 && minrow[colof[j]] == j) ? 1 : 0;
  int c = block_exclusive_scan(nrep, wsum, &total_sh);
  const int ncol = total_sh;
  for (int j = j0; j < j1; ++j)
    if (colof[j] >= 0 && minrow[colof[j]] == j) {
      cid[j] = c;
      T.rep[c] = j;
      crep[c] = j;
      ++c;
    }
  __syncthreads();
  for (int j = tid; j < nq; j += nt) {
    if (colof[j] < 0) continue;
    const int cc = cid[minrow[colof[j]]];
    colof[j] = cc;
    atomicAdd(&cnt[cc], 1);
    const int k = kk[j];
    if (k <= kmax) atomicMax(&kq[cc], k);
  }
  __syncthreads();
  // The columns in descending order of ||q|| (columns whose rows have no bound, k > k_max,
  // first; equal norms by first row): the user pass scores, per tile of users, only the
  // prefix of columns whose norm can reach the tile's bound.  A bitonic sort of
  // (key, column) pairs, then every table renumbered.
  int np = 1;                                     // the sort's width: a power of two >= ncol
  while (np < ncol) np <<= 1;
  (void)npow;                                     // (the shared memory is sized for the largest)
  for (int i = tid; i < np; i += nt) {
    skey[i] = i < ncol ? (kq[i] > 0 ? qn[crep[i]] : INFINITY) : -INFINITY;
    sidx[i] = i < ncol ? i : INT_MAX;
  }
  __syncthreads();
  for (int size = 2; size <= np; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      // a thread per compared pair (i, i + stride): i has a zero bit at the stride's position
      for (int pr = tid; pr < np / 2; pr += nt) {
        const int i = ((pr & ~(stride - 1)) << 1) | (pr & (stride - 1));
        const int j = i + stride;
        const float ki = skey[i], kj = skey[j];
        const int ii = sidx[i], ij = sidx[j];
        const bool i_first = ki > kj || (ki == kj && ii < ij);
        if (((i & size) == 0) != i_first) {
          skey[i] = kj;
          skey[j] = ki;
          sidx[i] = ij;
          sidx[j] = ii;
        }
      }
      __syncthreads();
    }
  }
  // position pos holds old column sidx[pos]: its first row, largest k and row count move
  // there (cid holds the counts from now on, minrow the old-to-new map)
  for (int pos = tid; pos < ncol; pos += nt) {
    const int old = sidx[pos];
    T.rep[pos] = crep[old];
    T.kq[pos] = kq[old];
    cid[pos] = cnt[old];
    minrow[old] = pos;
  }
  __syncthreads();
  for (int j = tid; j < nq; j += nt)
    if (colof[j] >= 0) colof[j] = minrow[colof[j]];
  // CSR starts of the columns' rows
  const int perc = (ncol + nt - 1) / nt;
  const int c0 = tid * perc, c1 = min(ncol, c0 + perc);
  int s = 0;
  for (int cc = c0; cc < c1; ++cc) s += cid[cc];
  int o = block_exclusive_scan(s, wsum, &total_sh);
  for (int cc = c0; cc < c1; ++cc) {
    T.start[cc] = o;
    const int x = cid[cc];
    cnt[cc] = o;
    o += x;
  }
  if (tid == 0) {
    T.start[ncol] = total_sh;
    T.ncol[0] = ncol;
    T.ncol[1] = 0;
  }
  __syncthreads();
  for (int j = tid; j < nq; j += nt) {
    const int cc = colof[j];
    T.colof[j] = cc;
    if (cc < 0) continue;
    const int k = kk[j];
    const int sa = (modes != nullptr && modes[j] == SAH_SAALSH && k <= kmax) ? 1 : 0;
    const float pk = k <= n ? pnorm[k - 1] : -INFINITY;
    T.rows[atomicAdd(&cnt[cc], 1)] = make_int4(j | (sa << 30), k, __float_as_int(pk), 0);
  }
  (void)crep;
}

// Every row against its column's first row, a 16-byte word per thread: any difference (two
// vectors that share a hash) raises the table's flag.
__global__ void column_check_kernel(const float* __restrict__ Qd, int nq, int dp, ColTable T) {
  const int dp4 = dp / 4;
  const int64_t total = (int64_t)nq * dp4;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(x / dp4), i = (int)(x - (int64_t)j * dp4);
    const int c = T.colof[j];
    if (c < 0) continue;
    const int r = T.rep[c];
    if (r == j) continue;
    const uint4 a = __ldcg(reinterpret_cast<const uint4*>(Qd + (int64_t)j * dp) + i);
    const uint4 b = __ldcg(reinterpret_cast<const uint4*>(Qd + (int64_t)r * dp) + i);
    if (a.x != b.x || a.y != b.y || a.z != b.z || a.w != b.w) T.ncol[1] = 1;
  }
}

// ---- The grid-wide table build.  col_init_kernel clears the work arrays.
__global__ void col_init_kernel(ColWork W, int nq, int ht) {
  const int64_t nz = 4 * (int64_t)nq + 8;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < ht + nz; x += (int64_t)gridDim.x * blockDim.x) {
    if (x < ht) {
      W.owner[x] = -1;
      W.minrow[x] = INT_MAX;
    } else {
      W.kqr[x - ht] = 0;   // kqr, cntr, rank, before, ctr: contiguous
    }
  }
}

// A thread per row: linear probing on (hash of the padded row's bits, k <= k_max) claims or
// finds the row's slot; the slot keeps its first row.  Rows with k outside 1..n get none.
__global__ void col_hash_kernel(const uint64_t* __restrict__ qh, const int32_t* __restrict__ kk, int nq, int kmax,
                                int64_t n, int ht, ColWork W) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nq) return;
  const int k = kk[j];
  int slot = -1;
  if (k >= 1 && k <= n) {
    const int cls = k <= kmax ? 0 : 1;
    const uint64_t key = qh[j];
    slot = (int)(splitmix64(key + (uint64_t)cls) & (uint64_t)(ht - 1));
    for (int probe = 0; probe < ht; ++probe) {
      const int cur = atomicCAS(&W.owner[slot], -1, j);
      if (cur == -1 || (qh[cur] == key && (kk[cur] <= kmax ? 0 : 1) == cls)) break;
      slot = (slot + 1) & (ht - 1);
    }
    atomicMin(&W.minrow[slot], j);
  }
  W.slot[j] = slot;
}

// A thread per row: its column's row count and largest k <= k_max accumulate at the
// column's first row, which lists itself.  The appends and the row total are counted per
// warp (every lane reaches the ballots).
__global__ void col_reps_kernel(const int32_t* __restrict__ kk, int nq, int kmax, ColWork W) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int s = j < nq ? W.slot[j] : -1;
  const int r = s >= 0 ? W.minrow[s] : -1;
  if (s >= 0) {
    atomicAdd(&W.cntr[r], 1);
    const int k = kk[j];
    if (k <= kmax) atomicMax(&W.kqr[r], k);
  }
  const unsigned has = __ballot_sync(0xffffffffu, s >= 0);
  const unsigned first = __ballot_sync(0xffffffffu, s >= 0 && r == j);
  int base = 0;
  if (lane == 0) {
    if (has) atomicAdd(&W.ctr[1], __popc(has));
    if (first) base = atomicAdd(&W.ctr[0], __popc(first));
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  if ((first >> lane) & 1u) W.reps[base + __popc(first & ((1u << lane) - 1u))] = j;
}

// A column's order key: ascending in it is descending in ||q|| (+inf for columns without a
// k <= k_max), then ascending in first row.  The norms are non-negative floats, whose bits
// order as their values.
__device__ __forceinline__ uint64_t col_order_key(const float* __restrict__ qn, const int32_t* __restrict__ kk,
                                                  int kmax, int r) {
  const float key = kk[r] <= kmax ? qn[r] : INFINITY;
  return ((uint64_t)(~__float_as_uint(key)) << 32) | (uint32_t)r;
}

// The order by counting: a column's place is the number of columns whose key is smaller,
// and its first entry in the row list the rows of those columns.  A CTA takes 1,024 listed
// columns (4 per thread) against a chunk of 512 staged in shared memory and adds its
// partial counts; the grid covers every (slice, chunk) pair of the sub-batch's rows, and
// the parts past the listed columns return at once.
constexpr int kRankOwn = 4;
constexpr int kRankThreads = 256;
constexpr int kRankChunk = 512;
__global__ void __launch_bounds__(kRankThreads)
col_rank_kernel(const float* __restrict__ qn, const int32_t* __restrict__ kk, int kmax, ColWork W) {
  __shared__ uint64_t ck[kRankChunk];
  __shared__ int cc[kRankChunk];
  const int ncol = *(volatile int32_t*)W.ctr;
  const int own0 = blockIdx.x * (kRankOwn * kRankThreads), oth0 = blockIdx.y * kRankChunk;
  if (own0 >= ncol || oth0 >= ncol) return;
  const int nch = min(kRankChunk, ncol - oth0);
  for (int i = threadIdx.x; i < nch; i += kRankThreads) {
    const int r = W.reps[oth0 + i];
    ck[i] = col_order_key(qn, kk, kmax, r);
    cc[i] = W.cntr[r];
  }
  uint64_t mine[kRankOwn];
#pragma unroll
  for (int t = 0; t < kRankOwn; ++t) {
    const int x = own0 + t * kRankThreads + threadIdx.x;
    mine[t] = x < ncol ? col_order_key(qn, kk, kmax, W.reps[x]) : 0ull;
  }
  __syncthreads();
  int rk[kRankOwn] = {}, bf[kRankOwn] = {};
  for (int i = 0; i < nch; ++i) {
    const uint64_t o = ck[i];
    const int w = cc[i];
#pragma unroll
    for (int t = 0; t < kRankOwn; ++t) {
      const bool ahead = o < mine[t];
      rk[t] += ahead ? 1 : 0;
      bf[t] += ahead ? w : 0;
    }
  }
#pragma unroll
  for (int t = 0; t < kRankOwn; ++t) {
    const int x = own0 + t * kRankThreads + threadIdx.x;
    if (x < ncol) {
      if (rk[t]) atomicAdd(&W.rank[x], rk[t]);
      if (bf[t]) atomicAdd(&W.before[x], bf[t]);
    }
  }
}

// A thread per listed column: the column moves to its place (first row, largest k, start
// of its rows); the table's counts and its flag are set.
__global__ void col_place_kernel(ColWork W, ColTable T) {
  const int ncol = *(volatile int32_t*)W.ctr;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x == 0) {
    T.ncol[0] = ncol;
    T.ncol[1] = 0;
    T.start[ncol] = W.ctr[1];
  }
  if (x >= ncol) return;
  const int pos = W.rank[x], r = W.reps[x];
  T.rep[pos] = r;
  T.kq[pos] = W.kqr[r];
  T.start[pos] = W.before[x];
  W.cursor[pos] = W.before[x];
  W.posr[r] = pos;
}

// A thread per (row, 16-byte word): the row's column and its entry in the column's rows
// (word 0), and the row against its column's first row bitwise: any difference (two
// vectors that share a hash) raises the table's flag.
__global__ void col_scatter_kernel(const float* __restrict__ Qd, const int32_t* __restrict__ kk,
                                   const int32_t* __restrict__ modes, int kmax, int64_t n,
                                   const float* __restrict__ pnorm, int nq, int dp, ColWork W, ColTable T) {
  const int dp4 = dp / 4;
  const int64_t total = (int64_t)nq * dp4;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(x / dp4), i = (int)(x - (int64_t)j * dp4);
    const int s = W.slot[j];
    if (s < 0) {
      if (i == 0) T.colof[j] = -1;
      continue;
    }
    const int r = W.minrow[s];
    if (i == 0) {
      const int c = W.posr[r];
      T.colof[j] = c;
      const int k = kk[j];
      const int sa = (modes != nullptr && modes[j] == SAH_SAALSH && k <= kmax) ? 1 : 0;
      const float pk = pnorm[k - 1];
      T.rows[atomicAdd(&W.cursor[c], 1)] = make_int4(j | (sa << 30), k, __float_as_int(pk), 0);
    }
    if (r == j) continue;
    const uint4 a = __ldcg(reinterpret_cast<const uint4*>(Qd + (int64_t)j * dp) + i);
    const uint4 b = __ldcg(reinterpret_cast<const uint4*>(Qd + (int64_t)r * dp) + i);
    if (a.x != b.x || a.y != b.y || a.z != b.z || a.w != b.w) T.ncol[1] = 1;
  }
}

// The columns' vectors transposed (16-byte words, dimension-major: the block filter reads a
// word of consecutive columns at once) and their norms.
__global__ void column_transpose_kernel(const float* __restrict__ Qd, const float* __restrict__ qn, int nq, int dp,
                                        ColTable T) {
  const int dp4 = dp / 4;
  const int ncol = T.ncol[0];
  const float4* Q4 = reinterpret_cast<const float4*>(Qd);
  const int64_t total = (int64_t)ncol * dp4;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(x / ncol), c = (int)(x - (int64_t)i * ncol);   // consecutive threads, consecutive columns
    T.qt[(int64_t)i * nq + c] = Q4[(int64_t)T.rep[c] * dp4 + i];
    if (i == 0) T.qnc[c] = qn[T.rep[c]];
  }
}

// A3 for the tensor-core user pass: Lemma 2 decides which 128-user tiles the GEMM scores.  A
// leaf is needed once one row (j, k) of one column passes its bound: ub >= L^k(B).  (A pair
// the bound prunes is decided "no" by the user pass's own tests anyway, which are tighter,
// so no per-row mask is kept.)  The <c_B, q> are a small GEMM (leaf centres x query
// columns): a CTA takes kBfLeaves leaves and runs over the sub-batch's columns in tiles of
// kBfCols, K in chunks of kBfK dimensions staged in shared memory, each thread accumulating
// 2 leaves x 8 columns; after every column tile the CTA stops if all its leaves are needed.
// With cos phi = <c_B, q> / ||q|| (c_B a unit vector; 1 / ||q|| taken once per column, its
// rounding far inside the slack) and the additive slack covering the FP32 dot and the cone:
//   ub = ||q|| (1 + slack)                                  if cos phi >= cos omega - slack
//   ub = ||q|| (cos phi cos omega + s_up sin omega + 2 slack)  otherwise,
// with s_up = sqrt(1 - (|cos phi| - slack)_+^2) >= sin phi.  The tiles of every needed leaf
// are flagged for the user pass, and leaf_flag[B] (zeroed before the launch) counts a
// leaf's users once.
constexpr int kBfLeaves = 32;
constexpr int kBfCols = 128;
constexpr int kBfK = 32;
constexpr int kBfRows = 512;    // rows of a column tile staged in shared memory (more: from memory)

__global__ void __launch_bounds__(256)
block_filter_cols_kernel(const float* __restrict__ bcent, const float* __restrict__ bcos,
                         const float* __restrict__ bsin, const float* __restrict__ LB, int nb, int kmax, int dp,
                         int nq, ColTable T, float slack, const int32_t* __restrict__ bstart,
                         uint8_t* __restrict__ tile_need, int32_t* __restrict__ leaf_flag,
                         unsigned long long* __restrict__ stats, int st_pairs, int st_users, int st_scored,
                         int st_colpairs) {
  __shared__ __align__(16) float As[kBfK][kBfLeaves];   // centres, dimension-major
  __shared__ __align__(16) float Bs[kBfK][kBfCols];     // columns, dimension-major
  __shared__ float lbs[kBfLeaves][65];                  // L^k(B), k = 1..64
  __shared__ float cws[kBfLeaves], sws[kBfLeaves];
  __shared__ int needed[kBfLeaves];
  __shared__ float cqn[kBfCols], cinv[kBfCols];         // the tile's columns: ||q||, 1 / ||q||
  __shared__ int cst[kBfCols + 1];                      // their rows: cst[c] .. cst[c + 1] (tile-relative)
  __shared__ int2 crw[kBfRows];                         // (j, k) of those rows
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int B0 = blockIdx.x * kBfLeaves;
  const int nl = min(kBfLeaves, nb - B0);
  const int ncol = *T.ncol;
  const int dp4 = dp / 4;
  const int k64 = min(kmax, 64);
  for (int i = tid; i < nl * k64; i += 256) {
    const int k = i / nl + 1, l = i - (k - 1) * nl;   // consecutive threads, consecutive leaves
    lbs[l][k] = LB[(int64_t)(k - 1) * nb + B0 + l];
  }
  if (tid < kBfLeaves) {
    cws[tid] = tid < nl ? bcos[B0 + tid] : -2.f;
    sws[tid] = tid < nl ? bsin[B0 + tid] : 0.f;
    needed[tid] = tid < nl ? 0 : 1;
  }
  int tiles_done = 0;
  for (int col0 = 0; col0 < ncol; col0 += kBfCols) {
    __syncthreads();
    const int nc = min(kBfCols, ncol - col0);
    const int rbase = T.start[col0];
    for (int c = tid; c <= nc; c += 256) {
      cst[c] = T.start[col0 + c] - rbase;
      if (c < nc) {
        const float nrm = T.qnc[col0 + c];
        cqn[c] = nrm;
        cinv[c] = nrm > 0.f ? 1.f / nrm : 0.f;
      }
    }
    const int nrw = T.start[col0 + nc] - rbase;
    for (int q = tid; q < min(nrw, kBfRows); q += 256) {
      const int4 rw = T.rows[rbase + q];
      crw[q] = make_int2(rw.x & 0x3fffffff, rw.y);
    }
    float acc[2][8];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    for (int k0 = 0; k0 < dp; k0 += kBfK) {
      __syncthreads();
      // centres: 16-byte words (4 dimensions) of kBfLeaves rows; consecutive threads take
      // consecutive leaves, so that the transposed stores hit distinct banks
      for (int i = tid; i < kBfLeaves * (kBfK / 4); i += 256) {
        const int l = i % kBfLeaves, w = i / kBfLeaves;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (l < nl && k0 + 4 * w < dp) v = *reinterpret_cast<const float4*>(bcent + (int64_t)(B0 + l) * dp + k0 + 4 * w);
        As[4 * w][l] = v.x;
        As[4 * w + 1][l] = v.y;
        As[4 * w + 2][l] = v.z;
        As[4 * w + 3][l] = v.w;
      }
      // columns: word w (4 dimensions) of column c from the transposed copy (coalesced)
      for (int i = tid; i < (kBfK / 4) * kBfCols; i += 256) {
        const int w = i / kBfCols, c = i % kBfCols;
        const int wg = k0 / 4 + w;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c < nc && wg < dp4) v = T.qt[(int64_t)wg * nq + col0 + c];
        Bs[4 * w][c] = v.x;
        Bs[4 * w + 1][c] = v.y;
        Bs[4 * w + 2][c] = v.z;
        Bs[4 * w + 3][c] = v.w;
      }
      __syncthreads();
#pragma unroll 4
      for (int k = 0; k < kBfK; ++k) {
        const float2 a = *reinterpret_cast<const float2*>(&As[k][2 * ty]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[k][4 * tx]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[k][64 + 4 * tx]);
        const float av[2] = {a.x, a.y};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
    }
    // Lemma 2 for the thread's (leaf, column) pairs of leaves not yet needed
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int l = 2 * ty + a;
      if (l >= nl) continue;
      const float cw = cws[l], sw = sws[l];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int c = b < 4 ? 4 * tx + b : 64 + 4 * tx + (b - 4);
        if (c >= nc || needed[l]) continue;
        const float nrm = cqn[c];
        float ub = INFINITY;   // no cone bound: every row kept
        if (!(cw < -1.5f) && nrm > 0.f) {
          const float cphi = fminf(1.f, fmaxf(-1.f, acc[a][b] * cinv[c]));
          const float cl = fmaxf(0.f, fabsf(cphi) - slack);
          const float sphi = sqrtf(fmaxf(0.f, fmaf(-cl, cl, 1.f)));
          if (cphi >= cw - slack) ub = nrm * (1.f + slack);
          else ub = nrm * (fmaf(cphi, cw, sphi * sw) + 2.f * slack);
        }
        for (int q = cst[c]; q < cst[c + 1]; ++q) {
          const int k = q < kBfRows ? crw[q].y : T.rows[rbase + q].y;
          const float lb = (k <= kmax) ? (k <= 64 ? lbs[l][k] : LB[(int64_t)(k - 1) * nb + B0 + l]) : -INFINITY;
          if (!(ub < lb)) {
            needed[l] = 1;
            break;
          }
        }
      }
    }
    ++tiles_done;
    if (__syncthreads_and(tid >= kBfLeaves || needed[tid])) break;   // every leaf needed
  }
  __syncthreads();
  // the user pass streams the 128-user tiles of every needed leaf
  if (tid < nl && needed[tid]) {
    const int t0 = bstart[B0 + tid] / kUM, t1 = (bstart[B0 + tid + 1] - 1) / kUM;
    for (int t = t0; t <= t1; ++t) tile_need[t] = 1;
  }
  if (tid == 0)
    atomicAdd(&stats[st_colpairs], (unsigned long long)nl * (unsigned long long)min(ncol, tiles_done * kBfCols));
  if (tid < 32) {
    // a needed leaf's users are scored against every column (and every row of the sub-batch)
    unsigned long long pairs = 0, users = 0, scored = 0;
    if (tid < nl && needed[tid]) {
      const unsigned long long u = (unsigned long long)(bstart[B0 + tid + 1] - bstart[B0 + tid]);
      pairs = (unsigned long long)T.start[ncol];
      scored = pairs * u;
      if (atomicExch(&leaf_flag[B0 + tid], 1) == 0) users = u;   // the leaf's users, once
    }
    for (int o = 16; o > 0; o >>= 1) {
      pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
      users += __shfl_xor_sync(0xffffffffu, users, o);
      scored += __shfl_xor_sync(0xffffffffu, scored, o);
    }
    if (tid == 0 && pairs) {
      atomicAdd(&stats[st_pairs], pairs);
      atomicAdd(&stats[st_users], users);
      atomicAdd(&stats[st_scored], scored);
    }
  }
}

struct UpParams {
  int64_t mz, n;
  int kmax, l_exact, dk;
  int slot_cap;                // lower-bound rows kept in shared memory per warp (<= k_max)
  int mask_words;              // words per leaf in kept_mask (the whole sub-batch)
  int ntiles;                  // tiles of all users (tile_need covers them all)
  int tile0, tile_end;         // this launch's tile range
  ColTable T;
  const uint16_t* Qhi;         // nq x dk
  const uint16_t* Qlo;
  const float* qn;
  const float* unorm;
  const float* Eu;
  const float* Lt;
  const float* pnorm;
  const int32_t* uid;
  const int32_t* ublock;
  const uint32_t* kept_mask;   // [nb][mask_words]
  const uint8_t* tile_need;    // [ntiles]
  float cband, gamma;          // score error factor of the MMA (times ||u|| ||q||); FP32 dot factor
  uint32_t* bitmap;
  int64_t words;
  Survivor* resc;
  unsigned long long* resc_count;
  int64_t resc_cap;            // also the capacity of the candidate list
  CandBlock* cand;             // candidate blocks (capacity resc_cap)
  unsigned long long* cand_count;
  unsigned long long* stats;
  int st_yes;
  int st_scores;               // stats slot: (user, column) scores computed
  int st_rows;                 // stats slot: user rows streamed (once per column set)
  int* timeout;
  int inject_stall;            // test hook: the MMA thread stops after its first tile
  int nring;                   // entries of the bound ring (3..kRingMax)
  // FP8 user pass: the columns' E4M3 rows and scales (column table), the users' scales
  const uint8_t* Q8;
  const float* qsc;
  const float* usc;
  // the tiles' bounds min over u of (L_u^k - E_u) / ||u|| ([k_max][ntiles]) and the factor
  // that turns one into the smallest ||q|| a column needs to reach the fast test
  const float* tile_lb;
  float prune_scale;
};

// 32 consecutive FP32 columns of this thread's TMEM lane, waited for; the wait names the
// registers, so that no use of them can be scheduled before it
__device__ __forceinline__ void tmem_ld32_wait(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 consecutive FP32 columns of this thread's TMEM lane, waited for
__device__ __forceinline__ void tmem_ld64_wait(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// one FP32 column of this thread's TMEM lane, waited for
__device__ __forceinline__ float tmem_ld1_wait(uint32_t taddr) {
  uint32_t r;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r)
      : "r"(taddr)
      : "memory");
  return __uint_as_float(r);
}

// Shared memory of the user pass.  A stage holds one 128-user tile (its hi K-blocks and,
// with PRODS = 3, its lo K-blocks); B holds the column set (up to SETN query vectors, hi
// and, with PRODS = 3, lo), resident while the set's tiles stream past.
template <int KB, int STAGES, int SETN, int PRODS, int NSLOT = 2>
struct UpSmem {
  static constexpr int kParts = PRODS == 3 ? 2 : 1;            // hi, or hi and lo
  static constexpr uint32_t kTile = kUM * 128;                  // one K-block of 128 user rows
  static constexpr uint32_t kStage = kParts * KB * kTile;
  static constexpr uint32_t kBPart = SETN * 128;                // one K-block of the set's columns
  static constexpr size_t kOperands = (size_t)STAGES * kStage + (size_t)kParts * KB * kBPart;
  // columns per slice: one MMA into one of NSLOT TMEM slots (512 columns in all; the two
  // epilogue groups take the slots alternately)
  static constexpr int kW = SETN < 512 / NSLOT ? SETN : 512 / NSLOT;
  static constexpr uint32_t kTmemCols = NSLOT * kW;
  // + the bound ring: nring entries of (slots + 5) rows of 128 words (the slots' lower
  // bounds, a -inf row, a +inf row, ||u||, E_u, the caller's user id)
  static constexpr size_t bytes(int slots, int nring) {
    return 1024 + kOperands + (size_t)nring * ((size_t)slots + 5) * 512;
  }
};

// Asynchronous global -> shared copies (no register involved); bytes past src_bytes are
// zero-filled, and src_bytes = 0 reads nothing.
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(tc::smem_addr(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_addr(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
// One arrival on the barrier once every earlier cp.async of this thread has completed
// (the barrier's expected count includes it).
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}

// Maximum of v[OFF .. OFF + 31] with three-input max instructions.
template <int OFF, int NV>
__device__ __forceinline__ float max32_at(const float (&v)[NV]) {
  float g[11];
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(v[OFF + 3 * i]), "f"(v[OFF + 3 * i + 1]), "f"(v[OFF + 3 * i + 2]));
    g[i] = r;
  }
  g[10] = fmaxf(v[OFF + 30], v[OFF + 31]);
  float a, b, c, r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(a) : "f"(g[0]), "f"(g[1]), "f"(g[2]));
  asm("max.f32 %0, %1, %2, %3;" : "=f"(b) : "f"(g[3]), "f"(g[4]), "f"(g[5]));
  asm("max.f32 %0, %1, %2, %3;" : "=f"(c) : "f"(g[6]), "f"(g[7]), "f"(g[8]));
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return fmaxf(r, fmaxf(g[9], g[10]));
}

// INL: candidates are resolved inside the epilogue (where they are dense: the paper's |P'|,
// whose lower bounds are loose) or written as candidate blocks for cand_resolve_kernel
// (where they are sparse: exact thresholds).
// F8: E4M3 operands with per-row scales (kind::f8f6f4, one 128-byte K-block, KB = 1): the
// accumulator times the column's and the user's scale is the score.
template <int KB, int STAGES, int SETN, int PRODS, bool INL, bool F8, int NSLOT>
__global__ void __launch_bounds__(kUThreads, 1)
user_pass_tc_kernel(const __grid_constant__ CUtensorMap tmapUhi, const __grid_constant__ CUtensorMap tmapUlo,
                    UpParams p) {
  using S = UpSmem<KB, STAGES, SETN, PRODS, NSLOT>;
  static_assert(NSLOT % 2 == 0, "the two epilogue groups take the slots alternately");
  constexpr int NROWS = INL ? (KB == 1 ? 512 : 128) : 1;   // rows of a set kept in shared memory
  constexpr int W = S::kW;
  constexpr int NG = SETN / 32;                     // 32-column groups of a set
  extern __shared__ uint8_t smem_raw[];
  // per slot: the MMA's commit (tfull) and the four epilogue warps of its group (tempty)
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[NSLOT], tempty_bar[NSLOT], done_bar;
  // bound ring: the loader fills an entry (ring_full), the eight epilogue warps release it
  __shared__ __align__(8) uint64_t ring_full[kRingMax], ring_empty[kRingMax];
  __shared__ uint32_t tmem_base_sh;
  __shared__ __align__(16) float2 cq[SETN];         // per column: ||q||, bound-table row of its largest k
  __shared__ float csq[F8 ? SETN : 1];              // per column: its E4M3 scale (F8)
  __shared__ int2 crows[INL ? SETN : 1];            // per column: first row (set-relative), row count
  // the set's rows: {j | sa << 30, bound-table row offset (-1: past the cap, -2: no bound),
  // bits of ||p_k||, k}
  __shared__ int4 srows[NROWS];
  __shared__ float2 gq[NG];                         // per 32 columns: largest ||q||, row of the smallest bound
  __shared__ int32_t kseen[65], kslot[65], kfast[65], klist[64], nsl_sh;
  __shared__ float ckey[SETN];                      // per column: ||q||, +inf without a bound (descending)
  __shared__ uint16_t tnc[kMaxTileList];            // per tile of the set: the columns it needs (a prefix)
  __shared__ int kmaxset_sh, nload_sh, njobs_sh, maxtnc_sh;
  __shared__ int32_t tlist[kMaxTileList];           // this CTA's needed tiles, in order
  __shared__ int32_t ntl_sh;
  __shared__ uint32_t tma_issued[STAGES];            // TMA loads issued per stage (teardown drain)
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;                               // [STAGES][hi kb.. | lo kb..]
  uint8_t* sB = base + STAGES * S::kStage;          // [hi kb.. | lo kb..], SETN rows each
  // ring entry e, for the tile's 128 users: row sl (< slot_cap) the lower bound L of slot
  // sl, row slot_cap -inf, row slot_cap + 1 +inf, row slot_cap + 2 ||u||, row slot_cap + 3
  // E_u, row slot_cap + 4 the caller's user id (users past m_nz read as 0); bound "offsets"
  // below are row * 128
  const int ring_rows = p.slot_cap + 5 + (F8 ? 1 : 0);   // F8: row slot_cap + 5 the user's scale
  const int nring = p.nring;
  float* ring = reinterpret_cast<float*>(base + S::kOperands);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&empty_bar[s], 1);
      tma_issued[s] = 0;
    }
    for (int a = 0; a < NSLOT; ++a) {
      tc::mbar_init(&tfull_bar[a], 1);
      tc::mbar_init(&tempty_bar[a], 4);
    }
    tc::mbar_init(&done_bar, 1);
    for (int e = 0; e < nring; ++e) {
      tc::mbar_init(&ring_full[e], 32);   // the loader's lanes, each once its copies land
      tc::mbar_init(&ring_empty[e], kEpiWarps);
    }
    tc::fence_mbar_init();
  }
  for (int i = tid; i < nring * 128; i += kUThreads) {
    float* ent = ring + (i / 128) * ring_rows * 128;
    ent[p.slot_cap * 128 + (i % 128)] = -INFINITY;
    ent[(p.slot_cap + 1) * 128 + (i % 128)] = INFINITY;
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_sh, S::kTmemCols);
    tc::tmem_relinquish();
    // the CTA's tiles of the range that hold a user of a kept leaf
    int cnt = 0;
    for (int b = 0;; b += 32) {
      if ((int64_t)p.tile0 + blockIdx.x + (int64_t)b * gridDim.x >= p.tile_end) break;
      const int64_t t = (int64_t)p.tile0 + blockIdx.x + (int64_t)(b + lane) * gridDim.x;
      const bool f = t < p.tile_end && p.tile_need[t];
      const unsigned m = __ballot_sync(0xffffffffu, f);
      const int pos = cnt + __popc(m & ((1u << lane) - 1u));
      if (f && pos < kMaxTileList) tlist[pos] = (int32_t)t;
      cnt += __popc(m);
    }
    if (lane == 0) ntl_sh = cnt < kMaxTileList ? cnt : kMaxTileList;
  }
  const int ncol = *p.T.ncol;
  int it_base = 0;     // tiles of earlier sets (the bound ring's running index)
  int ld_base = 0;     // tiles loaded for earlier sets (the stages' running index)
  int jbase = 0;       // jobs of earlier sets (the slots' running index)
  int mma_jobs = 0;    // the MMA thread: jobs issued so far
  unsigned long long yes_cnt = 0;   // "yes" taken in the epilogue (INL)
  bool failed = false;
  for (int c0 = 0; c0 < ncol; c0 += SETN) {
    const int nn = min(SETN, ncol - c0);
    // ---- the set's columns: distinct k of their rows, bound-table rows, B operand
    __syncthreads();   // the previous set is done with every shared table
    for (int k = tid; k <= 64; k += kUThreads) kseen[k] = 0;
    __syncthreads();
    const int rb = p.T.start[c0], re = p.T.start[c0 + nn];
    for (int i = rb + tid; i < re; i += kUThreads) {
      const int4 rw = p.T.rows[i];
      if (rw.y >= 1 && rw.y <= p.kmax) kseen[rw.y] = 1;
    }
    __syncthreads();
    if (tid == 0) {
      // the slotted k: every distinct k of the set, or, with more of them than slots, the
      // ranks ceil((i + 1) D / slots) (the largest k among them).  kslot[k]: k's own slot
      // (-1: its rows read their bound from global memory); kfast[k]: the slot of the
      // smallest slotted k' >= k, whose bound L^k' <= L^k serves the column's first test.
      int D = 0;
      for (int k = 1; k <= p.kmax; ++k)
        if (kseen[k]) kseen[k] = ++D;
      const int ns_ = D < p.slot_cap ? D : p.slot_cap;
      int i = 0;
      for (int k = 1; k <= p.kmax; ++k) {
        kslot[k] = -1;
        kfast[k] = -1;
        if (!kseen[k]) continue;
        const int rank = kseen[k];
        while (((i + 1) * D + ns_ - 1) / ns_ < rank) ++i;
        kfast[k] = i;
        if (((i + 1) * D + ns_ - 1) / ns_ == rank) {
          kslot[k] = i;
          klist[i] = k;
        }
      }
      nsl_sh = ns_;
      int km = 0;
      for (int k = p.kmax; k >= 1 && km == 0; --k)
        if (kseen[k]) km = k;
      kmaxset_sh = km;   // the set's largest k <= k_max (0: no row has a bound)
      nload_sh = 0;
      njobs_sh = 0;
      maxtnc_sh = 0;
    }
    __syncthreads();
    if (INL) {
      for (int i = rb + tid; i < re && i - rb < NROWS; i += kUThreads) {
        const int4 rw = p.T.rows[i];
        const int k = rw.y;
        const int sl = (k >= 1 && k <= p.kmax) ? kslot[k] : -1;
        srows[i - rb] = make_int4(rw.x, sl >= 0 ? 128 * sl : (k <= p.kmax ? -1 : -2), rw.z, k);
      }
      for (int c = tid; c < SETN; c += kUThreads)
        crows[INL ? c : 0] = c < nn ? make_int2(p.T.start[c0 + c] - rb, p.T.start[c0 + c + 1] - p.T.start[c0 + c])
                                   : make_int2(0, 0);
    }
    for (int c = tid; c < SETN; c += kUThreads) {
      float qn = 0.f;
      int row = p.slot_cap + 1;   // past nn: the +inf row, never a candidate
      if (c < nn) {
        const int kq = p.T.kq[c0 + c];
        const int sl = kq > 0 ? kfast[kq] : -1;
        qn = p.qn[p.T.rep[c0 + c]];
        // no bound row (only k > k_max rows, or past the cap): the -inf row, every user a candidate
        row = sl >= 0 ? sl : p.slot_cap;
      }
      cq[c] = make_float2(qn, __int_as_float(128 * row));
      ckey[c] = c < nn ? (p.T.kq[c0 + c] > 0 ? qn : INFINITY) : -INFINITY;
      if constexpr (F8) csq[c] = c < nn ? p.qsc[p.T.rep[c0 + c]] : 0.f;
    }
    __syncthreads();
    // Per tile, the columns it needs.  A column reaches the fast test of user u only if
    // (1 + 2c) ||u|| ||q|| >= L_u^k - E_u (the score is at most (1 + c) ||u|| ||q||), so
    // with the columns in descending order of ||q|| a tile needs the prefix with
    // ||q|| >= min over its users of (L_u^K - E_u) / ||u|| / (1 + 2c), K the set's largest
    // k (L falls as k grows); columns without a bound come first.  A tile that needs none is
    // not loaded at all.
    {
      unsigned long long scores = 0, rows = 0;
      for (int li = tid; li < ntl_sh; li += kUThreads) {
        const int t = tlist[li];
        int nc = nn;
        if (kmaxset_sh > 0) {
          const float tau = p.tile_lb[(int64_t)(kmaxset_sh - 1) * p.ntiles + t];
          if (tau > 0.f) {
            const float th = tau * p.prune_scale;
            int lo = 0, hi = nn;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (ckey[mid] >= th) lo = mid + 1;
              else hi = mid;
            }
            nc = lo;
          }
        }
        tnc[li] = (uint16_t)nc;
        if (nc > 0) {
          atomicMax(&maxtnc_sh, nc);
          atomicAdd(&nload_sh, 1);
          atomicAdd(&njobs_sh, (nc + W - 1) / W);
          const int64_t left = p.mz - (int64_t)t * kUM;
          const unsigned long long users = (unsigned long long)(left < kUM ? left : kUM);
          scores += users * (unsigned long long)nc;
          rows += users;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        scores += __shfl_xor_sync(0xffffffffu, scores, o);
        rows += __shfl_xor_sync(0xffffffffu, rows, o);
      }
      if (lane == 0 && scores) {
        atomicAdd(&p.stats[p.st_scores], scores);   // (user, column) scores computed
        atomicAdd(&p.stats[p.st_rows], rows);       // user rows streamed for them
      }
    }
    __syncthreads();
    // no tile of this CTA needs a column of the set (its norms are all too small): nothing
    // of it is staged, loaded or computed
    if (njobs_sh == 0) continue;
    if (tid < NG) {
      // the group's fast test: its largest ||q|| against its smallest bound, which belongs
      // to its largest k (bounds fall as k grows; slots follow k; the -inf row is last)
      float qmax = 0.f;
      int row = -1;
      for (int c = 32 * tid; c < min(nn, 32 * tid + 32); ++c) {
        qmax = fmaxf(qmax, cq[c].x);
        row = max(row, __float_as_int(cq[c].y) / 128);
      }
      gq[tid] = make_float2(qmax, __int_as_float(128 * (row < 0 ? p.slot_cap + 1 : row)));
    }
    const int Nfill = (maxtnc_sh + 15) & ~15;          // the widest prefix a tile of the CTA needs
    for (int i = tid; i < Nfill * KB * 8; i += kUThreads) {
      const int rr = i / (KB * 8), rem = i % (KB * 8), kb = rem / 8, ch = rem % 8;
      uint4 hi = make_uint4(0u, 0u, 0u, 0u), lo = hi;
      if (rr < nn) {
        if constexpr (F8) {
          hi = *reinterpret_cast<const uint4*>(p.Q8 + (int64_t)p.T.rep[c0 + rr] * 128 + ch * 16);
        } else {
          const int64_t off = (int64_t)p.T.rep[c0 + rr] * p.dk + kb * 64 + ch * 8;
          hi = *reinterpret_cast<const uint4*>(p.Qhi + off);
          if (PRODS == 3) lo = *reinterpret_cast<const uint4*>(p.Qlo + off);
        }
      }
      const uint32_t o = tc::sw128_offset(rr, ch);
      *reinterpret_cast<uint4*>(sB + kb * S::kBPart + o) = hi;
      if (PRODS == 3) *reinterpret_cast<uint4*>(sB + (KB + kb) * S::kBPart + o) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = tmem_base_sh;
    const int ntl = ntl_sh;

    if (warp == 0) {
      if (lane == 0) {
        // ---- TMA producer: the set's tiles in order, one stage each
        if (c0 == 0) {
          tc::prefetch_tensormap(&tmapUhi);
          if (PRODS == 3) tc::prefetch_tensormap(&tmapUlo);
        }
        int ld = 0;
        for (int li = 0; li < ntl; ++li) {
          if (tnc[li] == 0) continue;                   // a tile that needs no column
          const int it = ld_base + ld++, s = it % STAGES;
          if (it >= STAGES && !tc::mbar_wait(&empty_bar[s], ((it / STAGES) & 1) ^ 1, p.timeout, nullptr)) break;
          const int t = tlist[li];
          tc::mbar_arrive_expect_tx(&full_bar[s], S::kStage);
          uint8_t* dst = sA + s * S::kStage;
          for (int kb = 0; kb < KB; ++kb) {
            tc::tma_load_2d(dst + kb * S::kTile, &tmapUhi, &full_bar[s], kb * 64, t * kUM);
            if (PRODS == 3) tc::tma_load_2d(dst + (KB + kb) * S::kTile, &tmapUlo, &full_bar[s], kb * 64, t * kUM);
          }
          ++tma_issued[s];
        }
      }
    } else if (warp == 1) {
      if (lane == 0) {
        // ---- MMA issuer: the jobs (tile, slice of its column prefix) in order, job jr into
        // slot (jbase + jr) % NSLOT
        const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
        int ld = 0, jr = -1, li = -1, sc = 0, nst = 0, s = 0;
        for (;;) {
          if (++sc >= nst) {                            // the next tile with columns
            sc = 0;
            do {
              ++li;
            } while (li < ntl && tnc[li] == 0);
            if (li >= ntl) break;
            nst = (tnc[li] + W - 1) / W;
            const int it = ld_base + ld++;
            s = it % STAGES;
            if (p.inject_stall && mma_jobs >= 1) break;   // test hook: a partner that stops working
            if (!tc::mbar_wait(&full_bar[s], (it / STAGES) & 1, p.timeout, nullptr)) break;
          }
          ++jr;
          if (p.inject_stall && mma_jobs >= 1) break;
          const int jg = jbase + jr, slot = jg % NSLOT, u = jg / NSLOT;
          if (u >= 1 && !tc::mbar_wait(&tempty_bar[slot], (u - 1) & 1, p.timeout, nullptr)) break;
          tc::tc_fence_after();
          const int nh = min(W, (int)tnc[li] - sc * W);
          const int ns = nst;                             // slices of this tile's prefix
          const uint32_t idesc = F8 ? tc::idesc_e4m3_f32(kUM, (uint32_t)((nh + 15) & ~15))
                                    : tc::idesc_bf16_f32(kUM, (uint32_t)((nh + 15) & ~15));
          const uint32_t d = tbase + slot * W;
          const uint32_t aS = a0 + s * S::kStage;
          const uint32_t bS = b0 + sc * W * 128;           // rows sc W.. of each B K-block
          uint32_t acc = 0;
#pragma unroll
          for (int prod = 0; prod < PRODS; ++prod) {
            // (A, B) parts: (hi, hi), then with PRODS = 3 (hi, lo) and (lo, hi)
            const uint32_t ap = aS + (prod == 2 ? KB : 0) * S::kTile;
            const uint32_t bp = bS + (prod == 1 ? KB : 0) * S::kBPart;
#pragma unroll
            for (int kb = 0; kb < KB; ++kb)
#pragma unroll
              for (int k16 = 0; k16 < 4; ++k16) {
                // 32 bytes of K per instruction: 16 BF16 or 32 E4M3 values
                if constexpr (F8)
                  tc::umma_e4m3(d, tc::sw128_kmajor_desc(ap + kb * S::kTile + k16 * 32),
                                tc::sw128_kmajor_desc(bp + kb * S::kBPart + k16 * 32), idesc, acc);
                else
                  tc::umma_bf16(d, tc::sw128_kmajor_desc(ap + kb * S::kTile + k16 * 32),
                                tc::sw128_kmajor_desc(bp + kb * S::kBPart + k16 * 32), idesc, acc);
                acc = 1;
              }
          }
          tc::umma_commit(&tfull_bar[slot]);
          if (sc == ns - 1) tc::umma_commit(&empty_bar[s]);   // the tile's stage is free again
          ++mma_jobs;
        }
      }
    } else if (warp == kLoaderWarp) {
      // ---- bound loader: for each tile of the set, in order, the lower bounds of the set's k,
      // ||u||, E_u and the caller's id of its 128 users copied asynchronously into the ring, nring - 1 tiles
      // ahead of the epilogue; each lane's arrival on the entry's barrier waits for its copies
      const int nsl = nsl_sh;
      for (int li = 0; li < ntl; ++li) {
        const int rt = it_base + li, e = rt % nring;
        bool ok = true;
        if (rt >= nring) ok = tc::mbar_wait(&ring_empty[e], ((rt / nring) & 1) ^ 1, p.timeout, nullptr);
        if (!__all_sync(0xffffffffu, ok)) break;
        float* ent = ring + e * ring_rows * 128;
        const int64_t r0 = (int64_t)tlist[li] * kUM;
        {
          const int64_t u4 = r0 + 4 * lane;            // 16-byte chunk of 4 users
          const int nb = (int)std::min<int64_t>(16, std::max<int64_t>(0, (p.mz - u4) * 4));
          cp_async16(ent + (p.slot_cap + 2) * 128 + 4 * lane, nb ? (const void*)(p.unorm + u4) : (const void*)p.unorm, nb);
          cp_async16(ent + (p.slot_cap + 3) * 128 + 4 * lane, nb ? (const void*)(p.Eu + u4) : (const void*)p.Eu, nb);
          cp_async16(ent + (p.slot_cap + 4) * 128 + 4 * lane, nb ? (const void*)(p.uid + u4) : (const void*)p.uid, nb);
          if constexpr (F8)
            cp_async16(ent + (p.slot_cap + 5) * 128 + 4 * lane, nb ? (const void*)(p.usc + u4) : (const void*)p.usc, nb);
        }
        for (int sl = 0; sl < nsl; ++sl) {
          const float* Lrow = p.Lt + (int64_t)(klist[sl] - 1) * p.mz;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const int u = qq * 32 + lane;
            const bool v = r0 + u < p.mz;
            cp_async4(ent + sl * 128 + u, v ? (const void*)(Lrow + r0 + u) : (const void*)Lrow, v ? 4 : 0);
          }
        }
        cp_async_arrive(&ring_full[e]);
      }
      asm volatile("cp.async.wait_all;" ::: "memory");   // nothing in flight when the role ends
    } else {
      // ---- epilogue: group g (warps 2-5, 6-9) takes the jobs of slot g, so that two jobs'
      // epilogues overlap; a warp reads TMEM lane quadrant warp & 3, one user per lane.  The
      // users' bounds come from the loader's ring; ids and norms are read only by the rare
      // candidate path.
      const int ew = warp - 2, g = ew >> 2, quad = warp & 3;
      static_assert(W % 64 == 0, "the epilogue reads 64 columns at a time");
      const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
      const int ul = quad * 32 + lane;                 // this thread's user within the tile

      // ring entries: every epilogue warp takes and releases each tile of the set once, in
      // order (a tile without a job of this warp is taken and released at once)
      int held = -1, next_rel = 0;
      auto ring_take = [&](int li) -> bool {
        const int rt = it_base + li;
        return __all_sync(0xffffffffu, tc::mbar_wait(&ring_full[rt % nring], (rt / nring) & 1, p.timeout, nullptr));
      };
      auto ring_give = [&](int li) {
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&ring_empty[(it_base + li) % nring]);
      };
      auto advance_to = [&](int li) -> bool {   // release every tile before li, take li
        if (held >= 0) {
          ring_give(held);
          next_rel = held + 1;
          held = -1;
        }
        for (; next_rel < li; ++next_rel) {
          if (!ring_take(next_rel)) return false;
          ring_give(next_rel);
        }
        if (li < ntl) {
          if (!ring_take(li)) return false;
          held = li;
        }
        return true;
      };
      int cur_li = -1;
      const float* ent = ring;
      float cu = 0.f, E = 0.f, su = 1.f;
      int64_t r = 0;
      bool valid = false;
      // the bound L - E - 1e-30 (rounded down) of the ring row at `off` for user ul
      auto Lm = [&](int off, int u, float Eu_) { return __fsub_rd(__fsub_rd(ent[off + u], Eu_), 1e-30f); };
      // the jobs (tile, slice of its column prefix) in the MMA issuer's order; this group
      // takes those of its slot
      int jr = -1, li = -1, sc = 0, nst = 0;
      for (;;) {
        if (++sc >= nst) {                              // the next tile with columns
          sc = 0;
          do {
            ++li;
          } while (li < ntl && tnc[li] == 0);
          if (li >= ntl) break;
          nst = (tnc[li] + W - 1) / W;
        }
        ++jr;
        if (((jbase + jr) & 1) != g) continue;
        const int nct = tnc[li];                        // columns of the set this tile needs
        if (li != cur_li) {
          if (!advance_to(li)) {
            failed = true;
            break;
          }
          cur_li = li;
          ent = ring + ((it_base + li) % nring) * ring_rows * 128;
          r = (int64_t)tlist[li] * kUM + ul;
          valid = r < p.mz;
          cu = __fmul_ru(p.cband, ent[(p.slot_cap + 2) * 128 + ul]);
          E = ent[(p.slot_cap + 3) * 128 + ul];
          if constexpr (F8) su = ent[(p.slot_cap + 5) * 128 + ul];
        }
        const int jg = jbase + jr, slot = jg % NSLOT;  // slot % 2 == g
        if (!tc::mbar_wait(&tfull_bar[slot], (jg / NSLOT) & 1, p.timeout, nullptr)) {
          failed = true;
          break;
        }
        tc::tc_fence_after();
        const int cs0 = sc * W;                        // the slice's first column in the set
        // fast test of every 32 columns of the slice: their largest score against the smallest
        // bound of the 32 less their largest band, rounded down (so never above
        // L - E - c ||u|| ||q|| for any of the columns); "no" for all 32 unless it reaches
        constexpr int NG8 = W / 32;
        float thr[NG8];
#pragma unroll
        for (int q = 0; q < NG8; ++q) {
          const int cw = cs0 + 32 * q;
          thr[q] = INFINITY;
          if (cw < nct && valid) {
            const float2 gg = gq[cw >> 5];
            thr[q] = __fsub_rd(Lm(__float_as_int(gg.y), ul, E), __fmul_ru(cu, gg.x));
          }
        }
        const int rem = nct - cs0;                     // columns of the slice the MMA computed
        const uint32_t acc_addr = tbase + lane_addr + slot * W;   // the slice's first column
        if constexpr (INL) {
          // dense candidates: the 32-column groups some user passes are examined here
          uint32_t need = 0;
#pragma unroll
          for (int x2 = 0; x2 < W / 64; ++x2) {
            if (64 * x2 < rem) {
              float vv[64];
              tmem_ld64_wait(acc_addr + 64 * x2, vv);
              if constexpr (F8) {
#pragma unroll
                for (int i = 0; i < 64; ++i) vv[i] = (vv[i] * csq[cs0 + 64 * x2 + i]) * su;
              }
              if (64 * x2 + 64 > rem) {
#pragma unroll
                for (int i = 0; i < 64; ++i)
                  if (64 * x2 + i >= rem) vv[i] = -INFINITY;
              }
              const bool a0 = max32_at<0>(vv) >= thr[2 * x2];
              const bool a1 = max32_at<32>(vv) >= thr[2 * x2 + 1];
              if (__any_sync(0xffffffffu, a0 || a1))
                need |= ((__any_sync(0xffffffffu, a0) ? 1u : 0u) | (__any_sync(0xffffffffu, a1) ? 2u : 0u)) << (2 * x2);
            }
          }
          while (need) {
            const int x = __ffs(need) - 1;             // 32-column group of the slice
            need &= need - 1;
            const int cw = cs0 + 32 * x;               // set column of the group's first score
            const int left = nct - cw;
            float v[32];
            tmem_ld32_wait(acc_addr + 32 * x, v);
            if constexpr (F8) {
#pragma unroll
              for (int i = 0; i < 32; ++i) v[i] = (v[i] * csq[cw + i < SETN ? cw + i : SETN - 1]) * su;
            }
            uint32_t cand = 0;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const float2 c2 = cq[cw + i < SETN ? cw + i : SETN - 1];
              cand |= (i < left && __fmaf_ru(cu, c2.x, v[i]) >= Lm(__float_as_int(c2.y), ul, E) ? 1u : 0u) << i;
            }
            if (!valid) cand = 0u;
            // per candidate column: its rows for every candidate user, a (user, row) pair per
            // lane: the "no" test with the row's own k, then the "yes" tests (Alg. 5); what
            // stays open goes to the FP32 re-score.  L + E is bounded above from L - E - 1e-30
            // (rounded down) with four units in the last place and 2e-30 to spare.
            uint32_t uni = __reduce_or_sync(0xffffffffu, cand);
            while (uni) {
              const int i = __ffs(uni) - 1;
              uni &= uni - 1;
              float sv = tmem_ld1_wait(acc_addr + 32 * x + i);
              if constexpr (F8) sv = (sv * csq[cw + i]) * su;
              const unsigned cm = __ballot_sync(0xffffffffu, (cand >> i) & 1u);
              const int2 cr = crows[cw + i];
              const float qn = cq[cw + i].x;
              const int P = __popc(cm) * cr.y;
              for (int pb = 0; pb < P; pb += 32) {
                const int pp = pb + lane;
                const bool act = pp < P;
                const int ci = act ? pp / cr.y : 0, q = act ? pp % cr.y : 0;
                const int src = act ? (int)__fns(cm, 0, ci + 1) : lane;
                const float s_ = __shfl_sync(0xffffffffu, sv, src);
                const float cu_ = __shfl_sync(0xffffffffu, cu, src);
                const float E_ = __shfl_sync(0xffffffffu, E, src);
                const int r_ = __shfl_sync(0xffffffffu, (int)r, src);
                bool open = false;
                int jv = 0;
                if (act) {
                  int4 rw;
                  if (cr.x + q < NROWS) {
                    rw = srows[cr.x + q];
                  } else {
                    rw = p.T.rows[rb + cr.x + q];
                    const int sl3 = (rw.y >= 1 && rw.y <= p.kmax) ? kslot[rw.y] : -1;
                    rw = make_int4(rw.x, sl3 >= 0 ? 128 * sl3 : (rw.y <= p.kmax ? -1 : -2), rw.z, rw.y);
                  }
                  const int jr = rw.x & 0x3fffffff, k = rw.w;
                  jv = rw.x;
                  float Lq = -INFINITY;   // L - E - 1e-30 rounded down, or -inf without a bound
                  if (rw.y >= 0) {
                    Lq = Lm(rw.y, quad * 32 + src, E_);
                  } else if (rw.y == -1) {   // past the ring's slots
                    Lq = __fsub_rd(__fsub_rd(__ldg(&p.Lt[(int64_t)(k - 1) * p.mz + r_]), E_), 1e-30f);
                  }
                  if (!(__fmaf_ru(cu_, qn, s_) < Lq)) {   // not "no"
                    const float lo = __fsub_rd(s_, __fmul_ru(cu_, qn) + 1e-30f);
                    const float nun_ = __fmul_ru(ent[(p.slot_cap + 2) * 128 + quad * 32 + src], 1.f + 2.f * p.gamma);
                    bool yes = lo >= __fmul_ru(nun_, __int_as_float(rw.z));
                    if (!yes && p.l_exact && k <= p.kmax && Lq != -INFINITY)
                      yes = lo >= __fadd_ru(__fadd_ru(Lq, 2.f * E_), __fmaf_ru(fabsf(Lq), 0x1p-21f, 2e-30f));
                    if (yes) {
                      ++yes_cnt;
                      set_answer(p.bitmap, p.words, jr, __float_as_int(ent[(p.slot_cap + 4) * 128 + quad * 32 + src]));
                    } else {
                      open = true;
                    }
                  }
                }
                const unsigned m = __ballot_sync(0xffffffffu, open);
                if (m) {
                  unsigned long long b0 = 0;
                  if (lane == 0) b0 = atomicAdd(p.resc_count, (unsigned long long)__popc(m));
                  const unsigned long long sl_i = __shfl_sync(0xffffffffu, b0, 0) + __popc(m & ((1u << lane) - 1u));
                  if (open && (int64_t)sl_i < p.resc_cap) p.resc[sl_i] = Survivor{r_, jv, 0.f};
                }
              }
            }
          }
        } else {
          // sparse candidates: the hot loop only marks the 32-column groups some user of the
          // warp passes; those groups are read again from TMEM and every passing user writes
          // its 32 scores, as a candidate block, for the resolve kernel.  (Keeping the block
          // writes out of the unrolled loop keeps it small: with them inside, the pass took a
          // third longer although few groups pass.)
          uint32_t need = 0;
#pragma unroll
          for (int x2 = 0; x2 < W / 64; ++x2) {
            if (64 * x2 < rem) {
              float vv[64];
              tmem_ld64_wait(acc_addr + 64 * x2, vv);
              if constexpr (F8) {
#pragma unroll
                for (int i = 0; i < 64; ++i) vv[i] = (vv[i] * csq[cs0 + 64 * x2 + i]) * su;
              }
              if (64 * x2 + 64 > rem) {
#pragma unroll
                for (int i = 0; i < 64; ++i)
                  if (64 * x2 + i >= rem) vv[i] = -INFINITY;
              }
              const bool a0 = max32_at<0>(vv) >= thr[2 * x2];
              const bool a1 = max32_at<32>(vv) >= thr[2 * x2 + 1];
              need |= ((__any_sync(0xffffffffu, a0) ? 1u : 0u) | (__any_sync(0xffffffffu, a1) ? 2u : 0u)) << (2 * x2);
            }
          }
          while (need) {
            const int x = __ffs(need) - 1;             // 32-column group of the slice
            need &= need - 1;
            const int cw = cs0 + 32 * x;               // set column of the group's first score
            const int left = nct - cw;
            float v[32];
            tmem_ld32_wait(acc_addr + 32 * x, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              if constexpr (F8) v[i] = (v[i] * csq[cw + i < SETN ? cw + i : SETN - 1]) * su;
              if (i >= left) v[i] = -INFINITY;
            }
            // the group's threshold, as in the fast test
            const float2 gg = gq[cw >> 5];
            const float t = valid ? __fsub_rd(Lm(__float_as_int(gg.y), ul, E), __fmul_ru(cu, gg.x)) : INFINITY;
            const bool mine = max32_at<0>(v) >= t;
            const unsigned m = __ballot_sync(0xffffffffu, mine);
            if (m == 0u) continue;
            unsigned long long b0 = 0;
            if (lane == __ffs(m) - 1) b0 = atomicAdd(p.cand_count, (unsigned long long)__popc(m));
            const unsigned long long slot_i = __shfl_sync(0xffffffffu, b0, __ffs(m) - 1) + __popc(m & ((1u << lane) - 1u));
            if (mine && (int64_t)slot_i < p.resc_cap) {
              CandBlock* cb = p.cand + slot_i;
              reinterpret_cast<int4*>(cb)[0] = make_int4((int32_t)r, c0 + cw, 0, 0);
              float4* d4 = reinterpret_cast<float4*>(cb->s);
#pragma unroll
              for (int i = 0; i < 8; ++i) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&tempty_bar[slot]);
      }
      if (!failed && !advance_to(ntl)) failed = true;   // release the set's remaining tiles
    }
    it_base += ntl;
    ld_base += nload_sh;
    jbase += njobs_sh;
    tc::tc_fence_before();
    // a timed-out wait anywhere ends the pass for the whole CTA
    failed = __syncthreads_or(failed || *(volatile int*)p.timeout);
    if (failed) break;
  }
  // ---- teardown
  if (INL && warp >= 2) {
    for (int o = 16; o > 0; o >>= 1) yes_cnt += __shfl_xor_sync(0xffffffffu, yes_cnt, o);
    if (lane == 0 && yes_cnt) atomicAdd(&p.stats[p.st_yes], yes_cnt);
  }
  if (warp == 1 && lane == 0) tc::umma_commit(&done_bar);
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    if (lane == 0) {
      // every MMA this CTA issued, and every TMA load (a pass that stopped early may leave
      // loads that no MMA consumed), completes before TMEM is freed and the CTA exits
      tc::mbar_wait_drain(&done_bar, 0);
      for (int s = 0; s < STAGES; ++s)
        if (tma_issued[s] > 0) tc::mbar_wait_drain(&full_bar[s], (tma_issued[s] - 1) & 1);
    }
    __syncwarp();
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem_base_sh, S::kTmemCols);
  }
}


template <int KB, int STAGES, int SETN, int PRODS, bool INL, bool F8 = false, int NSLOT = 2>
sah_status launch_pass(Index* ix, UpParams p, int sms, cudaStream_t st, int* launches, const cudaEvent_t* ev) {
  using S = UpSmem<KB, STAGES, SETN, PRODS, NSLOT>;
  auto fn = user_pass_tc_kernel<KB, STAGES, SETN, PRODS, INL, F8, NSLOT>;
  constexpr int kFixedRows = 5 + (F8 ? 1 : 0);   // ring rows beside the bound slots
  // lower-bound rows per warp: what shared memory holds beside the operands
  int optin = 0;
  SAH_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ix->device));
  cudaFuncAttributes fa{};
  SAH_CUDA(cudaFuncGetAttributes(&fa, fn));
  // the ring: up to 8 slots of bounds and up to kRingMax entries, at least 3 entries
  const int64_t spare = (int64_t)optin - (int64_t)fa.sharedSizeBytes - (int64_t)S::bytes(0, 0);
  int slots = std::min({ix->kmax, 8, 64});
  while (slots > 1 && spare / ((int64_t)(slots + kFixedRows) * 512) < 3) --slots;
  const int nring = (int)std::min<int64_t>(kRingMax, spare / ((int64_t)(slots + kFixedRows) * 512));
  if (nring < 3) {
    set_error("tensor-core user pass: no shared memory left for the bound ring");
    return SAH_ERR_UNSUPPORTED;
  }
  p.slot_cap = slots;
  p.nring = nring;
  const size_t smem = S::bytes(p.slot_cap + kFixedRows - 5, p.nring);
  SAH_TRY(raise_smem_limit((const void*)fn, (size_t)((int)smem)));
  const unsigned grid = (unsigned)std::max(1, std::min(p.ntiles, sms));
  const int64_t seg = (int64_t)kMaxTileList * grid;   // tiles per launch: at most kMaxTileList per CTA
  for (int64_t t0 = 0; t0 < p.ntiles; t0 += seg) {
    p.tile0 = (int)t0;
    p.tile_end = (int)std::min<int64_t>(p.ntiles, t0 + seg);
    if (ev && t0 == 0) SAH_CUDA(cudaEventRecord(ev[0], st));
    if constexpr (F8) fn<<<grid, kUThreads, smem, st>>>(ix->tmap_U8, ix->tmap_U8, p);
    else fn<<<grid, kUThreads, smem, st>>>(ix->tmap_U, ix->tmap_Ulo, p);
    if (ev && t0 + seg >= p.ntiles) SAH_CUDA(cudaEventRecord(ev[1], st));
    SAH_CUDA(cudaGetLastError());
    if (launches) *launches += 1;
  }
  return SAH_OK;
}


// The per-row tests of Alg. 5 on the user pass's candidate blocks (one user, the tensor
// scores of 32 columns), a warp per block and a lane per column; the sub-batch's column table
// is read in place, the user's values come with the block.  With L = L_u^k, E its
// error and the band e = c ||u|| ||q|| (rounded up):
//   s + e <  L - E                                            -> "no" (k items beat <u,q>)
//   s - e >= ||u|| ||p_k|| (1 + 2 gamma)                       -> "yes" (Alg. 5)
//   s - e >= L + E, when L is the exact k-th score (|P'| = n)  -> "yes"
//   otherwise the pair is re-scored in FP32 (and FP64) by pair_rescore_kernel.
// L + E is bounded above from L - E - 1e-30 (rounded down) with four units in the last place
// and 2e-30 to spare.
constexpr int kResolveThreads = 512;
constexpr int kResolveCtasPerSm = 2;
__global__ void __launch_bounds__(kResolveThreads)
cand_resolve_kernel(const CandBlock* __restrict__ cand, const unsigned long long* __restrict__ cand_count,
                    int64_t cap, ColTable T, const float* __restrict__ Lt, const float* __restrict__ Eu,
                    const float* __restrict__ unorm, const int32_t* __restrict__ uid, int64_t mz, int kmax,
                    int l_exact, float cband, float gamma, uint32_t* __restrict__ bitmap, int64_t words,
                    Survivor* __restrict__ resc, unsigned long long* __restrict__ resc_count,
                    unsigned long long* __restrict__ stats, int st_yes, int st_cand, const int* __restrict__ timeout) {
  __shared__ int stop;
  if (threadIdx.x == 0) stop = *(volatile const int*)timeout;
  const int64_t total = block_count(cand_count, cap);   // synchronises the block
  if (stop || total == 0) return;   // after a timed-out wait the list may hold unwritten entries
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&stats[st_cand], (unsigned long long)total);
  const int ncol = *T.ncol;
  // the column table is read in place (it is small and stays in L2 and L1): staging all of
  // it in every CTA's shared memory cost more than the blocks' own work
  const int4* __restrict__ rows = T.rows;
  const int* __restrict__ start = T.start;
  const float* __restrict__ qnc = T.qnc;
  const int* __restrict__ kqc = T.kq;                        // the column's largest k <= k_max
  const int lane = threadIdx.x & 31;
  unsigned long long yes_cnt = 0;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < total; b += nw) {
    const int4 h0 = reinterpret_cast<const int4*>(cand + b)[0];
    const int64_t r = h0.x;
    const int c = h0.y + lane;
    const float s = cand[b].s[lane];
    const float nu = unorm[r], E = Eu[r];
    const int32_t uidv = uid[r];
    const float cu = __fmul_ru(cband, nu);
    const float nun = __fmul_ru(nu, 1.f + 2.f * gamma);
    const bool live = c < ncol;
    const float qn = live ? qnc[c] : 0.f;
    const float lo = __fsub_rd(s, __fmul_ru(cu, qn) + 1e-30f);
    // the column's own "no" first: its smallest bound belongs to its largest k (bounds fall as
    // k grows); below it, every row of the column is "no"
    // (a column holds rows of k <= k_max only, or rows of k > k_max only, which have no bound)
    bool cand_c = live;
    if (live) {
      const int kq = kqc[c];
      if (kq > 0) cand_c = !(__fmaf_ru(cu, qn, s) < __fsub_rd(__fsub_rd(Lt[(int64_t)(kq - 1) * mz + r], E), 1e-30f));
    }
    const int q0 = cand_c ? start[c] : 0, q1 = cand_c ? start[c + 1] : 0;
    const int nr = cand_c ? q1 - q0 : 0;
    const int nmax = __reduce_max_sync(0xffffffffu, nr);
    for (int t = 0; t < nmax; ++t) {
      bool open = false;
      int jv = 0;
      if (t < nr) {
        const int4 rw = rows[q0 + t];
        const int j = rw.x & 0x3fffffff, k = rw.y;
        jv = rw.x;
        float Lq = -INFINITY;   // L - E - 1e-30 rounded down, or -inf without a bound
        if (k <= kmax) Lq = __fsub_rd(__fsub_rd(Lt[(int64_t)(k - 1) * mz + r], E), 1e-30f);
        if (!(__fmaf_ru(cu, qn, s) < Lq)) {   // not "no"
          bool yes = lo >= __fmul_ru(nun, __int_as_float(rw.z));
          if (!yes && l_exact && k <= kmax && Lq != -INFINITY)
            yes = lo >= __fadd_ru(__fadd_ru(Lq, 2.f * E), __fmaf_ru(fabsf(Lq), 0x1p-21f, 2e-30f));
          if (yes) {
            ++yes_cnt;
            set_answer(bitmap, words, j, uidv);
          } else {
            open = true;
          }
        }
      }
      // open pairs: one append per warp
      const unsigned m = __ballot_sync(0xffffffffu, open);
      if (m) {
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(resc_count, (unsigned long long)__popc(m));
        const unsigned long long slot = __shfl_sync(0xffffffffu, b0, 0) + __popc(m & ((1u << lane) - 1u));
        if (open && (int64_t)slot < cap) resc[slot] = Survivor{(int32_t)r, jv, 0.f};
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) yes_cnt += __shfl_xor_sync(0xffffffffu, yes_cnt, o);
  if (lane == 0 && yes_cnt) atomicAdd(&stats[st_yes], yes_cnt);
}

}  // namespace

size_t user_pass_tc_scratch_bytes(int nq, int dp) { return col_table_bytes(nq, dp); }

sah_status prepare_user_pass_tc(Index* ix, const float* Qd, const float* qn, const uint64_t* qh, void* scratch,
                                const int32_t* kk, const int32_t* modes, int nq, cudaStream_t st, int* launches) {
  if (nq == 0 || ix->dk <= 0) return SAH_OK;
  if (nq > kMaxRows) {
    set_error("tensor-core user pass: sub-batch larger than its column table");
    return SAH_ERR_ARG;
  }
  // the distinct query vectors of the sub-batch
  const ColTable T = col_table_at(scratch, nq, ix->dp);
  int ht = 0, npow = 0;
  col_table_dims(nq, &ht, &npow);
  const ColWork W = col_work_at(T.scratch, nq, ht);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
  // the single CTA's work arrays: in shared memory up to 4,096 rows (180 KB), past that all
  // but the sort's (128 KB at 16,384 rows) in the table's scratch (a rebuild only)
  const size_t need = sizeof(int32_t) * (2 * (size_t)ht + 5 * (size_t)nq + 2 * (size_t)npow);
  const int in_global = need > 200 * 1024 ? 1 : 0;
  const size_t tsmem = in_global ? sizeof(int32_t) * 2 * (size_t)npow : need;
  SAH_TRY(raise_smem_limit((const void*)column_table_cta_kernel, tsmem));
  if (nq <= kSmallTable) {
    column_table_cta_kernel<<<1, 1024, tsmem, st>>>(Qd, qn, qh, nq, ix->dp, kk, modes, ix->kmax, ix->n, ix->pnorm,
                                                     ht, npow, T, 0, in_global);
    column_check_kernel<<<sms, 512, 0, st>>>(Qd, nq, ix->dp, T);
    if (launches) *launches += 2;
  } else {
    const unsigned rows_grid = (unsigned)((nq + 255) / 256);
    col_init_kernel<<<(unsigned)std::max(1, std::min(sms * 4, (ht + 4 * nq + 8 + 255) / 256)), 256, 0, st>>>(W, nq,
                                                                                                            ht);
    col_hash_kernel<<<rows_grid, 256, 0, st>>>(qh, kk, nq, ix->kmax, ix->n, ht, W);
    col_reps_kernel<<<rows_grid, 256, 0, st>>>(kk, nq, ix->kmax, W);
    const dim3 rank_grid((unsigned)((nq + kRankOwn * kRankThreads - 1) / (kRankOwn * kRankThreads)),
                         (unsigned)((nq + kRankChunk - 1) / kRankChunk));
    col_rank_kernel<<<rank_grid, kRankThreads, 0, st>>>(qn, kk, ix->kmax, W);
    col_place_kernel<<<rows_grid, 256, 0, st>>>(W, T);
    col_scatter_kernel<<<(unsigned)(sms * 4), 256, 0, st>>>(Qd, kk, modes, ix->kmax, ix->n, ix->pnorm, nq, ix->dp, W,
                                                            T);
    if (launches) *launches += 6;
  }
  // the rebuild (nothing unless a check raised the flag)
  column_table_cta_kernel<<<1, 1024, tsmem, st>>>(Qd, qn, qh, nq, ix->dp, kk, modes, ix->kmax, ix->n, ix->pnorm, ht,
                                                   npow, T, 1, in_global);
  column_transpose_kernel<<<sms, 512, 0, st>>>(Qd, qn, nq, ix->dp, T);
  SAH_CUDA(cudaGetLastError());
  if (launches) *launches += 2;
  if (ix->prm.tc_user_pass == 2) {
    // the FP8 user pass: every row of the sub-batch in E4M3 with its scale
    launch_e4m3_rows(Qd, nq, ix->dp, ix->d, T.q8, T.qsc, st);
    SAH_CUDA(cudaGetLastError());
    if (launches) *launches += 1;
  }
  return SAH_OK;
}

sah_status block_filter_tc(Index* ix, void* scratch, int nq, uint32_t* kept_mask, int mask_words, uint8_t* tile_need,
                           unsigned long long* stats, int st_pairs, int st_users, int st_scored, int st_colpairs,
                           cudaStream_t st) {
  if (ix->nb == 0 || nq == 0) return SAH_OK;
  const ColTable T = col_table_at(scratch, nq, ix->dp);
  // the leaf flags (after the kept-row words, which this path leaves unused) start zero
  int32_t* leaf_flag = reinterpret_cast<int32_t*>(kept_mask + (size_t)ix->nb * mask_words);
  SAH_CUDA(cudaMemsetAsync(leaf_flag, 0, sizeof(int32_t) * ix->nb, st));
  const unsigned grid = (unsigned)((ix->nb + kBfLeaves - 1) / kBfLeaves);
  block_filter_cols_kernel<<<grid, 256, 0, st>>>(ix->bcent, ix->bcos, ix->bsin, ix->LB, ix->nb, ix->kmax, ix->dp, nq, T,
                                                 ix->cone_slack, ix->bstart, tile_need, leaf_flag, stats, st_pairs,
                                                 st_users, st_scored, st_colpairs);
  SAH_CUDA(cudaGetLastError());
  return SAH_OK;
}

sah_status run_user_pass_tc(Index* ix, const float* Qd, uint16_t* Qsplit, void* scratch, const float* qn,
                            const int32_t* kk, int nq, const uint32_t* kept_mask, int mask_words, uint8_t* tile_need,
                            uint32_t* bitmap, int64_t words, Survivor* resc, unsigned long long* resc_count,
                            Survivor* cand, unsigned long long* cand_count,
                            Survivor* surv, unsigned long long* surv_count, int64_t surv_cap,
                            unsigned long long* stats, int st_yes, int st_fp64, int st_scores, int st_rows, int st_cand,
                            cudaStream_t st,
                            int* launches, const cudaEvent_t* ev) {
  if (ix->m_nz == 0 || nq == 0 || ix->dk <= 0) return SAH_OK;
  const uint16_t* Qhi = Qsplit;
  const uint16_t* Qlo = Qsplit + (size_t)nq * ix->dk;
  const ColTable T = col_table_at(scratch, nq, ix->dp);
  UpParams p{};
  p.mz = ix->m_nz;
  p.n = ix->n;
  p.kmax = ix->kmax;
  p.l_exact = ix->l_exact ? 1 : 0;
  p.dk = ix->dk;
  p.mask_words = mask_words;
  p.ntiles = (int)((ix->m_nz + kUM - 1) / kUM);
  p.tile0 = 0;
  p.tile_end = p.ntiles;
  p.T = T;
  p.Qhi = Qhi;
  p.Qlo = Qlo;
  p.qn = qn;
  p.unorm = ix->unorm;
  p.Eu = ix->Eu;
  p.Lt = ix->Lt;
  p.pnorm = ix->pnorm;
  p.uid = ix->uid;
  p.ublock = ix->ublock;
  p.kept_mask = kept_mask;
  p.tile_need = tile_need;
  // BF16 operands (u_hi = bf16(u), q_hi = bf16(q), each within 2^-8 of its value) and
  // FP32 accumulation of dk products, every addition allowed two units in the last place:
  // |s_tc - <u,q>| <= c_bf ||u|| ||q||
  p.cband = (float)(1.01 * (std::ldexp(1.0, -7) + std::ldexp(1.0, -16) + (2.0 * ix->dk + 16.0) * std::ldexp(1.0, -23)));
  const bool f8 = ix->prm.tc_user_pass == 2;
  p.tile_lb = ix->tile_lb;
  if (f8) {
    // E4M3 operands: every value y = x 448 / max|x_i| is rounded to within 2^-4 |y| + 2^-10
    // (half the subnormal spacing); over K = 128 products, with the scales at most
    // ||x|| / 448, the rounding is bounded by
    //   (2^-4 (1 + 2^-4) + 2^-4) ||u|| ||q|| + 2 (1 + 2^-4) 2^-10 sqrt(K) / 448 ||u|| ||q||
    //   + 2^-20 K / 448^2 ||u|| ||q||,
    // the FP32 accumulation of K products (two units in the last place per addition) and
    // the two scale multiplications and scale roundings by 1.13 ((K + 16) 2^-23 + 8 2^-24)
    // of it (the rounded operands' products sum to at most (1 + 2^-4)^2 ||u|| ||q||)
    const double K = 128.0;
    p.cband = (float)(1.01 * (std::ldexp(1.0, -4) * (2.0 + std::ldexp(1.0, -4)) +
                              2.0 * (1.0 + std::ldexp(1.0, -4)) * std::ldexp(1.0, -10) * std::sqrt(K) / 448.0 +
                              std::ldexp(1.0, -20) * K / (448.0 * 448.0) +
                              1.13 * ((K + 16.0) * std::ldexp(1.0, -23) + 8.0 * std::ldexp(1.0, -24))));
    p.Q8 = T.q8;
    p.qsc = T.qsc;
    p.usc = ix->usc;
  }
  p.gamma = ix->gamma;
  p.bitmap = bitmap;
  p.words = words;
  p.resc = resc;
  p.resc_count = resc_count;
  p.resc_cap = surv_cap;
  p.cand = reinterpret_cast<CandBlock*>(cand);
  p.cand_count = cand_count;
  p.stats = stats;
  p.st_yes = st_yes;
  p.st_scores = st_scores;
  p.st_rows = st_rows;
  p.timeout = ix->dev_timeout;
  p.inject_stall = ix->inject_site == SAH_INJECT_USER_PASS ? 1 : 0;
  // the smallest ||q|| a column needs against a tile bound tau is tau / ((1 + 2c)(1 + 2^-16)):
  // the 2^-16 covers the FP32 rounding of ||q||; the factor is rounded down again
  p.prune_scale = (float)(1.0 / ((1.0 + 2.0 * (double)p.cband) * (1.0 + std::ldexp(1.0, -16))) * (1.0 - std::ldexp(1.0, -20)));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
  // candidates are sparse against exact thresholds (|P'| = n): candidate blocks; dense
  // against the paper's |P'|: resolved in the epilogue
  if (f8) {
    if (ix->l_exact) SAH_TRY((launch_pass<1, 4, 512, 1, false, true>(ix, p, sms, st, launches, ev)));
    else SAH_TRY((launch_pass<1, 4, 512, 1, true, true>(ix, p, sms, st, launches, ev)));
  } else if (ix->dk == 64) {
    if (ix->l_exact) SAH_TRY((launch_pass<1, 4, 512, 1, false>(ix, p, sms, st, launches, ev)));
    else SAH_TRY((launch_pass<1, 4, 512, 1, true>(ix, p, sms, st, launches, ev)));
  } else {
    // d > 64: with exact thresholds the column prefixes are short and one set of 512 keeps the
    // users' rows streamed once (two stages fit beside it), with four TMEM slots of 128
    // columns; with the paper's |P'| the prefixes are long, and sets of 256 leave room for
    // four stages (measured on the 1M-item / 2M-user workload: 0.95 against 1.59 ms, and 4.0
    // against 5.1 ms)
    if (ix->l_exact) SAH_TRY((launch_pass<2, 2, 512, 1, false, false, 4>(ix, p, sms, st, launches, ev)));
    else SAH_TRY((launch_pass<2, 4, 256, 1, true>(ix, p, sms, st, launches, ev)));
  }
  {
    cand_resolve_kernel<<<sms * kResolveCtasPerSm, kResolveThreads, 0, st>>>(
        reinterpret_cast<const CandBlock*>(cand), cand_count, surv_cap, T, ix->Lt, ix->Eu, ix->unorm, ix->uid,
        ix->m_nz, ix->kmax, p.l_exact, p.cband, ix->gamma, bitmap, words, resc, resc_count, stats, st_yes, st_cand,
        ix->dev_timeout);
  }
  SAH_CUDA(cudaGetLastError());
  if (launches) *launches += 1;
  SAH_TRY(launch_pair_rescore(ix, resc, resc_count, surv_cap, Qd, qn, kk, bitmap, words, surv, surv_count, stats,
                               st_yes, st_fp64, nq, sms, st, nullptr, mask_words));
  SAH_CUDA(cudaGetLastError());
  if (launches) *launches += 1;
  return SAH_OK;
}

}  // namespace sah
