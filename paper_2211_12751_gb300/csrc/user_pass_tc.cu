// Tensor-core user pass (A4, with A8's batched score): S = U . Q^T over every user tile and
// the distinct query vectors of a sub-batch, on tcgen05, consumed in the epilogue by the A4
// tests and never written out.
//
// Columns.  The rows of a sub-batch are (q, k) requests; rows asking for the same vector q
// (with k <= k_max) share one GEMM column, so a batch that asks each item at several k
// costs one column per item.  column_table_kernel finds the distinct vectors (hash table in
// shared memory on a hash of each row's bits, then a bitwise check of the rows) and lists
// each column's rows.
//
// Operands.  BF16 alone carries 8 significant bits, which makes the score's error band
// (about 2^-7 ||u|| ||q||) so wide that many pairs would stay open.  Every FP32 vector x
// is therefore split into x_hi = bf16(x) and x_lo = bf16(x - x_hi) (x - x_hi is exact in
// FP32), and the MMA accumulates the three products that matter over a K three times as
// long:  u_hi q_hi + u_hi q_lo + u_lo q_hi.  Per coordinate the dropped parts are bounded
// by 3 * 2^-16 |u_i q_i| (u_lo q_lo and the two second-level rounding residues), so with
// the FP32 accumulation of 3K products
//   |s_tc - <u,q>| <= c_tc ||u|| ||q||,   c_tc = 1.01 (3 * 2^-16 + (6K + 16) 2^-23),
// where the accumulation term lets every addition inside the tensor core lose up to two
// units in the last place (no rounding mode is assumed).  That is about 1e-4 relative:
// the band holds few pairs.
//
// Tests per (user, row) whose leaf the node-level bound (Lemma 2) kept, with L = L_u^k,
// E the error of L, and the band e = c_tc ||u|| ||q||:
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
// Kernel shape: one persistent launch per sub-batch, one CTA per SM, 320 threads, looping
// over chunks of up to 256 columns.  Two groups of four epilogue warps (2-5, 6-9) take
// alternate 128-user tiles; each group owns a TMA stage and two TMEM slots, so the two
// pipelines never wait on each other.  One thread of warp 0 streams the tiles (hi and lo
// K-blocks) for both groups and one thread of warp 1 issues both groups' MMAs, each in a
// loop that polls the barriers without blocking on either group.  A chunk of up to 128
// columns puts a group's consecutive tiles into its two slots in turn, so the next tile's
// MMA runs while the current one is read; a wider chunk uses the two slots as halves of a
// tile.  An epilogue warp (one user per lane) keeps its users' lower bounds for the
// chunk's distinct k in shared memory and reads its TMEM lanes 32 columns at a time: one
// fused multiply-add and one compare per column find the users a column can concern;
// only those take the per-row tests.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cmath>

#include "sah_internal.cuh"
#include "tc.cuh"

namespace sah {
namespace {

constexpr int kUM = 128;             // users per tile (UMMA M)
constexpr int kUThreads = 320;       // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int kEpiWarps = 8;
constexpr int kMaxTileList = 1024;   // needed tiles per CTA and launch (the host splits longer ranges)
constexpr int kRowsSmem = 512;       // rows of a chunk kept in shared memory (more: read from global)
constexpr int kOpenBuf = 64;         // open pairs an epilogue warp buffers per tile
constexpr int kMaxRows = 4096;       // rows of a sub-batch the column table takes

// The columns of a sub-batch and their rows.
struct ColTable {
  int32_t* ncol;      // [1]
  int32_t* rep;       // [nq]: a row holding the column's vector
  int32_t* kq;        // [nq]: largest k <= k_max among the column's rows (0: none)
  int32_t* start;     // [nq + 1]: the column's rows in rows[start[c], start[c + 1])
  int4* rows;         // [nq]: {j | sa << 30, k, bits of ||p_k|| (-inf past n), 0}
  float* qnc;         // [nq]: ||q|| of each column
  float4* qt;         // [dp / 4][nq]: the columns' vectors, transposed (16-byte words)
};

size_t col_table_bytes(int nq, int dp) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return up(sizeof(int32_t)) + 3 * up(sizeof(int32_t) * (nq + 1)) + up(sizeof(int4) * (nq + 1)) +
         up(sizeof(float) * nq) + up(sizeof(float4) * (size_t)(dp / 4) * nq);
}

ColTable col_table_at(void* base, int nq) {
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
  return T;
}

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

// One CTA of 1024 threads.  Rows with k > n ask for every user and get no column.
__global__ void __launch_bounds__(1024, 1)
column_table_kernel(const float* __restrict__ Qd, const float* __restrict__ qn, const uint64_t* __restrict__ qh,
                    int nq, int dp, const int32_t* __restrict__ kk, const int32_t* __restrict__ modes, int kmax,
                    int64_t n, const float* __restrict__ pnorm, int ht, ColTable T) {
  extern __shared__ int32_t sm[];
  __shared__ int wsum[32];
  __shared__ int total_sh, collide_sh;
  int32_t* owner = sm;             // [ht] a row of the slot's vector, -1 empty
  int32_t* minrow = owner + ht;    // [ht] the first row of the slot's vector
  int32_t* colof = minrow + ht;    // [nq] slot, then column, of each row (-1: none)
  int32_t* cid = colof + nq;       // [nq] column of each first row
  int32_t* cnt = cid + nq;         // [nq] rows per column, then the scatter cursor
  int32_t* kq = cnt + nq;          // [nq] largest k <= k_max per column
  int32_t* crep = kq + nq;         // [nq] the first row of each column
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
  // slot's owner is a row of its vector.  Equal hashes are then checked bitwise (a 16-byte
  // word per thread and step, so that the loads coalesce); should two different vectors
  // share a hash, the table is built again with every probe comparing the rows bitwise.
  const int dp4 = dp / 4;
  if (tid == 0) collide_sh = 0;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      for (int i = tid; i < ht; i += nt) {
        owner[i] = -1;
        minrow[i] = INT_MAX;
      }
      __syncthreads();
    }
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
    if (pass == 1) break;
    for (int x0 = tid; x0 < nq * dp4; x0 += 4 * nt) {
      uint4 a[4], b[4];
      bool chk[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int x = x0 + e * nt;
        chk[e] = false;
        a[e] = b[e] = make_uint4(0u, 0u, 0u, 0u);
        if (x < nq * dp4) {
          const int j = x / dp4, i = x - j * dp4;
          const int sl = colof[j];
          const int o = sl >= 0 ? owner[sl] : j;
          if (o != j) {
            chk[e] = true;
            a[e] = __ldcg(reinterpret_cast<const uint4*>(Qd + (int64_t)j * dp) + i);
            b[e] = __ldcg(reinterpret_cast<const uint4*>(Qd + (int64_t)o * dp) + i);
          }
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (chk[e] && (a[e].x != b[e].x || a[e].y != b[e].y || a[e].z != b[e].z || a[e].w != b[e].w))
          collide_sh = 1;
    }
    __syncthreads();
    if (!collide_sh) break;
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
  // CSR starts of the columns' rows
  const int perc = (ncol + nt - 1) / nt;
  const int c0 = tid * perc, c1 = min(ncol, c0 + perc);
  int s = 0;
  for (int cc = c0; cc < c1; ++cc) s += cnt[cc];
  int o = block_exclusive_scan(s, wsum, &total_sh);
  for (int cc = c0; cc < c1; ++cc) {
    T.start[cc] = o;
    T.kq[cc] = kq[cc];
    const int x = cnt[cc];
    cnt[cc] = o;
    o += x;
  }
  if (tid == 0) {
    T.start[ncol] = total_sh;
    *T.ncol = ncol;
  }
  __syncthreads();
  for (int j = tid; j < nq; j += nt) {
    const int cc = colof[j];
    if (cc < 0) continue;
    const int k = kk[j];
    const int sa = (modes != nullptr && modes[j] == SAH_SAALSH && k <= kmax) ? 1 : 0;
    const float pk = k <= n ? pnorm[k - 1] : -INFINITY;
    T.rows[atomicAdd(&cnt[cc], 1)] = make_int4(j | (sa << 30), k, __float_as_int(pk), 0);
  }
  // the columns' vectors transposed (read row by row, so that the loads coalesce) and
  // their norms, for the block filter's thread-per-column reads
  const float4* Q4 = reinterpret_cast<const float4*>(Qd);
  for (int x = tid; x < ncol * dp4; x += nt) {
    const int c = x / dp4, i = x - c * dp4;
    T.qt[(int64_t)i * nq + c] = Q4[(int64_t)crep[c] * dp4 + i];
  }
  for (int c = tid; c < ncol; c += nt) T.qnc[c] = qn[crep[c]];
}

// A3 over the columns: Lemma 2 for every (leaf, distinct query vector) pair, then the bound
// compared with L^k(B) for each row of the column.  A CTA takes kFilterLeaves consecutive
// leaves (centres, cone angles and lower bounds staged in shared memory) and a thread a
// column, which it tests against each leaf in turn; the column vectors come from the
// column table's transposed copy, so that a warp's loads of a 16-byte word of 32 columns
// coalesce, and the (j, k) of the rows are staged in shared memory.  The leaf's decisions
// go to kept_mask[B] (bit j of word j / 32), as the row-wise block filter writes them.  The
// arithmetic of the bound is the row-wise kernel's.
constexpr int kFilterLeaves = 4;
constexpr int kFilterRows = 1024;   // rows staged in shared memory (the rest read from memory)

__global__ void __launch_bounds__(128)
block_filter_cols_kernel(const float* __restrict__ bcent, const float* __restrict__ bcos,
                         const float* __restrict__ bsin, const float* __restrict__ LB, int nb, int kmax, int dp,
                         int nq, ColTable T, float slack, uint32_t* __restrict__ kept_mask, int mask_words,
                         const int32_t* __restrict__ bstart, uint8_t* __restrict__ tile_need,
                         unsigned long long* __restrict__ stats, int st_pairs, int st_users, int st_scored) {
  extern __shared__ float4 cen[];   // [kFilterLeaves][dp / 4] the leaves' unit centres
  __shared__ int2 rs[kFilterRows];   // (j, k) of the rows
  __shared__ uint32_t kbits[kFilterLeaves][kMaxRows / 32];
  __shared__ float lbs[kFilterLeaves][65];   // the leaves' lower bounds L^k(B), k = 1..64
  __shared__ float cws[kFilterLeaves], sws[kFilterLeaves];
  __shared__ int kept_sh[kFilterLeaves];
  const int dp4 = dp / 4;
  const int B0 = blockIdx.x * kFilterLeaves;
  const int nl = min(kFilterLeaves, nb - B0);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ncol = *T.ncol;
  const int nrows = T.start[ncol];
  const float4* cg = reinterpret_cast<const float4*>(bcent + (int64_t)B0 * dp);
  for (int i = tid; i < nl * dp4; i += nt) cen[i] = cg[i];
  const int k64 = min(kmax, 64);
  for (int i = tid; i < nl * k64; i += nt) {
    const int k = i / nl + 1, l = i - (k - 1) * nl;   // consecutive threads, consecutive leaves
    lbs[l][k] = LB[(int64_t)(k - 1) * nb + B0 + l];
  }
  for (int q = tid; q < min(nrows, kFilterRows); q += nt) {
    const int4 rw = T.rows[q];
    rs[q] = make_int2(rw.x & 0x3fffffff, rw.y);
  }
  for (int i = tid; i < nl * mask_words; i += nt) kbits[i / mask_words][i % mask_words] = 0u;
  if (tid < nl) {
    cws[tid] = bcos[B0 + tid];
    sws[tid] = bsin[B0 + tid];
    kept_sh[tid] = 0;
  }
  __syncthreads();
  int kept[kFilterLeaves] = {};
  for (int c = tid; c < ncol; c += nt) {
    const float nrm = T.qnc[c];
    const int r0 = T.start[c], r1 = T.start[c + 1];
    const float4* qc = T.qt + c;   // word i at qc[i * nq]
#pragma unroll
    for (int l = 0; l < kFilterLeaves; ++l) {
      if (l >= nl) break;
      const float cw = cws[l], sw = sws[l];
      const float4* cl = cen + l * dp4;
      float ub = INFINITY;   // no cone bound: every row kept
      if (!(cw < -1.5f) && nrm > 0.f) {
        float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
#pragma unroll 4
        for (int i = 0; i < dp4; ++i) {
          const float4 a = cl[i], b = __ldg(qc + (int64_t)i * nq);
          d0 = fmaf(a.x, b.x, d0);
          d1 = fmaf(a.y, b.y, d1);
          d2 = fmaf(a.z, b.z, d2);
          d3 = fmaf(a.w, b.w, d3);
        }
        const float dq = (d0 + d1) + (d2 + d3);
        const float cphi = fminf(1.f, fmaxf(-1.f, dq / nrm));
        float sphi;
        if (cphi * cphi <= 0.5f) {
          sphi = sqrtf(fmaxf(0.f, fmaf(-cphi, cphi, 1.f)));
        } else {
          float o2 = 0.f;
          for (int i = 0; i < dp4; ++i) {
            const float4 a = cl[i], b = __ldg(qc + (int64_t)i * nq);
            float o;
            o = fmaf(-dq, a.x, b.x); o2 = fmaf(o, o, o2);
            o = fmaf(-dq, a.y, b.y); o2 = fmaf(o, o, o2);
            o = fmaf(-dq, a.z, b.z); o2 = fmaf(o, o, o2);
            o = fmaf(-dq, a.w, b.w); o2 = fmaf(o, o, o2);
          }
          sphi = fminf(1.f, sqrtf(o2) / nrm);
        }
        if (cphi >= cw - slack) ub = nrm * (1.f + slack);
        else ub = nrm * (fmaf(cphi, cw, sphi * sw) + 2.f * slack);
      }
      for (int q = r0; q < r1; ++q) {
        int2 jk;
        if (q < kFilterRows) {
          jk = rs[q];
        } else {
          const int4 rw = T.rows[q];
          jk = make_int2(rw.x & 0x3fffffff, rw.y);
        }
        const int j = jk.x, k = jk.y;
        const float lb = (k <= kmax) ? (k <= 64 ? lbs[l][k] : LB[(int64_t)(k - 1) * nb + B0 + l]) : -INFINITY;
        if (!(ub < lb)) {
          atomicOr(&kbits[l][j >> 5], 1u << (j & 31));
          ++kept[l];
        }
      }
    }
  }
#pragma unroll
  for (int l = 0; l < kFilterLeaves; ++l) {
    const int v = __reduce_add_sync(0xffffffffu, kept[l]);
    if ((tid & 31) == 0 && v) atomicAdd(&kept_sh[l], v);
  }
  __syncthreads();
  for (int i = tid; i < nl * mask_words; i += nt)
    kept_mask[(int64_t)B0 * mask_words + i] = kbits[i / mask_words][i % mask_words];
  // the user pass streams the 128-user tiles that hold a user of a leaf with a kept row
  if (tid < nl && kept_sh[tid] > 0) {
    const int t0 = bstart[B0 + tid] / kUM, t1 = (bstart[B0 + tid + 1] - 1) / kUM;
    for (int t = t0; t <= t1; ++t) tile_need[t] = 1;
  }
  if (tid == 0) {
    unsigned long long pairs = 0, users = 0, scored = 0;
    for (int l = 0; l < nl; ++l) {
      if (!kept_sh[l]) continue;
      const unsigned long long u = (unsigned long long)(bstart[B0 + l + 1] - bstart[B0 + l]);
      pairs += kept_sh[l];
      users += u;
      scored += (unsigned long long)kept_sh[l] * u;
    }
    if (pairs) {
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
  float ctc, gamma;
  uint32_t* bitmap;
  int64_t words;
  Survivor* resc;
  unsigned long long* resc_count;
  int64_t resc_cap;
  unsigned long long* stats;
  int st_yes;
  int* timeout;
  int inject_stall;            // test hook: the MMA thread stops after its first tile
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

template <int KB, int STAGES, int NMAX>
struct UpSmem {
  static constexpr uint32_t kTile = kUM * 128;             // one K-block of 128 user rows
  static constexpr uint32_t kStage = 2 * KB * kTile;       // hi and lo
  static constexpr uint32_t kBPart = NMAX * 128;           // one K-block of the columns
  static constexpr size_t kOperands = (size_t)STAGES * kStage + 2 * KB * (size_t)kBPart;
  // + per epilogue warp: (slots + 2) x 32 lower bounds, kOpenBuf open pairs, a 32-entry table
  static constexpr size_t bytes(int slots) {
    return 1024 + kOperands + (size_t)kEpiWarps * (32 * 4 * ((size_t)slots + 2) + 8 * kOpenBuf + 4 * 32);
  }
  // TMEM: two slots of kSW columns per epilogue group.  A chunk of up to kSW columns puts
  // consecutive tiles of a group into alternate slots (the next tile's MMA runs while the
  // current one is read); a wider chunk uses both slots of a tile as its halves.
  static constexpr int kSW = NMAX < 128 ? NMAX : 128;
  static constexpr uint32_t kTmemCols = 4 * kSW;
};

template <int KB, int STAGES, int NMAX>
__global__ void __launch_bounds__(kUThreads, 1)
user_pass_tc_kernel(const __grid_constant__ CUtensorMap tmapUhi, const __grid_constant__ CUtensorMap tmapUlo,
                    UpParams p) {
  using S = UpSmem<KB, STAGES, NMAX>;
  // the two epilogue groups run independent pipelines: group g owns the stages s = g mod 2
  static_assert(STAGES % 2 == 0, "stages are split between the two epilogue groups");
  extern __shared__ uint8_t smem_raw[];
  // accumulator barriers per (group, half of the columns): the MMA of a group's next tile
  // starts on a half as soon as the epilogue has read that half
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[2][2], tempty_bar[2][2], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ __align__(16) float2 cq[NMAX];         // per column: ||q||, bound-table row of its largest k
  __shared__ int2 crows[NMAX];                      // per column: first row in T.rows, row count
  // the chunk's rows: {j | sa << 30, bound-table row offset (-1: past the cap, -2: no
  // bound), bits of ||p_k||, k}
  __shared__ int4 srows[kRowsSmem];
  __shared__ int32_t wrow[NMAX / 32];               // per 32 columns: their common bound row, or -1
  __shared__ int32_t kseen[65], kslot[65], klist[64], nsl_sh;
  __shared__ int32_t tlist[kMaxTileList];           // this CTA's needed tiles, in order
  __shared__ int32_t ntl_sh, nopen_sh[kEpiWarps];
  __shared__ uint32_t tma_issued[STAGES];            // TMA loads issued per stage (teardown drain)
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;                               // [STAGES][hi kb.. | lo kb..]
  uint8_t* sB = base + STAGES * S::kStage;          // [hi kb.. | lo kb..]
  // per epilogue warp: [slot_cap + 2][32] lower bounds (row slot_cap -inf, row slot_cap + 1
  // +inf) and kOpenBuf open pairs
  float* Lsm = reinterpret_cast<float*>(base + S::kOperands);
  int2* Osm = reinterpret_cast<int2*>(Lsm + kEpiWarps * 32 * (p.slot_cap + 2));
  int32_t* Ism = reinterpret_cast<int32_t*>(Osm + kEpiWarps * kOpenBuf);   // per warp: 32 entries
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a)
      for (int h = 0; h < 2; ++h) {
        tc::mbar_init(&tfull_bar[a][h], 1);
        tc::mbar_init(&tempty_bar[a][h], 4);
      }
    tc::mbar_init(&done_bar, 1);
    for (int s = 0; s < STAGES; ++s) tma_issued[s] = 0;
    tc::fence_mbar_init();
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
  int it_base = 0;     // tiles processed by earlier chunks (all roles count the same)
  int use0 = 0, use1 = 0;   // epilogue: uses so far of its group's two TMEM slots
  int kt = 0;               // epilogue: tiles of its group so far
  int mkt[2] = {0, 0}, mu[2][2] = {{0, 0}, {0, 0}};   // the MMA thread's copies, per group
  int mma_tiles = 0;        // the MMA thread: accumulator slots committed so far
  unsigned long long yes_cnt = 0;
  bool failed = false;
  for (int c0 = 0; c0 < ncol; c0 += NMAX) {
    const int nn = min(NMAX, ncol - c0);
    const int N = (nn + 15) & ~15;
    const int H = N > S::kSW ? 2 : 1;   // TMEM slots per tile
    // ---- the chunk's columns: distinct k of their rows, bound-table rows, B operand
    __syncthreads();   // the previous chunk is done with every shared table
    for (int k = tid; k <= 64; k += kUThreads) kseen[k] = 0;
    __syncthreads();
    const int rb = p.T.start[c0], re = p.T.start[c0 + nn];
    for (int i = rb + tid; i < re; i += kUThreads) {
      const int4 rw = p.T.rows[i];
      if (rw.y >= 1 && rw.y <= p.kmax) kseen[rw.y] = 1;
    }
    __syncthreads();
    if (tid == 0) {
      int ns = 0;
      for (int k = 1; k <= p.kmax; ++k) {
        kslot[k] = -1;
        if (kseen[k]) {
          kslot[k] = ns < p.slot_cap ? ns : -1;   // past the cap: bounds read from global memory
          klist[ns++] = k;
        }
      }
      nsl_sh = ns < p.slot_cap ? ns : p.slot_cap;
    }
    __syncthreads();
    for (int i = rb + tid; i < re && i - rb < kRowsSmem; i += kUThreads) {
      const int4 rw = p.T.rows[i];
      const int k = rw.y;
      const int sl = (k >= 1 && k <= p.kmax) ? kslot[k] : -1;
      srows[i - rb] = make_int4(rw.x, sl >= 0 ? 32 * sl : (k <= p.kmax ? -1 : -2), rw.z, k);
    }
    for (int c = tid; c < NMAX; c += kUThreads) {
      float qn = 0.f;
      int row = p.slot_cap + 1;   // past nn: the +inf row, never a candidate
      int2 cr = make_int2(0, 0);
      if (c < nn) {
        const int kq = p.T.kq[c0 + c];
        const int sl = kq > 0 ? kslot[kq] : -1;
        qn = p.qn[p.T.rep[c0 + c]];
        // no bound row (only k > k_max rows, or past the cap): the -inf row, every user a candidate
        row = sl >= 0 ? sl : p.slot_cap;
        cr = make_int2(p.T.start[c0 + c] - rb, p.T.start[c0 + c + 1] - p.T.start[c0 + c]);   // chunk-relative
      }
      cq[c] = make_float2(qn, __int_as_float(32 * row));
      crows[c] = cr;
    }
    __syncthreads();
    if (tid < NMAX / 32) {
      // the columns < nn of the group share one bound row: the "no" test needs one table read
      int common = -1;
      bool same = true;
      for (int c = 32 * tid; c < min(nn, 32 * tid + 32); ++c) {
        const int off = __float_as_int(cq[c].y);
        if (common == -1) common = off;
        same = same && off == common;
      }
      wrow[tid] = same ? common : -1;
    }
    for (int i = tid; i < N * KB * 8; i += kUThreads) {
      const int rr = i / (KB * 8), rem = i % (KB * 8), kb = rem / 8, ch = rem % 8;
      uint4 hi = make_uint4(0u, 0u, 0u, 0u), lo = hi;
      if (rr < nn) {
        const int64_t off = (int64_t)p.T.rep[c0 + rr] * p.dk + kb * 64 + ch * 8;
        hi = *reinterpret_cast<const uint4*>(p.Qhi + off);
        lo = *reinterpret_cast<const uint4*>(p.Qlo + off);
      }
      const uint32_t o = tc::sw128_offset(rr, ch);
      *reinterpret_cast<uint4*>(sB + kb * S::kBPart + o) = hi;
      *reinterpret_cast<uint4*>(sB + (KB + kb) * S::kBPart + o) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = tmem_base_sh;
    const int ntl = ntl_sh;

    if (warp == 0) {
      if (lane == 0) {
        // TMA producer for both groups: one thread that never blocks on either, so a group
        // whose stage is still busy does not hold up the other
        if (c0 == 0) {
          tc::prefetch_tensormap(&tmapUhi);
          tc::prefetch_tensormap(&tmapUlo);
        }
        const int end = it_base + ntl;
        int nx[2] = {it_base + ((0 - it_base) & 1), it_base + ((1 - it_base) & 1)};
        uint32_t idle = 0;
        for (;;) {
          bool any_left = false, progressed = false;
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            if (nx[g] >= end) continue;
            any_left = true;
            const int s = nx[g] % STAGES;
            if (nx[g] >= STAGES && !tc::mbar_test_wait(&empty_bar[s], ((nx[g] / STAGES) & 1) ^ 1)) continue;
            const int t = tlist[nx[g] - it_base];
            tc::mbar_arrive_expect_tx(&full_bar[s], S::kStage);
            uint8_t* dst = sA + s * S::kStage;
            for (int kb = 0; kb < KB; ++kb) {
              tc::tma_load_2d(dst + kb * S::kTile, &tmapUhi, &full_bar[s], kb * 64, t * kUM);
              tc::tma_load_2d(dst + (KB + kb) * S::kTile, &tmapUlo, &full_bar[s], kb * 64, t * kUM);
            }
            ++tma_issued[s];
            nx[g] += 2;
            progressed = true;
          }
          if (!any_left) break;
          if (progressed) {
            idle = 0;
            continue;
          }
          if (++idle % tc::kFlagEvery == 0 && *(volatile int*)p.timeout) break;
          if (idle > tc::kSpinLimit) {
            atomicExch(p.timeout, 1);
            break;
          }
          if (idle > 32) __nanosleep(32);
        }
      }
    } else if (warp == 1) {
      if (lane == 0) {
        // MMA issuer for both groups (hi.hi + hi.lo + lo.hi into group g's TMEM slots), one
        // thread that never blocks on either group
        const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
        const int end = it_base + ntl;
        int nx[2] = {it_base + ((0 - it_base) & 1), it_base + ((1 - it_base) & 1)};
        int hh[2] = {0, 0};
        uint32_t idle = 0;
        for (;;) {
          // test hook: a partner that stops working; the epilogue's bounded wait runs out
          if (p.inject_stall && mma_tiles >= 1) break;
          bool any_left = false, progressed = false;
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            if (nx[g] >= end) continue;
            any_left = true;
            const int s = nx[g] % STAGES;
            if (hh[g] == 0 && !tc::mbar_test_wait(&full_bar[s], (nx[g] / STAGES) & 1)) continue;
            const int sl = H == 2 ? hh[g] : (mkt[g] & 1);
            const int u = mu[g][sl];
            if (u >= 1 && !tc::mbar_test_wait(&tempty_bar[g][sl], (u & 1) ^ 1)) continue;
            tc::tc_fence_after();
            const int nh = hh[g] == 0 ? (N < S::kSW ? N : S::kSW) : N - S::kSW;
            const uint32_t idesc = tc::idesc_bf16_f32(kUM, (uint32_t)nh);
            const uint32_t d = tbase + (2 * g + sl) * S::kSW;
            const uint32_t bh = b0 + hh[g] * S::kSW * 128;   // rows kSW hh.. of each B part
            const uint32_t aS = a0 + s * S::kStage;
            uint32_t acc = 0;
#pragma unroll
            for (int prod = 0; prod < 3; ++prod) {
              // (A, B) parts: (hi, hi), (hi, lo), (lo, hi)
              const uint32_t ap = aS + (prod == 2 ? KB : 0) * S::kTile;
              const uint32_t bp = bh + (prod == 1 ? KB : 0) * S::kBPart;
#pragma unroll
              for (int kb = 0; kb < KB; ++kb)
#pragma unroll
                for (int k16 = 0; k16 < 4; ++k16) {
                  tc::umma_bf16(d, tc::sw128_kmajor_desc(ap + kb * S::kTile + k16 * 32),
                                tc::sw128_kmajor_desc(bp + kb * S::kBPart + k16 * 32), idesc, acc);
                  acc = 1;
                }
            }
            tc::umma_commit(&tfull_bar[g][sl]);
            ++mu[g][sl];
            ++mma_tiles;
            if (++hh[g] == H) {
              tc::umma_commit(&empty_bar[s]);
              hh[g] = 0;
              ++mkt[g];
              nx[g] += 2;
            }
            progressed = true;
          }
          if (!any_left) break;
          if (progressed) {
            idle = 0;
            continue;
          }
          if (++idle % tc::kFlagEvery == 0 && *(volatile int*)p.timeout) break;
          if (idle > tc::kSpinLimit) {
            atomicExch(p.timeout, 1);
            break;
          }
          if (idle > 32) __nanosleep(32);
        }
      }
    } else {
      // ---- epilogue: group g takes the tiles it with it & 1 == g (accumulator g); a warp
      // reads TMEM lane quadrant warp & 3, one user per lane
      const int ew = warp - 2, g = ew >> 2, quad = warp & 3;
      const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
      const int inf_row = 32 * p.slot_cap;
      float* Lw = Lsm + ew * 32 * (p.slot_cap + 2);
      int2* Ob = Osm + ew * kOpenBuf;
      int32_t* Inv = Ism + ew * 32;
      Lw[inf_row + lane] = -INFINITY;
      Lw[inf_row + 32 + lane] = INFINITY;
      const int nsl = nsl_sh;
      const int wc = (nn + 31) >> 5;
      // values of the group's next tile, loaded while the current one is processed
      constexpr int kPre = 8;
      int Bu_n = 0, id_n = 0;
      float nu_n = 0.f, E_n = 0.f;
      float L_n[kPre];
      uint32_t kw0_n = 0;   // word `lane` of the kept bits of the warp's first leaf
      auto load_user = [&](int li) {
        Bu_n = 0;
        id_n = 0;
        nu_n = 0.f;
        E_n = 0.f;
#pragma unroll
        for (int j = 0; j < kPre; ++j) L_n[j] = 0.f;
        if (li < ntl) {
          const int64_t rr = (int64_t)tlist[li] * kUM + quad * 32 + lane;
          if (rr < p.mz) {
            Bu_n = p.ublock[rr];
            nu_n = p.unorm[rr];
            E_n = p.Eu[rr];
            id_n = p.uid[rr];
#pragma unroll
            for (int j = 0; j < kPre; ++j)
              if (j < nsl) L_n[j] = __ldg(&p.Lt[(int64_t)(klist[j] - 1) * p.mz + rr]);
          }
        }
      };
      // open pairs of a tile wait in Ob; their list slots are claimed with one atomic at
      // the end of the tile and written after the next wait
      int prev_n = 0;
      unsigned long long prev_base = 0;
      auto emit_prev = [&]() {
        if (prev_n == 0) return;
        const unsigned long long b0 = __shfl_sync(0xffffffffu, prev_base, 0);
        for (int i = lane; i < prev_n; i += 32) {
          const int2 e = Ob[i];
          if ((int64_t)(b0 + i) < p.resc_cap) p.resc[b0 + i] = Survivor{e.x, e.y, 0.f};
        }
        prev_n = 0;
        __syncwarp();
        if (lane == 0) nopen_sh[ew] = 0;
        __syncwarp();
      };
      // an open pair into the buffer; a full buffer goes out at once
      auto push_open = [&](int32_t upos, int32_t jv) {
        const int slot = atomicAdd(&nopen_sh[ew], 1);
        if (slot < kOpenBuf) {
          Ob[slot] = make_int2(upos, jv);
        } else {
          const unsigned long long gs = atomicAdd(p.resc_count, 1ull);
          if ((int64_t)gs < p.resc_cap) p.resc[gs] = Survivor{upos, jv, 0.f};
        }
      };
      // the kept words of the first leaf of the warp's users in the next tile
      auto load_words = [&](int li) {
        const int b0 = __shfl_sync(0xffffffffu, Bu_n, 0);
        kw0_n = 0u;
        if (li < ntl && lane < p.mask_words) kw0_n = __ldg(&p.kept_mask[(int64_t)b0 * p.mask_words + lane]);
      };
      if (lane == 0) nopen_sh[ew] = 0;
      __syncwarp();
      const int first = ((g - it_base) & 1);   // local index of the group's first tile
      load_user(first);
      load_words(first);
      for (int li = first; li < ntl; li += 2) {
        const int a = g;
        const int64_t r = (int64_t)tlist[li] * kUM + quad * 32 + lane;
        const bool valid = r < p.mz;
        const int Bu = Bu_n;
        const int B0 = __shfl_sync(0xffffffffu, Bu, 0);
        const uint32_t kw0 = kw0_n;
        const int32_t id = id_n;
        const float nu = nu_n, E = E_n;
        const float cu = __fmul_ru(p.ctc, nu);
        const float nun = __fmul_ru(nu, 1.f + 2.f * p.gamma);
        // this tile's lower bounds L - E (less the band's absolute slack) per distinct k
#pragma unroll
        for (int j = 0; j < kPre; ++j)
          if (j < nsl) Lw[32 * j + lane] = valid ? __fsub_rd(__fsub_rd(L_n[j], E), 1e-30f) : INFINITY;
        for (int sl = kPre; sl < nsl; ++sl) {
          float Llo = INFINITY;
          if (valid) Llo = __fsub_rd(__fsub_rd(__ldg(&p.Lt[(int64_t)(klist[sl] - 1) * p.mz + r]), E), 1e-30f);
          Lw[32 * sl + lane] = Llo;
        }
        __syncwarp();
        for (int h = 0; h < H; ++h) {
          const int sl = H == 2 ? h : (kt & 1);
          const int u = sl ? use1++ : use0++;
          // TMEM address of column 0 of this chunk, as seen from this half's slot
          const uint32_t acc_addr = tbase + lane_addr + (2 * a + sl) * S::kSW - h * S::kSW;
          if (!tc::mbar_wait(&tfull_bar[a][sl], u & 1, p.timeout, nullptr)) {
            failed = true;
            break;
          }
          tc::tc_fence_after();
          if (h == 0) {
            emit_prev();
            load_user(li + 2);
          }
          const int wend = h + 1 < H ? (S::kSW / 32) * (h + 1) : wc;
          for (int w = (S::kSW / 32) * h; w < wend; ++w) {
            float v[32];
            tmem_ld32_wait(acc_addr + 32 * w, v);
            // "no" unless s + c_tc ||u|| ||q|| (rounded up) reaches the column's lowest L - E
            bool any0 = false, any1 = false, any2 = false, any3 = false;
            const int wr = wrow[w];
            if (wr >= 0) {
              const float Lg = Lw[wr + lane];
#pragma unroll
              for (int i = 0; i < 32; i += 4) {
                const float4 ca = *reinterpret_cast<const float4*>(&cq[32 * w + i]);
                const float4 cb = *reinterpret_cast<const float4*>(&cq[32 * w + i + 2]);
                any0 |= __fmaf_ru(cu, ca.x, v[i]) >= Lg;
                any1 |= __fmaf_ru(cu, ca.z, v[i + 1]) >= Lg;
                any2 |= __fmaf_ru(cu, cb.x, v[i + 2]) >= Lg;
                any3 |= __fmaf_ru(cu, cb.z, v[i + 3]) >= Lg;
              }
            } else {
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
              const float4 ca = *reinterpret_cast<const float4*>(&cq[32 * w + i]);
              const float4 cb = *reinterpret_cast<const float4*>(&cq[32 * w + i + 2]);
              any0 |= __fmaf_ru(cu, ca.x, v[i]) >= Lw[__float_as_int(ca.y) + lane];
              any1 |= __fmaf_ru(cu, ca.z, v[i + 1]) >= Lw[__float_as_int(ca.w) + lane];
              any2 |= __fmaf_ru(cu, cb.x, v[i + 2]) >= Lw[__float_as_int(cb.y) + lane];
              any3 |= __fmaf_ru(cu, cb.z, v[i + 3]) >= Lw[__float_as_int(cb.w) + lane];
            }
            }
            if (!__any_sync(0xffffffffu, (any0 || any1) || (any2 || any3))) continue;
            uint32_t cand = 0;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const float2 c2 = cq[32 * w + i];
              cand |= (__fmaf_ru(cu, c2.x, v[i]) >= Lw[__float_as_int(c2.y) + lane] ? 1u : 0u) << i;
            }
            // per candidate column (the whole warp reads its score again from TMEM), the
            // column's rows whose leaf the block bound kept: the "no" test with the row's
            // own k, then the "yes" tests.  L + E is bounded above from the table's
            // L - E - 1e-30 (rounded down) with four units in the last place and 2e-30 to
            // spare.
            uint32_t uni = __reduce_or_sync(0xffffffffu, cand);
            while (uni) {
              const int i = __ffs(uni) - 1;
              uni &= uni - 1;
              const float sv = tmem_ld1_wait(acc_addr + 32 * w + i);
              const bool is_c = valid && ((cand >> i) & 1u);
              const unsigned cm = __ballot_sync(0xffffffffu, is_c);
              // candidate rank -> lane, through this warp's 32-entry table
              __syncwarp();
              if (is_c) Inv[__popc(cm & ((1u << lane) - 1u))] = lane;
              __syncwarp();
              const int2 cr = crows[32 * w + i];
              const float qn = cq[32 * w + i].x;
              // every (candidate user, row) pair of the column on its own lane
              const int P = __popc(cm) * cr.y;
              for (int pb = 0; pb < P; pb += 32) {
                const int pp = pb + lane;
                const bool act = pp < P;
                const int ci = act ? pp / cr.y : 0, q = act ? pp % cr.y : 0;
                const int src = act ? Inv[ci] : lane;
                const float s_ = __shfl_sync(0xffffffffu, sv, src);
                const float cu_ = __shfl_sync(0xffffffffu, cu, src);
                const float nun_ = __shfl_sync(0xffffffffu, nun, src);
                const float E_ = __shfl_sync(0xffffffffu, E, src);
                const int Bu_ = __shfl_sync(0xffffffffu, Bu, src);
                const int id_ = __shfl_sync(0xffffffffu, id, src);
                const int r_ = __shfl_sync(0xffffffffu, (int)r, src);
                int4 rw = make_int4(0, -2, 0, 0);
                if (act) {
                  if (cr.x + q < kRowsSmem) {
                    rw = srows[cr.x + q];
                  } else {
                    rw = p.T.rows[rb + cr.x + q];
                    const int sl3 = (rw.y >= 1 && rw.y <= p.kmax) ? kslot[rw.y] : -1;
                    rw = make_int4(rw.x, sl3 >= 0 ? 32 * sl3 : (rw.y <= p.kmax ? -1 : -2), rw.z, rw.y);
                  }
                }
                const int j = rw.x & 0x3fffffff, k = rw.w;
                // the kept bit: from the words of leaf B0 spread over the lanes, else memory
                uint32_t kwv = __shfl_sync(0xffffffffu, kw0, (j >> 5) & 31);
                if (!act) continue;
                if (Bu_ != B0 || (j >> 5) >= 32) kwv = __ldg(&p.kept_mask[(int64_t)Bu_ * p.mask_words + (j >> 5)]);
                if (!((kwv >> (j & 31)) & 1u)) continue;
                float Lq = -INFINITY;   // L - E - 1e-30 rounded down, or -inf without a bound
                if (rw.y >= 0) {
                  Lq = Lw[rw.y + src];
                } else if (rw.y == -1) {   // past the table's cap
                  Lq = __fsub_rd(__fsub_rd(__ldg(&p.Lt[(int64_t)(k - 1) * p.mz + r_]), E_), 1e-30f);
                }
                if (__fmaf_ru(cu_, qn, s_) < Lq) continue;   // "no"
                const float lo = __fsub_rd(s_, __fmul_ru(cu_, qn) + 1e-30f);
                bool yes = lo >= __fmul_ru(nun_, __int_as_float(rw.z));
                if (!yes && p.l_exact && k <= p.kmax && Lq != -INFINITY)
                  yes = lo >= __fadd_ru(__fadd_ru(Lq, 2.f * E_), __fmaf_ru(fabsf(Lq), 0x1p-21f, 2e-30f));
                if (yes) {
                  ++yes_cnt;
                  set_answer(p.bitmap, p.words, j, id_);
                } else {
                  push_open((int32_t)r_, rw.x);
                }
              }
            }
          }
          tc::tc_fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&tempty_bar[a][sl]);
        }
        ++kt;
        if (failed) break;
        // claim the re-score slots of this tile's open pairs (written after the next wait)
        __syncwarp();
        const int no = min(nopen_sh[ew], kOpenBuf);
        prev_n = no;
        if (no && lane == 0) prev_base = atomicAdd(p.resc_count, (unsigned long long)no);
        load_words(li + 2);
      }
      if (!failed) emit_prev();
    }
    it_base += ntl;
    tc::tc_fence_before();
    // a timed-out wait anywhere ends the pass for the whole CTA
    failed = __syncthreads_or(failed || *(volatile int*)p.timeout);
    if (failed) break;
  }
  // ---- teardown
  if (warp >= 2) {
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


template <int KB, int STAGES, int NMAX>
sah_status launch_pass(Index* ix, UpParams p, int sms, cudaStream_t st, int* launches, const cudaEvent_t* ev) {
  using S = UpSmem<KB, STAGES, NMAX>;
  auto fn = user_pass_tc_kernel<KB, STAGES, NMAX>;
  // lower-bound rows per warp: what shared memory holds beside the operands
  int optin = 0;
  SAH_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ix->device));
  cudaFuncAttributes fa{};
  SAH_CUDA(cudaFuncGetAttributes(&fa, fn));
  const int64_t spare = (int64_t)optin - (int64_t)fa.sharedSizeBytes - (int64_t)S::bytes(0);
  const int rows = (int)std::max<int64_t>(0, spare / (kEpiWarps * 32 * 4));
  p.slot_cap = std::min({ix->kmax, 64, rows});
  if (p.slot_cap < 1) {
    set_error("tensor-core user pass: no shared memory left for the lower bounds");
    return SAH_ERR_UNSUPPORTED;
  }
  const size_t smem = S::bytes(p.slot_cap);
  SAH_TRY(raise_smem_limit((const void*)fn, (size_t)((int)smem)));
  const unsigned grid = (unsigned)std::max(1, std::min(p.ntiles, sms));
  const int64_t seg = (int64_t)kMaxTileList * grid;   // tiles per launch: at most kMaxTileList per CTA
  for (int64_t t0 = 0; t0 < p.ntiles; t0 += seg) {
    p.tile0 = (int)t0;
    p.tile_end = (int)std::min<int64_t>(p.ntiles, t0 + seg);
    if (ev && t0 == 0) SAH_CUDA(cudaEventRecord(ev[0], st));
    fn<<<grid, kUThreads, smem, st>>>(ix->tmap_U, ix->tmap_Ulo, p);
    if (ev && t0 + seg >= p.ntiles) SAH_CUDA(cudaEventRecord(ev[1], st));
    SAH_CUDA(cudaGetLastError());
    if (launches) *launches += 1;
  }
  return SAH_OK;
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
  const ColTable T = col_table_at(scratch, nq);
  int ht = 64;
  while (ht < 2 * nq) ht <<= 1;
  const size_t tsmem = sizeof(int32_t) * (2 * (size_t)ht + 5 * (size_t)nq);
  SAH_TRY(raise_smem_limit((const void*)column_table_kernel, tsmem));
  column_table_kernel<<<1, 1024, tsmem, st>>>(Qd, qn, qh, nq, ix->dp, kk, modes, ix->kmax, ix->n, ix->pnorm, ht,
                                               T);
  SAH_CUDA(cudaGetLastError());
  if (launches) *launches += 1;
  return SAH_OK;
}

sah_status block_filter_tc(Index* ix, void* scratch, int nq, uint32_t* kept_mask, int mask_words, uint8_t* tile_need,
                           unsigned long long* stats, int st_pairs, int st_users, int st_scored,
                           cudaStream_t st) {
  if (ix->nb == 0 || nq == 0) return SAH_OK;
  const ColTable T = col_table_at(scratch, nq);
  block_filter_cols_kernel<<<(ix->nb + kFilterLeaves - 1) / kFilterLeaves, 128,
                             sizeof(float) * ix->dp * kFilterLeaves, st>>>(
      ix->bcent, ix->bcos, ix->bsin, ix->LB, ix->nb, ix->kmax, ix->dp, nq, T, ix->cone_slack, kept_mask, mask_words,
      ix->bstart, tile_need, stats, st_pairs, st_users, st_scored);
  SAH_CUDA(cudaGetLastError());
  return SAH_OK;
}

sah_status run_user_pass_tc(Index* ix, const float* Qd, uint16_t* Qsplit, void* scratch, const float* qn,
                            const int32_t* kk, int nq, const uint32_t* kept_mask, int mask_words, uint8_t* tile_need,
                            uint32_t* bitmap, int64_t words, Survivor* resc, unsigned long long* resc_count,
                            Survivor* surv, unsigned long long* surv_count, int64_t surv_cap,
                            unsigned long long* stats, int st_yes, int st_fp64, cudaStream_t st, int* launches,
                            const cudaEvent_t* ev) {
  if (ix->m_nz == 0 || nq == 0 || ix->dk <= 0) return SAH_OK;
  const uint16_t* Qhi = Qsplit;
  const uint16_t* Qlo = Qsplit + (size_t)nq * ix->dk;
  const ColTable T = col_table_at(scratch, nq);
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
  p.ctc = (float)(1.01 * (3.0 * std::ldexp(1.0, -16) + (6.0 * ix->dk + 16.0) * std::ldexp(1.0, -23)));
  p.gamma = ix->gamma;
  p.bitmap = bitmap;
  p.words = words;
  p.resc = resc;
  p.resc_count = resc_count;
  p.resc_cap = surv_cap;
  p.stats = stats;
  p.st_yes = st_yes;
  p.timeout = ix->dev_timeout;
  p.inject_stall = ix->inject_site == SAH_INJECT_USER_PASS ? 1 : 0;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
  if (ix->dk == 64) {
    SAH_TRY((launch_pass<1, 4, 128>(ix, p, sms, st, launches, ev)));
  } else {
    SAH_TRY((launch_pass<2, 2, 64>(ix, p, sms, st, launches, ev)));
  }
  SAH_TRY(launch_pair_rescore(ix, resc, resc_count, surv_cap, Qd, qn, kk, bitmap, words, surv, surv_count, stats,
                               st_yes, st_fp64, nq, sms, st));
  SAH_CUDA(cudaGetLastError());
  if (launches) *launches += 1;
  return SAH_OK;
}

}  // namespace sah
