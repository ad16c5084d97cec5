// SA-ALSH (Alg. 1, Alg. 2) on the items behind P'.
//
// Indexing (Alg. 1): the items are already in descending norm order; partition S_j opens
// at the largest remaining norm M_j and keeps every following item with ||p|| > b M_j
// (zero-norm items form one final partition).  Per partition: centroid c_j, radius
// R_j = max ||p - c_j||, the shifting-invariant transform I(p, c_j) =
// [p - c_j; sqrt(R_j^2 - ||p - c_j||^2)] (Eq. 6) and SRP codes of it (Eq. 1, Eq. 9): table t
// packs code_bits sign bits, bit b = [<a_{t,b}, I(p, c_j)> >= 0].  Items are sorted by
// code inside every (partition, table) so that a bucket is a contiguous range.
//
// The user transform U(u) = [R_j u / ||u||; 0] (Eq. 7) has the same signs for every
// partition with R_j > 0, so a user's codes are computed once; a partition with R_j = 0
// maps every item and user to the zero vector, where every code collides.
//
// Query (Alg. 2, one warp per survivor): phi is the k-th largest score over the
// candidate set C, kept in a k-slot list spread over the warp's lanes; C starts as P'
// (its k largest scores are the lower-bound array).  Per partition in descending M_j:
// "yes" once phi exceeds mu_j = M_j ||u||; otherwise the partition's candidates (items
// whose code is within Hamming probe_radius of the user's code in some table) are
// scored in FP32 and merged (each item once); "no" once <u,q> is certainly below phi.
// Scores carry the FP32 bound, so every "no" is backed by k items that certainly beat
// <u,q>: SA-ALSH answers are supersets of the exact answers.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <thread>
#include <vector>

#include "sah_internal.cuh"

namespace sah {
namespace {

inline unsigned grid_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

// Partial column sums of every partition's items, in chunks of 1024 items (double).
constexpr int kCentChunk = 1024;
__global__ void centroid_partial_kernel(const float* __restrict__ Ps, int dp, const int32_t* __restrict__ start,
                                        const int32_t* __restrict__ chunk_part, const int32_t* __restrict__ chunk_first,
                                        double* __restrict__ partial) {
  const int c = blockIdx.x;
  const int j = chunk_part[c];
  const int64_t i0 = chunk_first[c];
  const int64_t i1 = std::min<int64_t>(i0 + kCentChunk, start[j + 1]);
  for (int e = threadIdx.x; e < dp; e += blockDim.x) {
    double s = 0.0;
    for (int64_t i = i0; i < i1; ++i) s += (double)Ps[i * dp + e];
    partial[(int64_t)c * dp + e] = s;
  }
}

__global__ void centroid_final_kernel(const double* __restrict__ partial, const int32_t* __restrict__ part_chunk0,
                                      const int32_t* __restrict__ start, int dp, float* __restrict__ cent) {
  const int j = blockIdx.x;
  const int c0 = part_chunk0[j], c1 = part_chunk0[j + 1];
  const double cnt = (double)(start[j + 1] - start[j]);
  for (int e = threadIdx.x; e < dp; e += blockDim.x) {
    double s = 0.0;
    for (int c = c0; c < c1; ++c) s += partial[(int64_t)c * dp + e];
    cent[(int64_t)j * dp + e] = (float)(s / cnt);
  }
}

// R_j = max ||p - c_j|| (an order-independent max, so deterministic).
__global__ void radius_kernel(const float* __restrict__ Ps, int dp, int64_t first, int64_t n,
                              const int32_t* __restrict__ part_of, const float* __restrict__ cent,
                              unsigned int* __restrict__ Rbits) {
  const int64_t i = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = part_of[i - first];
  const float* p = Ps + i * dp;
  const float* c = cent + (int64_t)j * dp;
  float s = 0.f;
  for (int e = 0; e < dp; ++e) {
    const float t = p[e] - c[e];
    s = fmaf(t, t, s);
  }
  atomicMax(&Rbits[j], __float_as_uint(sqrtf(s)));
}

// Item codes (Eq. 6, Eq. 1, Eq. 9): one thread per (item, table).
__global__ void item_codes_kernel(const float* __restrict__ Ps, int d, int dp, int64_t first, int64_t n,
                                  const int32_t* __restrict__ part_of, const float* __restrict__ cent,
                                  const float* __restrict__ R, const float* __restrict__ A, int d1p, int K,
                                  int bits, uint16_t* __restrict__ codes) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cnt = n - first;
  if (g >= cnt * K) return;
  const int64_t it = g / K;
  const int t = (int)(g % K);
  const int64_t i = first + it;
  const int j = part_of[it];
  const float* p = Ps + i * dp;
  const float* c = cent + (int64_t)j * dp;
  float r2 = 0.f;
  for (int e = 0; e < d; ++e) {
    const float x = p[e] - c[e];
    r2 = fmaf(x, x, r2);
  }
  const float Rj = R[j];
  const float last = sqrtf(fmaxf(0.f, Rj * Rj - r2));
  uint32_t code = 0;
  for (int b = 0; b < bits; ++b) {
    const float* a = A + (int64_t)(t * bits + b) * d1p;
    float s = a[d] * last;
    for (int e = 0; e < d; ++e) s = fmaf(a[e], p[e] - c[e], s);
    code |= (s >= 0.f ? 1u : 0u) << b;
  }
  codes[it * K + t] = (uint16_t)code;
}

// User codes: signs of <a, u> (Eq. 7 up to a positive factor).  A CTA takes 128 users and
// kCodeTables tables: their projection rows and the users' rows are staged in shared
// memory (odd row stride: conflict-free), one thread per (user, table).
constexpr int kCodeUsers = 128;
constexpr int kCodeTables = 2;

__global__ void user_codes_kernel(const float* __restrict__ Ut, int d, int dp, int64_t m, const float* __restrict__ A,
                                  int d1p, int K, int bits, uint16_t* __restrict__ codes) {
  extern __shared__ float sh[];
  const int ds = d | 1;                                   // odd stride
  float* us = sh;                                         // kCodeUsers x ds
  float* as = sh + kCodeUsers * ds;                       // kCodeTables * bits x ds
  const int64_t u0 = (int64_t)blockIdx.x * kCodeUsers;
  const int t0 = blockIdx.y * kCodeTables;
  const int nt = min(kCodeTables, K - t0);
  for (int i = threadIdx.x; i < kCodeUsers * d; i += blockDim.x) {
    const int r = i / d, e = i % d;
    us[r * ds + e] = (u0 + r < m) ? Ut[(u0 + r) * dp + e] : 0.f;
  }
  for (int i = threadIdx.x; i < nt * bits * d; i += blockDim.x) {
    const int r = i / d, e = i % d;
    as[r * ds + e] = A[(int64_t)(t0 * bits + r) * d1p + e];
  }
  __syncthreads();
  const int r = threadIdx.x % kCodeUsers, tl = threadIdx.x / kCodeUsers;
  if (tl >= nt || u0 + r >= m) return;
  const float* x = us + r * ds;
  uint32_t code = 0;
  for (int b = 0; b < bits; ++b) {
    const float* a = as + (tl * bits + b) * ds;
    float s0 = 0.f, s1 = 0.f;
    int e = 0;
    for (; e + 1 < d; e += 2) {
      s0 = fmaf(a[e], x[e], s0);
      s1 = fmaf(a[e + 1], x[e + 1], s1);
    }
    if (e < d) s0 = fmaf(a[e], x[e], s0);
    code |= ((s0 + s1) >= 0.f ? 1u : 0u) << b;
  }
  codes[(u0 + r) * K + t0 + tl] = (uint16_t)code;
}

// The same codes without staging, for dimensions too large for the tile: one thread per
// (user, table).
__global__ void user_codes_simple_kernel(const float* __restrict__ Ut, int d, int dp, int64_t m,
                                         const float* __restrict__ A, int d1p, int K, int bits,
                                         uint16_t* __restrict__ codes) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= m * K) return;
  const int64_t u = g / K;
  const int t = (int)(g % K);
  const float* x = Ut + u * dp;
  uint32_t code = 0;
  for (int b = 0; b < bits; ++b) {
    const float* a = A + (int64_t)(t * bits + b) * d1p;
    float s = 0.f;
    for (int e = 0; e < d; ++e) s = fmaf(a[e], x[e], s);
    code |= (s >= 0.f ? 1u : 0u) << b;
  }
  codes[u * K + t] = (uint16_t)code;
}

// ---------------------------------------------------------------- Alg. 2
constexpr int kSaWarps = 4;
constexpr int kQueue = 512;   // candidate queue per warp

__device__ __forceinline__ void insert_with_id(float& a, float& b, int& ia, int& ib, float v, int id, int lane) {
  const int pos = __popc(__ballot_sync(0xffffffffu, a > v)) + __popc(__ballot_sync(0xffffffffu, b > v));
  const float prev_b = __shfl_up_sync(0xffffffffu, b, 1);
  const int prev_ib = __shfl_up_sync(0xffffffffu, ib, 1);
  const int s0 = 2 * lane, s1 = 2 * lane + 1;
  const float na = (s0 < pos) ? a : (s0 == pos ? v : prev_b);
  const int nia = (s0 < pos) ? ia : (s0 == pos ? id : prev_ib);
  const float nb = (s1 < pos) ? b : (s1 == pos ? v : a);
  const int nib = (s1 < pos) ? ib : (s1 == pos ? id : ia);
  a = na;
  b = nb;
  ia = nia;
  ib = nib;
}

__device__ __forceinline__ float slot_value(float a, float b, int slot) {
  const float va = __shfl_sync(0xffffffffu, a, slot >> 1);
  const float vb = __shfl_sync(0xffffffffu, b, slot >> 1);
  return (slot & 1) ? vb : va;
}

struct SaParams {
  const Survivor* rows;
  const unsigned long long* nrows_dev;
  int64_t cap;
  const float* Ut;
  const float* unorm;
  const int32_t* uid;
  const float* Eu;
  const float* Lt;
  int64_t mz;
  int pp;
  const float* Ps;
  int64_t n;
  int dp;
  const float* qn;
  const int32_t* kk;
  float gamma;
  int parts;
  const int32_t* start;
  const float* M;
  const float* R;
  const uint16_t* ucode;
  const int32_t* boff;
  const int32_t* rbin;
  int nbin, rshift;
  const uint16_t* bcode;
  const int32_t* bitem;
  const uint32_t* probes;
  int nprobes;
  int K;
  uint32_t* bitmap;
  int64_t words;
  unsigned long long* items_stat;
};

__device__ __forceinline__ int lower_bound_u16(const uint16_t* a, int lo, int hi, uint32_t key) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kSaWarps * 32) saalsh_decide_kernel(SaParams prm) {
  __shared__ int32_t queue[kSaWarps][kQueue];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kSaWarps + warp;
  const int64_t nw = (int64_t)gridDim.x * kSaWarps;
  int32_t* q = queue[warp];
  unsigned long long scored = 0;
  const int64_t nrows = block_count(prm.nrows_dev, prm.cap);
  for (int64_t r = gw; r < nrows; r += nw) {
    const Survivor S = prm.rows[r];
    const int k = prm.kk[S.j];
    const float* u = prm.Ut + (int64_t)S.upos * prm.dp;
    const float nu = prm.unorm[S.upos];
    const float E = prm.Eu[S.upos];
    const float eq = __fmul_ru(__fmul_ru(prm.gamma, nu), prm.qn[S.j]) + 1e-30f;
    const float hi = __fadd_ru(S.sq, eq);
    // C = P': its k largest FP32 scores (ids -1: P' never meets SA-ALSH's items)
    float a = -INFINITY, b = -INFINITY;
    int ia = -1, ib = -1;
    if (2 * lane < k) a = prm.Lt[(int64_t)(2 * lane) * prm.mz + S.upos];
    if (2 * lane + 1 < k) b = prm.Lt[(int64_t)(2 * lane + 1) * prm.mz + S.upos];
    float phi = slot_value(a, b, k - 1);
    bool yes = true;
    if (hi < __fsub_rd(phi, E)) {
      yes = false;
    } else {
      for (int j = 0; j < prm.parts; ++j) {
        const float mu = __fmul_ru(__fmul_ru(prm.M[j], nu), 1.f + 2.f * prm.gamma);
        if (__fsub_rd(phi, E) > mu) break;                         // "yes": nothing left can beat phi
        const int s0 = prm.start[j], s1 = prm.start[j + 1];
        const bool all = !(prm.R[j] > 0.f);                        // R_j = 0: every item collides
        // gather candidates table by table (lane t owns table t + 32 i) and score them
        const int ntasks = all ? 1 : prm.K * prm.nprobes;
        for (int base = 0; base < ntasks; base += 32) {
          const int task = base + lane;
          int lo = 0, len = 0;
          if (task < ntasks) {
            if (all) {
              lo = s0;
              len = s1 - s0;
            } else {
              const int t = task / prm.nprobes, pr = task % prm.nprobes;
              const uint32_t code = prm.ucode[(int64_t)S.upos * prm.K + t] ^ prm.probes[pr];
              const int seg = j * prm.K + t;
              const int b0 = prm.boff[seg];
              // the codes with the same top bits first (radix index), then a short search
              const int32_t* rb = prm.rbin + (int64_t)seg * (prm.nbin + 1);
              const int c8 = (int)(code >> prm.rshift);
              const int lo8 = b0 + rb[c8], hi8 = b0 + rb[c8 + 1];
              const int l = lower_bound_u16(prm.bcode, lo8, hi8, code);
              const int h = lower_bound_u16(prm.bcode, l, hi8, code + 1);
              lo = l;
              len = h - l;
            }
          }
          // prefix over lanes, then drain through the queue kQueue at a time
          int incl = len;
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
          }
          const int total = __shfl_sync(0xffffffffu, incl, 31);
          const int excl = incl - len;
          for (int q0 = 0; q0 < total; q0 += kQueue) {
            // my range's share of [q0, q0 + kQueue)
            const int from = max(excl, q0), to = min(excl + len, q0 + kQueue);
            for (int x = from; x < to; ++x) q[x - q0] = all ? (lo + (x - excl)) : prm.bitem[lo + (x - excl)];
            __syncwarp();
            const int qn_ = min(kQueue, total - q0);
            for (int c0 = 0; c0 < qn_; c0 += 32) {
              const int c = c0 + lane;
              float v = -INFINITY;
              int id = -1;
              if (c < qn_) {
                id = q[c];
                const float4* p4 = reinterpret_cast<const float4*>(prm.Ps + (int64_t)id * prm.dp);
                const float4* u4 = reinterpret_cast<const float4*>(u);
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 4
                for (int e = 0; e < prm.dp / 4; ++e) {
                  const float4 pa = p4[e], ua = u4[e];
                  s0 = fmaf(ua.x, pa.x, s0);
                  s1 = fmaf(ua.y, pa.y, s1);
                  s2 = fmaf(ua.z, pa.z, s2);
                  s3 = fmaf(ua.w, pa.w, s3);
                }
                v = (s0 + s1) + (s2 + s3);
              }
              scored += (c < qn_) ? 1 : 0;
              unsigned cand = __ballot_sync(0xffffffffu, v > phi);
              while (cand) {
                const int src = __ffs(cand) - 1;
                cand &= cand - 1;
                const float vv = __shfl_sync(0xffffffffu, v, src);
                const int iid = __shfl_sync(0xffffffffu, id, src);
                if (!(vv > phi)) continue;
                const bool dup = __any_sync(0xffffffffu, ia == iid || ib == iid);
                if (dup) continue;
                insert_with_id(a, b, ia, ib, vv, iid, lane);
                phi = slot_value(a, b, k - 1);
              }
            }
            __syncwarp();
          }
        }
        if (hi < __fsub_rd(phi, E)) {   // <u,q> certainly below the k-th largest found
          yes = false;
          break;
        }
      }
    }
    if (yes && lane == 0) {
      const int32_t id = prm.uid[S.upos];
      set_answer(prm.bitmap, prm.words, S.j, id);
    }
  }
  for (int o = 16; o > 0; o >>= 1) scored += __shfl_xor_sync(0xffffffffu, scored, o);
  if (lane == 0 && scored) atomicAdd(prm.items_stat, scored);
}

// Standalone kMIPS (Alg. 2's candidate loop without a query item), one warp per query
// vector: C is seeded with P' (positions 0 .. pp-1, scored exactly), then the partitions in
// order until phi, the k-th largest score in C, exceeds mu_j = M_j ||u|| (rounded up); each
// visited partition adds the items whose code is within the probe radius of the query's in
// some table.  The k-slot list is spread over the lanes (slots 2l, 2l + 1), positions as ids.
struct KmParams {
  const float* Q;            // nq x dp, padded
  const float* qn;           // ||u||
  const uint16_t* qcode;     // nq x K
  int nq, k, pp;
  const float* Ps;
  const int32_t* pid;
  int dp;
  float gamma;
  int parts;
  const int32_t* start;
  const float* M;
  const float* R;
  const int32_t* boff;
  const int32_t* rbin;
  int nbin, rshift;
  const uint16_t* bcode;
  const int32_t* bitem;
  const uint32_t* probes;
  int nprobes;
  int K;
  int32_t* out_ids;          // nq x k
  float* out_scores;         // nq x k, or null
  unsigned long long* items_stat;
};

__device__ __forceinline__ float dot_rows(const float* __restrict__ p, const float* __restrict__ u, int dp) {
  const float4* p4 = reinterpret_cast<const float4*>(p);
  const float4* u4 = reinterpret_cast<const float4*>(u);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 4
  for (int e = 0; e < dp / 4; ++e) {
    const float4 pa = p4[e], ua = u4[e];
    s0 = fmaf(ua.x, pa.x, s0);
    s1 = fmaf(ua.y, pa.y, s1);
    s2 = fmaf(ua.z, pa.z, s2);
    s3 = fmaf(ua.w, pa.w, s3);
  }
  return (s0 + s1) + (s2 + s3);
}

__global__ void __launch_bounds__(kSaWarps * 32) kmips_kernel(KmParams prm) {
  __shared__ int32_t queue[kSaWarps][kQueue];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kSaWarps + warp;
  const int64_t nw = (int64_t)gridDim.x * kSaWarps;
  int32_t* q = queue[warp];
  const int k = prm.k;
  unsigned long long scored = 0;
  for (int64_t r = gw; r < prm.nq; r += nw) {
    const float* u = prm.Q + r * prm.dp;
    const float nu = prm.qn[r];
    float a = -INFINITY, b = -INFINITY;
    int ia = -1, ib = -1;
    float phi = -INFINITY;
    // any candidate that beats phi enters the list (duplicates of listed items skipped)
    auto offer = [&](float v, int id) {
      unsigned cand = __ballot_sync(0xffffffffu, v > phi);
      while (cand) {
        const int src = __ffs(cand) - 1;
        cand &= cand - 1;
        const float vv = __shfl_sync(0xffffffffu, v, src);
        const int iid = __shfl_sync(0xffffffffu, id, src);
        if (!(vv > phi)) continue;
        if (__any_sync(0xffffffffu, ia == iid || ib == iid)) continue;
        insert_with_id(a, b, ia, ib, vv, iid, lane);
        phi = slot_value(a, b, k - 1);
      }
    };
    // C = P'
    for (int c0 = 0; c0 < prm.pp; c0 += 32) {
      const int c = c0 + lane;
      float v = -INFINITY;
      if (c < prm.pp) v = dot_rows(prm.Ps + (int64_t)c * prm.dp, u, prm.dp);
      scored += (c < prm.pp) ? 1 : 0;
      offer(v, c < prm.pp ? c : -1);
    }
    for (int j = 0; j < prm.parts; ++j) {
      const float mu = __fmul_ru(__fmul_ru(prm.M[j], nu), 1.f + 2.f * prm.gamma);
      if (phi > mu) break;                                       // nothing left beats phi
      const int s0 = prm.start[j], s1 = prm.start[j + 1];
      const bool all = !(prm.R[j] > 0.f);                        // R_j = 0: every item collides
      const int ntasks = all ? 1 : prm.K * prm.nprobes;
      for (int base = 0; base < ntasks; base += 32) {
        const int task = base + lane;
        int lo = 0, len = 0;
        if (task < ntasks) {
          if (all) {
            lo = s0;
            len = s1 - s0;
          } else {
            const int t = task / prm.nprobes, pr = task % prm.nprobes;
            const uint32_t code = prm.qcode[r * prm.K + t] ^ prm.probes[pr];
            const int seg = j * prm.K + t;
            const int b0 = prm.boff[seg];
            const int32_t* rb = prm.rbin + (int64_t)seg * (prm.nbin + 1);
            const int c8 = (int)(code >> prm.rshift);
            const int lo8 = b0 + rb[c8], hi8 = b0 + rb[c8 + 1];
            const int l = lower_bound_u16(prm.bcode, lo8, hi8, code);
            const int h = lower_bound_u16(prm.bcode, l, hi8, code + 1);
            lo = l;
            len = h - l;
          }
        }
        int incl = len;
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int excl = incl - len;
        for (int q0 = 0; q0 < total; q0 += kQueue) {
          const int from = max(excl, q0), to = min(excl + len, q0 + kQueue);
          for (int x = from; x < to; ++x) q[x - q0] = all ? (lo + (x - excl)) : prm.bitem[lo + (x - excl)];
          __syncwarp();
          const int qn_ = min(kQueue, total - q0);
          for (int c0 = 0; c0 < qn_; c0 += 32) {
            const int c = c0 + lane;
            float v = -INFINITY;
            int id = -1;
            if (c < qn_) {
              id = q[c];
              v = dot_rows(prm.Ps + (int64_t)id * prm.dp, u, prm.dp);
            }
            scored += (c < qn_) ? 1 : 0;
            offer(v, id);
          }
          __syncwarp();
        }
      }
    }
    // the k slots, best first: slot 2l in a, 2l + 1 in b
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int slot = 2 * lane + h;
      if (slot < k) {
        const int pos = h ? ib : ia;
        prm.out_ids[r * k + slot] = pos >= 0 ? prm.pid[pos] : -1;
        if (prm.out_scores) prm.out_scores[r * k + slot] = pos >= 0 ? (h ? b : a) : -INFINITY;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) scored += __shfl_xor_sync(0xffffffffu, scored, o);
  if (lane == 0 && scored && prm.items_stat) atomicAdd(prm.items_stat, scored);
}

// Query rows padded to dp with their norms; a non-finite value raises *bad.
__global__ void kmips_prep_kernel(const float* __restrict__ Q, int nq, int d, int dp, float* __restrict__ Qp,
                                  float* __restrict__ qn, int* __restrict__ bad) {
  const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= nq) return;
  float s = 0.f;
  bool fin = true;
  for (int e = lane; e < dp; e += 32) {
    const float x = e < d ? Q[(int64_t)r * d + e] : 0.f;
    fin &= isfinite(x);
    Qp[(int64_t)r * dp + e] = x;
    s = fmaf(x, x, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (!__all_sync(0xffffffffu, fin) && lane == 0) atomicExch(bad, 1);
  if (lane == 0) qn[r] = sqrtf(s);
}

// SRP projection vectors drawn from the seed when the caller gives none: SplitMix64
// uniforms through the Box-Muller transform.
std::vector<float> draw_srp(uint64_t seed, int rows, int cols) {
  std::vector<float> out((size_t)rows * cols);
  uint64_t state = splitmix64(seed ^ 0x5A5A5A5A5A5A5A5Aull);
  auto uni = [&]() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = splitmix64(state - 0x9E3779B97F4A7C15ull);
    return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  for (size_t i = 0; i < out.size(); i += 2) {
    const double u1 = uni(), u2 = uni();
    const double r = std::sqrt(-2.0 * std::log(u1));
    out[i] = (float)(r * std::cos(2.0 * M_PI * u2));
    if (i + 1 < out.size()) out[i + 1] = (float)(r * std::sin(2.0 * M_PI * u2));
  }
  return out;
}

}  // namespace

sah_status build_saalsh(Index* ix, const float* srp_host, cudaStream_t st) {
  const int64_t n = ix->n, first = ix->pp;
  ix->sa_parts = 0;
  if (first >= n || ix->prm.n_tables < 1) return SAH_OK;
  const int d = ix->d, dp = ix->dp;
  const int K = ix->prm.n_tables, bits = ix->prm.code_bits;
  ix->sa_K = K;
  ix->sa_bits = bits;
  ix->sa_d1p = (d + 1 + 3) / 4 * 4;
  // partitions (Alg. 1) from the descending norms
  std::vector<float> pn(n);
  SAH_CUDA(cudaMemcpyAsync(pn.data(), ix->pnorm, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
  SAH_CUDA(cudaStreamSynchronize(st));
  std::vector<int32_t> start;
  std::vector<float> M;
  for (int64_t i = first; i < n;) {
    const float Mj = pn[i];
    start.push_back((int32_t)i);
    M.push_back(Mj);
    if (!(Mj > 0.f)) {
      i = n;
    } else {
      const float lim = ix->prm.b * Mj;
      while (i < n && pn[i] > lim) ++i;
    }
  }
  start.push_back((int32_t)n);
  const int t = (int)M.size();
  ix->sa_parts = t;
  ix->sa_start_h = start;
  std::vector<int32_t> part_of(n - first);
  for (int j = 0; j < t; ++j)
    for (int64_t i = start[j]; i < start[j + 1]; ++i) part_of[i - first] = j;
  // chunks for the deterministic centroid sums
  std::vector<int32_t> chunk_part, chunk_first, part_chunk0;
  for (int j = 0; j < t; ++j) {
    part_chunk0.push_back((int32_t)chunk_part.size());
    for (int64_t i = start[j]; i < start[j + 1]; i += kCentChunk) {
      chunk_part.push_back(j);
      chunk_first.push_back((int32_t)i);
    }
  }
  part_chunk0.push_back((int32_t)chunk_part.size());
  const int nchunk = (int)chunk_part.size();

  SAH_TRY(dev_alloc(ix, (void**)&ix->sa_start, sizeof(int32_t) * (t + 1)));
  SAH_TRY(dev_alloc(ix, (void**)&ix->sa_M, sizeof(float) * t));
  SAH_TRY(dev_alloc(ix, (void**)&ix->sa_R, sizeof(float) * t));
  SAH_TRY(dev_alloc(ix, (void**)&ix->sa_cent, sizeof(float) * (size_t)t * dp));
  SAH_CUDA(cudaMemcpyAsync(ix->sa_start, start.data(), sizeof(int32_t) * (t + 1), cudaMemcpyHostToDevice, st));
  SAH_CUDA(cudaMemcpyAsync(ix->sa_M, M.data(), sizeof(float) * t, cudaMemcpyHostToDevice, st));
  int32_t *part_of_d = nullptr, *cpart_d = nullptr, *cfirst_d = nullptr, *pchunk_d = nullptr;
  double* partial = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&part_of_d, sizeof(int32_t) * (n - first), st));
  SAH_CUDA(cudaMallocAsync((void**)&cpart_d, sizeof(int32_t) * nchunk, st));
  SAH_CUDA(cudaMallocAsync((void**)&cfirst_d, sizeof(int32_t) * nchunk, st));
  SAH_CUDA(cudaMallocAsync((void**)&pchunk_d, sizeof(int32_t) * (t + 1), st));
  SAH_CUDA(cudaMallocAsync((void**)&partial, sizeof(double) * (size_t)nchunk * dp, st));
  SAH_CUDA(cudaMemcpyAsync(part_of_d, part_of.data(), sizeof(int32_t) * (n - first), cudaMemcpyHostToDevice, st));
  SAH_CUDA(cudaMemcpyAsync(cpart_d, chunk_part.data(), sizeof(int32_t) * nchunk, cudaMemcpyHostToDevice, st));
  SAH_CUDA(cudaMemcpyAsync(cfirst_d, chunk_first.data(), sizeof(int32_t) * nchunk, cudaMemcpyHostToDevice, st));
  SAH_CUDA(cudaMemcpyAsync(pchunk_d, part_chunk0.data(), sizeof(int32_t) * (t + 1), cudaMemcpyHostToDevice, st));
  centroid_partial_kernel<<<nchunk, 128, 0, st>>>(ix->Ps, dp, ix->sa_start, cpart_d, cfirst_d, partial);
  centroid_final_kernel<<<t, 128, 0, st>>>(partial, pchunk_d, ix->sa_start, dp, ix->sa_cent);
  SAH_CUDA(cudaMemsetAsync(ix->sa_R, 0, sizeof(float) * t, st));
  radius_kernel<<<grid_for(n - first, 256), 256, 0, st>>>(ix->Ps, dp, first, n, part_of_d, ix->sa_cent,
                                                          reinterpret_cast<unsigned int*>(ix->sa_R));
  SAH_CUDA(cudaGetLastError());
  if (ix->prm.transform == SAH_QNF) {
    // Eq. 3: no shift, every partition padded to its largest norm (c_j = 0, R_j = M_j)
    SAH_CUDA(cudaMemsetAsync(ix->sa_cent, 0, sizeof(float) * (size_t)t * dp, st));
    SAH_CUDA(cudaMemcpyAsync(ix->sa_R, M.data(), sizeof(float) * t, cudaMemcpyHostToDevice, st));
  }

  // SRP matrix, rows padded to d1p
  const int rows = K * bits;
  std::vector<float> A_h = srp_host ? std::vector<float>(srp_host, srp_host + (size_t)rows * (d + 1))
                                    : draw_srp(ix->prm.seed, rows, d + 1);
  std::vector<float> A_pad((size_t)rows * ix->sa_d1p, 0.f);
  for (int r = 0; r < rows; ++r)
    for (int e = 0; e <= d; ++e) A_pad[(size_t)r * ix->sa_d1p + e] = A_h[(size_t)r * (d + 1) + e];
  SAH_TRY(dev_alloc(ix, (void**)&ix->sa_A, sizeof(float) * A_pad.size()));
  SAH_CUDA(cudaMemcpyAsync(ix->sa_A, A_pad.data(), sizeof(float) * A_pad.size(), cudaMemcpyHostToDevice, st));

  // item codes, then buckets sorted by code inside every (partition, table)
  const int64_t ni = n - first;
  uint16_t* icodes = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&icodes, sizeof(uint16_t) * ni * K, st));
  if (ix->prm.precision == SAH_FP8) {
    // FP8 E4M3 projections on the tensor cores
    SAH_TRY(codes_f8(ix, ix->Ps, first, n, part_of_d, A_pad.data(), ix->sa_d1p, K, bits, icodes, st));
  } else if (ix->dk > 0 && d + 1 <= 128) {
    // BF16 precision: the projections on the tensor cores
    SAH_TRY(item_codes_tc(ix, first, part_of_d, A_pad.data(), ix->sa_d1p, K, bits, icodes, st));
  } else {
    item_codes_kernel<<<grid_for(ni * K, 256), 256, 0, st>>>(ix->Ps, d, dp, first, n, part_of_d, ix->sa_cent,
                                                             ix->sa_R, ix->sa_A, ix->sa_d1p, K, bits, icodes);
  }
  SAH_CUDA(cudaGetLastError());
  std::vector<uint16_t> ic((size_t)ni * K);
  SAH_CUDA(cudaMemcpyAsync(ic.data(), icodes, sizeof(uint16_t) * ic.size(), cudaMemcpyDeviceToHost, st));
  SAH_CUDA(cudaStreamSynchronize(st));
  std::vector<int32_t> boff((size_t)t * K + 1);
  std::vector<uint16_t> bcode((size_t)ni * K);
  std::vector<int32_t> bitem((size_t)ni * K);
  {
    // segment (partition j, table tb) starts at start[j] - first times K plus tb times |S_j|
    for (int j = 0; j < t; ++j)
      for (int tb = 0; tb < K; ++tb)
        boff[(size_t)j * K + tb] = (int32_t)((size_t)(start[j] - first) * K + (size_t)tb * (start[j + 1] - start[j]));
    boff[(size_t)t * K] = (int32_t)((size_t)ni * K);
    // every (partition, table) segment is sorted by code independently: spread them over threads
    const int nthreads = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int w = 0; w < nthreads; ++w) {
      pool.emplace_back([&, w]() {
        std::vector<int32_t> idx;
        for (int seg = w; seg < t * K; seg += nthreads) {
          const int j = seg / K, tb = seg % K;
          idx.resize(start[j + 1] - start[j]);
          std::iota(idx.begin(), idx.end(), start[j]);
          std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) {
            return ic[(size_t)(x - first) * K + tb] < ic[(size_t)(y - first) * K + tb];
          });
          size_t o = (size_t)boff[seg];
          for (int32_t x : idx) {
            bcode[o] = ic[(size_t)(x - first) * K + tb];
            bitem[o] = x;
            ++o;
          }
        }
      });
    }
    for (auto& th : pool) th.join();
  }
  // radix index of every segment on the codes' top bits (at most 8 of them)
  ix->sa_rshift = bits > 8 ? bits - 8 : 0;
  ix->sa_nbin = 1 << (bits - ix->sa_rshift);
  std::vector<int32_t> rbin((size_t)t * K * (ix->sa_nbin + 1));
  for (int seg = 0; seg < t * K; ++seg) {
    int32_t* rb = rbin.data() + (size_t)seg * (ix->sa_nbin + 1);
    const int32_t b0 = boff[seg], b1 = boff[seg + 1];
    int32_t o = b0;
    for (int c = 0; c <= ix->sa_nbin; ++c) {
      // first position of the segment whose code's top bits are >= c
      while (o < b1 && (int)(bcode[o] >> ix->sa_rshift) < c) ++o;
      rb[c] = o - b0;
    }
  }
  SAH_TRY(dev_alloc(ix, (void**)&ix->sa_rbin, sizeof(int32_t) * rbin.size()));
  SAH_CUDA(cudaMemcpyAsync(ix->sa_rbin, rbin.data(), sizeof(int32_t) * rbin.size(), cudaMemcpyHostToDevice, st));
  SAH_TRY(dev_alloc(ix, (void**)&ix->sa_boff, sizeof(int32_t) * boff.size()));
  SAH_TRY(dev_alloc(ix, (void**)&ix->sa_bcode, sizeof(uint16_t) * bcode.size()));
  SAH_TRY(dev_alloc(ix, (void**)&ix->sa_bitem, sizeof(int32_t) * bitem.size()));
  SAH_CUDA(cudaMemcpyAsync(ix->sa_boff, boff.data(), sizeof(int32_t) * boff.size(), cudaMemcpyHostToDevice, st));
  SAH_CUDA(cudaMemcpyAsync(ix->sa_bcode, bcode.data(), sizeof(uint16_t) * bcode.size(), cudaMemcpyHostToDevice, st));
  SAH_CUDA(cudaMemcpyAsync(ix->sa_bitem, bitem.data(), sizeof(int32_t) * bitem.size(), cudaMemcpyHostToDevice, st));

  // user codes (leaf order)
  if (ix->m_nz > 0) {
    SAH_TRY(dev_alloc(ix, (void**)&ix->sa_ucode, sizeof(uint16_t) * (size_t)ix->m_nz * K));
    const size_t smem = sizeof(float) * (size_t)(kCodeUsers + kCodeTables * bits) * (d | 1);
    if (ix->prm.precision == SAH_FP8) {
      SAH_TRY(codes_f8(ix, ix->Ut, 0, ix->m_nz, nullptr, A_pad.data(), ix->sa_d1p, K, bits, ix->sa_ucode, st));
    } else if (ix->dk == 64 || ix->dk == 128) {
      // BF16 precision: the projections on the tensor cores
      SAH_TRY(user_codes_tc(ix, A_pad.data(), ix->sa_d1p, K, bits, ix->sa_ucode, st));
    } else if (smem <= 160 * 1024) {
      if (smem > 48 * 1024)
        SAH_TRY(raise_smem_limit((const void*)user_codes_kernel, (size_t)((int)smem)));
      dim3 g(grid_for(ix->m_nz, kCodeUsers), (K + kCodeTables - 1) / kCodeTables);
      user_codes_kernel<<<g, kCodeUsers * kCodeTables, smem, st>>>(ix->Ut, d, dp, ix->m_nz, ix->sa_A, ix->sa_d1p, K,
                                                                  bits, ix->sa_ucode);
    } else {
      user_codes_simple_kernel<<<grid_for(ix->m_nz * K, 256), 256, 0, st>>>(ix->Ut, d, dp, ix->m_nz, ix->sa_A,
                                                                            ix->sa_d1p, K, bits, ix->sa_ucode);
    }
    SAH_CUDA(cudaGetLastError());
  }
  // Hamming probes: every mask over code_bits bits with popcount <= probe_radius
  std::vector<uint32_t> probes;
  for (uint32_t msk = 0; msk < (1u << bits); ++msk)
    if (__builtin_popcount(msk) <= ix->prm.probe_radius) probes.push_back(msk);
  ix->sa_nprobes = (int32_t)probes.size();
  SAH_TRY(dev_alloc(ix, (void**)&ix->sa_probes, sizeof(uint32_t) * probes.size()));
  SAH_CUDA(cudaMemcpyAsync(ix->sa_probes, probes.data(), sizeof(uint32_t) * probes.size(), cudaMemcpyHostToDevice,
                           st));
  SAH_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(part_of_d, st);
  cudaFreeAsync(cpart_d, st);
  cudaFreeAsync(cfirst_d, st);
  cudaFreeAsync(pchunk_d, st);
  cudaFreeAsync(partial, st);
  cudaFreeAsync(icodes, st);
  SAH_CUDA(cudaStreamSynchronize(st));
  return SAH_OK;
}

sah_status run_saalsh(Index* ix, const Survivor* surv, const unsigned long long* count_dev, int64_t cap,
                      const float* Qd, const float* qn, const int32_t* kk, uint32_t* bitmap, int64_t words,
                      unsigned long long* stats, int stat_items, cudaStream_t st, int* launches) {
  (void)Qd;
  if (cap <= 0) return SAH_OK;
  const int64_t ns = cap;
  SaParams p;
  p.rows = surv;
  p.nrows_dev = count_dev;
  p.cap = cap;
  p.Ut = ix->Ut;
  p.unorm = ix->unorm;
  p.uid = ix->uid;
  p.Eu = ix->Eu;
  p.Lt = ix->Lt;
  p.mz = ix->m_nz;
  p.pp = ix->pp;
  p.Ps = ix->Ps;
  p.n = ix->n;
  p.dp = ix->dp;
  p.qn = qn;
  p.kk = kk;
  p.gamma = ix->gamma;
  p.parts = ix->sa_parts;
  p.start = ix->sa_start;
  p.M = ix->sa_M;
  p.R = ix->sa_R;
  p.ucode = ix->sa_ucode;
  p.boff = ix->sa_boff;
  p.rbin = ix->sa_rbin;
  p.nbin = ix->sa_nbin;
  p.rshift = ix->sa_rshift;
  p.bcode = ix->sa_bcode;
  p.bitem = ix->sa_bitem;
  p.probes = ix->sa_probes;
  p.nprobes = ix->sa_nprobes;
  p.K = ix->sa_K;
  p.bitmap = bitmap;
  p.words = words;
  p.items_stat = stats + stat_items;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
  const unsigned grid = (unsigned)std::min<int64_t>((ns + kSaWarps - 1) / kSaWarps, (int64_t)sms * 16);
  saalsh_decide_kernel<<<grid, kSaWarps * 32, 0, st>>>(p);
  SAH_CUDA(cudaGetLastError());
  if (launches) *launches += 1;
  return SAH_OK;
}

sah_status run_kmips(Index* ix, const float* Q_dev, int32_t nq, int32_t k, int32_t* out_ids, float* out_scores,
                     cudaStream_t st) {
  if (nq == 0) return SAH_OK;
  const int d = ix->d, dp = ix->dp;
  const int K = ix->sa_parts > 0 ? ix->sa_K : 0;
  // workspace: padded rows, norms, codes, the non-finite flag, the scored-items counter
  const size_t b_rows = sizeof(float) * (size_t)nq * dp, b_qn = sizeof(float) * (size_t)nq,
               b_code = sizeof(uint16_t) * (size_t)nq * std::max(K, 1);
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t total = up(b_rows) + up(b_qn) + up(b_code) + 256;
  char* ws = nullptr;
  if (cudaMallocAsync((void**)&ws, total, st) != cudaSuccess) {
    cudaGetLastError();
    set_error("sah_kmips: workspace allocation failed");
    return SAH_ERR_OOM;
  }
  float* Qp = (float*)ws;
  float* qn = (float*)(ws + up(b_rows));
  uint16_t* qcode = (uint16_t*)(ws + up(b_rows) + up(b_qn));
  int* bad = (int*)(ws + up(b_rows) + up(b_qn) + up(b_code));
  unsigned long long* scored = (unsigned long long*)(bad + 2);
  sah_status s = SAH_OK;
  int bad_h = 0;
  unsigned long long scored_h = 0;
  do {
    if (cudaMemsetAsync(bad, 0, 256, st) != cudaSuccess) { s = SAH_ERR_CUDA; break; }
    kmips_prep_kernel<<<grid_for(nq, 8), 256, 0, st>>>(Q_dev, nq, d, dp, Qp, qn, bad);
    if (K > 0)
      user_codes_simple_kernel<<<grid_for((int64_t)nq * K, 256), 256, 0, st>>>(Qp, d, dp, nq, ix->sa_A, ix->sa_d1p,
                                                                               K, ix->sa_bits, qcode);
    KmParams p;
    p.Q = Qp;
    p.qn = qn;
    p.qcode = qcode;
    p.nq = nq;
    p.k = k;
    p.pp = ix->pp;
    p.Ps = ix->Ps;
    p.pid = ix->pid;
    p.dp = dp;
    p.gamma = ix->gamma;
    p.parts = ix->sa_parts;
    p.start = ix->sa_start;
    p.M = ix->sa_M;
    p.R = ix->sa_R;
    p.boff = ix->sa_boff;
    p.rbin = ix->sa_rbin;
    p.nbin = ix->sa_nbin;
    p.rshift = ix->sa_rshift;
    p.bcode = ix->sa_bcode;
    p.bitem = ix->sa_bitem;
    p.probes = ix->sa_probes;
    p.nprobes = ix->sa_nprobes;
    p.K = K;
    p.out_ids = out_ids;
    p.out_scores = out_scores;
    p.items_stat = scored;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
    const unsigned grid = (unsigned)std::min<int64_t>((nq + kSaWarps - 1) / kSaWarps, (int64_t)sms * 16);
    kmips_kernel<<<grid, kSaWarps * 32, 0, st>>>(p);
    if (cudaGetLastError() != cudaSuccess) { s = SAH_ERR_CUDA; break; }
    if (cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&scored_h, scored, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      s = SAH_ERR_CUDA;
      break;
    }
  } while (false);
  cudaFreeAsync(ws, st);
  if (s == SAH_ERR_CUDA) {
    set_error(std::string("sah_kmips: ") + cudaGetErrorString(cudaGetLastError()));
    return s;
  }
  if (bad_h) {
    set_error("sah_kmips: a query vector holds a non-finite value");
    return SAH_ERR_ARG;
  }
  // the call's counters: queries and the items scored (P' and the candidates)
  sah_stats stt{};
  stt.queries = nq;
  stt.items_scanned = (int64_t)scored_h;
  ix->main_ctx.stats = stt;
  return SAH_OK;
}

}  // namespace sah
