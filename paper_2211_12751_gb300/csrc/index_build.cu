// SAH indexing on the GPU (Alg. 4): item norms and descending-norm order, lower-bound
// arrays over the first |P'| items, the Cone-Tree over the users (Alg. 3) built level by
// level, and the per-leaf cone data used by the node- and vector-level upper bounds
// (Lemma 2, Lemma 3).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "sah_internal.cuh"

namespace sah {

namespace {

constexpr int kTile = 1024;  // Cone-Tree elements per CTA

// ---------------------------------------------------------------- A0: norms
// One warp per row: ||x|| in FP32 and a finiteness check.
__global__ void row_norms_kernel(const float* __restrict__ X, int64_t rows, int d,
                                 float* __restrict__ norms, int* __restrict__ bad) {
  int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const float* x = X + row * d;
  float s = 0.f;
  bool fin = true;
  for (int i = lane; i < d; i += 32) {
    float v = x[i];
    fin &= isfinite(v);
    s = fmaf(v, v, s);
  }
  s = warp_sum(s);
  bool allfin = __all_sync(0xffffffffu, fin);
  if (lane == 0) {
    norms[row] = sqrtf(s);
    if (!allfin) atomicExch(bad, 1);
  }
}

// dst[i] = src[idx[i]] with rows padded from d to dp floats (padding zero); optionally
// divided by the row norm (unit directions for the Cone-Tree).
__global__ void gather_rows_kernel(const float* __restrict__ src, int d, const int32_t* __restrict__ idx,
                                   int64_t rows, int dp, float* __restrict__ dst,
                                   const float* __restrict__ norms, int normalise) {
  int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= rows) return;
  int64_t s = idx[row];
  float inv = 1.f;
  if (normalise) inv = 1.f / norms[s];
  for (int i = lane; i < dp; i += 32) {
    float v = (i < d) ? src[s * d + i] : 0.f;
    dst[row * dp + i] = normalise ? v * inv : v;
  }
}

__global__ void gather_f32_kernel(const float* __restrict__ src, const int32_t* __restrict__ idx,
                                  int64_t n, float* __restrict__ dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

__global__ void gather_i32_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ idx,
                                  int64_t n, int32_t* __restrict__ dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

// Padded-row gather: dst[i] = src[idx[i]] (both dp wide).
__global__ void gather_padded_kernel(const float* __restrict__ src, const int32_t* __restrict__ idx,
                                     int64_t rows, int dp, float* __restrict__ dst) {
  int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const float4* s = reinterpret_cast<const float4*>(src + (int64_t)idx[row] * dp);
  float4* t = reinterpret_cast<float4*>(dst + row * dp);
  for (int i = lane; i < dp / 4; i += 32) t[i] = s[i];
}

__device__ inline float dot_padded(const float* __restrict__ a, const float* __restrict__ b, int dp) {
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  float s = 0.f;
  for (int i = 0; i < dp / 4; ++i) {
    float4 x = a4[i], y = b4[i];
    s = fmaf(x.x, y.x, s);
    s = fmaf(x.y, y.y, s);
    s = fmaf(x.z, y.z, s);
    s = fmaf(x.w, y.w, s);
  }
  return s;
}

// ---------------------------------------------------------------- A2: Cone-Tree levels
struct CtTile {
  int32_t seg;     // active segment this tile belongs to
  int32_t start;   // first position (in perm) of the tile
  int32_t len;     // elements in the tile (<= kTile)
  int32_t first;   // position of the tile's first element inside its segment
};

// argmin over each segment of <uhat_x, uhat_v[seg]>; ties go to the lowest position in
// the segment.  Result packed as (order key << 32 | position) with a 64-bit atomicMin.
__global__ void ct_argmin_kernel(const float* __restrict__ Uh, int dp, const int32_t* __restrict__ perm,
                                 const CtTile* __restrict__ tiles, const int32_t* __restrict__ pivot,
                                 unsigned long long* __restrict__ best) {
  CtTile t = tiles[blockIdx.x];
  const float* v = Uh + (int64_t)pivot[t.seg] * dp;
  unsigned long long key = ~0ull;
  for (int i = threadIdx.x; i < t.len; i += blockDim.x) {
    int32_t x = perm[t.start + i];
    float s = dot_padded(Uh + (int64_t)x * dp, v, dp);
    unsigned long long k = ((unsigned long long)float_order_key(s) << 32) | (uint32_t)(t.first + i);
    key = k < key ? k : key;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
    key = other < key ? other : key;
  }
  if ((threadIdx.x & 31) == 0) atomicMin(&best[t.seg], key);
}

// Split flag (left iff <uhat, u_l> >= <uhat, u_r>, Alg. 3) and each element's rank among
// the left elements of its tile; one count of left elements per tile.
__global__ void ct_split_kernel(const float* __restrict__ Uh, int dp, const int32_t* __restrict__ perm,
                                const CtTile* __restrict__ tiles, const int32_t* __restrict__ ul,
                                const int32_t* __restrict__ ur, int32_t* __restrict__ lrank,
                                int32_t* __restrict__ tile_left) {
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t carry;
  CtTile t = tiles[blockIdx.x];
  const float* a = Uh + (int64_t)ul[t.seg] * dp;
  const float* b = Uh + (int64_t)ur[t.seg] * dp;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < t.len; base += blockDim.x) {
    int i = base + threadIdx.x;
    bool left = false;
    if (i < t.len) {
      const float* x = Uh + (int64_t)perm[t.start + i] * dp;
      left = dot_padded(x, a, dp) >= dot_padded(x, b, dp);
    }
    unsigned m = __ballot_sync(0xffffffffu, left);
    int before = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[warp] = __popc(m);
    __syncthreads();
    int off = carry;
    for (int w = 0; w < warp; ++w) off += warp_tot[w];
    if (i < t.len) lrank[t.start + i] = left ? (off + before) : -1 - (off + before);
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < nw; ++w) tot += warp_tot[w];
      carry += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_left[blockIdx.x] = carry;
}

// Stable partition of every active segment: left elements first, in list order.
// lrank >= 0: rank among the tile's left elements; lrank < 0: -1 - (lefts before it).
__global__ void ct_scatter_kernel(const int32_t* __restrict__ perm, const CtTile* __restrict__ tiles,
                                  const int32_t* __restrict__ lrank, const int32_t* __restrict__ tile_loff,
                                  const int32_t* __restrict__ tile_roff, const int32_t* __restrict__ seg_start,
                                  const int32_t* __restrict__ seg_nleft, const int32_t* __restrict__ seg_halves,
                                  int32_t* __restrict__ perm_out) {
  CtTile t = tiles[blockIdx.x];
  int32_t s0 = seg_start[t.seg];
  for (int i = threadIdx.x; i < t.len; i += blockDim.x) {
    int32_t pos = t.start + i;
    int32_t dst;
    if (seg_halves[t.seg]) {
      dst = pos;
    } else {
      int32_t r = lrank[pos];
      if (r >= 0) {
        dst = s0 + tile_loff[blockIdx.x] + r;
      } else {
        int32_t lefts_before = -1 - r;
        dst = s0 + seg_nleft[t.seg] + tile_roff[blockIdx.x] + (i - lefts_before);
      }
    }
    perm_out[dst] = perm[pos];
  }
}

// ---------------------------------------------------------------- leaf (block) cones
// One CTA per leaf: centre c = mean of the unit users (Alg. 3), its direction, every
// member's cos/sin theta_u to it (sin from the orthogonal component, which stays accurate
// near theta = 0), and omega = max theta_u.  A zero centre marks the block with
// bcos = -2 (no cone bound for it or its users).
// norm_blocks (Simpfer's blocking): no cone at all; the block is given omega = pi around a
// zero centre and every user theta_u = pi/2, so that Lemma 2 and Lemma 3 both reduce to
// Cauchy-Schwarz, ||q|| for a unit user (cos phi = <0, q> = 0 and cos(phi - theta_u) = 1).
__global__ void leaf_stats_kernel(const float* __restrict__ Uh, int dp, const int32_t* __restrict__ bstart,
                                  float* __restrict__ bcent, float* __restrict__ bcos, float* __restrict__ bsin,
                                  float* __restrict__ ucos, float* __restrict__ usin, int norm_blocks) {
  extern __shared__ float cs[];   // dp floats
  __shared__ float red[32];
  __shared__ unsigned long long best;
  int B = blockIdx.x;
  int s = bstart[B], e = bstart[B + 1], cnt = e - s;
  if (norm_blocks) {
    for (int i = threadIdx.x; i < dp; i += blockDim.x) bcent[(int64_t)B * dp + i] = 0.f;
    for (int r = s + threadIdx.x; r < e; r += blockDim.x) {
      ucos[r] = 0.f;
      usin[r] = 1.f;
    }
    if (threadIdx.x == 0) {
      bcos[B] = -1.f;
      bsin[B] = 0.f;
    }
    return;
  }
  for (int i = threadIdx.x; i < dp; i += blockDim.x) {
    float acc = 0.f;
    for (int r = s; r < e; ++r) acc += Uh[(int64_t)r * dp + i];
    cs[i] = acc / (float)cnt;
  }
  if (threadIdx.x == 0) best = ~0ull;
  __syncthreads();
  float part = 0.f;
  for (int i = threadIdx.x; i < dp; i += blockDim.x) part = fmaf(cs[i], cs[i], part);
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  float nc2 = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) nc2 += red[w];
  float nc = sqrtf(nc2);
  bool degenerate = !(nc > 0.f) || !isfinite(nc);
  __syncthreads();
  for (int i = threadIdx.x; i < dp; i += blockDim.x) {
    float v = degenerate ? 0.f : cs[i] / nc;
    cs[i] = v;
    bcent[(int64_t)B * dp + i] = v;
  }
  __syncthreads();
  for (int r = s + threadIdx.x; r < e; r += blockDim.x) {
    const float* x = Uh + (int64_t)r * dp;
    float c = 0.f, sn = 0.f;
    if (!degenerate) {
      c = fminf(1.f, fmaxf(-1.f, dot_padded(x, cs, dp)));
      float p2 = 0.f;
      for (int i = 0; i < dp; ++i) {
        float o = fmaf(-c, cs[i], x[i]);
        p2 = fmaf(o, o, p2);
      }
      sn = fminf(1.f, sqrtf(p2));
      unsigned long long key = ((unsigned long long)float_order_key(c) << 32) | (uint32_t)(r - s);
      atomicMin(&best, key);
    }
    ucos[r] = c;
    usin[r] = sn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (degenerate) {
      bcos[B] = -2.f;
      bsin[B] = 0.f;
    } else {
      int r = s + (int)(best & 0xffffffffu);
      bcos[B] = ucos[r];
      bsin[B] = usin[r];
    }
  }
}

// ---------------------------------------------------------------- A1: lower bounds
// Top-k_max of <u,p> over the first pp items (descending norm order) for every user.
// A CTA holds 32 users (4 per warp); item tiles are staged in shared memory; each warp
// keeps one descending list of 64 slots per user spread over its lanes (slots 2l, 2l+1).
constexpr int kUsersPerWarp = 4;
constexpr int kTopkWarps = 8;

__device__ inline void list_insert(float& a, float& b, int& ia, int& ib, float v, int id, int lane) {
  int pos = __popc(__ballot_sync(0xffffffffu, a > v)) + __popc(__ballot_sync(0xffffffffu, b > v));
  float prev_b = __shfl_up_sync(0xffffffffu, b, 1);
  int prev_ib = __shfl_up_sync(0xffffffffu, ib, 1);
  int s0 = 2 * lane, s1 = 2 * lane + 1;
  float na = (s0 < pos) ? a : (s0 == pos ? v : prev_b);
  int nia = (s0 < pos) ? ia : (s0 == pos ? id : prev_ib);
  float nb = (s1 < pos) ? b : (s1 == pos ? v : a);
  int nib = (s1 < pos) ? ib : (s1 == pos ? id : ia);
  a = na;
  b = nb;
  ia = nia;
  ib = nib;
}

__device__ inline float list_get(float a, float b, int slot) {
  float va = __shfl_sync(0xffffffffu, a, slot >> 1);
  float vb = __shfl_sync(0xffffffffu, b, slot >> 1);
  return (slot & 1) ? vb : va;
}

__global__ void __launch_bounds__(kTopkWarps * 32)
topk_lower_bounds_kernel(const float* __restrict__ Ut, const float* __restrict__ Ps, int dp,
                         int64_t m, int pp, int kmax, int tile_items, int stride4,
                         float* __restrict__ Lt, int32_t* __restrict__ ids_out, float* __restrict__ vlast_out) {
  extern __shared__ float4 sm4[];
  float4* tileP = sm4;                                        // tile_items x stride4
  float4* us = sm4 + (size_t)tile_items * stride4;            // 32 users x (dp/4)
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int dp4 = dp / 4;
  int64_t u0 = (int64_t)blockIdx.x * (kTopkWarps * kUsersPerWarp);
  for (int i = threadIdx.x; i < kTopkWarps * kUsersPerWarp * dp4; i += blockDim.x) {
    int r = i / dp4, c = i % dp4;
    int64_t u = u0 + r;
    us[i] = (u < m) ? reinterpret_cast<const float4*>(Ut + u * dp)[c] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float la[kUsersPerWarp], lb[kUsersPerWarp], thr[kUsersPerWarp];
  int ia[kUsersPerWarp], ib[kUsersPerWarp];
  // with ids requested, all 64 slots are kept and the threshold is the 64th value
  const int keep = ids_out ? 64 : kmax;
#pragma unroll
  for (int w = 0; w < kUsersPerWarp; ++w) {
    la[w] = -INFINITY;
    lb[w] = -INFINITY;
    thr[w] = -INFINITY;
    ia[w] = -1;
    ib[w] = -1;
  }
  const float4* myu = us + (size_t)(warp * kUsersPerWarp) * dp4;
  for (int t0 = 0; t0 < pp; t0 += tile_items) {
    int tn = min(tile_items, pp - t0);
    __syncthreads();
    for (int i = threadIdx.x; i < tn * dp4; i += blockDim.x) {
      int r = i / dp4, c = i % dp4;
      tileP[r * stride4 + c] = reinterpret_cast<const float4*>(Ps + (int64_t)(t0 + r) * dp)[c];
    }
    __syncthreads();
    for (int base = 0; base < tn; base += 32) {
      int it = base + lane;
      float s[kUsersPerWarp];
#pragma unroll
      for (int w = 0; w < kUsersPerWarp; ++w) s[w] = 0.f;
      if (it < tn) {
        const float4* pr = tileP + it * stride4;
        for (int c = 0; c < dp4; ++c) {
          float4 p = pr[c];
#pragma unroll
          for (int w = 0; w < kUsersPerWarp; ++w) {
            float4 u = myu[w * dp4 + c];
            s[w] = fmaf(p.x, u.x, s[w]);
            s[w] = fmaf(p.y, u.y, s[w]);
            s[w] = fmaf(p.z, u.z, s[w]);
            s[w] = fmaf(p.w, u.w, s[w]);
          }
        }
      }
#pragma unroll
      for (int w = 0; w < kUsersPerWarp; ++w) {
        bool cand = (it < tn) && (s[w] > thr[w]);
        unsigned mask = __ballot_sync(0xffffffffu, cand);
        while (mask) {
          int src = __ffs(mask) - 1;
          float v = __shfl_sync(0xffffffffu, s[w], src);
          list_insert(la[w], lb[w], ia[w], ib[w], v, t0 + base + src, lane);
          thr[w] = list_get(la[w], lb[w], keep - 1);
          mask &= ~(1u << src);
          // drop candidates the new threshold already excludes
          mask &= __ballot_sync(0xffffffffu, cand && s[w] > thr[w]);
        }
      }
    }
  }
#pragma unroll
  for (int w = 0; w < kUsersPerWarp; ++w) {
    int64_t u = u0 + warp * kUsersPerWarp + w;
    const float last = list_get(la[w], lb[w], 63);
    if (u < m) {
      int s0 = 2 * lane, s1 = 2 * lane + 1;
      if (s0 < kmax) Lt[(int64_t)s0 * m + u] = la[w];
      if (s1 < kmax) Lt[(int64_t)s1 * m + u] = lb[w];
      if (ids_out) {
        ids_out[(int64_t)s0 * m + u] = ia[w];
        ids_out[(int64_t)s1 * m + u] = ib[w];
        if (lane == 0) vlast_out[u] = last;
      }
    }
  }
}

// Exact thresholds (all items in P'): the 64 listed items of every user re-scored in
// double precision in the order i = 0..d-1 and ranked; T64[k-1][u] is the k-th largest
// double-precision score whenever the list provably holds every item that can rank k or
// better: the 64th FP32 score plus twice the FP32 bound (and a margin for the double
// rounding) stays below the k-th FP32 score.  Otherwise T64 is NaN for that k.
__global__ void tau64_kernel(const float* __restrict__ Ut, const float* __restrict__ Ps, int d, int dp, int64_t m,
                             int kmax, const int32_t* __restrict__ ids, const float* __restrict__ vlast,
                             const float* __restrict__ Lt, const float* __restrict__ Eu,
                             const float* __restrict__ unorm, float mmax, double* __restrict__ T64) {
  __shared__ double sv[8][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t u = (int64_t)blockIdx.x * 8 + warp;
  if (u >= m) return;
  const float* ur = Ut + u * dp;
  double x[2];
  for (int h = 0; h < 2; ++h) {
    const int id = ids[(int64_t)(2 * lane + h) * m + u];
    x[h] = id >= 0 ? dot64_seq(ur, Ps + (int64_t)id * dp, d) : -INFINITY;
    sv[warp][2 * lane + h] = x[h];
  }
  __syncwarp();
  // rank of each value (ties broken by slot), then the sorted order
  double sorted_me[2];
  int rank[2];
  for (int h = 0; h < 2; ++h) {
    const int me = 2 * lane + h;
    int r = 0;
    for (int o = 0; o < 64; ++o) {
      const double y = sv[warp][o];
      r += (y > x[h]) || (y == x[h] && o < me);
    }
    rank[h] = r;
    sorted_me[h] = x[h];
  }
  __syncwarp();
  for (int h = 0; h < 2; ++h) sv[warp][rank[h]] = sorted_me[h];
  __syncwarp();
  const float E = Eu[u];
  const float last = vlast[u];
  const double margin = 1e-9 * (double)unorm[u] * (double)mmax;
  for (int k0 = lane; k0 < kmax; k0 += 32) {
    const float tk = Lt[(int64_t)k0 * m + u];
    const bool covered = (last == -INFINITY) || ((double)last + 2.0 * (double)E + margin < (double)tk);
    T64[(int64_t)k0 * m + u] = covered ? sv[warp][k0] : (double)NAN;
  }
}

// E_u bounds the FP32 error of any item score of u: gamma * ||u|| * max ||p||, rounded up.
__global__ void user_error_kernel(const float* __restrict__ unorm, int64_t m, float gamma, float mmax,
                                  float* __restrict__ Eu) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) Eu[i] = __fmul_ru(__fmul_ru(gamma, unorm[i]), mmax) + 1e-30f;
}

// L^k(B) = min over the block's users of (L_u^k - E_u) / ||u||, rounded down (Alg. 4,
// for unit users).
__global__ void block_lower_bounds_kernel(const float* __restrict__ Lt, const float* __restrict__ Eu,
                                          const float* __restrict__ unorm, const int32_t* __restrict__ bstart,
                                          int nb, int64_t m, int kmax, float* __restrict__ LB) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nb * kmax) return;
  int k = (int)(t / nb), B = (int)(t % nb);
  float mn = INFINITY;
  for (int r = bstart[B]; r < bstart[B + 1]; ++r) {
    float L = Lt[(int64_t)k * m + r];
    float v = (L == -INFINITY) ? -INFINITY : __fdiv_rd(__fsub_rd(L, Eu[r]), unorm[r]);
    mn = fminf(mn, v);
  }
  LB[(int64_t)k * nb + B] = mn;
}

// The same minimum, min over u of (L_u^k - E_u) / ||u|| rounded down, over each tile of 128
// consecutive user positions (the tensor-core user pass's tiles).
__global__ void tile_lower_bounds_kernel(const float* __restrict__ Lt, const float* __restrict__ Eu,
                                         const float* __restrict__ unorm, int64_t m, int kmax, int ntiles,
                                         float* __restrict__ TLB) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ntiles * kmax) return;
  const int k = (int)(t / ntiles), tile = (int)(t % ntiles);
  float mn = INFINITY;
  const int64_t r1 = m < (int64_t)(tile + 1) * 128 ? m : (int64_t)(tile + 1) * 128;
  for (int64_t r = (int64_t)tile * 128; r < r1; ++r) {
    const float L = Lt[(int64_t)k * m + r];
    const float v = (L == -INFINITY) ? -INFINITY : __fdiv_rd(__fsub_rd(L, Eu[r]), unorm[r]);
    mn = fminf(mn, v);
  }
  TLB[(int64_t)k * ntiles + tile] = mn;
}

// leaf (block) of every user position
__global__ void user_block_kernel(const int32_t* __restrict__ bstart, int nb, int32_t* __restrict__ ublock) {
  const int B = blockIdx.x;
  if (B >= nb) return;
  for (int r = bstart[B] + threadIdx.x; r < bstart[B + 1]; r += blockDim.x) ublock[r] = B;
}

__global__ void fill_i32_kernel(int32_t* p, int64_t n, int32_t v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

inline unsigned grid_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

struct Seg {
  int32_t start, len;
  uint64_t key;
};

}  // namespace

// Builds every device array of the index from U (m x d) and P (n x d) on the device.
sah_status build_index_device(Index* ix, const float* U_dev, const float* P_dev, cudaStream_t st) {
  const int64_t n = ix->n, m = ix->m;
  const int d = ix->d, dp = ix->dp;
  int* bad = nullptr;
  SAH_TRY(dev_alloc(ix, (void**)&bad, sizeof(int)));
  SAH_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  SAH_TRY(dev_alloc(ix, (void**)&ix->dev_timeout, sizeof(int)));
  SAH_CUDA(cudaMemsetAsync(ix->dev_timeout, 0, sizeof(int), st));

  // ---- A0: item norms, descending order (ties: lower id first), padded rows
  float* pn_raw = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&pn_raw, sizeof(float) * n, st));
  row_norms_kernel<<<grid_for(n, 8), 256, 0, st>>>(P_dev, n, d, pn_raw, bad);
  float* un_raw = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&un_raw, sizeof(float) * m, st));
  row_norms_kernel<<<grid_for(m, 8), 256, 0, st>>>(U_dev, m, d, un_raw, bad);
  SAH_CUDA(cudaGetLastError());
  std::vector<float> pn_h(n), un_h(m);
  int bad_h = 0;
  SAH_CUDA(cudaMemcpyAsync(pn_h.data(), pn_raw, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
  SAH_CUDA(cudaMemcpyAsync(un_h.data(), un_raw, sizeof(float) * m, cudaMemcpyDeviceToHost, st));
  SAH_CUDA(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  SAH_CUDA(cudaStreamSynchronize(st));
  if (bad_h) {
    cudaFreeAsync(pn_raw, st);
    cudaFreeAsync(un_raw, st);
    set_error("sah_build_index: U or P holds a non-finite value");
    return SAH_ERR_ARG;
  }
  std::vector<int32_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return pn_h[a] > pn_h[b]; });
  int32_t* order_d = nullptr;
  SAH_TRY(dev_alloc(ix, (void**)&ix->pid, sizeof(int32_t) * n));
  order_d = ix->pid;
  SAH_CUDA(cudaMemcpyAsync(order_d, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
  SAH_TRY(dev_alloc(ix, (void**)&ix->Ps, sizeof(float) * n * dp));
  SAH_TRY(dev_alloc(ix, (void**)&ix->pnorm, sizeof(float) * n));
  gather_rows_kernel<<<grid_for(n, 8), 256, 0, st>>>(P_dev, d, order_d, n, dp, ix->Ps, nullptr, 0);
  gather_f32_kernel<<<grid_for(n, 256), 256, 0, st>>>(pn_raw, order_d, n, ix->pnorm);
  SAH_CUDA(cudaGetLastError());
  ix->mmax = pn_h[order[0]];

  // ---- users: zero-norm users answer "yes" always and stay out of the tree
  std::vector<int32_t> nz, zero;
  nz.reserve(m);
  for (int64_t i = 0; i < m; ++i) (un_h[i] > 0.f ? nz : zero).push_back((int32_t)i);
  ix->m_nz = (int64_t)nz.size();
  ix->nzero = (int64_t)zero.size();
  if (!zero.empty()) {
    SAH_TRY(dev_alloc(ix, (void**)&ix->zero_uid, sizeof(int32_t) * zero.size()));
    SAH_CUDA(cudaMemcpyAsync(ix->zero_uid, zero.data(), sizeof(int32_t) * zero.size(),
                             cudaMemcpyHostToDevice, st));
  }
  const int64_t mz = ix->m_nz;
  if (mz == 0) {
    SAH_CUDA(cudaStreamSynchronize(st));
    cudaFreeAsync(pn_raw, st);
    cudaFreeAsync(un_raw, st);
    ix->nb = 0;
    SAH_TRY(dev_alloc(ix, (void**)&ix->bstart, sizeof(int32_t)));
    SAH_CUDA(cudaMemsetAsync(ix->bstart, 0, sizeof(int32_t), st));
    return SAH_OK;
  }
  int32_t* nz_d = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&nz_d, sizeof(int32_t) * mz, st));
  SAH_CUDA(cudaMemcpyAsync(nz_d, nz.data(), sizeof(int32_t) * mz, cudaMemcpyHostToDevice, st));
  float* Uh = nullptr;   // unit directions, compacted order
  SAH_CUDA(cudaMallocAsync((void**)&Uh, sizeof(float) * mz * dp, st));
  gather_rows_kernel<<<grid_for(mz, 8), 256, 0, st>>>(U_dev, d, nz_d, mz, dp, Uh, un_raw, 1);
  SAH_CUDA(cudaGetLastError());

  // ---- A2: Cone-Tree, level by level.  perm holds positions into the compacted users.
  int32_t *perm = nullptr, *perm2 = nullptr, *lrank = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&perm, sizeof(int32_t) * mz, st));
  SAH_CUDA(cudaMallocAsync((void**)&perm2, sizeof(int32_t) * mz, st));
  SAH_CUDA(cudaMallocAsync((void**)&lrank, sizeof(int32_t) * mz, st));
  {
    std::vector<int32_t> id(mz);
    std::iota(id.begin(), id.end(), 0);
    SAH_CUDA(cudaMemcpyAsync(perm, id.data(), sizeof(int32_t) * mz, cudaMemcpyHostToDevice, st));
    SAH_CUDA(cudaStreamSynchronize(st));
  }
  const int N0 = ix->prm.leaf_size;
  const uint64_t seed_mix = splitmix64(ix->prm.seed);
  std::vector<Seg> leaves, active;
  const bool norm_blocks = ix->prm.blocking == SAH_BLOCK_NORM;
  if (norm_blocks) {
    // Simpfer's blocks: the users in descending norm order (ties: lower id first), cut into
    // consecutive runs of N0
    std::vector<int32_t> id(mz);
    std::iota(id.begin(), id.end(), 0);
    std::stable_sort(id.begin(), id.end(), [&](int32_t a, int32_t b) { return un_h[nz[a]] > un_h[nz[b]]; });
    SAH_CUDA(cudaMemcpyAsync(perm, id.data(), sizeof(int32_t) * mz, cudaMemcpyHostToDevice, st));
    SAH_CUDA(cudaStreamSynchronize(st));
    for (int64_t s0 = 0; s0 < mz; s0 += N0)
      leaves.push_back(Seg{(int32_t)s0, (int32_t)std::min<int64_t>(N0, mz - s0), 0ull});
  } else {
    Seg root{0, (int32_t)mz, 1ull};
    (root.len > N0 ? active : leaves).push_back(root);
  }
  // scratch sized for the largest level: at most mz / kTile + #segments tiles
  const int64_t max_tiles = mz / kTile + mz / (N0 + 1) + 2;
  const int64_t max_segs = mz / (N0 + 1) + 2;
  CtTile* tiles_d = nullptr;
  int32_t *seg_i32 = nullptr, *tile_i32 = nullptr;
  unsigned long long* best_d = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&tiles_d, sizeof(CtTile) * max_tiles, st));
  SAH_CUDA(cudaMallocAsync((void**)&seg_i32, sizeof(int32_t) * max_segs * 6, st));
  SAH_CUDA(cudaMallocAsync((void**)&tile_i32, sizeof(int32_t) * max_tiles * 3, st));
  SAH_CUDA(cudaMallocAsync((void**)&best_d, sizeof(unsigned long long) * max_segs, st));
  int32_t* pivot_d = seg_i32;
  int32_t* ul_d = seg_i32 + max_segs;
  int32_t* ur_d = seg_i32 + 2 * max_segs;
  int32_t* sstart_d = seg_i32 + 3 * max_segs;
  int32_t* snleft_d = seg_i32 + 4 * max_segs;
  int32_t* shalves_d = seg_i32 + 5 * max_segs;
  int32_t* tleft_d = tile_i32;
  int32_t* tloff_d = tile_i32 + max_tiles;
  int32_t* troff_d = tile_i32 + 2 * max_tiles;
  std::vector<int32_t> perm_h;   // host copy, only read for pivot lookups
  while (!active.empty()) {
    const int ns = (int)active.size();
    std::vector<CtTile> tiles;
    std::vector<int32_t> sstart(ns), pivpos(ns);
    for (int s = 0; s < ns; ++s) {
      const Seg& g = active[s];
      sstart[s] = g.start;
      pivpos[s] = (int32_t)(splitmix64(seed_mix ^ g.key) % (uint64_t)g.len);
      for (int32_t f = 0; f < g.len; f += kTile)
        tiles.push_back(CtTile{s, g.start + f, std::min<int32_t>(kTile, g.len - f), f});
    }
    const int nt = (int)tiles.size();
    perm_h.resize(mz);
    SAH_CUDA(cudaMemcpyAsync(perm_h.data(), perm, sizeof(int32_t) * mz, cudaMemcpyDeviceToHost, st));
    SAH_CUDA(cudaMemcpyAsync(tiles_d, tiles.data(), sizeof(CtTile) * nt, cudaMemcpyHostToDevice, st));
    SAH_CUDA(cudaMemcpyAsync(sstart_d, sstart.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st));
    SAH_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> piv(ns);
    for (int s = 0; s < ns; ++s) piv[s] = perm_h[sstart[s] + pivpos[s]];
    SAH_CUDA(cudaMemcpyAsync(pivot_d, piv.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st));
    // u_l = argmin <u, v>
    SAH_CUDA(cudaMemsetAsync(best_d, 0xff, sizeof(unsigned long long) * ns, st));
    ct_argmin_kernel<<<nt, 256, 0, st>>>(Uh, dp, perm, tiles_d, pivot_d, best_d);
    SAH_CUDA(cudaGetLastError());
    std::vector<unsigned long long> best(ns);
    SAH_CUDA(cudaMemcpyAsync(best.data(), best_d, sizeof(unsigned long long) * ns, cudaMemcpyDeviceToHost, st));
    SAH_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> ulh(ns), urh(ns);
    for (int s = 0; s < ns; ++s) ulh[s] = perm_h[sstart[s] + (int32_t)(best[s] & 0xffffffffu)];
    SAH_CUDA(cudaMemcpyAsync(ul_d, ulh.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st));
    // u_r = argmin <u, u_l>
    SAH_CUDA(cudaMemsetAsync(best_d, 0xff, sizeof(unsigned long long) * ns, st));
    ct_argmin_kernel<<<nt, 256, 0, st>>>(Uh, dp, perm, tiles_d, ul_d, best_d);
    SAH_CUDA(cudaGetLastError());
    SAH_CUDA(cudaMemcpyAsync(best.data(), best_d, sizeof(unsigned long long) * ns, cudaMemcpyDeviceToHost, st));
    SAH_CUDA(cudaStreamSynchronize(st));
    for (int s = 0; s < ns; ++s) urh[s] = perm_h[sstart[s] + (int32_t)(best[s] & 0xffffffffu)];
    SAH_CUDA(cudaMemcpyAsync(ur_d, urh.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st));
    // split flags, per-tile left counts
    ct_split_kernel<<<nt, 256, 0, st>>>(Uh, dp, perm, tiles_d, ul_d, ur_d, lrank, tleft_d);
    SAH_CUDA(cudaGetLastError());
    std::vector<int32_t> tleft(nt);
    SAH_CUDA(cudaMemcpyAsync(tleft.data(), tleft_d, sizeof(int32_t) * nt, cudaMemcpyDeviceToHost, st));
    SAH_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> nleft(ns, 0), halves(ns, 0), tloff(nt), troff(nt);
    for (int t = 0; t < nt; ++t) nleft[tiles[t].seg] += tleft[t];
    {
      std::vector<int32_t> accl(ns, 0), accr(ns, 0);
      for (int t = 0; t < nt; ++t) {
        int s = tiles[t].seg;
        tloff[t] = accl[s];
        troff[t] = accr[s];
        accl[s] += tleft[t];
        accr[s] += tiles[t].len - tleft[t];
      }
    }
    std::vector<Seg> next;
    for (int s = 0; s < ns; ++s) {
      const Seg& g = active[s];
      int32_t nl = nleft[s];
      if (nl == 0 || nl == g.len) {   // all users on one side: split the list in halves
        halves[s] = 1;
        nl = g.len / 2;
      }
      Seg L{g.start, nl, 2 * g.key}, R{g.start + nl, g.len - nl, 2 * g.key + 1};
      (L.len > N0 ? next : leaves).push_back(L);
      (R.len > N0 ? next : leaves).push_back(R);
    }
    SAH_CUDA(cudaMemcpyAsync(tloff_d, tloff.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, st));
    SAH_CUDA(cudaMemcpyAsync(troff_d, troff.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, st));
    SAH_CUDA(cudaMemcpyAsync(snleft_d, nleft.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st));
    SAH_CUDA(cudaMemcpyAsync(shalves_d, halves.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st));
    SAH_CUDA(cudaMemcpyAsync(perm2, perm, sizeof(int32_t) * mz, cudaMemcpyDeviceToDevice, st));
    ct_scatter_kernel<<<nt, 256, 0, st>>>(perm, tiles_d, lrank, tloff_d, troff_d, sstart_d, snleft_d,
                                         shalves_d, perm2);
    SAH_CUDA(cudaGetLastError());
    std::swap(perm, perm2);
    active.swap(next);
  }
  std::sort(leaves.begin(), leaves.end(), [](const Seg& a, const Seg& b) { return a.start < b.start; });
  ix->nb = (int32_t)leaves.size();
  std::vector<int32_t> bstart(ix->nb + 1);
  for (int i = 0; i < ix->nb; ++i) bstart[i] = leaves[i].start;
  bstart[ix->nb] = (int32_t)mz;

  // ---- users in leaf order
  SAH_TRY(dev_alloc(ix, (void**)&ix->Ut, sizeof(float) * mz * dp));
  SAH_TRY(dev_alloc(ix, (void**)&ix->unorm, sizeof(float) * mz));
  SAH_TRY(dev_alloc(ix, (void**)&ix->uid, sizeof(int32_t) * mz));
  SAH_TRY(dev_alloc(ix, (void**)&ix->ucos, sizeof(float) * mz));
  SAH_TRY(dev_alloc(ix, (void**)&ix->usin, sizeof(float) * mz));
  int32_t* orig_of_pos = nullptr;   // caller id of each tree position
  SAH_CUDA(cudaMallocAsync((void**)&orig_of_pos, sizeof(int32_t) * mz, st));
  gather_i32_kernel<<<grid_for(mz, 256), 256, 0, st>>>(nz_d, perm, mz, ix->uid);
  gather_rows_kernel<<<grid_for(mz, 8), 256, 0, st>>>(U_dev, d, ix->uid, mz, dp, ix->Ut, nullptr, 0);
  gather_f32_kernel<<<grid_for(mz, 256), 256, 0, st>>>(un_raw, ix->uid, mz, ix->unorm);
  float* Uh_t = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&Uh_t, sizeof(float) * mz * dp, st));
  gather_padded_kernel<<<grid_for(mz, 8), 256, 0, st>>>(Uh, perm, mz, dp, Uh_t);
  SAH_CUDA(cudaGetLastError());

  SAH_TRY(dev_alloc(ix, (void**)&ix->bstart, sizeof(int32_t) * (ix->nb + 1)));
  SAH_CUDA(cudaMemcpyAsync(ix->bstart, bstart.data(), sizeof(int32_t) * (ix->nb + 1),
                           cudaMemcpyHostToDevice, st));
  SAH_TRY(dev_alloc(ix, (void**)&ix->bcent, sizeof(float) * (size_t)ix->nb * dp));
  SAH_TRY(dev_alloc(ix, (void**)&ix->bcos, sizeof(float) * ix->nb));
  SAH_TRY(dev_alloc(ix, (void**)&ix->bsin, sizeof(float) * ix->nb));
  leaf_stats_kernel<<<ix->nb, 256, sizeof(float) * dp, st>>>(Uh_t, dp, ix->bstart, ix->bcent, ix->bcos,
                                                             ix->bsin, ix->ucos, ix->usin, norm_blocks ? 1 : 0);
  SAH_CUDA(cudaGetLastError());
  SAH_TRY(dev_alloc(ix, (void**)&ix->ublock, sizeof(int32_t) * mz));
  user_block_kernel<<<ix->nb, 256, 0, st>>>(ix->bstart, ix->nb, ix->ublock);
  SAH_CUDA(cudaGetLastError());

  // ---- A1: lower-bound arrays over P' and the per-block bounds
  const int kmax = ix->kmax;
  int32_t* ids64 = nullptr;
  float* vlast = nullptr;
  SAH_TRY(dev_alloc(ix, (void**)&ix->Lt, sizeof(float) * (size_t)kmax * mz));
  SAH_TRY(dev_alloc(ix, (void**)&ix->Eu, sizeof(float) * mz));
  {
    int stride4 = (dp / 4) | 1;
    int tile_items = 128;
    while (tile_items > 32 && (size_t)tile_items * stride4 * 16 > 96 * 1024) tile_items -= 32;
    size_t smem = ((size_t)tile_items * stride4 + (size_t)kTopkWarps * kUsersPerWarp * (dp / 4)) * 16;
    SAH_TRY(raise_smem_limit((const void*)topk_lower_bounds_kernel, (size_t)((int)smem)));
    unsigned grid = grid_for(mz, kTopkWarps * kUsersPerWarp);
    if (ix->prm.precision != SAH_FP32) SAH_TRY(build_bf16_copies(ix, st));
    if (ix->prm.precision != SAH_FP32 && ix->prm.tc_user_pass == 2) SAH_TRY(build_fp8_users(ix, st));
    if (ix->pp > 0) {
      if (ix->l_exact) {
        SAH_CUDA(cudaMallocAsync((void**)&ids64, sizeof(int32_t) * 64 * (size_t)mz, st));
        SAH_CUDA(cudaMallocAsync((void**)&vlast, sizeof(float) * (size_t)mz, st));
      }
      // tensor cores: a floor from the largest-norm items, then the items up to each user's
      // cut through tcgen05 (a higher floor keeps fewer candidates and ends the scans sooner)
      const int kFloorItems = (int)std::min<int64_t>(2048, std::max<int64_t>(256, ix->n / 8));
      if (ix->l_exact && ix->dk > 0 && ix->n > kFloorItems) {
        topk_lower_bounds_kernel<<<grid, kTopkWarps * 32, smem, st>>>(ix->Ut, ix->Ps, dp, mz, kFloorItems, kmax,
                                                                      tile_items, stride4, ix->Lt, ids64, vlast);
        SAH_CUDA(cudaGetLastError());
        SAH_TRY(topk_full_tc(ix, vlast, ids64, st, nullptr));
      } else {
        topk_lower_bounds_kernel<<<grid, kTopkWarps * 32, smem, st>>>(ix->Ut, ix->Ps, dp, mz, ix->pp, kmax,
                                                                      tile_items, stride4, ix->Lt, ids64, vlast);
      }
    } else {
      // no P': every lower bound is -inf
      fill_i32_kernel<<<grid_for((int64_t)kmax * mz, 256), 256, 0, st>>>(
          reinterpret_cast<int32_t*>(ix->Lt), (int64_t)kmax * mz, (int32_t)0xff800000u);
    }
    SAH_CUDA(cudaGetLastError());
  }
  user_error_kernel<<<grid_for(mz, 256), 256, 0, st>>>(ix->unorm, mz, ix->gamma, ix->mmax, ix->Eu);
  if (ids64) {
    SAH_TRY(dev_alloc(ix, (void**)&ix->T64, sizeof(double) * (size_t)kmax * mz));
    tau64_kernel<<<grid_for(mz, 8), 256, 0, st>>>(ix->Ut, ix->Ps, ix->d, dp, mz, kmax, ids64, vlast, ix->Lt, ix->Eu,
                                                  ix->unorm, ix->mmax, ix->T64);
    SAH_CUDA(cudaGetLastError());
  }
  SAH_TRY(dev_alloc(ix, (void**)&ix->LB, sizeof(float) * (size_t)kmax * ix->nb));
  block_lower_bounds_kernel<<<grid_for((int64_t)kmax * ix->nb, 256), 256, 0, st>>>(
      ix->Lt, ix->Eu, ix->unorm, ix->bstart, ix->nb, mz, kmax, ix->LB);
  SAH_CUDA(cudaGetLastError());
  {
    const int ntiles = (int)((mz + 127) / 128);
    SAH_TRY(dev_alloc(ix, (void**)&ix->tile_lb, sizeof(float) * (size_t)kmax * ntiles));
    tile_lower_bounds_kernel<<<grid_for((int64_t)kmax * ntiles, 256), 256, 0, st>>>(ix->Lt, ix->Eu, ix->unorm, mz,
                                                                                   kmax, ntiles, ix->tile_lb);
    SAH_CUDA(cudaGetLastError());
  }
  SAH_CUDA(cudaStreamSynchronize(st));

  cudaFreeAsync(pn_raw, st);
  cudaFreeAsync(un_raw, st);
  cudaFreeAsync(nz_d, st);
  cudaFreeAsync(Uh, st);
  cudaFreeAsync(Uh_t, st);
  cudaFreeAsync(perm, st);
  cudaFreeAsync(perm2, st);
  cudaFreeAsync(lrank, st);
  cudaFreeAsync(tiles_d, st);
  cudaFreeAsync(seg_i32, st);
  cudaFreeAsync(tile_i32, st);
  cudaFreeAsync(best_d, st);
  cudaFreeAsync(orig_of_pos, st);
  if (ids64) cudaFreeAsync(ids64, st);
  if (vlast) cudaFreeAsync(vlast, st);
  SAH_CUDA(cudaStreamSynchronize(st));
  return SAH_OK;
}

}  // namespace sah
