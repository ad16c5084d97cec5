// Tensor-core kMIPS decision for the survivors of the user pass (A5 on tcgen05), and the
// boundary re-score of what its error band leaves open (A6).
//
// Per survivor row (u, q, <u,q>, k) the exact decision counts the items p with
// <u,p> > <u,q>, in descending norm order, stopping "no" at k items and stopping the
// scan once ||u|| ||p_i|| cannot reach <u,q> (the mu_j rule of Alg. 2; items are sorted
// by norm as in Alg. 1 and Alg. 4).  Here 128 survivors form the A operand of a
// 128 x 128 x K UMMA and the items stream through TMA as the B operand, in tiles of 128.
//
// Operands are split as in the tensor-core user pass: x_hi = bf16(x), x_lo = bf16(x - x_hi)
// for both users and items, and the MMA accumulates u_hi p_hi + u_hi p_lo + u_lo p_hi in
// FP32, so that
//     |s - <u,p>| <= c ||u|| ||p||,   c = 1.01 (3 * 2^-16 + (6K + 16) 2^-23)
// (about 1e-4 for K = 64).  With BF16 operands alone the bound is near 2^-7, and about
// one item per row and tile would fall inside it: each such item costs the epilogue far
// more than the two extra MMAs cost the tensor pipe.  The epilogue reads each row's
// scores from TMEM, skips groups of 32 items whose maximum is below the row's band, counts
// the items that are certainly above <u,q> and remembers the few it cannot separate.
// Rows finish independently; a CTA stops streaming tiles when all its rows are done.
// Survivors are first sorted by the tile where their norm cut falls, so that rows in
// one CTA need similar numbers of tiles.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "sah_internal.cuh"
#include "tc.cuh"

namespace sah {
namespace {

constexpr int kTileN = 128;       // items per tile (UMMA N)
constexpr int kRows = 128;        // survivors per CTA (UMMA M)
constexpr int kBandCap = 32;      // band items remembered per row
constexpr int kThreads = 192;     // warp 0 TMA producer, warp 1 MMA issuer, warps 2-5 epilogue
constexpr uint32_t kTmemCols = 2 * kTileN;   // two score slots

enum RowStatus : int32_t { ROW_YES = 1, ROW_NO = 2, ROW_BAND = 3, ROW_FULL = 4 };

// lo = bf16(x - bf16(x)) of every row: the low half of the split operands
__global__ void f32_to_bf16_lo_rows_kernel(const float* __restrict__ src, int64_t rows, int dp, int d, int dk,
                                           uint16_t* __restrict__ dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * dk) return;
  int64_t r = i / dk;
  int c = (int)(i % dk);
  float v = c < d ? src[r * dp + c] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
  dst[i] = __bfloat16_as_ushort(l);
}

__global__ void f32_to_bf16_rows_kernel(const float* __restrict__ src, int64_t rows, int dp, int d, int dk,
                                        uint16_t* __restrict__ dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * dk) return;
  int64_t r = i / dk;
  int c = (int)(i % dk);
  float v = c < d ? src[r * dp + c] : 0.f;
  __nv_bfloat16 b = __float2bfloat16_rn(v);
  dst[i] = *reinterpret_cast<uint16_t*>(&b);
}

// Tile (of kTileN items) at which a row's norm cut falls: the first t with
// ||u|| ||p_{t kTileN}|| (1 + 2 gamma) <= <u,q> - e_q; ntiles when it never falls.
__device__ __forceinline__ int cut_of(const Survivor& S, const float* __restrict__ unorm,
                                      const float* __restrict__ pnorm, const float* __restrict__ qn, float gamma,
                                      int ntiles) {
  const float nu = unorm[S.upos];
  const float eq = __fmul_ru(__fmul_ru(gamma, nu), qn[S.j]) + 1e-30f;
  const float lo = __fsub_rd(S.sq, eq);
  const float scale = __fmul_ru(nu, 1.f + 2.f * gamma);
  int a = 0, b = ntiles;   // first t in [0, ntiles] whose test holds (monotone in t)
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (__fmul_ru(scale, pnorm[(int64_t)mid * kTileN]) <= lo) b = mid;
    else a = mid + 1;
  }
  return a;
}

// The contiguous range of the survivor list that block b of the grid owns.
__device__ __forceinline__ void block_range(int64_t ns, int64_t& lo, int64_t& hi) {
  const int64_t per = (ns + gridDim.x - 1) / gridDim.x;
  lo = std::min<int64_t>((int64_t)blockIdx.x * per, ns);
  hi = std::min<int64_t>(lo + per, ns);
}

// Cut of every survivor, and the histogram of the cuts: counted per block in shared
// memory (nbins = ntiles + 1 counters), then one global addition per bin and block
// (SMEM = false, for more bins than shared memory holds: global additions only).
template <bool SMEM>
__global__ void cut_kernel(const Survivor* __restrict__ surv, const unsigned long long* __restrict__ count,
                           int64_t cap, const float* __restrict__ unorm, const float* __restrict__ pnorm,
                           const float* __restrict__ qn, float gamma, int ntiles, int32_t* __restrict__ cut,
                           int32_t* __restrict__ hist) {
  extern __shared__ int32_t sh_hist[];
  const int nbins = ntiles + 1;
  if (SMEM)
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) sh_hist[i] = 0;
  const int64_t ns = block_count(count, cap);   // synchronises the block
  int64_t lo, hi;
  block_range(ns, lo, hi);
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const int a = cut_of(surv[i], unorm, pnorm, qn, gamma, ntiles);
    cut[i] = a;
    atomicAdd(SMEM ? &sh_hist[a] : &hist[a], 1);
  }
  if (!SMEM) return;
  __syncthreads();
  for (int i = threadIdx.x; i < nbins; i += blockDim.x)
    if (sh_hist[i]) atomicAdd(&hist[i], sh_hist[i]);
}

// Exclusive prefix sum of count values in place, by one block of 1024 threads.
__global__ void __launch_bounds__(1024) exclusive_scan_small_kernel(int32_t* __restrict__ v, int count) {
  __shared__ int32_t warp_sum[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int per = (count + 1023) / 1024;
  const int b = std::min(t * per, count), e = std::min(b + per, count);
  int32_t s = 0;
  for (int i = b; i < e; ++i) s += v[i];
  int32_t x = s;   // inclusive scan of the per-thread sums
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t ws = warp_sum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, ws, o);
      if (lane >= o) ws += y;
    }
    warp_sum[lane] = ws;
  }
  __syncthreads();
  int32_t acc = x - s + (w > 0 ? warp_sum[w - 1] : 0);
  for (int i = b; i < e; ++i) {
    const int32_t y = v[i];
    v[i] = acc;
    acc += y;
  }
}

// Survivors reordered by cut (counting sort): each block counts its range per bin in
// shared memory, reserves its share of every bin with one global addition, then places
// its rows (SMEM = false: one global addition per row).  Order within a bin is arbitrary.
template <bool SMEM>
__global__ void sort_by_cut_kernel(const Survivor* __restrict__ surv, const int32_t* __restrict__ cut,
                                   const unsigned long long* __restrict__ count, int64_t cap, int ntiles,
                                   int32_t* __restrict__ off, Survivor* __restrict__ out_rows,
                                   int32_t* __restrict__ out_cut) {
  extern __shared__ int32_t sh_sort[];   // [nbins] counts, then [nbins] bases
  const int nbins = ntiles + 1;
  int32_t* cnt = sh_sort;
  int32_t* base = sh_sort + nbins;
  if (SMEM)
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) cnt[i] = 0;
  const int64_t ns = block_count(count, cap);   // synchronises the block
  int64_t lo, hi;
  block_range(ns, lo, hi);
  if (!SMEM) {
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const int32_t c = cut[i];
      const int32_t p = atomicAdd(&off[c], 1);
      out_rows[p] = surv[i];
      out_cut[p] = c;
    }
    return;
  }
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&cnt[cut[i]], 1);
  __syncthreads();
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
    base[i] = cnt[i] ? atomicAdd(&off[i], cnt[i]) : 0;
    cnt[i] = 0;
  }
  __syncthreads();
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const int32_t c = cut[i];
    const int32_t p = base[c] + atomicAdd(&cnt[c], 1);
    out_rows[p] = surv[i];
    out_cut[p] = c;
  }
}

__device__ __forceinline__ bool epilogue_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, 1, 128, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ float max3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

struct TcParams {
  const Survivor* rows;
  const int32_t* cut;
  const unsigned long long* nrows_dev;   // survivors, read on the device
  int64_t cap;
  const uint16_t* Ub;
  const uint16_t* Ulo;
  int dk;
  const float* unorm;
  const float* pnorm;
  int64_t n;
  const float* qn;
  const int32_t* kk;
  float gamma;
  float cbf;
  int32_t* status;
  int32_t* certain_out;
  int32_t* band_out;
  int32_t* band_items;
  unsigned long long* items_stat;
  int* timeout;
};

// One CTA per 128 survivor rows.  Warp 0 (one thread) streams the item tiles by TMA,
// warp 1 (one thread) issues the MMAs, warps 2-5 read the scores from TMEM, one thread
// per row.  Operands are split: A = (u_hi, u_lo) gathered from the BF16 copies of the
// users, B = (p_hi, p_lo) tiles of the items, and every K block accumulates
// u_hi p_hi + u_hi p_lo + u_lo p_hi into the tile's TMEM slot (two slots alternate, so
// the MMAs of tile t+1 run while tile t is read).
template <int KB, int STAGES, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
verify_tc_kernel(const __grid_constant__ CUtensorMap tmapPhi, const __grid_constant__ CUtensorMap tmapPlo,
                 TcParams prm) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[2], tempty_bar[2], done_bar,
      a_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int stop_flag, p_issued, p_done;

  constexpr uint32_t kABytes = kRows * 128;          // one 64-wide K block of A (hi or lo)
  constexpr uint32_t kBBytes = kTileN * 128;         // one 64-wide K block of a B tile (hi or lo)
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;                                // [hi | lo][KB]
  uint8_t* sB = base + 2 * KB * kABytes;             // [stage][hi | lo][KB]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  const int64_t nrows_all = block_count(prm.nrows_dev, prm.cap);
  if (r0 >= nrows_all) return;                          // the grid is sized for the list's capacity
  const int64_t nrows_cta = std::min<int64_t>(kRows, nrows_all - r0);
  const int T = prm.cut[r0 + nrows_cta - 1];          // rows are sorted by cut: the last needs most

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&tfull_bar[a], 1);
      tc::mbar_init(&tempty_bar[a], 4);
    }
    tc::mbar_init(&done_bar, 1);
    tc::mbar_init(&a_bar, 128);                      // every epilogue thread, once its row is in place
    stop_flag = 0;
    p_issued = 0;
    p_done = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_sh, kTmemCols);
    tc::tmem_relinquish();
  }
  // The item tiles do not depend on the rows: the producer starts streaming them while
  // the epilogue warps gather the A operand.
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_base_sh;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      tc::prefetch_tensormap(&tmapPhi);
      tc::prefetch_tensormap(&tmapPlo);
      int issued = 0;
      for (int t = 0; t < T; ++t) {
        const int s = t % STAGES;
        if (t >= STAGES && !tc::mbar_wait(&empty_bar[s], ((t / STAGES) & 1) ^ 1, prm.timeout, nullptr)) break;
        if (stop_flag) break;
        tc::mbar_arrive_expect_tx(&full_bar[s], 2 * KB * kBBytes);
        uint8_t* dst = sB + (size_t)s * 2 * KB * kBBytes;
        for (int kb = 0; kb < KB; ++kb) {
          tc::tma_load_2d(dst + kb * kBBytes, &tmapPhi, &full_bar[s], kb * 64, t * kTileN);
          tc::tma_load_2d(dst + (KB + kb) * kBBytes, &tmapPlo, &full_bar[s], kb * 64, t * kTileN);
        }
        issued = t + 1;
      }
      p_issued = issued;
      __threadfence_block();
      p_done = 1;
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(kRows, kTileN);
      const uint32_t a_addr = tc::smem_addr(sA);
      const uint32_t b_addr = tc::smem_addr(sB);
      if (!tc::mbar_wait(&a_bar, 0, prm.timeout, nullptr)) stop_flag = 1;
      for (int t = 0;; ++t) {
        const int s = t % STAGES, a = t & 1;
        bool got = false, finished = false;
        for (uint32_t i = 0; i < tc::kSpinLimit; ++i) {
          if (tc::mbar_try_wait(&full_bar[s], (t / STAGES) & 1)) {
            got = true;
            break;
          }
          if (p_done && t >= p_issued) {
            finished = true;
            break;
          }
          if (i % tc::kFlagEvery == tc::kFlagEvery - 1 && *(volatile int*)prm.timeout) break;
          if (i > 32) __nanosleep(32);
        }
        if (!got) {
          if (!finished && !*(volatile int*)prm.timeout) atomicExch(prm.timeout, 1);
          break;
        }
        bool do_mma = !stop_flag;
        if (do_mma && t >= 2)
          do_mma = tc::mbar_wait(&tempty_bar[a], ((t >> 1) & 1) ^ 1, prm.timeout, &stop_flag);
        if (do_mma) {
          tc::tc_fence_after();
          const uint32_t bs = b_addr + (uint32_t)s * 2 * KB * kBBytes;
#pragma unroll
          for (int kb = 0; kb < KB; ++kb)
#pragma unroll
            for (int k16 = 0; k16 < 4; ++k16) {
              const uint64_t ah = tc::sw128_kmajor_desc(a_addr + kb * kABytes + k16 * 32);
              const uint64_t al = tc::sw128_kmajor_desc(a_addr + (KB + kb) * kABytes + k16 * 32);
              const uint64_t bh = tc::sw128_kmajor_desc(bs + kb * kBBytes + k16 * 32);
              const uint64_t bl = tc::sw128_kmajor_desc(bs + (KB + kb) * kBBytes + k16 * 32);
              const uint32_t d = tbase + a * kTileN;
              tc::umma_bf16(d, ah, bh, idesc, (kb | k16) ? 1u : 0u);
              tc::umma_bf16(d, ah, bl, idesc, 1u);
              tc::umma_bf16(d, al, bh, idesc, 1u);
            }
          tc::umma_commit(&empty_bar[s]);
          tc::umma_commit(&tfull_bar[a]);
        } else {
          tc::mbar_arrive(&empty_bar[s]);
        }
      }
      tc::umma_commit(&done_bar);
    }
  } else {
    // ------------------------------------------------ epilogue: one thread per row
    const int quad = warp & 3;                  // TMEM lanes this warp may read
    const int row = quad * 32 + lane;
    const int64_t gi = r0 + row;
    const bool valid = row < nrows_cta;
    Survivor S{};
    if (valid) S = prm.rows[gi];
    {
      // A operand: this thread's survivor row (high and low parts) into the
      // 128-byte-swizzled K-major layout
      uint4 vh[KB * 8], vl[KB * 8];
      const int64_t off = (int64_t)S.upos * prm.dk;
#pragma unroll
      for (int c = 0; c < KB * 8; ++c) {
        vh[c] = valid ? *reinterpret_cast<const uint4*>(prm.Ub + off + c * 8) : make_uint4(0u, 0u, 0u, 0u);
        vl[c] = valid ? *reinterpret_cast<const uint4*>(prm.Ulo + off + c * 8) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int c = 0; c < KB * 8; ++c) {
        const int kb = c / 8;
        *reinterpret_cast<uint4*>(sA + kb * kABytes + tc::sw128_offset(row, c % 8)) = vh[c];
        *reinterpret_cast<uint4*>(sA + (KB + kb) * kABytes + tc::sw128_offset(row, c % 8)) = vl[c];
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::mbar_arrive(&a_bar);
    }
    int k = 0, cut_r = 0;
    float nu = 0.f, hi = 0.f, lo = 0.f;
    if (valid) {
      k = prm.kk[S.j];
      cut_r = prm.cut[gi];
      nu = prm.unorm[S.upos];
      float eq = __fmul_ru(__fmul_ru(prm.gamma, nu), prm.qn[S.j]) + 1e-30f;
      hi = __fadd_ru(S.sq, eq);
      lo = __fsub_rd(S.sq, eq);
    }
    const float cbu = __fmul_ru(prm.cbf, nu);
    float pn_next = T > 0 ? prm.pnorm[0] : 0.f;
    int certain = 0, band = 0;
    bool decided = !valid, failed = false;
    unsigned long long scanned = 0;
    for (int t = 0; t < T; ++t) {
      const int a = t & 1;
      if (!failed && !tc::mbar_wait(&tfull_bar[a], (t >> 1) & 1, prm.timeout, nullptr)) {
        failed = true;
        stop_flag = 1;
      }
      tc::tc_fence_after();
      const bool need = !failed && !decided && t < cut_r;
      const float pn_tile = pn_next;                       // ||p|| of the tile's first (largest) item
      if (t + 1 < T) pn_next = prm.pnorm[(int64_t)(t + 1) * kTileN];
      if (__any_sync(0xffffffffu, need)) {
        // every item of the tile has ||p|| <= pn_tile, so E bounds its score error
        const float E = __fmul_ru(cbu, pn_tile) + 1e-30f;
        const float thb = __fsub_rd(lo, E);                // at or below: certainly not above <u,q>
        const float thc = __fadd_ru(hi, E);                // above: certainly above <u,q>
        const int ncols = (int)std::min<int64_t>(kTileN, prm.n - (int64_t)t * kTileN);
        if (need) scanned += ncols;
        const uint32_t taddr = tbase + ((uint32_t)(quad * 32) << 16) + a * kTileN;
        // the maximum of every group of 32 items: a group whose maximum is at or below
        // the band holds no item that counts
        float gmax[kTileN / 32];
        {
          float v[kTileN];
          tc::tmem_ld128(taddr, v);
          tc::tmem_ld_wait();
#pragma unroll
          for (int c0 = 0; c0 < kTileN; c0 += 32) {
            float g[11];
#pragma unroll
            for (int i = 0; i < 10; ++i) g[i] = max3(v[c0 + 3 * i], v[c0 + 3 * i + 1], v[c0 + 3 * i + 2]);
            g[10] = fmaxf(v[c0 + 30], v[c0 + 31]);
            gmax[c0 / 32] = max3(max3(g[0], g[1], g[2]), max3(g[3], g[4], g[5]),
                                 max3(max3(g[6], g[7], g[8]), g[9], g[10]));
          }
        }
        // the few groups that hold such an item (for some row of the warp) are read again
        // from TMEM under a warp-uniform branch; the items are classified into bit masks
        uint32_t mine = 0;
#pragma unroll
        for (int j = 0; j < kTileN / 32; ++j) mine |= (need && gmax[j] > thb) ? 1u << j : 0u;
        uint32_t todo = __reduce_or_sync(0xffffffffu, mine);
        while (todo) {
          const int gi32 = __ffs(todo) - 1;
          todo &= todo - 1;
          float w[32];
          tc::tmem_ld32(taddr + gi32 * 32, w);
          tc::tmem_ld_wait();
          if ((mine >> gi32) & 1u) {
            uint32_t above = 0, inband = 0;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              above |= (w[i] > thc) ? 1u << i : 0u;
              inband |= (w[i] > thb) ? 1u << i : 0u;
            }
            const int left = ncols - gi32 * 32;           // items of the group inside P
            const uint32_t valid = left >= 32 ? 0xffffffffu : left <= 0 ? 0u : (1u << left) - 1u;
            above &= valid;
            inband &= valid & ~above;
            certain += __popc(above);
            while (inband) {
              const int i = __ffs(inband) - 1;
              inband &= inband - 1;
              if (band < kBandCap) prm.band_items[gi * kBandCap + band] = t * kTileN + gi32 * 32 + i;
              ++band;
            }
          }
        }
        if (need && certain >= k) decided = true;
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty_bar[a]);
      const bool row_done = failed || decided || (t + 1 >= cut_r);
      if (epilogue_all(row_done)) {
        if (t + 1 < T) stop_flag = 1;
        break;
      }
    }
    if (valid) {
      int32_t st;
      if (certain >= k) st = ROW_NO;
      else if (failed) st = ROW_FULL;
      else if (certain + band < k) st = ROW_YES;
      else if (band <= kBandCap) st = ROW_BAND;
      else st = ROW_FULL;
      prm.status[gi] = st;
      prm.certain_out[gi] = certain;
      prm.band_out[gi] = band;
    }
    for (int o = 16; o > 0; o >>= 1) scanned += __shfl_xor_sync(0xffffffffu, scanned, o);
    if (lane == 0 && scanned) atomicAdd(prm.items_stat, scanned);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    if (lane == 0) tc::mbar_wait(&done_bar, 0, prm.timeout, nullptr);
    __syncwarp();
    tc::tc_fence_after();
    tc::tmem_dealloc(tbase, kTmemCols);
  }
}

// Decides every row of the tensor-core pass: "yes"/"no" as found, band items (or, when
// the band overflowed, the whole row) in FP32 with the bound and in double precision
// where the bound cannot separate.  One warp per row.
__global__ void resolve_kernel(const Survivor* __restrict__ rows, const unsigned long long* __restrict__ count,
                               int64_t cap, const int32_t* __restrict__ status,
                               const int32_t* __restrict__ certain_in, const int32_t* __restrict__ band_in,
                               const int32_t* __restrict__ band_items, const float* __restrict__ Ut,
                               const float* __restrict__ unorm, const int32_t* __restrict__ uid,
                               const float* __restrict__ Ps, const float* __restrict__ pnorm, int64_t n, int d,
                               int dp, const float* __restrict__ Qd, const float* __restrict__ qn,
                               const int32_t* __restrict__ kk, float gamma, uint32_t* __restrict__ bitmap,
                               int64_t words, unsigned long long* __restrict__ fp64_stat,
                               unsigned long long* __restrict__ items_stat) {
  const int lane = threadIdx.x & 31;
  const int64_t nrows = block_count(count, cap);
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long fp64 = 0, scanned = 0;
  for (int64_t r = gw; r < nrows; r += nw) {
    const int32_t st = status[r];
    if (st == ROW_NO) continue;
    const Survivor S = rows[r];
    bool yes = st == ROW_YES;
    if (st == ROW_BAND || st == ROW_FULL) {
      const int k = kk[S.j];
      const float* u = Ut + (int64_t)S.upos * dp;
      const float nu = unorm[S.upos];
      const float eq = __fmul_ru(__fmul_ru(gamma, nu), qn[S.j]) + 1e-30f;
      const float hi = __fadd_ru(S.sq, eq), lo = __fsub_rd(S.sq, eq);
      const float gnu = __fmul_ru(gamma, nu);
      // <u,q> in double precision, computed once per row and only if some item needs it
      bool have64 = false;
      double s64q = 0.0;
      auto need64 = [&](bool any) {
        if (any && !have64) {
          double v64 = 0.0;
          if (lane == 0) v64 = dot64_seq(u, Qd + (int64_t)S.j * dp, d);
          s64q = __shfl_sync(0xffffffffu, v64, 0);
          have64 = true;
        }
      };
      int c;
      if (st == ROW_BAND) {
        c = certain_in[r];
        const int nb = band_in[r];
        bool gt = false, amb = false;
        const float* p = nullptr;
        if (lane < nb) {
          const int64_t it = band_items[r * kBandCap + lane];
          p = Ps + it * dp;
          float s = 0.f;
          for (int i = 0; i < dp; ++i) s = fmaf(u[i], p[i], s);
          const float ep = __fmul_ru(gnu, pnorm[it]) + 1e-30f;
          if (__fsub_rd(s, ep) > hi) gt = true;
          else amb = __fadd_ru(s, ep) > lo;
        }
        need64(__any_sync(0xffffffffu, amb));
        if (amb) gt = dot64_seq(u, p, d) > s64q;
        c += __popc(__ballot_sync(0xffffffffu, gt));
        if (have64) ++fp64;
      } else {
        // whole row: certain counts in FP32, everything undecided in double precision
        const float scale = __fmul_ru(nu, 1.f + 2.f * gamma);
        c = 0;
        for (int64_t b0 = 0; b0 < n && c < k; b0 += 32) {
          if (__fmul_ru(scale, pnorm[b0]) <= lo) break;
          const int64_t i = b0 + lane;
          bool gt = false, amb = false;
          const float* p = Ps + i * dp;
          if (i < n) {
            float s = 0.f;
            for (int e = 0; e < dp; ++e) s = fmaf(u[e], p[e], s);
            const float ep = __fmul_ru(gnu, pnorm[i]) + 1e-30f;
            if (__fsub_rd(s, ep) > hi) gt = true;
            else amb = __fadd_ru(s, ep) > lo;
          }
          need64(__any_sync(0xffffffffu, amb));
          if (amb) gt = dot64_seq(u, p, d) > s64q;
          c += __popc(__ballot_sync(0xffffffffu, gt));
          scanned += 32;
        }
        ++fp64;
      }
      yes = c < k;
    }
    if (yes && lane == 0) {
      const int32_t id = uid[S.upos];
      atomicOr(&bitmap[(int64_t)S.j * words + (id >> 5)], 1u << (id & 31));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    fp64 += __shfl_xor_sync(0xffffffffu, fp64, o);
    scanned += __shfl_xor_sync(0xffffffffu, scanned, o);
  }
  if (lane == 0) {
    if (fp64) atomicAdd(fp64_stat, fp64 / 32);
    if (scanned) atomicAdd(items_stat, scanned / 32);
  }
}

inline unsigned grid_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

template <int KB, int STAGES>
constexpr size_t tc_smem_bytes() {
  return 2 * ((size_t)KB * kRows * 128 + (size_t)STAGES * KB * kTileN * 128) + 1024;
}

}  // namespace

// BF16 copies of the users and items (K padded to 64 or 128) and the TMA map of the
// items, for the tensor-core path.
sah_status build_bf16_copies(Index* ix, cudaStream_t st) {
  if (ix->d > 128) {
    ix->dk = 0;
    return SAH_OK;
  }
  ix->dk = ix->d <= 64 ? 64 : 128;
  const int dk = ix->dk;
  SAH_TRY(dev_alloc(ix, (void**)&ix->Ub, sizeof(uint16_t) * (size_t)std::max<int64_t>(ix->m_nz, 1) * dk));
  SAH_TRY(dev_alloc(ix, (void**)&ix->Ulo, sizeof(uint16_t) * (size_t)std::max<int64_t>(ix->m_nz, 1) * dk));
  SAH_TRY(dev_alloc(ix, (void**)&ix->Pb, sizeof(uint16_t) * (size_t)ix->n * dk));
  SAH_TRY(dev_alloc(ix, (void**)&ix->Plo, sizeof(uint16_t) * (size_t)ix->n * dk));
  if (ix->m_nz > 0) {
    f32_to_bf16_rows_kernel<<<grid_for(ix->m_nz * dk, 256), 256, 0, st>>>(ix->Ut, ix->m_nz, ix->dp, ix->d, dk,
                                                                          ix->Ub);
    f32_to_bf16_lo_rows_kernel<<<grid_for(ix->m_nz * dk, 256), 256, 0, st>>>(ix->Ut, ix->m_nz, ix->dp, ix->d, dk,
                                                                             ix->Ulo);
  }
  f32_to_bf16_rows_kernel<<<grid_for(ix->n * dk, 256), 256, 0, st>>>(ix->Ps, ix->n, ix->dp, ix->d, dk, ix->Pb);
  f32_to_bf16_lo_rows_kernel<<<grid_for(ix->n * dk, 256), 256, 0, st>>>(ix->Ps, ix->n, ix->dp, ix->d, dk, ix->Plo);
  SAH_CUDA(cudaGetLastError());
  auto encode = get_encode_fn();
  if (!encode) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return SAH_ERR_UNSUPPORTED;
  }
  cuuint64_t dims[2] = {(cuuint64_t)dk, (cuuint64_t)ix->n};
  cuuint64_t strides[1] = {(cuuint64_t)dk * 2};
  cuuint32_t box[2] = {64, 256};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(&ix->tmap_P, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ix->Pb, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return SAH_ERR_CUDA;
  }
  // the verify pass's item tiles: kTileN items of the high and the low parts
  cuuint32_t vbox[2] = {64, (cuuint32_t)kTileN};
  r = encode(&ix->tmap_Pv, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ix->Pb, dims, strides, vbox, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r == CUDA_SUCCESS)
    r = encode(&ix->tmap_Plo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ix->Plo, dims, strides, vbox, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (verify item tiles) failed with code " + std::to_string((int)r));
    return SAH_ERR_CUDA;
  }
  if (ix->m_nz > 0) {
    cuuint64_t udims[2] = {(cuuint64_t)dk, (cuuint64_t)ix->m_nz};
    cuuint32_t ubox[2] = {64, 128};
    r = encode(&ix->tmap_U, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ix->Ub, udims, strides, ubox, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error("cuTensorMapEncodeTiled (users) failed with code " + std::to_string((int)r));
      return SAH_ERR_CUDA;
    }
    r = encode(&ix->tmap_Ulo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ix->Ulo, udims, strides, ubox, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error("cuTensorMapEncodeTiled (user low parts) failed with code " + std::to_string((int)r));
      return SAH_ERR_CUDA;
    }
  }
  return SAH_OK;
}

sah_status run_verify_tc(Index* ix, CallCtx* cx, const Survivor* surv, const unsigned long long* count_dev,
                         int64_t ns, const float* Qd, const float* qn, const int32_t* kk, uint32_t* bitmap,
                         int64_t words, unsigned long long* stats, int stat_fp64, int stat_items,
                         cudaStream_t st, int* launches, const cudaEvent_t* ev) {
  // ns is the capacity of the survivor list; the number of survivors stays on the device
  if (ns <= 0) return SAH_OK;
  const int ntiles = (int)((ix->n + kTileN - 1) / kTileN);
  // scratch: cut, hist, sorted rows, sorted cut, status, certain, band, band items
  size_t need = 0;
  auto take = [&](size_t b) { size_t o = need; need = (need + b + 255) & ~(size_t)255; return o; };
  const size_t o_cut = take(sizeof(int32_t) * ns), o_hist = take(sizeof(int32_t) * (ntiles + 2)),
               o_rows = take(sizeof(Survivor) * ns), o_scut = take(sizeof(int32_t) * ns),
               o_stat = take(sizeof(int32_t) * ns), o_cert = take(sizeof(int32_t) * ns),
               o_band = take(sizeof(int32_t) * ns), o_items = take(sizeof(int32_t) * ns * kBandCap);
  if (cx->tcws.bytes < need) {
    SAH_CUDA(cudaStreamSynchronize(st));
    if (cx->tcws.base) cudaFree(cx->tcws.base);
    cx->tcws.base = nullptr;
    cx->tcws.bytes = 0;
    cudaError_t e = cudaMalloc(&cx->tcws.base, need + need / 4);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("tensor-core verify workspace allocation failed");
      return SAH_ERR_OOM;
    }
    cx->tcws.bytes = need + need / 4;
  }
  char* w = (char*)cx->tcws.base;
  int32_t* cut = (int32_t*)(w + o_cut);
  int32_t* hist = (int32_t*)(w + o_hist);
  Survivor* rows = (Survivor*)(w + o_rows);
  int32_t* scut = (int32_t*)(w + o_scut);
  int32_t* status = (int32_t*)(w + o_stat);
  int32_t* cert = (int32_t*)(w + o_cert);
  int32_t* band = (int32_t*)(w + o_band);
  int32_t* items = (int32_t*)(w + o_items);

  SAH_CUDA(cudaMemsetAsync(hist, 0, sizeof(int32_t) * (ntiles + 2), st));
  {
    // per-block histograms in shared memory: one block per SM, each over a contiguous range
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
    const size_t hsmem = sizeof(int32_t) * (size_t)(ntiles + 1), ssmem = 2 * hsmem;
    if (ssmem <= 200 * 1024) {
      if (hsmem > 48 * 1024) SAH_TRY(raise_smem_limit((const void*)cut_kernel<true>, hsmem));
      if (ssmem > 48 * 1024) SAH_TRY(raise_smem_limit((const void*)sort_by_cut_kernel<true>, ssmem));
      const unsigned hb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(sms, grid_for(ns, 1024)));
      cut_kernel<true><<<hb, 512, hsmem, st>>>(surv, count_dev, ns, ix->unorm, ix->pnorm, qn, ix->gamma, ntiles,
                                               cut, hist);
      exclusive_scan_small_kernel<<<1, 1024, 0, st>>>(hist, ntiles + 1);
      sort_by_cut_kernel<true><<<hb, 512, ssmem, st>>>(surv, cut, count_dev, ns, ntiles, hist, rows, scut);
    } else {
      cut_kernel<false><<<grid_for(ns, 256), 256, 0, st>>>(surv, count_dev, ns, ix->unorm, ix->pnorm, qn,
                                                           ix->gamma, ntiles, cut, hist);
      exclusive_scan_small_kernel<<<1, 1024, 0, st>>>(hist, ntiles + 1);
      sort_by_cut_kernel<false><<<grid_for(ns, 256), 256, 0, st>>>(surv, cut, count_dev, ns, ntiles, hist, rows,
                                                                   scut);
    }
  }
  SAH_CUDA(cudaGetLastError());

  TcParams prm;
  prm.rows = rows;
  prm.cut = scut;
  prm.nrows_dev = count_dev;
  prm.cap = ns;
  prm.Ub = ix->Ub;
  prm.Ulo = ix->Ulo;
  prm.dk = ix->dk;
  prm.unorm = ix->unorm;
  prm.pnorm = ix->pnorm;
  prm.n = ix->n;
  prm.qn = qn;
  prm.kk = kk;
  prm.gamma = ix->gamma;
  // score error of the split product over K = dk (three products per coordinate)
  prm.cbf = (float)(1.01 * (3.0 * std::ldexp(1.0, -16) + (6.0 * ix->dk + 16.0) * std::ldexp(1.0, -23)));
  prm.status = status;
  prm.certain_out = cert;
  prm.band_out = band;
  prm.band_items = items;
  prm.items_stat = stats + stat_items;
  prm.timeout = ix->dev_timeout;
  const unsigned grid = grid_for(ns, kRows);
  if (ev) SAH_CUDA(cudaEventRecord(ev[0], st));
  if (ix->dk == 64) {
    // 97 KB of shared memory and 256 TMEM columns: two CTAs per SM
    constexpr size_t smem = tc_smem_bytes<1, 2>();
    SAH_TRY(raise_smem_limit((const void*)verify_tc_kernel<1, 2, 2>, smem));
    verify_tc_kernel<1, 2, 2><<<grid, kThreads, smem, st>>>(ix->tmap_Pv, ix->tmap_Plo, prm);
  } else {
    constexpr size_t smem = tc_smem_bytes<2, 2>();
    SAH_TRY(raise_smem_limit((const void*)verify_tc_kernel<2, 2, 1>, smem));
    verify_tc_kernel<2, 2, 1><<<grid, kThreads, smem, st>>>(ix->tmap_Pv, ix->tmap_Plo, prm);
  }
  SAH_CUDA(cudaGetLastError());
  if (ev) SAH_CUDA(cudaEventRecord(ev[1], st));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
  resolve_kernel<<<sms * 8, 256, 0, st>>>(rows, count_dev, ns, status, cert, band, items, ix->Ut, ix->unorm, ix->uid, ix->Ps,
                                          ix->pnorm, ix->n, ix->d, ix->dp, Qd, qn, kk, ix->gamma, bitmap, words,
                                          stats + stat_fp64, stats + stat_items);
  SAH_CUDA(cudaGetLastError());
  if (launches) *launches += 6;
  return SAH_OK;
}

}  // namespace sah
