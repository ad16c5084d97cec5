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
#include <cuda_fp8.h>
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
  // phase of the scan: tiles [t_begin, t_end) for the rows of list (positions in the
  // cut-sorted rows; all rows in order when list is null).  A row that is still open at
  // t_end keeps its counts in certain_out / band_out and sets its flag.
  const int32_t* list;
  int t_begin, t_end;
  uint8_t* flags;
  int inject_stall;   // test hook: the MMA thread stops after its first tile
};

// Persistent: a CTA takes row blocks blockIdx.x, blockIdx.x + gridDim.x, ... (128 survivor
// rows each).  Warp 0 (one thread) streams the item tiles by TMA, warp 1 (one thread)
// issues the MMAs, warps 2-5 read the scores from TMEM, one thread per row.  Operands are
// split: A = (u_hi, u_lo) gathered from the BF16 copies of the users, B = (p_hi, p_lo)
// tiles of the items, and every K block accumulates u_hi p_hi + u_hi p_lo + u_lo p_hi into
// the tile's TMEM slot (two slots alternate, so the MMAs of tile t+1 run while tile t is
// read).  The barriers are set up once; stages and slots run on counters across blocks
// (P tiles streamed, M tiles consumed, C tiles computed, E tiles read), and at the end of a
// block the epilogue also takes the (at most two) computed tiles it did not need, so the
// counters stay in step and the A buffer is free for the next block.
template <int KB, int STAGES, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
verify_tc_kernel(const __grid_constant__ CUtensorMap tmapPhi, const __grid_constant__ CUtensorMap tmapPlo,
                 TcParams prm) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[2], tempty_bar[2], a_bar, done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int stop_flag, p_issued, p_done, quit_sh;
  __shared__ volatile uint32_t c_sh;

  constexpr uint32_t kABytes = kRows * 128;          // one 64-wide K block of A (hi or lo)
  constexpr uint32_t kBBytes = kTileN * 128;         // one 64-wide K block of a B tile (hi or lo)
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;                                // [hi | lo][KB]
  uint8_t* sB = base + 2 * KB * kABytes;             // [stage][hi | lo][KB]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nrows_all = block_count(prm.nrows_dev, prm.cap);
  if ((int64_t)blockIdx.x * kRows >= nrows_all) return;   // no block for this CTA

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&tfull_bar[a], 1);
      tc::mbar_init(&tempty_bar[a], 4);
    }
    tc::mbar_init(&a_bar, 128);                      // every epilogue thread, once its row is in place
    tc::mbar_init(&done_bar, 1);                     // teardown: every MMA of the CTA has completed
    stop_flag = 0;
    p_issued = 0;
    p_done = 0;
    quit_sh = 0;
    c_sh = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_sh, kTmemCols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_base_sh;
  if (warp == 0 && lane == 0) {
    tc::prefetch_tensormap(&tmapPhi);
    tc::prefetch_tensormap(&tmapPlo);
  }

  uint32_t P = 0, M = 0, C = 0, E = 0;               // running counters (each kept by its role)
  int it = 0;                                        // blocks done by this CTA
  const int t0 = prm.t_begin;
  for (int64_t blk = blockIdx.x; blk * kRows < nrows_all; blk += gridDim.x, ++it) {
    const int64_t r0 = blk * kRows;
    const int64_t nrows_cta = std::min<int64_t>(kRows, nrows_all - r0);
    // rows are sorted by cut (lists keep that order): the last needs most
    const int64_t last = prm.list ? prm.list[r0 + nrows_cta - 1] : r0 + nrows_cta - 1;
    const int T = std::max(t0, std::min(prm.cut[last], prm.t_end));

    // The item tiles do not depend on the rows: the producer streams them while the
    // epilogue warps gather the A operand.
    if (warp == 0) {
      // ------------------------------------------------ TMA producer
      if (lane == 0) {
        int issued = 0;
        for (int i = 0; i < T - t0; ++i, ++P) {       // item tile t0 + i
          const uint32_t s = P % STAGES;
          if (P >= STAGES && !tc::mbar_wait(&empty_bar[s], ((P / STAGES) & 1) ^ 1, prm.timeout, nullptr)) break;
          if (stop_flag) break;
          tc::mbar_arrive_expect_tx(&full_bar[s], 2 * KB * kBBytes);
          uint8_t* dst = sB + (size_t)s * 2 * KB * kBBytes;
          const int y = (t0 + i) * kTileN;
          for (int kb = 0; kb < KB; ++kb) {
            tc::tma_load_2d(dst + kb * kBBytes, &tmapPhi, &full_bar[s], kb * 64, y);
            tc::tma_load_2d(dst + (KB + kb) * kBBytes, &tmapPlo, &full_bar[s], kb * 64, y);
          }
          issued = i + 1;
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
        if (!tc::mbar_wait(&a_bar, it & 1, prm.timeout, nullptr)) stop_flag = 1;
        for (int i = 0;; ++i) {                       // the block's i-th tile
          // test hook: a partner that stops working; the epilogue's bounded wait runs out
          if (prm.inject_stall && C >= 1) break;
          const uint32_t s = M % STAGES;
          bool got = false, finished = false;
          for (uint32_t w = 0; w < tc::kSpinLimit; ++w) {
            if (tc::mbar_try_wait(&full_bar[s], (M / STAGES) & 1)) {
              got = true;
              break;
            }
            if (p_done && i >= p_issued) {
              finished = true;
              break;
            }
            if (w % tc::kFlagEvery == tc::kFlagEvery - 1 && *(volatile int*)prm.timeout) break;
            if (w > 32) __nanosleep(32);
          }
          if (!got) {
            if (!finished && !*(volatile int*)prm.timeout) atomicExch(prm.timeout, 1);
            break;
          }
          ++M;
          const uint32_t a = C & 1;
          bool do_mma = !stop_flag;
          if (do_mma && C >= 2)
            do_mma = tc::mbar_wait(&tempty_bar[a], ((C >> 1) & 1) ^ 1, prm.timeout, &stop_flag);
          if (do_mma) {
            tc::tc_fence_after();
            const uint32_t bs = b_addr + s * 2 * KB * kBBytes;
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
            ++C;
          } else {
            tc::mbar_arrive(&empty_bar[s]);
          }
        }
        c_sh = C;
      }
    } else {
      // ------------------------------------------------ epilogue: one thread per row
      const int quad = warp & 3;                  // TMEM lanes this warp may read
      const int row = quad * 32 + lane;
      const bool valid = row < nrows_cta;
      const int64_t gi = !valid ? 0 : prm.list ? (int64_t)prm.list[r0 + row] : r0 + row;
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
      float pn_next = T > t0 ? prm.pnorm[(int64_t)t0 * kTileN] : 0.f;
      int certain = 0, band = 0;
      if (valid && prm.list) {
        certain = prm.certain_out[gi];
        band = prm.band_out[gi];
      }
      bool decided = !valid || band > kBandCap, failed = false;
      unsigned long long scanned = 0;
      for (int t = t0; t < T; ++t) {
        const uint32_t a = E & 1;
        if (!failed && !tc::mbar_wait(&tfull_bar[a], (E >> 1) & 1, prm.timeout, nullptr)) {
          failed = true;
          stop_flag = 1;
        }
        ++E;
        tc::tc_fence_after();
        const bool need = !failed && !decided && t < cut_r;
        const float pn_tile = pn_next;                       // ||p|| of the tile's first (largest) item
        if (t + 1 < T) pn_next = prm.pnorm[(int64_t)(t + 1) * kTileN];
        if (__any_sync(0xffffffffu, need)) {
          // every item of the tile has ||p|| <= pn_tile, so E_t bounds its score error
          const float Et = __fmul_ru(cbu, pn_tile) + 1e-30f;
          const float thb = __fsub_rd(lo, Et);               // at or below: certainly not above <u,q>
          const float thc = __fadd_ru(hi, Et);               // above: certainly above <u,q>
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
          // the few groups that hold such an item (for some row of the warp) are read
          // again from TMEM under a warp-uniform branch; items are classified into masks
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
              const uint32_t inside = left >= 32 ? 0xffffffffu : left <= 0 ? 0u : (1u << left) - 1u;
              above &= inside;
              inband &= inside & ~above;
              certain += __popc(above);
              while (inband) {
                const int i = __ffs(inband) - 1;
                inband &= inband - 1;
                if (band < kBandCap) prm.band_items[gi * kBandCap + band] = t * kTileN + gi32 * 32 + i;
                ++band;
              }
            }
          }
          // a row whose band overflowed is re-scanned whole by the resolve pass
          if (need && (certain >= k || band > kBandCap)) decided = true;
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
        // open: not decided, and items before the row's cut lie beyond this phase
        const bool open = !failed && certain < k && band <= kBandCap && cut_r > prm.t_end;
        if (!open) {
          int32_t st;
          if (certain >= k) st = ROW_NO;
          else if (failed) st = ROW_FULL;
          else if (certain + band < k) st = ROW_YES;
          else if (band <= kBandCap) st = ROW_BAND;
          else st = ROW_FULL;
          prm.status[gi] = st;
        }
        prm.certain_out[gi] = certain;
        prm.band_out[gi] = band;
        prm.flags[gi] = open ? 1 : 0;
      }
      for (int o = 16; o > 0; o >>= 1) scanned += __shfl_xor_sync(0xffffffffu, scanned, o);
      if (lane == 0 && scanned) atomicAdd(prm.items_stat, scanned);
    }
    tc::tc_fence_before();
    __syncthreads();
    // every role is done with the block: the epilogue takes the tiles computed after its
    // rows had finished (their MMAs complete before the next block's rows replace A), and
    // the per-block flags are reset
    if (warp >= 2) {
      const uint32_t c = c_sh;
      if (lane == 0)
        for (uint32_t e = E; e < c; ++e) {
          if (!tc::mbar_wait(&tfull_bar[e & 1], (e >> 1) & 1, prm.timeout, nullptr)) break;
          tc::mbar_arrive(&tempty_bar[e & 1]);
        }
      __syncwarp();
      E = c;
    }
    if (threadIdx.x == 0) {
      stop_flag = 0;
      p_issued = 0;
      p_done = 0;
      quit_sh = *(volatile int*)prm.timeout;
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (quit_sh) break;
  }
  // teardown: every MMA this CTA issued, and every TMA load (a block that stopped early may
  // leave loads that no MMA consumed), completes before TMEM is freed and the CTA exits
  if (warp == 1 && lane == 0) tc::umma_commit(&done_bar);
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    if (lane == 0) {
      tc::mbar_wait_drain(&done_bar, 0);
      for (uint32_t s = 0; s < STAGES && s < P; ++s) {
        const uint32_t issued = P / STAGES + (s < P % STAGES ? 1u : 0u);   // loads on stage s
        tc::mbar_wait_drain(&full_bar[s], (issued - 1) & 1);
      }
    }
    __syncwarp();
    tc::tc_fence_after();
    tc::tmem_dealloc(tbase, kTmemCols);
  }
}

// Positions (in the cut-sorted rows) of the rows whose flag is set, in ascending order,
// so that the next phase's list stays sorted by cut: per-block counts, then each block
// places its rows after those of the blocks before it.
constexpr int kCompactPer = 8192;   // rows per block: 8 consecutive rows per thread

__device__ __forceinline__ int32_t block_sum_1024(int32_t v, int32_t* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int32_t t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __syncthreads();
  return t;
}

__device__ __forceinline__ uint32_t flags8(const uint8_t* __restrict__ flags, int64_t r, int64_t ns) {
  uint32_t m = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) m |= (r + i < ns && flags[r + i]) ? 1u << i : 0u;
  return m;
}

__global__ void __launch_bounds__(1024) flag_count_kernel(const uint8_t* __restrict__ flags,
                                                          const unsigned long long* __restrict__ count, int64_t cap,
                                                          int32_t* __restrict__ bcount) {
  __shared__ int32_t sh[32];
  const int64_t ns = block_count(count, cap);
  const int64_t r = (int64_t)blockIdx.x * kCompactPer + threadIdx.x * 8;
  const int32_t c = block_sum_1024(__popc(flags8(flags, r, ns)), sh);
  if (threadIdx.x == 0) bcount[blockIdx.x] = c;
}

__global__ void __launch_bounds__(1024) flag_scatter_kernel(const uint8_t* __restrict__ flags,
                                                            const unsigned long long* __restrict__ count,
                                                            int64_t cap, const int32_t* __restrict__ bcount,
                                                            int32_t* __restrict__ list,
                                                            unsigned long long* __restrict__ list_count) {
  __shared__ int32_t sh[32];
  const int64_t ns = block_count(count, cap);
  int32_t before = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) before += bcount[b];
  before = block_sum_1024(before, sh);
  const int64_t r = (int64_t)blockIdx.x * kCompactPer + threadIdx.x * 8;
  const uint32_t m = flags8(flags, r, ns);
  // exclusive scan of the per-thread counts over the block
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t c = __popc(m);
  int32_t x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t t = sh[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sh[lane] = t;
  }
  __syncthreads();
  int32_t pos = before + x - c + (w > 0 ? sh[w - 1] : 0);
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if ((m >> i) & 1u) list[pos++] = (int32_t)(r + i);
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *list_count = (unsigned long long)(before + sh[31]);
}

// FP32 inner product of two padded rows (dp a multiple of 4, 16-byte aligned): four
// partial sums over float4 loads.  Its error is within gamma_d sum |u_i p_i| whatever the
// order of the additions.
__device__ __forceinline__ float dot32_rows(const float* __restrict__ u, const float* __restrict__ p, int dp) {
  const float4* u4 = reinterpret_cast<const float4*>(u);
  const float4* p4 = reinterpret_cast<const float4*>(p);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 4
  for (int c = 0; c < dp / 4; ++c) {
    const float4 a = u4[c], b = p4[c];
    s0 = fmaf(a.x, b.x, s0);
    s1 = fmaf(a.y, b.y, s1);
    s2 = fmaf(a.z, b.z, s2);
    s3 = fmaf(a.w, b.w, s3);
  }
  return (s0 + s1) + (s2 + s3);
}

// Whether two rows hold the same d floats bit for bit.  An item equal to the query
// vector scores exactly <u,q>, which is not above it: no double-precision score needed.
__device__ __forceinline__ bool same_vector(const float* __restrict__ a, const float* __restrict__ b, int d) {
  bool eq = true;
  int i = 0;
  for (; i + 4 <= d; i += 4) {
    const uint4 x = *reinterpret_cast<const uint4*>(a + i), y = *reinterpret_cast<const uint4*>(b + i);
    eq &= x.x == y.x && x.y == y.y && x.z == y.z && x.w == y.w;
  }
  for (; i < d; ++i) eq &= __float_as_uint(a[i]) == __float_as_uint(b[i]);
  return eq;
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
  // 32 rows per warp step: statuses and "yes" rows lane-parallel, rows with band items
  // (or a whole-row re-scan) one after another with the whole warp
  for (int64_t r0 = gw * 32; r0 < nrows; r0 += nw * 32) {
    const int64_t rl = r0 + lane;
    const int32_t st_l = rl < nrows ? status[rl] : (int32_t)ROW_NO;
    if (st_l == ROW_YES) {
      const Survivor S = rows[rl];
      const int32_t id = uid[S.upos];
      set_answer(bitmap, words, S.j, id);
    }
    uint32_t open = __ballot_sync(0xffffffffu, st_l == ROW_BAND || st_l == ROW_FULL);
    while (open) {
      const int src = __ffs(open) - 1;
      open &= open - 1;
      const int64_t r = r0 + src;
      const int32_t st = __shfl_sync(0xffffffffu, st_l, src);
      const Survivor S = rows[r];
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
          const float s = dot32_rows(u, p, dp);
          const float ep = __fmul_ru(gnu, pnorm[it]) + 1e-30f;
          if (__fsub_rd(s, ep) > hi) gt = true;
          else amb = __fadd_ru(s, ep) > lo && !same_vector(p, Qd + (int64_t)S.j * dp, d);
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
            const float s = dot32_rows(u, p, dp);
            const float ep = __fmul_ru(gnu, pnorm[i]) + 1e-30f;
            if (__fsub_rd(s, ep) > hi) gt = true;
            else amb = __fadd_ru(s, ep) > lo && !same_vector(p, Qd + (int64_t)S.j * dp, d);
          }
          need64(__any_sync(0xffffffffu, amb));
          if (amb) gt = dot64_seq(u, p, d) > s64q;
          c += __popc(__ballot_sync(0xffffffffu, gt));
          scanned += 32;
        }
        ++fp64;
      }
      if (c < k && lane == 0) {
        const int32_t id = uid[S.upos];
        set_answer(bitmap, words, S.j, id);
      }
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

__global__ void e4m3_rows_kernel(const float* __restrict__ X, int64_t rows, int dp, int d, uint8_t* __restrict__ out,
                                 float* __restrict__ scale) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  float x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = lane * 4 + q;
    x[q] = e < d ? X[r * dp + e] : 0.f;
  }
  float mx = fmaxf(fmaxf(fabsf(x[0]), fabsf(x[1])), fmaxf(fabsf(x[2]), fabsf(x[3])));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float inv = mx > 0.f ? 448.f / mx : 0.f;
  uint32_t packed = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_fp8_e4m3 v(x[q] * inv);
    packed |= (uint32_t)v.__x << (8 * q);
  }
  reinterpret_cast<uint32_t*>(out + r * 128)[lane] = packed;
  if (lane == 0) scale[r] = mx / 448.f;
}

}  // namespace

void launch_e4m3_rows(const float* X, int64_t rows, int dp, int d, uint8_t* out, float* scale, cudaStream_t st) {
  if (rows > 0) e4m3_rows_kernel<<<grid_for(rows, 8), 256, 0, st>>>(X, rows, dp, d, out, scale);
}

sah_status build_fp8_users(Index* ix, cudaStream_t st) {
  if (ix->d > 128 || ix->m_nz == 0) return SAH_OK;
  SAH_TRY(dev_alloc(ix, (void**)&ix->U8, (size_t)ix->m_nz * 128));
  SAH_TRY(dev_alloc(ix, (void**)&ix->usc, sizeof(float) * (size_t)ix->m_nz));
  launch_e4m3_rows(ix->Ut, ix->m_nz, ix->dp, ix->d, ix->U8, ix->usc, st);
  SAH_CUDA(cudaGetLastError());
  auto encode = get_encode_fn();
  if (!encode) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return SAH_ERR_UNSUPPORTED;
  }
  cuuint64_t dims[2] = {128, (cuuint64_t)ix->m_nz};
  cuuint64_t strides[1] = {128};
  cuuint32_t box[2] = {128, 128};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(&ix->tmap_U8, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, ix->U8, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (E4M3 users) failed with code " + std::to_string((int)r));
    return SAH_ERR_CUDA;
  }
  return SAH_OK;
}

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
  const int64_t nbc = (ns + kCompactPer - 1) / kCompactPer;
  const size_t o_flags = take(ns), o_lists = take(sizeof(int32_t) * 2 * ns), o_bcount = take(sizeof(int32_t) * nbc),
               o_lcount = take(sizeof(unsigned long long) * 2);
  if (cx->tcws.bytes < need) {
    SAH_CUDA(cudaStreamSynchronize(st));
    if (cx->tcws.base) cudaFree(cx->tcws.base);
    cx->tcws.base = nullptr;
    cx->tcws.bytes = 0;
    ++cx->alloc_epoch;
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
  uint8_t* flags = (uint8_t*)(w + o_flags);
  int32_t* lists = (int32_t*)(w + o_lists);
  int32_t* bcount = (int32_t*)(w + o_bcount);
  unsigned long long* lcount = (unsigned long long*)(w + o_lcount);

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
  prm.flags = flags;
  prm.inject_stall = ix->inject_site == SAH_INJECT_VERIFY ? 1 : 0;
  // Two phases of the scan over item tiles, [0,8) and [8, end): rows still open after the
  // first go on, compacted, to the second, so that its (longer) CTAs hold only rows that
  // still need the items.  Every phase boundary costs a fill and drain of the CTAs and
  // the gather of their rows: with more phases ([4,8,16,32] was tried) that cost exceeds
  // the saving.  With exact thresholds (|P'| = n) the user pass decides nearly every pair,
  // the list is short or empty, and one phase costs fewer launches.
  std::vector<int> bounds{0};
  if (!ix->l_exact && 8 < ntiles) bounds.push_back(8);
  bounds.push_back(ntiles);
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ix->device);
  // persistent CTAs (two per SM when they fit), each over several row blocks
  const unsigned grid = (unsigned)std::min<int64_t>(grid_for(ns, kRows), (ix->dk == 64 ? 2 : 1) * (int64_t)nsm);
  if (ev) SAH_CUDA(cudaEventRecord(ev[0], st));
  int nlaunch = 0;
  for (size_t ph = 0; ph + 1 < bounds.size(); ++ph) {
    prm.t_begin = bounds[ph];
    prm.t_end = bounds[ph + 1];
    prm.list = ph == 0 ? nullptr : lists + (ph & 1) * ns;
    prm.nrows_dev = ph == 0 ? count_dev : lcount + (ph & 1);
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
    ++nlaunch;
    if (ph + 2 < bounds.size()) {
      const int nx = (int)((ph + 1) & 1);
      flag_count_kernel<<<(unsigned)nbc, 1024, 0, st>>>(flags, count_dev, ns, bcount);
      flag_scatter_kernel<<<(unsigned)nbc, 1024, 0, st>>>(flags, count_dev, ns, bcount, lists + nx * ns,
                                                          lcount + nx);
      SAH_CUDA(cudaGetLastError());
      nlaunch += 2;
    }
  }
  if (ev) SAH_CUDA(cudaEventRecord(ev[1], st));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
  resolve_kernel<<<sms * 8, 256, 0, st>>>(rows, count_dev, ns, status, cert, band, items, ix->Ut, ix->unorm, ix->uid, ix->Ps,
                                          ix->pnorm, ix->n, ix->d, ix->dp, Qd, qn, kk, ix->gamma, bitmap, words,
                                          stats + stat_fp64, stats + stat_items);
  SAH_CUDA(cudaGetLastError());
  if (launches) *launches += 4 + nlaunch;
  return SAH_OK;
}

}  // namespace sah
