// Tensor-core user pass (A4, with A8's batched score): S = U . Q^T for the batch's queries
// over every user tile, on tcgen05, consumed in the epilogue by the A4 tests and never
// written out.
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
// Tests per (user, query) whose leaf the node-level bound (Lemma 2) kept, with L = L_u^k,
// E the error of L, and the band e = c_tc ||u|| ||q||:
//   s + e <  L - E                                            -> "no" (k items beat <u,q>)
//   s - e >= L + E, when L is the exact k-th score (|P'| = n)  -> "yes"
//   s - e >= ||u|| ||p_k|| (1 + 2 gamma)                       -> "yes" (Alg. 5)
//   otherwise the pair is re-scored in FP32 (and in FP64 against the exact threshold) by
//   pair_rescore_kernel, which lists what stays open for the kMIPS decision.
// Lemma 3 (the vector-level bound) is not applied here: with the score coming from the
// tensor cores it would cost more than it saves.
//
// Kernel shape: persistent, one CTA per SM, 320 threads.  Warp 0 streams 128-user tiles
// (hi and lo K-blocks) through a TMA ring, warp 1 issues the MMAs into two TMEM
// accumulators in turn, and two groups of four epilogue warps (2-5, 6-9) take the tiles
// of accumulator 0 and 1.  The launch's queries (up to 256) stay in shared memory for the
// whole launch.  An epilogue warp (one user per lane) keeps, per tile, its users' lower
// bounds for the launch's distinct k in shared memory and reads its TMEM lanes 32 columns
// at a time: one fused multiply-add and one compare per column mark the pairs the "no"
// test cannot settle; those of kept (leaf, query) pairs take the full tests.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cmath>

#include "sah_internal.cuh"
#include "tc.cuh"

namespace sah {
namespace {

constexpr int kUM = 128;          // users per tile (UMMA M)
constexpr int kUThreads = 320;    // warp 0 TMA producer, warp 1 MMA issuer, warps 2-9 epilogue
constexpr int kEpiWarps = 8;
constexpr int kMaxTileList = 1024;
constexpr int kHalf = 128;           // accumulator columns per half   // needed tiles per CTA and launch (the host splits longer ranges)

struct ColInfo {
  float qn;        // ||q||
  float pk;        // ||p_k|| (-inf past n)
  int32_t krow;    // k - 1 when k <= k_max (the row of L), else -1
  int32_t j;       // query row in the sub-batch, bit 30: SA-ALSH row
};

struct UpParams {
  int64_t mz, n;
  int kmax, l_exact, dk;
  int j0, nn, N;               // this launch's query rows [j0, j0 + nn); MMA N = roundup(nn, 16)
  int slot_cap;                // lower-bound rows kept in shared memory per warp (<= k_max)
  int mask_words;              // words per leaf in kept_mask (the whole sub-batch)
  int ntiles;                  // tiles of all users (tile_need covers them all)
  int tile0, tile_end;         // this launch's tile range
  const uint16_t* Qhi;         // nq x dk
  const uint16_t* Qlo;
  const float* qn;
  const int32_t* kk;
  const int32_t* modes;
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
  int st_scored, st_yes;
  int* timeout;
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
  static constexpr uint32_t kBPart = NMAX * 128;           // one K-block of the queries
  static constexpr size_t kOperands = (size_t)STAGES * kStage + 2 * KB * (size_t)kBPart;
  static constexpr int kWords = NMAX / 32;                 // kept-bit words per launch
  // + per epilogue warp: (slots + 2) x 32 lower bounds and kWords x 32 kept words
  static constexpr size_t bytes(int slots) {
    return 1024 + kOperands + (size_t)kEpiWarps * 32 * 4 * ((size_t)slots + 2 + kWords);
  }
  static constexpr uint32_t kTmemCols = 2 * NMAX <= 256 ? 256 : 512;
  static constexpr uint32_t kAccStride = kTmemCols / 2;
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
  __shared__ ColInfo cols[NMAX];
  __shared__ __align__(16) float2 cq[NMAX];                       // per column: ||q||, row offset in a warp's bound table
  __shared__ int32_t kseen[65], kslot[65], klist[64], nsl_sh;
  __shared__ int32_t tlist[kMaxTileList];           // this CTA's needed tiles, in order
  __shared__ int32_t ntl_sh;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;                               // [STAGES][hi kb.. | lo kb..]
  uint8_t* sB = base + STAGES * S::kStage;          // [hi kb.. | lo kb..]
  // per epilogue warp: [slot_cap + 2][32] lower bounds (row slot_cap -inf, row slot_cap + 1
  // +inf), [kWords][32] kept words
  float* Lsm = reinterpret_cast<float*>(base + S::kOperands);
  uint32_t* Ksm = reinterpret_cast<uint32_t*>(Lsm + kEpiWarps * 32 * (p.slot_cap + 2));
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
    tc::mbar_init(&done_bar, 2);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_sh, S::kTmemCols);
    tc::tmem_relinquish();
    // the CTA's tiles of the range that hold a user of a kept leaf
    int cnt = 0;
    for (int base = 0;; base += 32) {
      const int64_t t = (int64_t)p.tile0 + blockIdx.x + (int64_t)(base + lane) * gridDim.x;
      if ((int64_t)p.tile0 + blockIdx.x + (int64_t)base * gridDim.x >= p.tile_end) break;
      const bool f = t < p.tile_end && p.tile_need[t];
      const unsigned m = __ballot_sync(0xffffffffu, f);
      const int pos = cnt + __popc(m & ((1u << lane) - 1u));
      if (f && pos < kMaxTileList) tlist[pos] = (int32_t)t;
      cnt += __popc(m);
    }
    if (lane == 0) ntl_sh = cnt < kMaxTileList ? cnt : kMaxTileList;
  }
  // the distinct k <= k_max among the launch's queries (their lower-bound rows are
  // prefetched a tile ahead)
  for (int k = tid; k <= 64; k += kUThreads) kseen[k] = 0;
  __syncthreads();
  for (int c = tid; c < p.nn; c += kUThreads) {
    const int k = p.kk[p.j0 + c];
    if (k >= 1 && k <= p.kmax) kseen[k] = 1;
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
  // the launch's queries: per-column records and the hi / lo operand rows (zero past nn)
  for (int c = tid; c < NMAX; c += kUThreads) {
    ColInfo ci{0.f, -INFINITY, -1, 0};
    if (c < p.nn) {
      const int j = p.j0 + c;
      const int k = p.kk[j];
      const int sa = (p.modes != nullptr && p.modes[j] == SAH_SAALSH && k <= p.kmax) ? 1 : 0;
      ci.qn = p.qn[j];
      ci.pk = (k >= 1 && k <= p.n) ? p.pnorm[k - 1] : -INFINITY;
      ci.krow = (k >= 1 && k <= p.kmax) ? k - 1 : -1;
      ci.j = j | (sa << 30);
    }
    cols[c] = ci;
    // columns without a bound row in the table (k > k_max, past the cap) point at the -inf
    // row: every pair of theirs takes the full tests; columns past nn at the +inf row
    const int sl = (c < p.nn && ci.krow >= 0) ? kslot[ci.krow + 1] : -1;
    const int row = c >= p.nn ? p.slot_cap + 1 : (sl >= 0 ? sl : p.slot_cap);
    cq[c] = make_float2(ci.qn, __int_as_float(32 * row));
  }
  for (int i = tid; i < p.N * KB * 8; i += kUThreads) {
    const int rr = i / (KB * 8), rem = i % (KB * 8), kb = rem / 8, ch = rem % 8;
    uint4 hi = make_uint4(0u, 0u, 0u, 0u), lo = hi;
    if (rr < p.nn) {
      const int64_t off = (int64_t)(p.j0 + rr) * p.dk + kb * 64 + ch * 8;
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

  if (warp == 0) {
    if (lane < 2) {   // TMA producers, lane g for the tiles of epilogue group g
      if (lane == 0) {
        tc::prefetch_tensormap(&tmapUhi);
        tc::prefetch_tensormap(&tmapUlo);
      }
      const int ntl = ntl_sh;
      for (int it = lane; it < ntl; it += 2) {
        const int t = tlist[it];
        const int s = it % STAGES;
        if (it >= STAGES && !tc::mbar_wait(&empty_bar[s], ((it / STAGES) & 1) ^ 1, p.timeout, nullptr)) break;
        tc::mbar_arrive_expect_tx(&full_bar[s], S::kStage);
        uint8_t* dst = sA + s * S::kStage;
        for (int kb = 0; kb < KB; ++kb) {
          tc::tma_load_2d(dst + kb * S::kTile, &tmapUhi, &full_bar[s], kb * 64, t * kUM);
          tc::tma_load_2d(dst + (KB + kb) * S::kTile, &tmapUlo, &full_bar[s], kb * 64, t * kUM);
        }
      }
    }
  } else if (warp == 1) {
    if (lane < 2) {   // MMA issuers, lane g: hi.hi + hi.lo + lo.hi into accumulator g, by halves
      const int H = p.N > kHalf ? 2 : 1;
      const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
      const int ntl = ntl_sh;
      bool ok = true;
      for (int it = lane; ok && it < ntl; it += 2) {
        const int s = it % STAGES, a = lane;
        if (!tc::mbar_wait(&full_bar[s], (it / STAGES) & 1, p.timeout, nullptr)) break;
        const uint32_t aS = a0 + s * S::kStage;
        for (int h = 0; h < H; ++h) {
          if (it >= 2 && !tc::mbar_wait(&tempty_bar[a][h], ((it >> 1) & 1) ^ 1, p.timeout, nullptr)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const int nh = h == 0 ? (p.N < kHalf ? p.N : kHalf) : p.N - kHalf;
          const uint32_t idesc = tc::idesc_bf16_f32(kUM, (uint32_t)nh);
          const uint32_t d = tbase + a * S::kAccStride + h * kHalf;
          const uint32_t bh = b0 + h * kHalf * 128;   // rows 128 h.. of each B part
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
          tc::umma_commit(&tfull_bar[a][h]);
        }
        if (ok) tc::umma_commit(&empty_bar[s]);
      }
      tc::umma_commit(&done_bar);
    }
  } else {
    // epilogue: two groups of four warps take alternate tiles (accumulator g = it & 1); a
    // warp reads TMEM lane quadrant warp & 3, one user per lane
    const int ew = warp - 2, g = ew >> 2, quad = warp & 3;
    const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
    const int w0 = p.j0 >> 5, wc = (p.nn + 31) >> 5;
    const int H = p.N > kHalf ? 2 : 1;
    const uint32_t tail = (p.nn & 31) ? ((1u << (p.nn & 31)) - 1u) : 0xffffffffu;
    const int inf_row = 32 * p.slot_cap;
    float* Lw = Lsm + ew * 32 * (p.slot_cap + 2);
    uint32_t* Kw = Ksm + ew * 32 * S::kWords;   // kept words of the tile; then its open pairs
    Lw[inf_row + lane] = -INFINITY;
    Lw[inf_row + 32 + lane] = INFINITY;
    const int nsl = nsl_sh, ntl = ntl_sh;
    // Values of the group's next tile travel in registers, loaded while the current tile is
    // processed: per user its leaf, norm, bound error and id, the lower bounds of the first
    // kPre distinct k, and (once the leaf is known) its leaf's kept-query words.
    constexpr int kPre = 8;
    int Bu_n = 0, id_n = 0;
    float nu_n = 0.f, E_n = 0.f;
    float L_n[kPre];
    uint4 K_lo = make_uint4(0u, 0u, 0u, 0u), K_hi = K_lo;   // kept words 0-3 and 4-7
    auto load_user = [&](int idx) {
      Bu_n = 0;
      id_n = 0;
      nu_n = 0.f;
      E_n = 0.f;
#pragma unroll
      for (int j = 0; j < kPre; ++j) L_n[j] = 0.f;
      if (idx < ntl) {
        const int64_t rr = (int64_t)tlist[idx] * kUM + quad * 32 + lane;
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
    auto load_words = [&](int idx) {
      const bool ok = idx < ntl && (int64_t)tlist[idx] * kUM + quad * 32 + lane < p.mz;
      const uint32_t* km = p.kept_mask + (int64_t)Bu_n * p.mask_words + w0;
      K_lo.x = (ok && 0 < wc) ? __ldg(km + 0) : 0u;
      K_lo.y = (ok && 1 < wc) ? __ldg(km + 1) : 0u;
      K_lo.z = (ok && 2 < wc) ? __ldg(km + 2) : 0u;
      K_lo.w = (ok && 3 < wc) ? __ldg(km + 3) : 0u;
      if (S::kWords > 4) {
        K_hi.x = (ok && 4 < wc) ? __ldg(km + 4) : 0u;
        K_hi.y = (ok && 5 < wc) ? __ldg(km + 5) : 0u;
        K_hi.z = (ok && 6 < wc) ? __ldg(km + 6) : 0u;
        K_hi.w = (ok && 7 < wc) ? __ldg(km + 7) : 0u;
      }
    };
    // open pairs of the previous tile (masks left in Kw) go to the re-score list after
    // the next wait; the list's slots were claimed with one atomic at the end of that tile
    int64_t r_prev = 0;
    int prev_excl = 0, prev_total = 0;
    unsigned long long prev_base = 0;
    auto emit_prev = [&]() {
      if (prev_total == 0) return;
      const unsigned long long base0 = __shfl_sync(0xffffffffu, prev_base, 31);
      unsigned long long slot = base0 + (unsigned long long)prev_excl;
      for (int w = 0; w < wc; ++w) {
        uint32_t om = Kw[32 * w + lane];
        while (om) {
          const int i = __ffs(om) - 1;
          om &= om - 1;
          if ((int64_t)slot < p.resc_cap) p.resc[slot] = Survivor{(int32_t)r_prev, cols[32 * w + i].j, 0.f};
          ++slot;
        }
      }
      prev_total = 0;
    };
    load_user(g);
    load_words(g);
    unsigned long long scored = 0, yes_cnt = 0;
    bool failed = false;
    for (int it = g; it < ntl; it += 2) {
      const int a = g;
      const int64_t r = (int64_t)tlist[it] * kUM + quad * 32 + lane;
      const bool valid = r < p.mz;
      const int32_t id = id_n;
      const float nu = nu_n, E = E_n;
      const float cu = __fmul_ru(p.ctc, nu);
      const float nun = __fmul_ru(nu, 1.f + 2.f * p.gamma);
      const uint4 klo = K_lo, khi = K_hi;
      // this tile's lower bounds L - E (less the band's absolute slack) per distinct k
#pragma unroll
      for (int j = 0; j < kPre; ++j)
        if (j < nsl) Lw[32 * j + lane] = valid ? __fsub_rd(__fsub_rd(L_n[j], E), 1e-30f) : INFINITY;
      for (int sl = kPre; sl < nsl; ++sl) {
        float Llo = INFINITY;
        if (valid) Llo = __fsub_rd(__fsub_rd(__ldg(&p.Lt[(int64_t)(klist[sl] - 1) * p.mz + r]), E), 1e-30f);
        Lw[32 * sl + lane] = Llo;
      }
      const uint32_t acc_addr = tbase + lane_addr + a * S::kAccStride;
      int open_cnt = 0;
      for (int h = 0; h < H; ++h) {
        if (!tc::mbar_wait(&tfull_bar[a][h], (it >> 1) & 1, p.timeout, nullptr)) {
          failed = true;
          break;
        }
        tc::tc_fence_after();
        if (h == 0) {
          // the previous tile's open pairs, then this tile's kept words, then the next
          // tile's values start loading
          emit_prev();
#pragma unroll
          for (int w = 0; w < S::kWords; ++w) {
            const uint32_t kv = w == 0 ? klo.x : w == 1 ? klo.y : w == 2 ? klo.z : w == 3 ? klo.w
                              : w == 4 ? khi.x : w == 5 ? khi.y : w == 6 ? khi.z : khi.w;
            if (w < wc) Kw[32 * w + lane] = (w == wc - 1) ? (kv & tail) : kv;
          }
          __syncwarp();
          load_user(it + 2);
        }
        const int wend = h + 1 < H ? 4 * (h + 1) : wc;
        for (int w = 4 * h; w < wend; ++w) {
          const uint32_t kw = Kw[32 * w + lane];
          Kw[32 * w + lane] = 0u;
          if (!__any_sync(0xffffffffu, kw)) continue;
          scored += __popc(kw);
          float v[32];
          tmem_ld32_wait(acc_addr + 32 * w, v);
          // "no" unless s + c_tc ||u|| ||q|| (rounded up) reaches L - E, for any column
          bool any = false;
#pragma unroll
          for (int i = 0; i < 32; i += 2) {
            const float4 c4 = *reinterpret_cast<const float4*>(&cq[32 * w + i]);
            any |= __fmaf_ru(cu, c4.x, v[i]) >= Lw[__float_as_int(c4.y) + lane];
            any |= __fmaf_ru(cu, c4.z, v[i + 1]) >= Lw[__float_as_int(c4.w) + lane];
          }
          if (!__any_sync(0xffffffffu, any)) continue;
          // which kept columns
          uint32_t cand = 0;
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float2 c2 = cq[32 * w + i];
            cand |= (__fmaf_ru(cu, c2.x, v[i]) >= Lw[__float_as_int(c2.y) + lane] ? 1u : 0u) << i;
          }
          cand &= kw;
          if (!__any_sync(0xffffffffu, cand)) continue;
          // the "yes" tests of the FP32 user pass with the tensor-core band, one candidate
          // column at a time.  L + E is bounded above from the table's L - E - 1e-30
          // (rounded down) with four units in the last place and 2e-30 to spare.
          uint32_t open_m = 0;
          uint32_t uni = __reduce_or_sync(0xffffffffu, cand);
          while (uni) {
            const int i = __ffs(uni) - 1;
            uni &= uni - 1;
            const float sv = tmem_ld1_wait(acc_addr + 32 * w + i);   // the whole warp reads column i
            if (!((cand >> i) & 1u)) continue;
            const ColInfo ci = cols[32 * w + i];
            const int off = __float_as_int(cq[32 * w + i].y);
            const float lo = __fsub_rd(sv, __fmul_ru(cu, ci.qn) + 1e-30f);
            bool yes = lo >= __fmul_ru(nun, ci.pk);
            if (!yes && p.l_exact && ci.krow >= 0) {
              float Lhi;
              if (off != inf_row) {
                const float Lq = Lw[off + lane];
                Lhi = Lq == -INFINITY ? INFINITY
                                      : __fadd_ru(__fadd_ru(Lq, 2.f * E), __fmaf_ru(fabsf(Lq), 0x1p-21f, 2e-30f));
              } else {
                Lhi = __fadd_ru(__ldg(&p.Lt[(int64_t)ci.krow * p.mz + r]), E);   // past the table's cap
              }
              yes = lo >= Lhi;
            }
            if (yes) {
              ++yes_cnt;
              atomicOr(&p.bitmap[(int64_t)(ci.j & 0x3fffffff) * p.words + (id >> 5)], 1u << (id & 31));
            } else {
              open_m |= 1u << i;
            }
          }
          Kw[32 * w + lane] = open_m;
          open_cnt += __popc(open_m);
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&tempty_bar[a][h]);
      }
      if (failed) break;
      // claim the re-score slots of this tile's open pairs (written after the next wait)
      int incl = open_cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
      }
      prev_total = __shfl_sync(0xffffffffu, incl, 31);
      prev_excl = incl - open_cnt;
      r_prev = r;
      if (prev_total && lane == 31) prev_base = atomicAdd(p.resc_count, (unsigned long long)prev_total);
      load_words(it + 2);
    }
    if (!failed) emit_prev();
    for (int o = 16; o > 0; o >>= 1) {
      scored += __shfl_xor_sync(0xffffffffu, scored, o);
      yes_cnt += __shfl_xor_sync(0xffffffffu, yes_cnt, o);
    }
    if (lane == 0) {
      if (scored) atomicAdd(&p.stats[p.st_scored], scored);
      if (yes_cnt) atomicAdd(&p.stats[p.st_yes], yes_cnt);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    if (lane == 0) tc::mbar_wait(&done_bar, 0, p.timeout, nullptr);
    __syncwarp();
    tc::tc_fence_after();
    tc::tmem_dealloc(tbase, S::kTmemCols);
  }
}

// Which 128-user tiles hold a user of a leaf with a kept pair among the launch's queries
// (one warp per tile).
__global__ void tile_need_kernel(const int32_t* __restrict__ ublock, int64_t mz,
                                 const uint32_t* __restrict__ kept_mask, int mask_words, int w0, int wc,
                                 int ntiles, uint8_t* __restrict__ need) {
  const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (t >= ntiles) return;
  const int64_t r0 = (int64_t)t * kUM;
  const int64_t r1 = (r0 + kUM < mz ? r0 + kUM : mz) - 1;
  const int Bf = ublock[r0], Bl = ublock[r1];
  bool any = false;
  for (int64_t i = lane; i < (int64_t)(Bl - Bf + 1) * wc; i += 32) {
    const int64_t B = Bf + i / wc;
    const int w = (int)(i % wc);
    any |= kept_mask[B * mask_words + w0 + w] != 0u;
  }
  any = __any_sync(0xffffffffu, any);
  if (lane == 0) need[t] = any ? 1 : 0;
}

// FP32 re-score of the pairs the tensor-core band left open; the same decisions as the
// FP32 user pass.  Grid-stride, one thread per pair.
__global__ void pair_rescore_kernel(const Survivor* __restrict__ pairs, const unsigned long long* __restrict__ count,
                                    int64_t cap, const float* __restrict__ Ut, const float* __restrict__ unorm,
                                    const int32_t* __restrict__ uid, const float* __restrict__ Lt,
                                    const float* __restrict__ Eu, const float* __restrict__ pnorm, int64_t n,
                                    int64_t mz, int kmax, int l_exact, int d, int dp, const float* __restrict__ Qd,
                                    const float* __restrict__ qn, const int32_t* __restrict__ kk, float gamma,
                                    const double* __restrict__ T64, uint32_t* __restrict__ bitmap, int64_t words,
                                    Survivor* __restrict__ surv, unsigned long long* __restrict__ surv_count,
                                    int64_t surv_cap, unsigned long long* __restrict__ stats, int st_yes,
                                    int st_fp64, int nq, const int* __restrict__ timeout) {
  // after a timed-out wait of the pass the list may hold unwritten entries: nothing is read
  if (*(volatile const int*)timeout) return;
  const int64_t total = min((int64_t)*count, cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const Survivor P = pairs[i];
    const int r = P.upos;
    const int j = P.j & 0x3fffffff;
    if (r < 0 || r >= mz || j >= nq) continue;
    const bool sa_row = (P.j >> 30) & 1;
    const int k = kk[j];
    const float4* u4 = reinterpret_cast<const float4*>(Ut + (int64_t)r * dp);
    const float4* q4 = reinterpret_cast<const float4*>(Qd + (int64_t)j * dp);
    float acc = 0.f;
    for (int c = 0; c < dp / 4; ++c) {
      const float4 a = u4[c], b = q4[c];
      acc = fmaf(a.x, b.x, acc);
      acc = fmaf(a.y, b.y, acc);
      acc = fmaf(a.z, b.z, acc);
      acc = fmaf(a.w, b.w, acc);
    }
    const float nu = unorm[r], E = Eu[r];
    const float L = (k <= kmax) ? Lt[(int64_t)(k - 1) * mz + r] : -INFINITY;
    const float Llo = (L == -INFINITY) ? -INFINITY : __fsub_rd(L, E);
    const float eq = __fmul_ru(__fmul_ru(gamma, nu), qn[j]) + 1e-30f;
    const float hi = __fadd_ru(acc, eq), lo = __fsub_rd(acc, eq);
    bool yes = false, surv_flag = false;
    if (hi < Llo) {
    } else if (l_exact && k <= kmax && lo >= __fadd_ru(L, E)) {
      yes = true;
    } else if (lo >= __fmul_ru(__fmul_ru(nu, pnorm[k - 1]), 1.f + 2.f * gamma)) {
      yes = true;
    } else if (T64 != nullptr && k <= kmax && !sa_row) {
      const double t64 = T64[(int64_t)(k - 1) * mz + r];
      if (t64 == t64) {
        atomicAdd(&stats[st_fp64], 1ull);
        yes = dot64_seq(Ut + (int64_t)r * dp, Qd + (int64_t)j * dp, d) >= t64;
      } else {
        surv_flag = true;
      }
    } else {
      surv_flag = true;
    }
    if (yes) {
      const int32_t id = uid[r];
      atomicOr(&bitmap[(int64_t)j * words + (id >> 5)], 1u << (id & 31));
      atomicAdd(&stats[st_yes], 1ull);
    } else if (surv_flag) {
      const unsigned long long slot = atomicAdd(surv_count + (sa_row ? 1 : 0), 1ull);
      if ((int64_t)slot < surv_cap) surv[(sa_row ? surv_cap : 0) + slot] = Survivor{r, j, acc};
    }
  }
}

// hi = bf16(x), lo = bf16(x - hi) of the queries, K padded to dk with zeros
__global__ void split_queries_kernel(const float* __restrict__ Qd, int nq, int d, int dp, int dk,
                                     uint16_t* __restrict__ Qhi, uint16_t* __restrict__ Qlo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nq * dk) return;
  const int64_t j = i / dk;
  const int c = (int)(i % dk);
  const float v = c < d ? Qd[j * dp + c] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
  Qhi[i] = __bfloat16_as_ushort(h);
  Qlo[i] = __bfloat16_as_ushort(l);
}

inline unsigned grid_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

template <int KB, int STAGES, int NMAX>
sah_status launch_chunks(Index* ix, UpParams p, int nq, uint8_t* tile_need, int sms, cudaStream_t st,
                         int* launches) {
  using S = UpSmem<KB, STAGES, NMAX>;
  auto fn = user_pass_tc_kernel<KB, STAGES, NMAX>;
  p.slot_cap = std::min(ix->kmax, KB == 1 ? 64 : 48);   // what shared memory holds
  const size_t smem = S::bytes(p.slot_cap);
  SAH_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)std::max(1, std::min(p.ntiles, sms));
  const int64_t seg = (int64_t)kMaxTileList * grid;   // tiles per launch: at most kMaxTileList per CTA
  for (int j0 = 0; j0 < nq; j0 += NMAX) {
    p.j0 = j0;
    p.nn = std::min(NMAX, nq - j0);
    p.N = (p.nn + 15) & ~15;
    tile_need_kernel<<<grid_for(p.ntiles, 8), 256, 0, st>>>(ix->ublock, ix->m_nz, p.kept_mask, p.mask_words,
                                                            j0 >> 5, (p.nn + 31) >> 5, p.ntiles, tile_need);
    if (launches) *launches += 1;
    for (int64_t t0 = 0; t0 < p.ntiles; t0 += seg) {
      p.tile0 = (int)t0;
      p.tile_end = (int)std::min<int64_t>(p.ntiles, t0 + seg);
      fn<<<grid, kUThreads, smem, st>>>(ix->tmap_U, ix->tmap_Ulo, p);
      SAH_CUDA(cudaGetLastError());
      if (launches) *launches += 1;
    }
  }
  return SAH_OK;
}

}  // namespace

sah_status run_user_pass_tc(Index* ix, const float* Qd, uint16_t* Qsplit, const float* qn, const int32_t* kk,
                            const int32_t* modes, int nq, const uint32_t* kept_mask, int mask_words,
                            uint8_t* tile_need, uint32_t* bitmap, int64_t words, Survivor* resc,
                            unsigned long long* resc_count, Survivor* surv, unsigned long long* surv_count,
                            int64_t surv_cap, unsigned long long* stats, int st_scored, int st_yes, int st_fp64,
                            cudaStream_t st, int* launches) {
  if (ix->m_nz == 0 || nq == 0 || ix->dk <= 0) return SAH_OK;
  uint16_t* Qhi = Qsplit;
  uint16_t* Qlo = Qsplit + (size_t)nq * ix->dk;
  split_queries_kernel<<<grid_for((int64_t)nq * ix->dk, 256), 256, 0, st>>>(Qd, nq, ix->d, ix->dp, ix->dk, Qhi,
                                                                           Qlo);
  SAH_CUDA(cudaGetLastError());
  if (launches) *launches += 1;
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
  p.Qhi = Qhi;
  p.Qlo = Qlo;
  p.qn = qn;
  p.kk = kk;
  p.modes = modes;
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
  p.st_scored = st_scored;
  p.st_yes = st_yes;
  p.timeout = ix->dev_timeout;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
  if (ix->dk == 64) {
    SAH_TRY((launch_chunks<1, 2, 256>(ix, p, nq, tile_need, sms, st, launches)));
  } else {
    SAH_TRY((launch_chunks<2, 2, 64>(ix, p, nq, tile_need, sms, st, launches)));
  }
  pair_rescore_kernel<<<sms * 4, 256, 0, st>>>(resc, resc_count, surv_cap, ix->Ut, ix->unorm, ix->uid, ix->Lt,
                                               ix->Eu, ix->pnorm, ix->n, ix->m_nz, ix->kmax, ix->l_exact ? 1 : 0,
                                               ix->d, ix->dp, Qd, qn, kk, ix->gamma, ix->T64, bitmap, words, surv,
                                               surv_count, surv_cap, stats, st_yes, st_fp64, nq, ix->dev_timeout);
  SAH_CUDA(cudaGetLastError());
  if (launches) *launches += 1;
  return SAH_OK;
}

}  // namespace sah
