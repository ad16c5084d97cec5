// Tensor-core kMIPS decision for the survivors of the user pass (A5 on tcgen05), and the
// boundary re-score of what its error band leaves open (A6).
//
// Per survivor row (u, q, <u,q>, k) the exact decision counts the items p with
// <u,p> > <u,q>, in descending norm order, stopping "no" at k items and stopping the
// scan once ||u|| ||p_i|| cannot reach <u,q> (the mu_j rule of Alg. 2; items are sorted
// by norm as in Alg. 1 and Alg. 4).  Here 128 survivors form the A operand of a
// 128 x 256 x K UMMA (BF16 in, FP32 accumulated in TMEM) and the items stream through
// TMA as the B operand.  The epilogue reads each row's scores from TMEM and, with the
// a-priori bound of BF16 rounding plus FP32 accumulation,
//     |s_bf - <u,p>| <= c_bf ||u|| ||p||,  c_bf = 1.01 (2^-7 + 2^-16 + (K + 8) 2^-23),
// counts items that are certainly above <u,q> and remembers the few it cannot separate.
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

constexpr int kTileN = 256;       // items per tile (UMMA N)
constexpr int kRows = 128;        // survivors per CTA (UMMA M)
constexpr int kBandCap = 32;      // band items remembered per row
constexpr int kThreads = 192;     // warp 0 TMA producer, warp 1 MMA issuer, warps 2-5 epilogue
constexpr uint32_t kTmemCols = 512;

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
__global__ void cut_kernel(const Survivor* __restrict__ surv, const unsigned long long* __restrict__ count,
                           int64_t cap, const float* __restrict__ unorm, const float* __restrict__ pnorm, int64_t n,
                           const float* __restrict__ qn, float gamma, int ntiles, int32_t* __restrict__ cut,
                           int32_t* __restrict__ hist) {
  const int64_t ns = block_count(count, cap);
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns) return;
  Survivor S = surv[i];
  float nu = unorm[S.upos];
  float eq = __fmul_ru(__fmul_ru(gamma, nu), qn[S.j]) + 1e-30f;
  float lo = __fsub_rd(S.sq, eq);
  float scale = __fmul_ru(nu, 1.f + 2.f * gamma);
  int a = 0, b = ntiles;   // first t in [0, ntiles] whose test holds (monotone in t)
  while (a < b) {
    int mid = (a + b) >> 1;
    if (__fmul_ru(scale, pnorm[(int64_t)mid * kTileN]) <= lo) b = mid;
    else a = mid + 1;
  }
  cut[i] = a;
  atomicAdd(&hist[a], 1);
}

__global__ void exclusive_scan_small_kernel(int32_t* __restrict__ v, int count) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int32_t acc = 0;
    for (int i = 0; i < count; ++i) {
      int32_t x = v[i];
      v[i] = acc;
      acc += x;
    }
  }
}

__global__ void sort_by_cut_kernel(const Survivor* __restrict__ surv, const int32_t* __restrict__ cut,
                                   const unsigned long long* __restrict__ count, int64_t cap,
                                   int32_t* __restrict__ off, Survivor* __restrict__ out_rows,
                                   int32_t* __restrict__ out_cut) {
  const int64_t ns = block_count(count, cap);
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns) return;
  int32_t c = cut[i];
  int32_t p = atomicAdd(&off[c], 1);
  out_rows[p] = surv[i];
  out_cut[p] = c;
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

template <int KB, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
verify_tc_kernel(const __grid_constant__ CUtensorMap tmapP, TcParams prm) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[2], tempty_bar[2], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int stop_flag, p_issued, p_done;

  constexpr uint32_t kABytes = kRows * 128;          // one 64-wide K block of A
  constexpr uint32_t kBBytes = kTileN * 128;         // one 64-wide K block of a B tile
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + KB * kABytes;

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
    stop_flag = 0;
    p_issued = 0;
    p_done = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_sh, kTmemCols);
    tc::tmem_relinquish();
  }
  // A operand: the CTA's survivor rows, gathered into the 128-byte-swizzled K-major layout
  for (int i = threadIdx.x; i < kRows * KB * 8; i += kThreads) {
    int r = i / (KB * 8), rem = i % (KB * 8), kb = rem / 8, c = rem % 8;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r < nrows_cta) {
      int64_t up = prm.rows[r0 + r].upos;
      v = *reinterpret_cast<const uint4*>(prm.Ub + up * prm.dk + kb * 64 + c * 8);
    }
    *reinterpret_cast<uint4*>(sA + kb * kABytes + tc::sw128_offset(r, c)) = v;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_base_sh;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      tc::prefetch_tensormap(&tmapP);
      int issued = 0;
      for (int t = 0; t < T; ++t) {
        const int s = t % STAGES;
        if (t >= STAGES && !tc::mbar_wait(&empty_bar[s], ((t / STAGES) & 1) ^ 1, prm.timeout, nullptr)) break;
        if (stop_flag) break;
        tc::mbar_arrive_expect_tx(&full_bar[s], KB * kBBytes);
        for (int kb = 0; kb < KB; ++kb)
          tc::tma_load_2d(sB + (s * KB + kb) * kBBytes, &tmapP, &full_bar[s], kb * 64, t * kTileN);
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
          if (i > 32) __nanosleep(64);
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
#pragma unroll
          for (int kb = 0; kb < KB; ++kb)
#pragma unroll
            for (int k16 = 0; k16 < 4; ++k16) {
              uint64_t ad = tc::sw128_kmajor_desc(a_addr + kb * kABytes + k16 * 32);
              uint64_t bd = tc::sw128_kmajor_desc(b_addr + (s * KB + kb) * kBBytes + k16 * 32);
              tc::umma_bf16(tbase + a * kTileN, ad, bd, idesc, (kb | k16) ? 1u : 0u);
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
    int k = 0, cut_r = 0;
    float nu = 0.f, hi = 0.f, lo = 0.f;
    if (valid) {
      Survivor S = prm.rows[gi];
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
      const float pn_tile = pn_next;                       // ||p|| of the tile's first item
      if (t + 1 < T) pn_next = prm.pnorm[(int64_t)(t + 1) * kTileN];
      if (__any_sync(0xffffffffu, need)) {
        const float E = __fmul_ru(cbu, pn_tile) + 1e-30f;
        const float thb = __fsub_rd(lo, E);
        const int ncols = (int)std::min<int64_t>(kTileN, prm.n - (int64_t)t * kTileN);
        if (need) scanned += ncols;
#pragma unroll 1
        for (int h = 0; h < kTileN; h += 128) {
          float v[128];
          tc::tmem_ld128(tbase + ((uint32_t)(quad * 32) << 16) + a * kTileN + h, v);
          tc::tmem_ld_wait();
          if (need) {
#pragma unroll
            for (int c0 = 0; c0 < 128; c0 += 32) {
              float g[11];
#pragma unroll
              for (int i = 0; i < 10; ++i) g[i] = max3(v[c0 + 3 * i], v[c0 + 3 * i + 1], v[c0 + 3 * i + 2]);
              g[10] = fmaxf(v[c0 + 30], v[c0 + 31]);
              const float gm = max3(max3(g[0], g[1], g[2]), max3(g[3], g[4], g[5]),
                                    max3(max3(g[6], g[7], g[8]), g[9], g[10]));
              if (gm > thb) {
                // per item: the bound of its own norm (items fall in norm within a tile)
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                  const int col = h + c0 + i;
                  if (col < ncols && v[c0 + i] > thb) {
                    const float Ei = __fmul_ru(cbu, prm.pnorm[(int64_t)t * kTileN + col]) + 1e-30f;
                    if (__fsub_rd(v[c0 + i], Ei) > hi) {
                      ++certain;
                    } else if (__fadd_ru(v[c0 + i], Ei) > lo) {
                      if (band < kBandCap) prm.band_items[gi * kBandCap + band] = t * kTileN + col;
                      ++band;
                    }
                  }
                }
              }
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
  return (size_t)KB * kRows * 128 + (size_t)STAGES * KB * kTileN * 128 + 1024;
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
  if (ix->m_nz > 0) {
    f32_to_bf16_rows_kernel<<<grid_for(ix->m_nz * dk, 256), 256, 0, st>>>(ix->Ut, ix->m_nz, ix->dp, ix->d, dk,
                                                                          ix->Ub);
    f32_to_bf16_lo_rows_kernel<<<grid_for(ix->m_nz * dk, 256), 256, 0, st>>>(ix->Ut, ix->m_nz, ix->dp, ix->d, dk,
                                                                             ix->Ulo);
  }
  f32_to_bf16_rows_kernel<<<grid_for(ix->n * dk, 256), 256, 0, st>>>(ix->Ps, ix->n, ix->dp, ix->d, dk, ix->Pb);
  SAH_CUDA(cudaGetLastError());
  auto encode = get_encode_fn();
  if (!encode) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return SAH_ERR_UNSUPPORTED;
  }
  cuuint64_t dims[2] = {(cuuint64_t)dk, (cuuint64_t)ix->n};
  cuuint64_t strides[1] = {(cuuint64_t)dk * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)kTileN};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(&ix->tmap_P, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ix->Pb, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
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
                         cudaStream_t st, int* launches) {
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
  cut_kernel<<<grid_for(ns, 256), 256, 0, st>>>(surv, count_dev, ns, ix->unorm, ix->pnorm, ix->n, qn, ix->gamma,
                                                ntiles, cut, hist);
  exclusive_scan_small_kernel<<<1, 32, 0, st>>>(hist, ntiles + 1);
  sort_by_cut_kernel<<<grid_for(ns, 256), 256, 0, st>>>(surv, cut, count_dev, ns, hist, rows, scut);
  SAH_CUDA(cudaGetLastError());

  TcParams prm;
  prm.rows = rows;
  prm.cut = scut;
  prm.nrows_dev = count_dev;
  prm.cap = ns;
  prm.Ub = ix->Ub;
  prm.dk = ix->dk;
  prm.unorm = ix->unorm;
  prm.pnorm = ix->pnorm;
  prm.n = ix->n;
  prm.qn = qn;
  prm.kk = kk;
  prm.gamma = ix->gamma;
  prm.cbf = (float)(1.01 * (std::ldexp(1.0, -7) + std::ldexp(1.0, -16) + (ix->dk + 8) * std::ldexp(1.0, -23)));
  prm.status = status;
  prm.certain_out = cert;
  prm.band_out = band;
  prm.band_items = items;
  prm.items_stat = stats + stat_items;
  prm.timeout = ix->dev_timeout;
  const unsigned grid = grid_for(ns, kRows);
  if (ix->dk == 64) {
    constexpr size_t smem = tc_smem_bytes<1, 4>();
    SAH_TRY(raise_smem_limit((const void*)verify_tc_kernel<1, 4>, smem));
    verify_tc_kernel<1, 4><<<grid, kThreads, smem, st>>>(ix->tmap_P, prm);
  } else {
    constexpr size_t smem = tc_smem_bytes<2, 2>();
    SAH_TRY(raise_smem_limit((const void*)verify_tc_kernel<2, 2>, smem));
    verify_tc_kernel<2, 2><<<grid, kThreads, smem, st>>>(ix->tmap_P, prm);
  }
  SAH_CUDA(cudaGetLastError());
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
