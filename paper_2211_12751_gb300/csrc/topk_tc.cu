// Index-time exact thresholds on the tensor cores (Alg. 4 with |P'| = n): for every user,
// the 64 largest FP32 scores over all items (their ids too), from which the lower-bound
// arrays L_u^1..k_max and the double-precision thresholds are taken.
//
// 1. A certified floor: V_u, the 64th largest FP32 score of u over the first items (a
//    subset of P, so V_u cannot exceed the 64th largest over P).
// 2. topk_tc_kernel: S = U . P^T on tcgen05 (BF16 in, FP32 in TMEM), 128 users x 256 items
//    per MMA tile, items streamed by TMA through a 4-stage ring, a double-buffered TMEM
//    accumulator and a warp-specialised pipeline.  The epilogue keeps, per user, every
//    item whose BF16 score can still reach V_u:  s_bf >= V_u - (c_bf + gamma) ||u|| ||p_t||,
//    where ||p_t|| is the largest norm of the tile (items arrive in descending norm order)
//    and the two terms bound the BF16 and the FP32 errors of those items' scores.
//    Every item whose FP32 score is >= V_u is kept, so the kept set holds the 64 largest.
//    Items arrive in descending norm order, so a tile whose largest norm ||p_t|| gives
//    ||u|| ||p_t|| (1 + 2 (c_bf + gamma)) < V_u holds no item that can be kept, and neither
//    does any later tile (the mu_j rule of Alg. 2): a user's scan ends at its cut, the first
//    such tile, and a CTA streams the tiles up to the largest cut of its 128 users.
// 3. topk_refine_kernel: the kept items re-scored in FP32 and ranked (64 slots per user
//    spread over a warp); a user whose candidate list overflowed is scanned in full up to
//    its cut (every item after it scores below V_u in FP32 too).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "sah_internal.cuh"
#include "tc.cuh"

namespace sah {
namespace {

constexpr int kTN = 256;
constexpr int kTM = 128;
constexpr int kTThreads = 192;
constexpr uint32_t kTTmem = 512;

struct TopkParams {
  int64_t mz, n;
  const float* vfloor;     // per user: V_u, the 64th largest FP32 score over the first items
  const float* unorm;
  const float* pnorm;      // descending item norms: a tile's first one bounds the tile
  float cb;                // c_bf + gamma
  int32_t* cand;           // [users in chunk][cap]
  int32_t* cand_cnt;       // [users in chunk]
  int32_t* cut_out;        // [users in chunk]: the user's cut (tiles of kTN items)
  float cut_factor;        // 1 + 2 (c_bf + gamma), rounded up, with room for the norms' rounding
  int32_t cap;
  int64_t u_first;         // first user of this launch
  int64_t u_count;         // users in this launch
  int* timeout;
};

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

template <int KB, int STAGES>
__global__ void __launch_bounds__(kTThreads, 1)
topk_tc_kernel(const __grid_constant__ CUtensorMap tmapU, const __grid_constant__ CUtensorMap tmapP, TopkParams p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[2], tempty_bar[2], a_bar, done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int tcut_sh;
  constexpr uint32_t kABytes = kTM * 128, kBBytes = kTN * 128;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + KB * kABytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = p.u_first + (int64_t)blockIdx.x * kTM;
  const int T_all = (int)((p.n + kTN - 1) / kTN);
  // each user's cut: the first tile t with ||u|| ||p_t|| cut_factor < V_u (binary search
  // over the descending tile norms); the CTA streams tiles [0, largest cut)
  int my_cut = 0;
  if (threadIdx.x == 0) tcut_sh = 0;
  if (warp >= 2) {
    const int64_t r = r0 + (warp & 3) * 32 + lane;
    if ((r - p.u_first) < p.u_count && r < p.mz) {
      const float V = p.vfloor[r];
      const float nu = p.unorm[r];
      int lo = 0, hi = T_all;   // tiles [0, lo) may hold a kept item; [hi, T_all) hold none
      if (V == -INFINITY || !(nu > 0.f)) {
        lo = T_all;
      } else {
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          const float bound = __fmul_ru(__fmul_ru(nu, p.pnorm[(int64_t)mid * kTN]), p.cut_factor);
          if (bound >= V) lo = mid + 1;
          else hi = mid;
        }
      }
      my_cut = lo;
      p.cut_out[r - p.u_first] = lo;
    }
  }
  __syncthreads();
  if (warp >= 2) atomicMax(&tcut_sh, my_cut);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&tfull_bar[a], 1);
      tc::mbar_init(&tempty_bar[a], 4);
    }
    tc::mbar_init(&a_bar, 1);
    tc::mbar_init(&done_bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_sh, kTTmem);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_base_sh;
  const int T = tcut_sh;

  int tiles_issued = 0;   // the producer: item tiles loaded (teardown drain)
  if (warp == 0) {
    if (lane == 0) {   // TMA producer: the users once, then the item tiles
      tc::prefetch_tensormap(&tmapU);
      tc::prefetch_tensormap(&tmapP);
      tc::mbar_arrive_expect_tx(&a_bar, KB * kABytes);
      for (int kb = 0; kb < KB; ++kb) tc::tma_load_2d(sA + kb * kABytes, &tmapU, &a_bar, kb * 64, (int32_t)r0);
      for (int t = 0; t < T; ++t) {
        const int s = t % STAGES;
        if (t >= STAGES && !tc::mbar_wait(&empty_bar[s], ((t / STAGES) & 1) ^ 1, p.timeout, nullptr)) break;
        tc::mbar_arrive_expect_tx(&full_bar[s], KB * kBBytes);
        for (int kb = 0; kb < KB; ++kb)
          tc::tma_load_2d(sB + (s * KB + kb) * kBBytes, &tmapP, &full_bar[s], kb * 64, t * kTN);
        tiles_issued = t + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      constexpr uint32_t idesc = tc::idesc_bf16_f32(kTM, kTN);
      const uint32_t a_addr = tc::smem_addr(sA), b_addr = tc::smem_addr(sB);
      bool ok = tc::mbar_wait(&a_bar, 0, p.timeout, nullptr);
      for (int t = 0; ok && t < T; ++t) {
        const int s = t % STAGES, a = t & 1;
        if (!tc::mbar_wait(&full_bar[s], (t / STAGES) & 1, p.timeout, nullptr)) break;
        if (t >= 2 && !tc::mbar_wait(&tempty_bar[a], ((t >> 1) & 1) ^ 1, p.timeout, nullptr)) break;
        tc::tc_fence_after();
#pragma unroll
        for (int kb = 0; kb < KB; ++kb)
#pragma unroll
          for (int k16 = 0; k16 < 4; ++k16)
            tc::umma_bf16(tbase + a * kTN, tc::sw128_kmajor_desc(a_addr + kb * kABytes + k16 * 32),
                          tc::sw128_kmajor_desc(b_addr + (s * KB + kb) * kBBytes + k16 * 32), idesc,
                          (kb | k16) ? 1u : 0u);
        tc::umma_commit(&empty_bar[s]);
        tc::umma_commit(&tfull_bar[a]);
      }
      tc::umma_commit(&done_bar);
    }
  } else {
    // epilogue: one thread per user row
    const int quad = warp & 3;
    const int row = quad * 32 + lane;
    const int64_t r = r0 + row;
    const bool valid = (r - p.u_first) < p.u_count && r < p.mz;
    const float V = valid ? p.vfloor[r] : INFINITY;
    const float cbu = valid ? __fmul_ru(p.cb, p.unorm[r]) : 0.f;
    const int64_t slot0 = (r - p.u_first) * p.cap;
    int cnt = 0;
    float pn_next = T > 0 ? p.pnorm[0] : 0.f;
    for (int t = 0; t < T; ++t) {
      const int a = t & 1;
      // keep threshold of this tile: V_u minus the BF16 and FP32 bounds for its largest norm
      const float thr = (V == -INFINITY) ? -INFINITY : __fsub_rd(V, __fmul_ru(cbu, pn_next));
      if (t + 1 < T) pn_next = p.pnorm[(int64_t)(t + 1) * kTN];
      if (!tc::mbar_wait(&tfull_bar[a], (t >> 1) & 1, p.timeout, nullptr)) break;
      tc::tc_fence_after();
      const int ncols = (int)std::min<int64_t>(kTN, p.n - (int64_t)t * kTN);
#pragma unroll 1
      for (int h = 0; h < kTN; h += 128) {
        float v[128];
        tc::tmem_ld128(tbase + ((uint32_t)(quad * 32) << 16) + a * kTN + h, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int c0 = 0; c0 < 128; c0 += 32) {
          float g[11];
#pragma unroll
          for (int i = 0; i < 10; ++i) g[i] = max3f(v[c0 + 3 * i], v[c0 + 3 * i + 1], v[c0 + 3 * i + 2]);
          g[10] = fmaxf(v[c0 + 30], v[c0 + 31]);
          const float gm = max3f(max3f(g[0], g[1], g[2]), max3f(g[3], g[4], g[5]),
                                 max3f(max3f(g[6], g[7], g[8]), g[9], g[10]));
          if (gm >= thr) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const int col = h + c0 + i;
              if (col < ncols && v[c0 + i] >= thr) {
                if (cnt < p.cap) p.cand[slot0 + cnt] = t * kTN + col;
                ++cnt;
              }
            }
          }
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty_bar[a]);
    }
    if (valid) p.cand_cnt[r - p.u_first] = cnt;
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    if (lane == 0) {
      // every MMA and every TMA load of the CTA completes before TMEM is freed and the CTA
      // exits, also when a bounded wait gave up early
      tc::mbar_wait_drain(&done_bar, 0);
      tc::mbar_wait_drain(&a_bar, 0);
      for (int s = 0; s < STAGES && s < tiles_issued; ++s) {
        const int issued = tiles_issued / STAGES + (s < tiles_issued % STAGES ? 1 : 0);
        tc::mbar_wait_drain(&full_bar[s], (uint32_t)((issued - 1) & 1));
      }
    }
    __syncwarp();
    tc::tc_fence_after();
    tc::tmem_dealloc(tbase, kTTmem);
  }
}

__device__ __forceinline__ void list_insert_id(float& a, float& b, int& ia, int& ib, float v, int id, int lane) {
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

__device__ __forceinline__ float slot_get(float a, float b, int slot) {
  const float va = __shfl_sync(0xffffffffu, a, slot >> 1);
  const float vb = __shfl_sync(0xffffffffu, b, slot >> 1);
  return (slot & 1) ? vb : va;
}

__device__ __forceinline__ float dot_f32(const float* __restrict__ u, const float* __restrict__ p, int dp) {
  const float4* a4 = reinterpret_cast<const float4*>(u);
  const float4* b4 = reinterpret_cast<const float4*>(p);
  float s = 0.f;
  for (int c = 0; c < dp / 4; ++c) {
    const float4 x = a4[c], y = b4[c];
    s = fmaf(y.x, x.x, s);
    s = fmaf(y.y, x.y, s);
    s = fmaf(y.z, x.z, s);
    s = fmaf(y.w, x.w, s);
  }
  return s;
}

// One warp per user: FP32 scores of the kept items (or of all items when the list
// overflowed), the 64 largest with their ids, written like the FP32 top-k pass writes them.
__global__ void topk_refine_kernel(const float* __restrict__ Ut, const float* __restrict__ Ps, int dp, int64_t n,
                                   int64_t mz, int kmax, int64_t u_first, int64_t u_count,
                                   const int32_t* __restrict__ cand, const int32_t* __restrict__ cand_cnt,
                                   const int32_t* __restrict__ cut, int cap,
                                   float* __restrict__ Lt, int32_t* __restrict__ ids_out, float* __restrict__ vlast_out,
                                   unsigned long long* __restrict__ overflow_rows) {
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= u_count) return;
  const int64_t r = u_first + w;
  const float* u = Ut + r * dp;
  float a = -INFINITY, b = -INFINITY;
  int ia = -1, ib = -1;
  float thr = -INFINITY;
  const int cnt = cand_cnt[w];
  const bool full = cnt > cap;
  if (full && lane == 0) atomicAdd(overflow_rows, 1ull);
  const int64_t total = full ? std::min<int64_t>(n, (int64_t)cut[w] * kTN) : cnt;
  for (int64_t base = 0; base < total; base += 32) {
    const int64_t i = base + lane;
    float s = -INFINITY;
    int id = -1;
    if (i < total) {
      id = full ? (int)i : cand[w * cap + i];
      s = dot_f32(u, Ps + (int64_t)id * dp, dp);
    }
    unsigned m = __ballot_sync(0xffffffffu, s > thr);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const float v = __shfl_sync(0xffffffffu, s, src);
      const int vid = __shfl_sync(0xffffffffu, id, src);
      if (!(v > thr)) continue;
      list_insert_id(a, b, ia, ib, v, vid, lane);
      thr = slot_get(a, b, 63);
    }
  }
  const int s0 = 2 * lane, s1 = 2 * lane + 1;
  if (s0 < kmax) Lt[(int64_t)s0 * mz + r] = a;
  if (s1 < kmax) Lt[(int64_t)s1 * mz + r] = b;
  ids_out[(int64_t)s0 * mz + r] = ia;
  ids_out[(int64_t)s1 * mz + r] = ib;
  const float last = slot_get(a, b, 63);
  if (lane == 0) vlast_out[r] = last;
}

template <int KB, int STAGES>
constexpr size_t topk_smem_bytes() {
  return (size_t)KB * kTM * 128 + (size_t)STAGES * KB * kTN * 128 + 1024;
}

inline unsigned grid_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

// Fills Lt (k_max rows), ids64 (64 rows) and vlast for every user with the 64 largest
// FP32 scores over all n items; vlast must hold V_u (the 64th largest over the first
// items) on entry.  Returns the GEMM's CUDA-event time in *gemm_ms.
sah_status topk_full_tc(Index* ix, float* vlast, int32_t* ids64, cudaStream_t st, double* gemm_ms) {
  const int64_t mz = ix->m_nz, n = ix->n;
  const float cbf = (float)(1.01 * (std::ldexp(1.0, -7) + std::ldexp(1.0, -16) + (ix->dk + 8) * std::ldexp(1.0, -23)));
  // the floors V_u are read by every chunk's GEMM, while the refine kernel overwrites vlast
  float* vfloor = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&vfloor, sizeof(float) * mz, st));
  SAH_CUDA(cudaMemcpyAsync(vfloor, vlast, sizeof(float) * mz, cudaMemcpyDeviceToDevice, st));
  const int cap = 256;
  const int64_t chunk = std::min<int64_t>(mz, (int64_t)1 << 18);   // users per launch (candidate buffer 256 MiB)
  const int64_t chunk_rows = (chunk + kTM - 1) / kTM * kTM;
  int32_t *cand = nullptr, *cnt = nullptr, *cut = nullptr;
  unsigned long long* ovf = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&cand, sizeof(int32_t) * (size_t)chunk_rows * cap, st));
  SAH_CUDA(cudaMallocAsync((void**)&cnt, sizeof(int32_t) * (size_t)chunk_rows, st));
  SAH_CUDA(cudaMallocAsync((void**)&cut, sizeof(int32_t) * (size_t)chunk_rows, st));
  SAH_CUDA(cudaMallocAsync((void**)&ovf, sizeof(unsigned long long), st));
  SAH_CUDA(cudaMemsetAsync(ovf, 0, sizeof(unsigned long long), st));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms_total = 0.f;
  for (int64_t u0 = 0; u0 < mz; u0 += chunk) {
    const int64_t uc = std::min(chunk, mz - u0);
    // c_bf + gamma, rounded up on the host (one ulp up covers the float rounding of the sum)
    const float cb = std::nextafter(cbf + ix->gamma, INFINITY);
    // the cut's factor: 1 + 2 cb, rounded up, plus 2^-20 for the rounding of ||u|| and ||p||
    const float cut_factor = std::nextafter(1.f + 2.f * cb + 0x1p-20f, INFINITY);
    TopkParams p{mz, n, vfloor, ix->unorm, ix->pnorm, cb, cand, cnt, cut, cut_factor, cap, u0, uc,
                 ix->dev_timeout};
    const unsigned grid = grid_for(uc, kTM);
    cudaEventRecord(e0, st);
    if (ix->dk == 64) {
      constexpr size_t smem = topk_smem_bytes<1, 4>();
      SAH_TRY(raise_smem_limit((const void*)topk_tc_kernel<1, 4>, smem));
      topk_tc_kernel<1, 4><<<grid, kTThreads, smem, st>>>(ix->tmap_U, ix->tmap_P, p);
    } else {
      constexpr size_t smem = topk_smem_bytes<2, 2>();
      SAH_TRY(raise_smem_limit((const void*)topk_tc_kernel<2, 2>, smem));
      topk_tc_kernel<2, 2><<<grid, kTThreads, smem, st>>>(ix->tmap_U, ix->tmap_P, p);
    }
    cudaEventRecord(e1, st);
    SAH_CUDA(cudaGetLastError());
    topk_refine_kernel<<<grid_for(uc * 32, 256), 256, 0, st>>>(ix->Ut, ix->Ps, ix->dp, n, mz, ix->kmax, u0, uc, cand,
                                                               cnt, cut, cap, ix->Lt, ids64, vlast, ovf);
    SAH_CUDA(cudaGetLastError());
    SAH_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms_total += ms;
  }
  unsigned long long ovf_h = 0;
  SAH_CUDA(cudaMemcpyAsync(&ovf_h, ovf, sizeof(ovf_h), cudaMemcpyDeviceToHost, st));
  SAH_CUDA(cudaStreamSynchronize(st));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(vfloor, st);
  cudaFreeAsync(cand, st);
  cudaFreeAsync(cnt, st);
  cudaFreeAsync(cut, st);
  cudaFreeAsync(ovf, st);
  ix->build_gemm_ms = ms_total;
  ix->build_overflow_rows = (int64_t)ovf_h;
  if (gemm_ms) *gemm_ms = ms_total;
  int to = 0;
  SAH_CUDA(cudaMemcpy(&to, ix->dev_timeout, sizeof(int), cudaMemcpyDeviceToHost));
  if (to) {
    cudaMemset(ix->dev_timeout, 0, sizeof(int));
    set_error("a bounded device-side wait of the index-time GEMM ran out");
    return SAH_ERR_DEVICE_TIMEOUT;
  }
  return SAH_OK;
}

}  // namespace sah
