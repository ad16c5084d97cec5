// Tensor-core user pass (A4 as the batched score GEMM of a tick): for every Cone-Tree
// leaf, S = U_leaf . Q_kept^T on tcgen05 (BF16 in, FP32 in TMEM), where Q_kept are the
// queries that survived the leaf's node-level bound (Lemma 2).  Users are the 128-row A
// operand (TMA tiles of the leaf-ordered BF16 users), the leaf's queries the B operand
// (gathered rows, up to 256 per MMA).  The epilogue takes, per (user, query):
//   Lemma 3 (vector-level bound) against the lower bound L_u^k  -> "no";
//   the BF16 score with its a-priori bound  |s_bf - <u,q>| <= c_bf ||u|| ||q||:
//     certainly below L_u^k                                   -> "no",
//     certainly above the exact threshold (|P'| = n)          -> "yes",
//     certainly above ||u|| ||p_k||                           -> "yes" (Alg. 5);
//   anything else is re-scored in FP32 by pair_rescore_kernel, which applies the same
//   tests as the FP32 user pass (and the double-precision threshold where it exists) and
//   lists the survivors for the kMIPS decision.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

#include "sah_internal.cuh"
#include "tc.cuh"

namespace sah {
namespace {

constexpr int kUpRows = 128;
constexpr int kUpN = 256;
constexpr int kUpThreads = 128;

struct UpPair {
  int32_t j;      // query (bit 30: SA-ALSH row)
  int32_t slot;   // lower-bound slot of k (-1: k > k_max)
  int32_t k;
  float cphi, sphi, nrm, pk;   // cos/sin phi, ||q||, ||p_k|| (-inf past n)
};

struct UpParams {
  const float* Ut;
  const float* unorm;
  const float* ucos;
  const float* usin;
  const int32_t* uid;
  const int32_t* bstart;
  const float* Lt;
  const float* Eu;
  const float* pnorm;
  int64_t n, mz;
  int kmax, l_exact, dk;
  const uint16_t* Qb;
  const float* qn;
  const int32_t* kk;
  const int32_t* modes;
  int nq;
  const int32_t* pairs_j;       // PairEntry array viewed as 3 x int32 records
  const int32_t* pcount;
  float gamma, slack, cbf;
  uint32_t* bitmap;
  int64_t words;
  Survivor* resc;               // pairs to re-score in FP32
  unsigned long long* resc_count;
  int64_t resc_cap;
  unsigned long long* stats;
  int st_scored, st_yes, st_kept;
  int* timeout;
};

template <int KB>
__global__ void __launch_bounds__(kUpThreads, 1)
user_pass_tc_kernel(const __grid_constant__ CUtensorMap tmapU, UpParams p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t tma_bar, mma_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int32_t kslot[65], klist[64];
  __shared__ int32_t nslots;
  constexpr uint32_t kABytes = kUpRows * 128, kBBytes = kUpN * 128;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = sA + KB * kABytes;
  float* Ls = reinterpret_cast<float*>(sB + KB * kBBytes);            // [64][128]
  UpPair* pin = reinterpret_cast<UpPair*>(Ls + 64 * kUpRows);          // [256]

  const int Bk = blockIdx.x;
  const int npairs = p.pcount[Bk];
  if (npairs == 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = p.bstart[Bk], e = p.bstart[Bk + 1], cnt = e - s;
  if (tid == 0) {
    tc::mbar_init(&tma_bar, 1);
    tc::mbar_init(&mma_bar, 1);
    tc::fence_mbar_init();
    atomicAdd(&p.stats[p.st_kept], (unsigned long long)cnt);
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_sh, kUpN);
    tc::tmem_relinquish();
  }
  // lower-bound slots of the k values this leaf's queries ask for
  for (int k = tid; k <= 64; k += kUpThreads) kslot[k] = -1;
  __syncthreads();
  const int3* pr = reinterpret_cast<const int3*>(p.pairs_j) + (int64_t)Bk * p.nq;
  for (int i = tid; i < npairs; i += kUpThreads) {
    const int k = p.kk[pr[i].x];
    if (k <= p.kmax) kslot[k] = 0;
  }
  __syncthreads();
  if (tid == 0) {
    int ns = 0;
    for (int k = 1; k <= p.kmax; ++k)
      if (kslot[k] == 0) {
        kslot[k] = ns;
        klist[ns++] = k;
      }
    nslots = ns;
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_base_sh;
  unsigned long long scored = 0, yes_cnt = 0;
  uint32_t mma_phase = 0;
  bool failed_all = false;
  for (int mb = 0; mb * kUpRows < cnt && !failed_all; ++mb) {
    // users mb*128 .. of the leaf: TMA tile of the leaf-ordered BF16 rows
    if (tid == 0) {
      tc::mbar_arrive_expect_tx(&tma_bar, KB * kABytes);
      for (int kb = 0; kb < KB; ++kb)
        tc::tma_load_2d(sA + kb * kABytes, &tmapU, &tma_bar, kb * 64, s + mb * kUpRows);
    }
    const int row = mb * kUpRows + tid;
    const bool active = row < cnt;
    const int64_t r = s + (active ? row : 0);
    float nu = 0.f, ct = 0.f, st_ = 0.f, E = 0.f;
    int32_t id = 0;
    if (active) {
      nu = p.unorm[r];
      ct = p.ucos[r];
      st_ = p.usin[r];
      E = p.Eu[r];
      id = p.uid[r];
    }
    for (int sl = 0; sl < nslots; ++sl)
      Ls[sl * kUpRows + tid] = active ? p.Lt[(int64_t)(klist[sl] - 1) * p.mz + r] : -INFINITY;
    const float cbu = __fmul_ru(p.cbf, nu);
    const float nuu = __fmul_ru(nu, 1.f + 2.f * p.gamma);
    // a failed (timed-out) wait ends the CTA's work for every thread together
    if (__syncthreads_or(!tc::mbar_wait(&tma_bar, mb & 1, p.timeout, nullptr))) break;
    for (int n0 = 0; n0 < npairs; n0 += kUpN) {
      const int nn = min(kUpN, npairs - n0);
      const int Npad = max(16, (nn + 15) & ~15);
      __syncthreads();   // the previous tile's epilogue is done with pin and sB
      for (int i = tid; i < nn; i += kUpThreads) {
        const int3 raw = pr[n0 + i];
        const int j = raw.x;
        const int k = p.kk[j];
        const int sa = (p.modes != nullptr && p.modes[j] == SAH_SAALSH && k <= p.kmax) ? 1 : 0;
        UpPair u;
        u.j = j | (sa << 30);
        u.slot = k <= p.kmax ? kslot[k] : -1;
        u.k = k;
        u.cphi = __int_as_float(raw.y);
        u.sphi = __int_as_float(raw.z);
        u.nrm = p.qn[j];
        u.pk = k <= p.n ? p.pnorm[k - 1] : -INFINITY;
        pin[i] = u;
      }
      __syncthreads();
      for (int i = tid; i < Npad * KB * 8; i += kUpThreads) {
        const int rr = i / (KB * 8), rem = i % (KB * 8), kb = rem / 8, c = rem % 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (rr < nn) {
          const int j = pin[rr].j & 0x3fffffff;
          v = *reinterpret_cast<const uint4*>(p.Qb + (int64_t)j * p.dk + kb * 64 + c * 8);
        }
        *reinterpret_cast<uint4*>(sB + kb * kBBytes + tc::sw128_offset(rr, c)) = v;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc::tc_fence_after();
        const uint32_t idesc = tc::idesc_bf16_f32(kUpRows, (uint32_t)Npad);
        const uint32_t a_addr = tc::smem_addr(sA), b_addr = tc::smem_addr(sB);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb)
#pragma unroll
          for (int k16 = 0; k16 < 4; ++k16)
            tc::umma_bf16(tbase, tc::sw128_kmajor_desc(a_addr + kb * kABytes + k16 * 32),
                          tc::sw128_kmajor_desc(b_addr + kb * kBBytes + k16 * 32), idesc, (kb | k16) ? 1u : 0u);
        tc::umma_commit(&mma_bar);
      }
      const bool mma_ok = tc::mbar_wait(&mma_bar, mma_phase & 1, p.timeout, nullptr);
      ++mma_phase;
      if (__syncthreads_or(!mma_ok)) {
        failed_all = true;
        break;
      }
      tc::tc_fence_after();
      for (int c0 = 0; c0 < Npad; c0 += 32) {
        float v[32];
        tc::tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + c0, v);
        tc::tmem_ld_wait();
        if (!active) continue;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int col = c0 + i;
          if (col >= nn) continue;
          const UpPair u = pin[col];
          const float L = u.slot >= 0 ? Ls[u.slot * kUpRows + tid] : -INFINITY;
          const float Llo = (L == -INFINITY) ? -INFINITY : __fsub_rd(L, E);
          if (u.cphi <= 1.5f) {   // Lemma 3 with the slack of the FP32 terms
            const float ub = __fmul_ru(__fmul_ru(nu, u.nrm), fmaf(u.cphi, ct, u.sphi * st_) + 2.f * p.slack);
            if (ub < Llo) continue;
          }
          ++scored;
          const float Eb = __fmul_ru(cbu, u.nrm) + 1e-30f;
          const float hi = __fadd_ru(v[i], Eb), lo = __fsub_rd(v[i], Eb);
          bool yes = false, resc = false;
          if (hi < Llo) {
            // "no": at least k items of P' certainly beat <u,q>
          } else if (p.l_exact && u.slot >= 0 && lo >= __fadd_ru(L, E)) {
            yes = true;
          } else if (lo >= __fmul_ru(nuu, u.pk)) {
            yes = true;
          } else {
            resc = true;
          }
          const int j = u.j & 0x3fffffff;
          if (yes) {
            ++yes_cnt;
            atomicOr(&p.bitmap[(int64_t)j * p.words + (id >> 5)], 1u << (id & 31));
          } else if (resc) {
            const unsigned long long slot = atomicAdd(p.resc_count, 1ull);
            if ((int64_t)slot < p.resc_cap) p.resc[slot] = Survivor{(int32_t)r, u.j, 0.f};
          }
        }
      }
      tc::tc_fence_before();
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    scored += __shfl_xor_sync(0xffffffffu, scored, o);
    yes_cnt += __shfl_xor_sync(0xffffffffu, yes_cnt, o);
  }
  if (lane == 0) {
    if (scored) atomicAdd(&p.stats[p.st_scored], scored);
    if (yes_cnt) atomicAdd(&p.stats[p.st_yes], yes_cnt);
  }
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tbase, kUpN);
  }
}

// FP32 re-score of the pairs the BF16 bound left open; the same decisions as the FP32
// user pass.  One thread per pair.
__global__ void pair_rescore_kernel(const Survivor* __restrict__ pairs, const unsigned long long* __restrict__ count,
                                    int64_t cap, const float* __restrict__ Ut, const float* __restrict__ unorm,
                                    const int32_t* __restrict__ uid, const float* __restrict__ Lt,
                                    const float* __restrict__ Eu, const float* __restrict__ pnorm, int64_t n,
                                    int64_t mz, int kmax, int l_exact, int d, int dp, const float* __restrict__ Qd,
                                    const float* __restrict__ qn, const int32_t* __restrict__ kk, float gamma,
                                    const double* __restrict__ T64, uint32_t* __restrict__ bitmap, int64_t words,
                                    Survivor* __restrict__ surv, unsigned long long* __restrict__ surv_count,
                                    int64_t surv_cap, unsigned long long* __restrict__ stats, int st_yes,
                                    int st_fp64) {
  const int64_t total = min((int64_t)*count, cap);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const Survivor P = pairs[i];
  const int r = P.upos;
  const int j = P.j & 0x3fffffff;
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

__global__ void queries_to_bf16_kernel(const float* __restrict__ Qd, int nq, int d, int dp, int dk,
                                       uint16_t* __restrict__ Qb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nq * dk) return;
  const int64_t j = i / dk;
  const int c = (int)(i % dk);
  const float v = c < d ? Qd[j * dp + c] : 0.f;
  __nv_bfloat16 b = __float2bfloat16_rn(v);
  Qb[i] = *reinterpret_cast<uint16_t*>(&b);
}

template <int KB>
constexpr size_t up_smem_bytes() {
  return (size_t)KB * kUpRows * 128 + (size_t)KB * kUpN * 128 + 64 * kUpRows * 4 + kUpN * sizeof(UpPair) + 1024;
}

inline unsigned grid_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

sah_status run_user_pass_tc(Index* ix, const float* Qd, uint16_t* Qb, const float* qn, const int32_t* kk,
                            const int32_t* modes, int nq, const void* pairs, const int32_t* pcount, uint32_t* bitmap,
                            int64_t words, Survivor* resc, unsigned long long* resc_count, Survivor* surv,
                            unsigned long long* surv_count, int64_t surv_cap, unsigned long long* stats,
                            int st_scored, int st_yes, int st_kept, int st_fp64, cudaStream_t st, int* launches) {
  queries_to_bf16_kernel<<<grid_for((int64_t)nq * ix->dk, 256), 256, 0, st>>>(Qd, nq, ix->d, ix->dp, ix->dk, Qb);
  UpParams p;
  p.Ut = ix->Ut;
  p.unorm = ix->unorm;
  p.ucos = ix->ucos;
  p.usin = ix->usin;
  p.uid = ix->uid;
  p.bstart = ix->bstart;
  p.Lt = ix->Lt;
  p.Eu = ix->Eu;
  p.pnorm = ix->pnorm;
  p.n = ix->n;
  p.mz = ix->m_nz;
  p.kmax = ix->kmax;
  p.l_exact = ix->l_exact ? 1 : 0;
  p.dk = ix->dk;
  p.Qb = Qb;
  p.qn = qn;
  p.kk = kk;
  p.modes = modes;
  p.nq = nq;
  p.pairs_j = reinterpret_cast<const int32_t*>(pairs);
  p.pcount = pcount;
  p.gamma = ix->gamma;
  p.slack = ix->cone_slack;
  p.cbf = (float)(1.01 * (std::ldexp(1.0, -7) + std::ldexp(1.0, -16) + (ix->dk + 8) * std::ldexp(1.0, -23)));
  p.bitmap = bitmap;
  p.words = words;
  p.resc = resc;
  p.resc_count = resc_count;
  p.resc_cap = surv_cap;
  p.stats = stats;
  p.st_scored = st_scored;
  p.st_yes = st_yes;
  p.st_kept = st_kept;
  p.timeout = ix->dev_timeout;
  if (ix->dk == 64) {
    constexpr size_t smem = up_smem_bytes<1>();
    SAH_CUDA(cudaFuncSetAttribute(user_pass_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    user_pass_tc_kernel<1><<<ix->nb, kUpThreads, smem, st>>>(ix->tmap_U, p);
  } else {
    constexpr size_t smem = up_smem_bytes<2>();
    SAH_CUDA(cudaFuncSetAttribute(user_pass_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    user_pass_tc_kernel<2><<<ix->nb, kUpThreads, smem, st>>>(ix->tmap_U, p);
  }
  SAH_CUDA(cudaGetLastError());
  pair_rescore_kernel<<<grid_for(surv_cap, 256), 256, 0, st>>>(
      resc, resc_count, surv_cap, ix->Ut, ix->unorm, ix->uid, ix->Lt, ix->Eu, ix->pnorm, ix->n, ix->m_nz, ix->kmax,
      ix->l_exact ? 1 : 0, ix->d, ix->dp, Qd, qn, kk, ix->gamma, ix->T64, bitmap, words, surv, surv_count, surv_cap,
      stats, st_yes, st_fp64);
  SAH_CUDA(cudaGetLastError());
  if (launches) *launches += 3;
  return SAH_OK;
}

}  // namespace sah
