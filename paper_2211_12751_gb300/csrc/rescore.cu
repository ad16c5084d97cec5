// FP32 re-score (A6) of the (user, request) pairs the tensor-core user pass left inside
// its band: the same decisions as the FP32 user pass (Alg. 5 with the bounds of Lemma 3
// replaced by the FP32 score and its a-priori error), and with exact thresholds a
// double-precision dot summed i = 0..d-1 for what FP32 cannot separate.  Pairs still open
// go to the survivor lists of the kMIPS decision.  Grid-stride, one thread per pair.
#include <climits>
#include <cmath>

#include "sah_internal.cuh"

namespace sah {
namespace {

// DP4 > 0: user rows of at most 4 DP4 floats, held in registers for the FP32 dot; DP4 = 0:
// any width, read as needed.  The double-precision dot reads both rows again (from L1).
template <int DP4>
__global__ void pair_rescore_kernel(const Survivor* __restrict__ pairs, const unsigned long long* __restrict__ count,
                                    int64_t cap, const float* __restrict__ Ut, const float* __restrict__ unorm,
                                    const int32_t* __restrict__ uid, const float* __restrict__ Lt,
                                    const float* __restrict__ Eu, const float* __restrict__ pnorm, int64_t n,
                                    int64_t mz, int kmax, int l_exact, int d, int dp, const float* __restrict__ Qd,
                                    const float* __restrict__ qn, const int32_t* __restrict__ kk, float gamma,
                                    const double* __restrict__ T64, uint32_t* __restrict__ bitmap, int64_t words,
                                    Survivor* __restrict__ surv, unsigned long long* __restrict__ surv_count,
                                    int64_t surv_cap, unsigned long long* __restrict__ stats, int st_yes,
                                    int st_fp64, int nq, const int* __restrict__ timeout,
                                    const uint32_t* __restrict__ kept_mask, int mask_words,
                                    const int32_t* __restrict__ ublock) {
  // after a timed-out wait of the pass the list may hold unwritten entries: nothing is read
  __shared__ int stop;
  if (threadIdx.x == 0) stop = *(volatile const int*)timeout;
  const int64_t total = block_count(count, cap);   // synchronises the block
  if (stop) return;
  // warp-strided, so that every lane runs the same iterations and the appends to the
  // lists and counters go out once per warp; consecutive 32-pair chunks go to warps of
  // different CTAs, so that a short list still spreads over the SMs
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t wid = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  for (int64_t w0 = wid * 32; w0 < total; w0 += nw * 32) {
    const int64_t i = w0 + lane;
    bool yes = false, surv_flag = false, sa_row = false, fp64 = false;
    int r = 0, j = 0;
    float acc = 0.f;
    if (i < total) {
      const Survivor P = pairs[i];
      r = P.upos;
      j = P.j & 0x3fffffff;
      // with kept_mask: a pair whose leaf the node-level bound (Lemma 2) pruned for its row
      // cannot answer "yes"; it is dropped before any arithmetic
      const bool kept = kept_mask == nullptr ||
                        (r >= 0 && r < mz && j < nq &&
                         ((__ldg(&kept_mask[(int64_t)__ldg(&ublock[r]) * mask_words + (j >> 5)]) >> (j & 31)) & 1u));
      if (kept && r >= 0 && r < mz && j < nq) {
        sa_row = (P.j >> 30) & 1;
        const int k = kk[j];
        const float4* u4 = reinterpret_cast<const float4*>(Ut + (int64_t)r * dp);
        const float4* q4 = reinterpret_cast<const float4*>(Qd + (int64_t)j * dp);
        float4 ur[DP4 > 0 ? DP4 : 1];
        if (DP4 > 0) {
#pragma unroll
          for (int c = 0; c < DP4; ++c) ur[c] = c < dp / 4 ? u4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int c = 0; c < DP4; ++c) {
            const float4 b = c < dp / 4 ? __ldg(q4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            acc = fmaf(ur[c].x, b.x, acc);
            acc = fmaf(ur[c].y, b.y, acc);
            acc = fmaf(ur[c].z, b.z, acc);
            acc = fmaf(ur[c].w, b.w, acc);
          }
        } else {
          for (int c = 0; c < dp / 4; ++c) {
            const float4 a = u4[c], b = q4[c];
            acc = fmaf(a.x, b.x, acc);
            acc = fmaf(a.y, b.y, acc);
            acc = fmaf(a.z, b.z, acc);
            acc = fmaf(a.w, b.w, acc);
          }
        }
        const float nu = unorm[r], E = Eu[r];
        const float L = (k <= kmax) ? Lt[(int64_t)(k - 1) * mz + r] : -INFINITY;
        const float Llo = (L == -INFINITY) ? -INFINITY : __fsub_rd(L, E);
        const float eq = __fmul_ru(__fmul_ru(gamma, nu), qn[j]) + 1e-30f;
        const float hi = __fadd_ru(acc, eq), lo = __fsub_rd(acc, eq);
        if (hi < Llo) {
        } else if (l_exact && k <= kmax && lo >= __fadd_ru(L, E)) {
          yes = true;
        } else if (lo >= __fmul_ru(__fmul_ru(nu, pnorm[k - 1]), 1.f + 2.f * gamma)) {
          yes = true;
        } else if (T64 != nullptr && k <= kmax && !sa_row) {
          const double t64 = T64[(int64_t)(k - 1) * mz + r];
          if (t64 == t64) {
            fp64 = true;
            // the sequential double-precision sum i = 0..d-1, as a rolled loop (the rows
            // are in L1 by now): unrolled over the registers it was so long that the warps
            // waited on instruction fetch
            const double s64 = dot64_seq(Ut + (int64_t)r * dp, Qd + (int64_t)j * dp, d);
            yes = s64 >= t64;
          } else {
            surv_flag = true;
          }
        } else {
          surv_flag = true;
        }
      }
    }
    if (yes) {
      const int32_t id = uid[r];
      set_answer(bitmap, words, j, id);
    }
    const unsigned myes = __ballot_sync(0xffffffffu, yes), mf = __ballot_sync(0xffffffffu, fp64);
    if (lane == 0) {
      if (myes) atomicAdd(&stats[st_yes], (unsigned long long)__popc(myes));
      if (mf) atomicAdd(&stats[st_fp64], (unsigned long long)__popc(mf));
    }
#pragma unroll
    for (int sa = 0; sa < 2; ++sa) {
      const bool mine = surv_flag && (sa_row == (sa == 1));
      const unsigned m = __ballot_sync(0xffffffffu, mine);
      if (m) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(surv_count + sa, (unsigned long long)__popc(m));
        b = __shfl_sync(0xffffffffu, b, 0);
        if (mine) {
          const unsigned long long slot = b + __popc(m & ((1u << lane) - 1u));
          if ((int64_t)slot < surv_cap) surv[(sa ? surv_cap : 0) + slot] = Survivor{r, j, acc};
        }
      }
    }
  }
}

}  // namespace

sah_status launch_pair_rescore(Index* ix, const Survivor* pairs, const unsigned long long* count, int64_t cap,
                               const float* Qd, const float* qn, const int32_t* kk, uint32_t* bitmap, int64_t words,
                               Survivor* surv, unsigned long long* surv_count, unsigned long long* stats, int st_yes,
                               int st_fp64, int nq, int sms, cudaStream_t st, const uint32_t* kept_mask,
                               int mask_words) {
  // rows in registers pay off where most pairs also take the double-precision dot (exact
  // thresholds); otherwise the narrower kernel keeps more warps in flight
  auto fn = (ix->T64 != nullptr && ix->dp <= 64) ? pair_rescore_kernel<16> : pair_rescore_kernel<0>;
  // one wave: the CTAs that fit on an SM at once (the register-resident rows allow fewer),
  // each warp taking its pairs in one or a few strides; CTAs of a second wave would only
  // find the list already done
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
  fn<<<sms * per_sm, 256, 0, st>>>(pairs, count, cap, ix->Ut, ix->unorm, ix->uid, ix->Lt, ix->Eu, ix->pnorm, ix->n,
                              ix->m_nz, ix->kmax, ix->l_exact ? 1 : 0, ix->d, ix->dp, Qd, qn, kk, ix->gamma, ix->T64,
                              bitmap, words, surv, surv_count, cap, stats, st_yes, st_fp64, nq, ix->dev_timeout,
                              kept_mask, mask_words, ix->ublock);
  SAH_CUDA(cudaGetLastError());
  return SAH_OK;
}

}  // namespace sah
