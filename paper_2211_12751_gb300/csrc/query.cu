// SAH query (Alg. 5) for a batch of queries, exact mode.
//
//   A3  block pass: node-level bound (Lemma 2) of every (leaf, query) pair against the
//       block lower bound L^k(B) (Alg. 4); surviving pairs are listed per leaf.
//   A4  user pass: vector-level bound (Lemma 3), then <u,q> with its FP32 error bound,
//       then the lower bound L_u^k ("no"), the exact-threshold upper bound when |P'| = n
//       ("yes") and the ||p_k|| bound ("yes", Alg. 5); the rest become survivors.
//   A5  verify: per survivor, items in descending norm order, counting items whose FP32
//       score is certainly above <u,q>, keeping the few inside the error band, and
//       stopping at k certain items ("no") or when ||u|| ||p_i|| can no longer reach
//       <u,q> (the mu_j rule of Alg. 2).
//   A6  the open cases are decided in double precision, summed i = 0..d-1.
//   A7  answers are set in a per-query bitmap over the caller's user ids and emitted in
//       ascending id order.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "sah_internal.cuh"

namespace sah {

namespace {

struct PairEntry {
  int32_t j;      // query within the sub-batch
  float cphi;     // cos(angle(q, block centre)); > 1.5 means "no cone bound"
  float sphi;     // sin of that angle
};

enum StatSlot {
  ST_PAIRS_KEPT = 0,
  ST_USERS_SCORED,
  ST_YES_EARLY,
  ST_FP64,
  ST_KEPT_USERS,
  ST_ITEMS,
  ST_BAD_Q,
  ST_BAD_K,
  ST_EMIT_OVERFLOW,
  ST_TC_SCORES,      // (user, column) scores of the tensor-core user pass
  ST_BF_COLPAIRS,    // (leaf, distinct column) pairs of the tensor-core block filter
  ST_TC_ROWS,        // user rows the tensor-core user pass streamed (once per column set)
  ST_CAND_BLOCKS,    // candidate blocks (a user's 32 scores) the tensor-core user pass wrote
  ST_COUNT
};


inline unsigned grid_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

// ---------------------------------------------------------------- query preparation
// A row with an invalid k or mode is counted (the call then fails) and its k set to
// INT_MAX, which no kernel uses as an index: such a row asks for every user.
// (with Qhi non-null, also the split BF16 copy of the tensor-core user pass: hi = bf16(x),
// lo = bf16(x - hi), K padded to dk with zeros, lo at Qhi + nq dk)
__global__ void prep_queries_kernel(const float* __restrict__ Q, int nq, int d, int dp,
                                    float* __restrict__ Qd, float* __restrict__ qn,
                                    const int32_t* __restrict__ ks, int32_t* __restrict__ kk,
                                    const int32_t* __restrict__ modes, unsigned long long* __restrict__ stats,
                                    uint16_t* __restrict__ Qhi, int dk, uint64_t* __restrict__ qh, int collide) {
  int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (j >= nq) return;
  const int32_t kj = ks[j];
  const bool bad_k = kj < 1 || (modes && modes[j] != SAH_EXACT && modes[j] != SAH_SAALSH);
  if (lane == 0) {
    kk[j] = bad_k ? INT_MAX : kj;
    if (bad_k) atomicAdd(&stats[ST_BAD_K], 1ull);
  }
  float s = 0.f;
  bool fin = true;
  uint64_t h = 0;   // sum over i of a mix of (i, bits of the padded row's element i)
  for (int i = lane; i < dp; i += 32) {
    float v = (i < d) ? Q[(int64_t)j * d + i] : 0.f;
    fin &= isfinite(v);
    Qd[(int64_t)j * dp + i] = v;
    s = fmaf(v, v, s);
    h += splitmix64(((uint64_t)i << 32) | __float_as_uint(v));
  }
  if (qh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if (lane == 0) qh[j] = collide ? 0ull : h;   // (a test hook makes every row collide)
  }
  if (Qhi) {
    uint16_t* Qlo = Qhi + (int64_t)nq * dk;
    for (int i = lane; i < dk; i += 32) {
      const float v = (i < d) ? Q[(int64_t)j * d + i] : 0.f;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
      Qhi[(int64_t)j * dk + i] = __bfloat16_as_ushort(h);
      Qlo[(int64_t)j * dk + i] = __bfloat16_as_ushort(l);
    }
  }
  s = warp_sum(s);
  bool ok = __all_sync(0xffffffffu, fin);
  if (lane == 0) {
    qn[j] = sqrtf(s);
    if (!ok) atomicAdd(&stats[ST_BAD_Q], 1ull);
  }
}

// ---------------------------------------------------------------- A3: block pass
// One CTA per leaf, one thread per (leaf, query) pair.  cos phi = <c, q> / ||q|| with
// the unit centre c.  sin phi = sqrt(1 - cos^2 phi) while cos^2 phi <= 1/2, where that
// formula is well conditioned (|d sin / d cos| <= 1); closer to the centre it comes
// from the norm of q's component orthogonal to c.  Upper bound (Lemma 2), unit users:
//   ||q||                                           if phi <= omega
//   ||q|| (cos phi cos omega + sin phi sin omega)   otherwise,
// plus an additive slack that covers the FP32 error of every term.
__global__ void block_filter_kernel(const float* __restrict__ bcent, const float* __restrict__ bcos,
                                    const float* __restrict__ bsin, const float* __restrict__ LB,
                                    int nb, int kmax, int64_t n, int dp,
                                    const float* __restrict__ Qd, const float* __restrict__ qn,
                                    const int32_t* __restrict__ kk, int nq, float slack,
                                    PairEntry* __restrict__ pairs, int32_t* __restrict__ pcount,
                                    unsigned long long* __restrict__ stats, uint32_t* __restrict__ kept_mask,
                                    int mask_words, const int32_t* __restrict__ bstart, int count_pairs) {
  extern __shared__ float4 c4s[];   // the leaf's unit centre
  __shared__ int32_t cnt;
  const int B = blockIdx.x;
  const int lane = threadIdx.x & 31;
  const int dp4 = dp / 4;
  if (threadIdx.x == 0) cnt = 0;
  for (int i = threadIdx.x; i < dp4; i += blockDim.x)
    c4s[i] = reinterpret_cast<const float4*>(bcent + (int64_t)B * dp)[i];
  __syncthreads();
  const float cw = bcos[B], sw = bsin[B];
  const bool degenerate = cw < -1.5f;
  for (int j0 = 0; j0 < nq; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    bool keep = false;
    float cphi = 2.f, sphi = 0.f;
    if (j < nq) {
      const int k = kk[j];
      const float nrm = qn[j];
      if (k <= n) {                     // k > n: every user answers "yes" elsewhere
        if (degenerate || !(nrm > 0.f)) {
          keep = true;
        } else {
          const float4* q4 = reinterpret_cast<const float4*>(Qd + (int64_t)j * dp);
          float dq = 0.f;
          for (int i = 0; i < dp4; ++i) {
            const float4 a = c4s[i], b = __ldg(q4 + i);
            dq = fmaf(a.x, b.x, dq);
            dq = fmaf(a.y, b.y, dq);
            dq = fmaf(a.z, b.z, dq);
            dq = fmaf(a.w, b.w, dq);
          }
          cphi = fminf(1.f, fmaxf(-1.f, dq / nrm));
          if (cphi * cphi <= 0.5f) {
            sphi = sqrtf(fmaxf(0.f, fmaf(-cphi, cphi, 1.f)));
          } else {
            float o2 = 0.f;
            for (int i = 0; i < dp4; ++i) {
              const float4 a = c4s[i], b = __ldg(q4 + i);
              float o;
              o = fmaf(-dq, a.x, b.x); o2 = fmaf(o, o, o2);
              o = fmaf(-dq, a.y, b.y); o2 = fmaf(o, o, o2);
              o = fmaf(-dq, a.z, b.z); o2 = fmaf(o, o, o2);
              o = fmaf(-dq, a.w, b.w); o2 = fmaf(o, o, o2);
            }
            sphi = fminf(1.f, sqrtf(o2) / nrm);
          }
          float ub;
          if (cphi >= cw - slack) ub = nrm * (1.f + slack);
          else ub = nrm * (fmaf(cphi, cw, sphi * sw) + 2.f * slack);
          const float lb = (k <= kmax) ? LB[(int64_t)(k - 1) * nb + B] : -INFINITY;
          keep = !(ub < lb);
        }
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    // the same decisions as a dense bitmask per leaf: bit j of word j / 32
    if (kept_mask && lane == 0 && (j0 + threadIdx.x) / 32 < mask_words)
      kept_mask[(int64_t)B * mask_words + (j0 + threadIdx.x) / 32] = m;
    if (m) {
      int base = 0;
      const int leader = __ffs(m) - 1;
      if (lane == leader) base = atomicAdd(&cnt, __popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (keep) pairs[(int64_t)B * nq + base + __popc(m & ((1u << lane) - 1u))] = PairEntry{j, cphi, sphi};
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    pcount[B] = cnt;
    if (cnt) {
      const int users = bstart[B + 1] - bstart[B];
      atomicAdd(&stats[ST_PAIRS_KEPT], (unsigned long long)cnt);
      atomicAdd(&stats[ST_KEPT_USERS], (unsigned long long)users);
      // the tensor-core user pass scores every (user, query) pair of the kept leaves
      if (count_pairs) atomicAdd(&stats[ST_USERS_SCORED], (unsigned long long)cnt * users);
    }
  }
}

// ---------------------------------------------------------------- A4: user pass
// One CTA per leaf, one thread per user; the leaf's user rows are staged in shared
// memory (odd float4 stride: conflict-free 16-byte loads), and so are the leaf's
// surviving (query, k, ||q||, cos phi, sin phi) records, 512 at a time.  The lower bound
// of the next record is loaded one iteration ahead.
struct PairInfo {
  int32_t j, k;
  float cphi, sphi, nrm;
};
constexpr int kPairChunk = 512;

__global__ void user_scan_kernel(const float* __restrict__ Ut, const float* __restrict__ unorm,
                                 const float* __restrict__ ucos, const float* __restrict__ usin,
                                 const int32_t* __restrict__ uid, const int32_t* __restrict__ bstart,
                                 const float* __restrict__ Lt, const float* __restrict__ Eu,
                                 const float* __restrict__ pnorm, int64_t n, int64_t mz, int kmax,
                                 int l_exact, int dp, const float* __restrict__ Qd,
                                 const float* __restrict__ qn, const int32_t* __restrict__ kk, int nq,
                                 const PairEntry* __restrict__ pairs, const int32_t* __restrict__ pcount,
                                 float gamma, float slack, uint32_t* __restrict__ bitmap, int64_t words,
                                 Survivor* __restrict__ surv, unsigned long long* __restrict__ surv_count,
                                 int64_t surv_cap, unsigned long long* __restrict__ stats, int stage,
                                 const int32_t* __restrict__ modes, const double* __restrict__ T64, int d) {
  // survivors of exact-mode queries go to surv[0, surv_cap) (counter surv_count[0]),
  // those of SA-ALSH-mode queries with k <= k_max to surv[surv_cap, 2 surv_cap)
  extern __shared__ float4 us4[];
  const int B = blockIdx.x;
  const int npairs = pcount[B];
  if (npairs == 0) return;
  const int s = bstart[B], e = bstart[B + 1];
  const int cnt = e - s;
  const int dp4 = dp / 4, stride4 = dp4 | 1;
  PairInfo* pinfo = reinterpret_cast<PairInfo*>(us4 + (stage ? (size_t)blockDim.x * stride4 : 0));
  if (stage) {
    for (int i = threadIdx.x; i < cnt * dp4; i += blockDim.x) {
      const int r = i / dp4, c = i % dp4;
      us4[r * stride4 + c] = reinterpret_cast<const float4*>(Ut + (int64_t)(s + r) * dp)[c];
    }
  }
  const int t = threadIdx.x;
  const bool active = t < cnt;
  const int r = s + t;
  float nu = 0.f, ct = 0.f, st_ = 0.f, E = 0.f;
  int32_t id = 0;
  if (active) {
    nu = unorm[r];
    ct = ucos[r];
    st_ = usin[r];
    E = Eu[r];
    id = uid[r];
  }
  // rows too wide to stage for the whole leaf are read from global memory (L1/L2)
  const float4* myu = stage ? us4 + t * stride4
                            : reinterpret_cast<const float4*>(Ut + (int64_t)(active ? r : s) * dp);
  unsigned long long scored = 0, yes_early = 0, fp64_here = 0;
  const int lane = threadIdx.x & 31;
  for (int p0 = 0; p0 < npairs; p0 += kPairChunk) {
    const int pn = min(kPairChunk, npairs - p0);
    __syncthreads();
    for (int i = threadIdx.x; i < pn; i += blockDim.x) {
      const PairEntry pe = pairs[(int64_t)B * nq + p0 + i];
      const int kj = kk[pe.j];
      const int sa = (modes != nullptr && modes[pe.j] == SAH_SAALSH && kj <= kmax) ? 1 : 0;
      pinfo[i] = PairInfo{pe.j | (sa << 30), kj, pe.cphi, pe.sphi, qn[pe.j]};
    }
    __syncthreads();
    float Lnext = 0.f;
    if (active) {
      const int k0 = pinfo[0].k;
      Lnext = (k0 <= kmax) ? Lt[(int64_t)(k0 - 1) * mz + r] : -INFINITY;
    }
    for (int pi = 0; pi < pn; ++pi) {
      const PairInfo pe = pinfo[pi];
      const float L = Lnext;
      if (active && pi + 1 < pn) {
        const int k1 = pinfo[pi + 1].k;
        Lnext = (k1 <= kmax) ? Lt[(int64_t)(k1 - 1) * mz + r] : -INFINITY;
      }
      const int j = pe.j & 0x3fffffff, k = pe.k;
      const bool sa_row = (pe.j >> 30) & 1;
      const float nrm = pe.nrm;
      bool surv_flag = false, yes = false;
      float sq = 0.f;
      if (active) {
        const float Llo = (L == -INFINITY) ? -INFINITY : __fsub_rd(L, E);
        bool pruned = false;
        if (pe.cphi <= 1.5f) {   // Lemma 3 with the slack of the FP32 terms
          const float ub = __fmul_ru(__fmul_ru(nu, nrm), fmaf(pe.cphi, ct, pe.sphi * st_) + 2.f * slack);
          pruned = ub < Llo;
        }
        if (!pruned) {
          ++scored;
          const float4* q4 = reinterpret_cast<const float4*>(Qd + (int64_t)j * dp);
          float acc = 0.f;
          for (int c = 0; c < dp4; ++c) {
            const float4 a = myu[c], b = __ldg(q4 + c);
            acc = fmaf(a.x, b.x, acc);
            acc = fmaf(a.y, b.y, acc);
            acc = fmaf(a.z, b.z, acc);
            acc = fmaf(a.w, b.w, acc);
          }
          sq = acc;
          const float eq = __fmul_ru(__fmul_ru(gamma, nu), nrm) + 1e-30f;
          const float hi = __fadd_ru(sq, eq), lo = __fsub_rd(sq, eq);
          if (hi < Llo) {
            // "no": at least k items of P' score above <u,q>
          } else if (l_exact && k <= kmax && lo >= __fadd_ru(L, E)) {
            yes = true;                        // <u,q> >= exact k-th largest score
          } else if (lo >= __fmul_ru(__fmul_ru(nu, pnorm[k - 1]), 1.f + 2.f * gamma)) {
            yes = true;                        // <u,q> >= ||u|| ||p_k|| >= k-th largest score
          } else if (T64 != nullptr && k <= kmax && !sa_row) {
            // exact thresholds: the count rule in double precision is <u,q> >= tau_u(k)
            const double t64 = T64[(int64_t)(k - 1) * mz + r];
            if (t64 == t64) {
              ++fp64_here;
              yes = dot64_seq(reinterpret_cast<const float*>(Ut + (int64_t)r * dp), Qd + (int64_t)j * dp, d) >= t64;
            } else {
              surv_flag = true;
            }
          } else {
            surv_flag = true;
          }
        }
      }
      if (yes) {
        ++yes_early;
        set_answer(bitmap, words, j, id);
      }
      // every record in this loop iteration belongs to one query, so one list per warp step
      const unsigned m = __ballot_sync(0xffffffffu, surv_flag);
      if (m) {
        unsigned long long base = 0;
        const int leader = __ffs(m) - 1;
        if (lane == leader) base = atomicAdd(surv_count + (sa_row ? 1 : 0), (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (surv_flag) {
          const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
          if ((int64_t)slot < surv_cap) surv[(sa_row ? surv_cap : 0) + slot] = Survivor{r, j, sq};
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    scored += __shfl_xor_sync(0xffffffffu, scored, o);
    yes_early += __shfl_xor_sync(0xffffffffu, yes_early, o);
    fp64_here += __shfl_xor_sync(0xffffffffu, fp64_here, o);
  }
  if (lane == 0) {
    if (scored) atomicAdd(&stats[ST_USERS_SCORED], scored);
    if (yes_early) atomicAdd(&stats[ST_YES_EARLY], yes_early);
    if (fp64_here) atomicAdd(&stats[ST_FP64], fp64_here);
  }
}

// Register-tiled form of the user pass for d <= 128: each thread keeps its user's row in
// registers; the leaf's surviving queries are staged in shared memory kQChunk at a time
// and scored kQG at a time (kQG FMAs per broadcast shared-memory load).  Every (user,
// query) decision is the same as in user_scan_kernel: Lemma 3 first, then the FP32
// score against the lower bound, the exact threshold and the ||p_k|| bound.
constexpr int kQG = 4;
constexpr int kQChunk = 128;

template <int DP4MAX>
__global__ void __launch_bounds__(256)
user_scan_reg_kernel(const float* __restrict__ Ut, const float* __restrict__ unorm,
                     const float* __restrict__ ucos, const float* __restrict__ usin,
                     const int32_t* __restrict__ uid, const int32_t* __restrict__ bstart,
                     const float* __restrict__ Lt, const float* __restrict__ Eu,
                     const float* __restrict__ pnorm, int64_t n, int64_t mz, int kmax,
                     int l_exact, int dp, const float* __restrict__ Qd,
                     const float* __restrict__ qn, const int32_t* __restrict__ kk, int nq,
                     const PairEntry* __restrict__ pairs, const int32_t* __restrict__ pcount,
                     float gamma, float slack, uint32_t* __restrict__ bitmap, int64_t words,
                     Survivor* __restrict__ surv, unsigned long long* __restrict__ surv_count,
                     int64_t surv_cap, unsigned long long* __restrict__ stats,
                     const int32_t* __restrict__ modes, const double* __restrict__ T64, int d) {
  extern __shared__ float4 sq4[];
  __shared__ int32_t kslot[65], klist[64];
  __shared__ int32_t nslots;
  const int B = blockIdx.x;
  const int npairs = pcount[B];
  if (npairs == 0) return;
  const int s = bstart[B], e = bstart[B + 1];
  const int cnt = e - s;
  const int dp4 = dp / 4;
  float4* qs = sq4;                                              // kQChunk x dp4
  PairInfo* pinfo = reinterpret_cast<PairInfo*>(qs + (size_t)kQChunk * dp4);
  float* Ls = reinterpret_cast<float*>(pinfo + kQChunk);         // [nslots][blockDim]
  const int t = threadIdx.x;
  const bool active = t < cnt;
  const int r = s + (active ? t : 0);
  // lower bounds of the k values this leaf's queries ask for, one row per distinct k
  for (int k = t; k <= 64; k += blockDim.x) kslot[k] = -1;
  __syncthreads();
  for (int i = t; i < npairs; i += blockDim.x) {
    const int k = kk[pairs[(int64_t)B * nq + i].j];
    if (k <= kmax) kslot[k] = 0;
  }
  __syncthreads();
  if (t == 0) {
    int ns = 0;
    for (int k = 1; k <= kmax; ++k)
      if (kslot[k] == 0) {
        kslot[k] = ns;
        klist[ns++] = k;
      }
    nslots = ns;
  }
  __syncthreads();
  for (int sl = 0; sl < nslots; ++sl)
    Ls[sl * blockDim.x + t] = active ? Lt[(int64_t)(klist[sl] - 1) * mz + r] : -INFINITY;
  float4 ur[DP4MAX];
#pragma unroll
  for (int c = 0; c < DP4MAX; ++c)
    ur[c] = (c < dp4 && active) ? reinterpret_cast<const float4*>(Ut + (int64_t)r * dp)[c]
                                : make_float4(0.f, 0.f, 0.f, 0.f);
  float nu = 0.f, ct = 0.f, st_ = 0.f, E = 0.f;
  int32_t id = 0;
  if (active) {
    nu = unorm[r];
    ct = ucos[r];
    st_ = usin[r];
    E = Eu[r];
    id = uid[r];
  }
  const float nun = __fmul_ru(nu, 1.f + 2.f * gamma);
  unsigned long long scored = 0, yes_early = 0, fp64_here = 0;
  const int lane = threadIdx.x & 31;
  for (int p0 = 0; p0 < npairs; p0 += kQChunk) {
    const int pn = min(kQChunk, npairs - p0);
    __syncthreads();
    for (int i = threadIdx.x; i < pn; i += blockDim.x) {
      const PairEntry pe = pairs[(int64_t)B * nq + p0 + i];
      const int kj = kk[pe.j];
      const int sa = (modes != nullptr && modes[pe.j] == SAH_SAALSH && kj <= kmax) ? 1 : 0;
      // k is stored with its lower-bound slot in the high bits
      const int slot = kj <= kmax ? kslot[kj] : 63;
      pinfo[i] = PairInfo{pe.j | (sa << 30), kj | (slot << 24), pe.cphi, pe.sphi, qn[pe.j]};
    }
    __syncthreads();
    for (int i = threadIdx.x; i < pn * dp4; i += blockDim.x) {
      const int row = i / dp4, c = i % dp4;
      qs[i] = reinterpret_cast<const float4*>(Qd + (int64_t)(pinfo[row].j & 0x3fffffff) * dp)[c];
    }
    __syncthreads();
    for (int pi = 0; pi < pn; pi += kQG) {
      // Lemma 3 first: groups no lane of the warp needs are not scored at all
      float Lg[kQG], Llo[kQG];
      bool need[kQG];
#pragma unroll
      for (int g = 0; g < kQG; ++g) {
        const int col = min(pi + g, pn - 1);
        const PairInfo pe = pinfo[col];
        const int k = pe.k & 0xffffff, slot = pe.k >> 24;
        Lg[g] = (k <= kmax) ? Ls[slot * blockDim.x + t] : -INFINITY;
        Llo[g] = (Lg[g] == -INFINITY) ? -INFINITY : __fsub_rd(Lg[g], E);
        bool pruned = false;
        if (pe.cphi <= 1.5f) {
          const float ub = __fmul_ru(__fmul_ru(nu, pe.nrm), fmaf(pe.cphi, ct, pe.sphi * st_) + 2.f * slack);
          pruned = ub < Llo[g];
        }
        need[g] = active && (pi + g < pn) && !pruned;
      }
      const bool any = __any_sync(0xffffffffu, need[0] || need[1] || need[2] || need[3]);
      if (!any) continue;
      // four partial sums per query (one per float4 lane): 16 independent FMA chains
      float ax[kQG], ay[kQG], az[kQG], aw[kQG];
#pragma unroll
      for (int g = 0; g < kQG; ++g) ax[g] = ay[g] = az[g] = aw[g] = 0.f;
#pragma unroll
      for (int c = 0; c < DP4MAX; ++c) {
        if (c < dp4) {
          const float4 a = ur[c];
#pragma unroll
          for (int g = 0; g < kQG; ++g) {
            const float4 b = qs[(pi + g) * dp4 + c];
            ax[g] = fmaf(a.x, b.x, ax[g]);
            ay[g] = fmaf(a.y, b.y, ay[g]);
            az[g] = fmaf(a.z, b.z, az[g]);
            aw[g] = fmaf(a.w, b.w, aw[g]);
          }
        }
      }
#pragma unroll
      for (int g = 0; g < kQG; ++g) {
        if (pi + g >= pn) break;
        const PairInfo pe = pinfo[pi + g];
        const int j = pe.j & 0x3fffffff, k = pe.k & 0xffffff;
        const bool sa_row = (pe.j >> 30) & 1;
        bool surv_flag = false, yes = false;
        const float sq = (ax[g] + ay[g]) + (az[g] + aw[g]);
        if (need[g]) {
          ++scored;
          const float L = Lg[g];
          const float eq = __fmul_ru(__fmul_ru(gamma, nu), pe.nrm) + 1e-30f;
          const float hi = __fadd_ru(sq, eq), lo = __fsub_rd(sq, eq);
          if (hi < Llo[g]) {
            // "no": at least k items of P' score above <u,q>
          } else if (l_exact && k <= kmax && lo >= __fadd_ru(L, E)) {
            yes = true;
          } else if (lo >= __fmul_ru(nun, pnorm[k - 1])) {
            yes = true;
          } else if (T64 != nullptr && k <= kmax && !sa_row) {
            const double t64 = T64[(int64_t)(k - 1) * mz + r];
            if (t64 == t64) {
              ++fp64_here;
              yes = dot64_seq(Ut + (int64_t)r * dp, Qd + (int64_t)j * dp, d) >= t64;
            } else {
              surv_flag = true;
            }
          } else {
            surv_flag = true;
          }
        }
        if (yes) {
          ++yes_early;
          set_answer(bitmap, words, j, id);
        }
        const unsigned m = __ballot_sync(0xffffffffu, surv_flag);
        if (m) {
          unsigned long long base = 0;
          const int leader = __ffs(m) - 1;
          if (lane == leader) base = atomicAdd(surv_count + (sa_row ? 1 : 0), (unsigned long long)__popc(m));
          base = __shfl_sync(0xffffffffu, base, leader);
          if (surv_flag) {
            const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
            if ((int64_t)slot < surv_cap) surv[(sa_row ? surv_cap : 0) + slot] = Survivor{r, j, sq};
          }
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    scored += __shfl_xor_sync(0xffffffffu, scored, o);
    yes_early += __shfl_xor_sync(0xffffffffu, yes_early, o);
    fp64_here += __shfl_xor_sync(0xffffffffu, fp64_here, o);
  }
  if (lane == 0) {
    if (scored) atomicAdd(&stats[ST_USERS_SCORED], scored);
    if (yes_early) atomicAdd(&stats[ST_YES_EARLY], yes_early);
    if (fp64_here) atomicAdd(&stats[ST_FP64], fp64_here);
  }
}

// ---------------------------------------------------------------- A5 + A6: verify
// One warp per survivor.  Item scores in FP32 with the a-priori bound
//   |fl(<u,p>) - <u,p>| <= gamma ||u|| ||p||;
// an item is certainly above <u,q> when s_p - e_p > s_q + e_q, certainly not when
// s_p + e_p <= s_q - e_q, and in the band otherwise.  Band items (up to 32) are decided
// in double precision; a larger band falls back to a full double-precision count.
constexpr int kVerifyWarps = 8;

__global__ void __launch_bounds__(kVerifyWarps * 32)
verify_exact_kernel(const Survivor* __restrict__ surv, const unsigned long long* __restrict__ surv_count,
                    int64_t surv_cap, const float* __restrict__ Ut, const float* __restrict__ unorm,
                    const int32_t* __restrict__ uid, const float* __restrict__ Ps,
                    const float* __restrict__ pnorm, int64_t n, int d, int dp,
                    const float* __restrict__ Qd, const float* __restrict__ qn,
                    const int32_t* __restrict__ kk, float gamma, uint32_t* __restrict__ bitmap,
                    int64_t words, unsigned long long* __restrict__ stats) {
  extern __shared__ float4 vs4[];            // kVerifyWarps x dp4 user rows
  __shared__ int32_t band_list[kVerifyWarps][32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int dp4 = dp / 4;
  float4* myu = vs4 + warp * dp4;
  int64_t total = block_count(surv_count, surv_cap);
  int64_t gw = (int64_t)blockIdx.x * kVerifyWarps + warp;
  int64_t nwarps = (int64_t)gridDim.x * kVerifyWarps;
  unsigned long long fp64_cnt = 0, scanned = 0;
  for (int64_t si = gw; si < total; si += nwarps) {
    Survivor S = surv[si];
    int k = kk[S.j];
    const float* urow = Ut + (int64_t)S.upos * dp;
    for (int c = lane; c < dp4; c += 32) myu[c] = reinterpret_cast<const float4*>(urow)[c];
    __syncwarp();
    float nu = unorm[S.upos];
    float eq = __fmul_ru(__fmul_ru(gamma, nu), qn[S.j]) + 1e-30f;
    float hi = __fadd_ru(S.sq, eq), lo = __fsub_rd(S.sq, eq);
    float gnu = __fmul_ru(gamma, nu);
    float cut_scale = __fmul_ru(nu, 1.f + 2.f * gamma);
    int above = 0, band = 0;
    for (int64_t base = 0; base < n; base += 32) {
      if (__fmul_ru(cut_scale, pnorm[base]) <= lo) break;   // no later item can beat <u,q>
      int64_t i = base + lane;
      bool is_above = false, is_band = false;
      if (i < n) {
        const float4* p4 = reinterpret_cast<const float4*>(Ps + i * dp);
        float acc = 0.f;
        for (int c = 0; c < dp4; ++c) {
          float4 a = myu[c], b = __ldg(p4 + c);
          acc = fmaf(a.x, b.x, acc);
          acc = fmaf(a.y, b.y, acc);
          acc = fmaf(a.z, b.z, acc);
          acc = fmaf(a.w, b.w, acc);
        }
        float ep = __fmul_ru(gnu, pnorm[i]) + 1e-30f;
        is_above = __fsub_rd(acc, ep) > hi;
        is_band = !is_above && __fadd_ru(acc, ep) > lo;
      }
      above += __popc(__ballot_sync(0xffffffffu, is_above));
      unsigned bm = __ballot_sync(0xffffffffu, is_band);
      if (is_band) {
        int slot = band + __popc(bm & ((1u << lane) - 1u));
        if (slot < 32) band_list[warp][slot] = (int32_t)i;
      }
      band += __popc(bm);
      scanned += (unsigned long long)((n - base) < 32 ? (n - base) : 32);
      if (above >= k) break;
    }
    __syncwarp();
    bool yes;
    if (above >= k) {
      yes = false;
    } else if (above + band < k) {
      yes = true;
    } else {
      ++fp64_cnt;
      const float* urow_f = Ut + (int64_t)S.upos * dp;
      const float* q = Qd + (int64_t)S.j * dp;
      double s64q = dot64_seq(urow_f, q, d);
      int c = above;
      if (band <= 32) {
        bool gt = false;
        if (lane < band) gt = dot64_seq(urow_f, Ps + (int64_t)band_list[warp][lane] * dp, d) > s64q;
        c += __popc(__ballot_sync(0xffffffffu, gt));
      } else {
        c = 0;
        for (int64_t base = 0; base < n && c < k; base += 32) {
          int64_t i = base + lane;
          bool gt = (i < n) && dot64_seq(urow_f, Ps + i * dp, d) > s64q;
          c += __popc(__ballot_sync(0xffffffffu, gt));
        }
      }
      yes = c < k;
    }
    if (yes && lane == 0) {
      int32_t id = uid[S.upos];
      set_answer(bitmap, words, S.j, id);
    }
    __syncwarp();
  }
  if (lane == 0 && fp64_cnt) atomicAdd(&stats[ST_FP64], fp64_cnt);
  if (lane == 0 && scanned) atomicAdd(&stats[ST_ITEMS], scanned);
}

// ---------------------------------------------------------------- A7: special users, compaction
__global__ void zero_users_kernel(const int32_t* __restrict__ zid, int64_t nz, int nq,
                                  uint32_t* __restrict__ bitmap, int64_t words) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nz * nq) return;
  int j = (int)(t / nz);
  int32_t id = zid[t % nz];
  set_answer(bitmap, words, j, id);
}

// Answers per summary word, then their scan.  Per query j: a summary word sw that marks any
// bitmap word gets its count of answers; the exclusive prefix of the counts within the query
// is written to wpre[j * nsw + sw] and the word is appended to list; cnt[j] gets the query's
// total; a row with k > n counts every summary word's users.  The last CTA of the second
// kernel (a ticket taken after a fence) turns the totals into the offsets: offsets[j] = base
// + the answers of the queries before j, offsets[nq] the end (also into offsets2 when
// given).
//
// answer_count_light_kernel, a warp per query (kAnswerWarps per CTA): the lanes read the top
// words and count the summary words they mark; a query with at most kLightWords of them is
// counted here, one summary word per lane and round (a lane finds its word from the scan of
// the top words' bit counts), every other query (and every row with k > n) goes to the heavy
// list.  answer_count_heavy_kernel, a CTA of kHeavyThreads per listed query (the CTAs loop
// over the list): the marked summary words dealt out the same way, a thread per word and
// kHeavyThreads words per step, a block scan per step (a row with k > n: every summary
// word).  Either way a summary word's bitmap words are read by predicated loads that all go
// out before any is used.
constexpr int kAnswerWarps = 8;
constexpr int kLightWords = 64;
constexpr int kHeavyThreads = 512;

__device__ __forceinline__ int warp_inclusive_scan(int x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Position of the n-th set bit of x (n counted from 0, n < popc(x)): halving the word.
__device__ __forceinline__ int nth_set_bit(uint32_t x, int n) {
  int pos = 0;
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const int c = __popc(x & ((1u << h) - 1u));
    if (n >= c) {
      n -= c;
      x >>= h;
      pos += h;
    }
  }
  return pos;
}

// The answers in the bitmap words p[b] whose bit b of sm is set: 32 predicated loads issued
// back to back, then their bit counts.
__device__ __forceinline__ int count_marked_words(const uint32_t* p, uint32_t sm) {
  uint32_t v[32];
#pragma unroll
  for (int b = 0; b < 32; ++b) {
    v[b] = 0u;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.u32 %0, [%1];\n\t}"
        : "+r"(v[b])
        : "l"(p + b), "r"(sm & (1u << b)));
  }
  int c = 0;
#pragma unroll
  for (int b = 0; b < 32; ++b) c += __popc(v[b]);
  return c;
}

// Users a summary word of a k > n row holds.
__device__ __forceinline__ int all_users_in(int sw, int64_t m) {
  return (int)std::max<int64_t>(0, std::min<int64_t>(1024, m - (int64_t)sw * 1024));
}

__global__ void __launch_bounds__(kAnswerWarps * 32)
answer_count_light_kernel(const uint32_t* __restrict__ bitmap, int64_t stride, const int32_t* __restrict__ kk,
                          int64_t n, int32_t* __restrict__ wpre, int32_t* __restrict__ list,
                          unsigned int* __restrict__ list_count, int32_t* __restrict__ cnt,
                          int32_t* __restrict__ heavy, unsigned int* __restrict__ heavy_count, int nq) {
  const int64_t w = answer_words(stride);
  const int nsw = (int)(w / 32), ntop = (int)(w / 1024);
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * kAnswerWarps + (threadIdx.x >> 5);
  if (j >= nq) return;   // warp-uniform; no block barrier follows
  const uint32_t* row = bitmap + (int64_t)j * stride;
  int marked = 0;
  if (kk[j] <= n) {
    for (int t0 = 0; t0 < ntop; t0 += 32) marked += __popc(t0 + lane < ntop ? row[w + nsw + t0 + lane] : 0u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) marked += __shfl_xor_sync(0xffffffffu, marked, o);
  }
  if (kk[j] > n || marked > kLightWords) {
    if (lane == 0) heavy[atomicAdd(heavy_count, 1u)] = j;
    return;
  }
  const int64_t g0 = (int64_t)j * nsw;
  int carry = 0;
  for (int t0 = 0; t0 < ntop && marked > 0; t0 += 32) {
    const uint32_t top = t0 + lane < ntop ? row[w + nsw + t0 + lane] : 0u;
    const int pc = __popc(top);
    const int incl = warp_inclusive_scan(pc, lane);
    const int excl = incl - pc;
    const int here = __shfl_sync(0xffffffffu, incl, 31);
    marked -= here;
    for (int r0 = 0; r0 < here; r0 += 32) {
      // this lane's summary word, the r-th marked one: its top word is the first lane's with
      // incl > r (a binary search over the lanes' inclusive counts, every lane taking part)
      const int r = r0 + lane;
      int lo = 0, hi = 31;
#pragma unroll
      for (int step = 0; step < 5; ++step) {
        const int mid = (lo + hi) >> 1;
        const int im = __shfl_sync(0xffffffffu, incl, mid);
        if (im > r) hi = mid; else lo = mid + 1;
      }
      const uint32_t tl = __shfl_sync(0xffffffffu, top, lo);
      const int el = __shfl_sync(0xffffffffu, excl, lo);
      int c = 0, sw = 0;
      if (r < here) {
        sw = (t0 + lo) * 32 + nth_set_bit(tl, r - el);
        c = count_marked_words(row + (int64_t)sw * 32, row[w + sw]);
      }
      const int ci = warp_inclusive_scan(c, lane);
      const unsigned mk = __ballot_sync(0xffffffffu, c > 0);
      unsigned b0 = 0;
      if (lane == 0 && mk) b0 = atomicAdd(list_count, (unsigned)__popc(mk));
      b0 = __shfl_sync(0xffffffffu, b0, 0);
      if (c > 0) {
        const int g = (int)(g0 + sw);
        wpre[g] = carry + ci - c;
        list[b0 + __popc(mk & ((1u << lane) - 1u))] = g;
      }
      carry += __shfl_sync(0xffffffffu, ci, 31);
    }
  }
  if (lane == 0) cnt[j] = carry;
}

__device__ inline int block_exclusive_scan(int v, int* total) {
  __shared__ int wsum[32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  int nw = blockDim.x >> 5;
  int before = 0, all = 0;
  for (int w = 0; w < nw; ++w) {
    if (w < warp) before += wsum[w];
    all += wsum[w];
  }
  __syncthreads();
  *total = all;
  return before + x - v;
}

// One step of a heavy query: each thread's count c of word g; its prefix (carry + the block's
// exclusive scan) for the listed words and the list entries; returns the step's total.
__device__ __forceinline__ int heavy_step(int c, int g, int carry, int lane, int32_t* __restrict__ wpre,
                                          int32_t* __restrict__ list, unsigned int* __restrict__ list_count) {
  int tot;
  const int pre = block_exclusive_scan(c, &tot);
  if (c > 0) wpre[g] = carry + pre;
  const unsigned mk = __ballot_sync(0xffffffffu, c > 0);
  if (mk) {
    unsigned b0 = 0;
    if (lane == 0) b0 = atomicAdd(list_count, (unsigned)__popc(mk));
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    if (c > 0) list[b0 + __popc(mk & ((1u << lane) - 1u))] = g;
  }
  return tot;
}

__global__ void __launch_bounds__(kHeavyThreads)
answer_count_heavy_kernel(const uint32_t* __restrict__ bitmap, int64_t stride, const int32_t* __restrict__ kk,
                          int64_t n, int64_t m, int32_t* __restrict__ wpre, int32_t* __restrict__ list,
                          unsigned int* __restrict__ list_count, int32_t* __restrict__ cnt,
                          const int32_t* __restrict__ heavy, const unsigned int* __restrict__ heavy_count, int nq,
                          int64_t base, int64_t* __restrict__ offsets, int64_t* __restrict__ offsets2,
                          unsigned int* __restrict__ ticket) {
  const int64_t w = answer_words(stride);
  const int nsw = (int)(w / 32), ntop = (int)(w / 1024);
  const int lane = threadIdx.x & 31;
  const int nh = (int)*heavy_count;
  __shared__ uint32_t tw[kHeavyThreads];   // a chunk of top words
  __shared__ int tpre[kHeavyThreads];      // the exclusive prefix of their bit counts
  for (int h = blockIdx.x; h < nh; h += gridDim.x) {
    const int j = heavy[h];
    const uint32_t* row = bitmap + (int64_t)j * stride;
    const int64_t g0 = (int64_t)j * nsw;
    int carry = 0;
    if (kk[j] > n) {
      // every user: each summary word's users, kHeavyThreads words per step
      for (int c0 = 0; c0 < nsw; c0 += kHeavyThreads) {
        const int sw = c0 + threadIdx.x;
        const int c = sw < nsw ? all_users_in(sw, m) : 0;
        carry += heavy_step(c, (int)(g0 + sw), carry, lane, wpre, list, list_count);
      }
    } else {
      // the summary words the top words mark, dealt out in ascending order: a thread per
      // marked word and step, which finds its top word by a binary search over the prefix
      for (int t0 = 0; t0 < ntop; t0 += kHeavyThreads) {
        const int nt = min(kHeavyThreads, ntop - t0);
        const uint32_t top = (int)threadIdx.x < nt ? row[w + nsw + t0 + threadIdx.x] : 0u;
        int marked;
        const int ex = block_exclusive_scan(__popc(top), &marked);
        tw[threadIdx.x] = top;
        tpre[threadIdx.x] = ex;
        __syncthreads();
        for (int r0 = 0; r0 < marked; r0 += kHeavyThreads) {
          const int r = r0 + threadIdx.x;
          int c = 0, sw = 0;
          if (r < marked) {
            int lo = 0, hi = nt - 1;   // the last top word whose prefix is <= r holds it
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (tpre[mid] <= r) lo = mid; else hi = mid - 1;
            }
            sw = (t0 + lo) * 32 + nth_set_bit(tw[lo], r - tpre[lo]);
            c = count_marked_words(row + (int64_t)sw * 32, row[w + sw]);
          }
          carry += heavy_step(c, (int)(g0 + sw), carry, lane, wpre, list, list_count);
        }
        __syncthreads();   // the chunk's top words are read until here
      }
    }
    if (threadIdx.x == 0) cnt[j] = carry;
  }
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the query offsets, in 64 bits: a contiguous run of queries per thread (loads from L2,
  // where the other CTAs' totals are), then a block scan
  __shared__ long long wtot[kHeavyThreads / 32];
  const int warp = threadIdx.x >> 5;
  const int qper = (nq + blockDim.x - 1) / blockDim.x;
  const int q0 = min((int)threadIdx.x * qper, nq), q1 = min(q0 + qper, nq);
  long long t = 0;
  for (int q = q0; q < q1; ++q) t += __ldcg(&cnt[q]);
  long long x = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtot[warp] = x;
  __syncthreads();
  long long before = base, all = base;
  for (int v = 0; v < kHeavyThreads / 32; ++v) {
    if (v < warp) before += wtot[v];
    all += wtot[v];
  }
  long long o = before + x - t;
  for (int q = q0; q < q1; ++q) {
    offsets[q] = o;
    if (offsets2) offsets2[q] = o;
    o += __ldcg(&cnt[q]);
  }
  if (threadIdx.x == 0) {
    offsets[nq] = all;
    if (offsets2) offsets2[nq] = all;
  }
}

// Emission, a warp per batch of kEmitBatch listed summary words (query j, word sw): lanes
// 0..kEmitBatch-1 read the words' list entries, summaries and output positions, then every
// lane l reads bitmap word 32 sw + l of each listed word (all loads in flight at once) and
// writes its ids at offsets[j] plus the scanned count before the summary word plus the
// lane's share, in ascending order, clearing the words it read so that the bitmap is zero
// for the next call.  A row with k > n writes the summary word's 1024 users.  Only if the
// call's total fits in out_cap; otherwise it raises *overflow and leaves the bitmap as it is.
constexpr int kEmitBatch = 8;

__global__ void answer_emit_kernel(uint32_t* __restrict__ bitmap, int64_t stride,
                                   const int32_t* __restrict__ kk, int64_t n, int64_t m,
                                   const int32_t* __restrict__ wpre, const int32_t* __restrict__ list,
                                   const unsigned int* __restrict__ list_count,
                                   const int64_t* __restrict__ offsets, int nq, int32_t* __restrict__ out,
                                   int64_t out_cap, unsigned long long* __restrict__ overflow) {
  const int lane = threadIdx.x & 31;
  const int64_t w = answer_words(stride);
  const int nsw = (int)(w / 32);
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (offsets[nq] > out_cap) {
    if (gw == 0 && lane == 0) atomicExch(overflow, 1ull);
    return;
  }
  const int64_t nl = *list_count;
  for (int64_t e0 = gw * kEmitBatch; e0 < nl; e0 += nwarps * kEmitBatch) {
    int g = -1;
    uint32_t sm = 0;
    int64_t dst = 0;
    int all = 0;
    if (lane < kEmitBatch && e0 + lane < nl) {
      g = list[e0 + lane];
      const int j = g / nsw, sw = g - j * nsw;
      sm = bitmap[(int64_t)j * stride + w + sw];
      dst = offsets[j] + wpre[g];
      all = kk[j] > n ? 1 : 0;
    }
    uint32_t v[kEmitBatch];
#pragma unroll
    for (int e = 0; e < kEmitBatch; ++e) {
      const int ge = __shfl_sync(0xffffffffu, g, e);
      const uint32_t se = __shfl_sync(0xffffffffu, sm, e);
      v[e] = 0u;
      if (ge >= 0 && ((se >> lane) & 1u)) {
        const int je = ge / nsw, swe = ge - je * nsw;
        v[e] = bitmap[(int64_t)je * stride + (int64_t)swe * 32 + lane];
      }
    }
#pragma unroll
    for (int e = 0; e < kEmitBatch; ++e) {
      const int ge = __shfl_sync(0xffffffffu, g, e);
      const uint32_t se = __shfl_sync(0xffffffffu, sm, e);
      const int64_t de = __shfl_sync(0xffffffffu, dst, e);
      const int ae = __shfl_sync(0xffffffffu, all, e);
      if (ge < 0) continue;   // warp-uniform
      const int je = ge / nsw, swe = ge - je * nsw;
      uint32_t* row = bitmap + (int64_t)je * stride;
      if ((se >> lane) & 1u) row[(int64_t)swe * 32 + lane] = 0u;
      if (lane == 0 && se) {
        row[w + swe] = 0u;
        row[w + nsw + (swe >> 5)] = 0u;   // the top word (every listed word under it clears it)
      }
      if (ae) {
        const int64_t lo = (int64_t)swe * 1024, hi = std::min<int64_t>(m, lo + 1024);
        for (int64_t i = lo + lane; i < hi; i += 32) out[de + (i - lo)] = (int32_t)i;
        continue;
      }
      uint32_t x = v[e];
      const int pc = __popc(x);
      int incl = pc;   // inclusive scan over the lanes
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      int64_t p = de + incl - pc;
      const int32_t base_id = (int32_t)(((int64_t)swe * 32 + lane) * 32);
      while (x) {
        const int i = __ffs(x) - 1;
        x &= x - 1;
        out[p++] = base_id + i;
      }
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- workspace
namespace {

constexpr int kCtlCounters = 7;   // survivor counts (4), answer-list length, scan ticket, heavy-list length

struct WsLayout {
  size_t qd, qb, qn, qh, kk, pairs, pcount, kmask, tneed, tneed_end, coltab, survcnt, alist_n, ticket, heavy_n, bitmap, chunk,
      offsets, stats, total;
};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

WsLayout layout_for(const Index* ix, int qb) {
  WsLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes); return r; };
  // the answer bitmaps first: the part of the workspace that stays zero between calls
  L.bitmap = take(sizeof(uint32_t) * (size_t)qb * answer_stride(ix->m));
  L.qd = take(sizeof(float) * (size_t)qb * ix->dp);
  L.qb = take(2 * sizeof(uint16_t) * (size_t)qb * std::max(ix->dk, 1));   // hi and lo parts
  L.qn = take(sizeof(float) * qb);
  L.qh = take(sizeof(uint64_t) * qb);
  L.kk = take(sizeof(int32_t) * qb);
  // the per-leaf pair lists of the CUDA-core user pass (the tensor-core pass keeps a bitmask)
  const bool tc_pass = ix->nb > 0 && ix->dk > 0 && ix->prm.tc_user_pass && ix->m_nz > 0;
  L.pairs = take(tc_pass ? 0 : sizeof(PairEntry) * (size_t)std::max(ix->nb, 1) * qb);
  L.pcount = take(sizeof(int32_t) * std::max(ix->nb, 1));
  // kept bits per (leaf, row), then one flag per leaf (the tensor-core block filter's)
  L.kmask = take(sizeof(uint32_t) * (size_t)std::max(ix->nb, 1) * ((qb + 31) / 32) + sizeof(int32_t) * std::max(ix->nb, 1));
  L.coltab = take(user_pass_tc_scratch_bytes(qb, ix->dp));
  // per-word prefixes (qb nsw) | per-query counts (qb) | listed words (qb nsw) | heavy rows (qb)
  L.chunk = take(sizeof(int32_t) * ((size_t)qb * (2 * (answer_words(answer_stride(ix->m)) / 32) + 2)));
  // the control block, contiguous so that one memset clears its counters (and, with the
  // tensor-core user pass, the tile flags) and one copy reads it back: stats[ST_COUNT] |
  // survivor counts[3] | answer-list length (u64) | scan ticket (u64) | offsets[qb + 1] |
  // one byte per 128-user tile (set by the block filter for the tiles of kept leaves)
  const size_t ntiles = (size_t)std::max<int64_t>((ix->m_nz + 127) / 128, 1);
  L.stats = take(sizeof(unsigned long long) * (ST_COUNT + kCtlCounters) + sizeof(int64_t) * (size_t)(qb + 1) + ntiles);
  L.survcnt = L.stats + sizeof(unsigned long long) * ST_COUNT;
  L.alist_n = L.survcnt + 4 * sizeof(unsigned long long);
  L.ticket = L.alist_n + sizeof(unsigned long long);
  L.heavy_n = L.ticket + sizeof(unsigned long long);
  L.offsets = L.heavy_n + sizeof(unsigned long long);
  L.tneed = L.offsets + sizeof(int64_t) * (size_t)(qb + 1);
  L.tneed_end = L.tneed + ntiles;
  L.total = o;
  return L;
}

sah_status ensure_buf(Workspace* b, size_t bytes, cudaStream_t st) {
  if (b->bytes >= bytes) return SAH_OK;
  SAH_CUDA(cudaStreamSynchronize(st));
  if (b->base) cudaFree(b->base);
  b->base = nullptr;
  b->bytes = 0;
  cudaError_t e = cudaMalloc(&b->base, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("workspace allocation failed");
    return SAH_ERR_OOM;
  }
  b->bytes = bytes;
  return SAH_OK;
}

sah_status ensure_ws(CallCtx* cx, size_t bytes, cudaStream_t st) {
  if (cx->ws.bytes >= bytes) return SAH_OK;
  ++cx->alloc_epoch;
  return ensure_buf(&cx->ws, bytes, st);
}

// three lists of cap entries: exact-mode survivors, SA-ALSH survivors, and the pairs the
// tensor-core user pass leaves to the FP32 re-score
sah_status ensure_surv(CallCtx* cx, int64_t cap, cudaStream_t st) {
  // exact survivors, SA-ALSH survivors, open pairs of the tensor-core user pass (cap entries
  // each), then its candidate blocks (cap blocks of 144 bytes)
  const size_t bytes = (3 * sizeof(Survivor) + 144) * (size_t)std::max<int64_t>(cap, 1);
  if (cx->surv.bytes >= bytes) return SAH_OK;
  ++cx->alloc_epoch;
  return ensure_buf(&cx->surv, bytes, st);
}

// Captures (begin, enqueue, end, instantiate) never overlap in one process: the server's
// workers each own a context and may replay their graphs concurrently, but one capture at a
// time.  Replays and direct launch sequences of other threads are not held up.
std::mutex g_capture_mu;

// Runs a sub-batch's launch sequence (enqueue) for the given key of shapes and buffers: the
// first time directly, the second time captured into a CUDA graph, which later calls with
// the same key replay as one launch.  A capture that fails (an operation that cannot be
// captured) marks the key, which then always runs directly.
template <class F>
sah_status run_captured(CallCtx* cx, const std::vector<uint64_t>& key, F&& enqueue, cudaStream_t st) {
  constexpr size_t kMaxGraphs = 8;
  GraphEntry* e = nullptr;
  for (GraphEntry& g : cx->graphs)
    if (g.key == key) e = &g;
  ++cx->graph_clock;
  if (!e) {
    if (cx->graphs.size() >= kMaxGraphs) {
      // the least recently used entry makes room
      size_t lru = 0;
      for (size_t i = 1; i < cx->graphs.size(); ++i)
        if (cx->graphs[i].last_use < cx->graphs[lru].last_use) lru = i;
      if (cx->graphs[lru].exec) cudaGraphExecDestroy(cx->graphs[lru].exec);
      cx->graphs.erase(cx->graphs.begin() + (std::ptrdiff_t)lru);
    }
    GraphEntry g;
    g.key = key;
    g.last_use = cx->graph_clock;
    cx->graphs.push_back(g);
    return enqueue();   // first sighting: direct (it also sizes every workspace)
  }
  e->last_use = cx->graph_clock;
  if (e->bad) return enqueue();
  if (!e->exec) {
    std::lock_guard<std::mutex> lk(g_capture_mu);
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      e->bad = true;
      return enqueue();
    }
    const sah_status s = enqueue();
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    cudaError_t ie = cudaErrorUnknown;
    if (s == SAH_OK && ce == cudaSuccess && graph) ie = cudaGraphInstantiate(&e->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (s != SAH_OK || ce != cudaSuccess || ie != cudaSuccess) {
      cudaGetLastError();
      e->exec = nullptr;
      e->bad = true;
      return enqueue();
    }
  }
  SAH_CUDA(cudaGraphLaunch(e->exec, st));
  return SAH_OK;
}

// CUDA events around each stage, on the call's stream (only when timing is enabled).
struct StageTimer {
  static constexpr int kStages = 8;
  bool on = false;
  cudaStream_t st = nullptr;
  cudaEvent_t b[kStages] = {}, e[kStages] = {};
  bool used[kStages] = {};
  double ms[kStages] = {};
  int64_t launches[kStages] = {};
  StageTimer(bool enable, cudaStream_t s) : on(enable), st(s) {
    if (!on) return;
    for (int i = 0; i < kStages; ++i) {
      cudaEventCreate(&b[i]);
      cudaEventCreate(&e[i]);
    }
  }
  ~StageTimer() {
    if (!on) return;
    for (int i = 0; i < kStages; ++i) {
      cudaEventDestroy(b[i]);
      cudaEventDestroy(e[i]);
    }
  }
  void begin(int i) { if (on) cudaEventRecord(b[i], st); }
  // the begin / end events of slot i for a launcher to record itself (nullptr when off)
  const cudaEvent_t* slot(int i) {
    if (!on) return nullptr;
    used[i] = true;
    pair[0] = b[i];
    pair[1] = e[i];
    return pair;
  }
  cudaEvent_t pair[2] = {};
  void end(int i, int nlaunch) {
    launches[i] += nlaunch;
    if (on) {
      cudaEventRecord(e[i], st);
      used[i] = true;
    }
  }
  // after a stream synchronisation: fold the recorded intervals into ms[]
  void collect() {
    if (!on) return;
    for (int i = 0; i < kStages; ++i)
      if (used[i]) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, b[i], e[i]) == cudaSuccess) ms[i] += t;
        else cudaGetLastError();   // a slot whose launcher recorded nothing
        used[i] = false;
      }
  }
};

}  // namespace

// Runs Alg. 5 for nq queries.  Results go to out_ids_dev (cap entries, device) and the
// offsets to offsets_host (nq + 1, host).  Queries are processed in sub-batches sized
// so that the workspace stays bounded; every sub-batch's ids are emitted into the
// index's internal result buffer first, so the caller's buffer is only written once the
// total is known to fit.
void free_ctx(CallCtx* cx) {
  for (GraphEntry& g : cx->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  cx->graphs.clear();
  for (Workspace* w : {&cx->ws, &cx->surv, &cx->res, &cx->tcws}) {
    if (w->base) cudaFree(w->base);
    w->base = nullptr;
    w->bytes = 0;
  }
  if (cx->pin) cudaFreeHost(cx->pin);
  cx->pin = nullptr;
  cx->pin_bytes = 0;
}

size_t ctx_bytes(const CallCtx* cx) { return cx->ws.bytes + cx->surv.bytes + cx->res.bytes + cx->tcws.bytes; }

size_t batch_workspace_bytes(const Index* ix, int32_t nq) {
  return layout_for(ix, std::max(nq, 1)).total;
}

sah_status run_batch(Index* ix, CallCtx* cx, const float* Q_dev, int32_t nq, const int32_t* ks_dev,
                     const int32_t* modes_dev, int32_t* out_dev, int64_t out_cap, int64_t* offsets_dev,
                     int64_t* offsets_host, bool* wrote_out, cudaStream_t st) {
  // row stride of the answer bitmaps (the kernels that set answers take it as "words")
  const int64_t words = answer_stride(ix->m);
  const int64_t nsw = answer_words(words) / 32;   // summary words per query
  // sub-batch size: with the tensor-core user pass up to the column table's 16,384 rows and
  // about 8 GiB of answer bitmaps (every sub-batch streams all users' rows once); otherwise a
  // bounded pair list and bitmap (about 1 GiB together) and 4,096 rows
  const bool tc_pass_q = ix->nb > 0 && ix->dk > 0 && ix->prm.tc_user_pass && ix->m_nz > 0;
  const size_t per_q = (tc_pass_q ? 0 : sizeof(PairEntry) * (size_t)std::max(ix->nb, 1)) + sizeof(uint32_t) * words +
                       sizeof(int32_t) * (nsw + 1) + sizeof(float) * ix->dp + 16;
  const size_t ws_cap = tc_pass_q ? (size_t(8) << 30) : (size_t(1) << 30);
  int qb = (int)std::max<size_t>(1, std::min<size_t>((size_t)nq, ws_cap / per_q));
  qb = std::min(qb, tc_pass_q ? kTcMaxRows : 4096);
  const bool direct = out_dev != nullptr && qb >= nq;   // one sub-batch: emit into the caller's buffer
  *wrote_out = false;
  // survivor-list capacity used by this call: twice the last call's count (at least 64k),
  // grown and re-run if a sub-batch exceeds it
  // capacities are multiples of 16 entries: the candidate blocks after the three lists are
  // written as 16-byte words
  int64_t surv_cap = (std::max<int64_t>(cx->surv_hint, 1 << 16) + 15) & ~int64_t(15);
  int64_t surv_call_max = 0;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);

  sah_stats agg{};
  agg.queries = nq;
  StageTimer tm(ix->timing, st);
  int64_t res_total = 0;
  std::vector<int64_t> offs(nq + 1, 0);

  for (int q0 = 0; q0 < nq; q0 += qb) {
    const int nqb = std::min(qb, nq - q0);
    const int32_t* modes_q = modes_dev ? modes_dev + q0 : nullptr;
    for (int attempt = 0;; ++attempt) {
      WsLayout L = layout_for(ix, nqb);
      SAH_TRY(ensure_ws(cx, L.total, st));
      // the answer bitmaps must start zero: the emit pass of a completed call leaves them
      // so; after a reallocation, a larger sub-batch or a call that stopped early, clear them
      const size_t bm_bytes = sizeof(uint32_t) * (size_t)nqb * words;
      const unsigned emit_grid = (unsigned)std::max(1, sms * 8);             // warps over the listed words
      if (cx->bm_clean_base != cx->ws.base || cx->bm_clean_bytes < bm_bytes) {
        SAH_CUDA(cudaMemsetAsync((char*)cx->ws.base + L.bitmap, 0, bm_bytes, st));
        cx->bm_clean_base = cx->ws.base;
        cx->bm_clean_bytes = bm_bytes;
      }
      // until this sub-batch has emitted (and so cleared) its answers, nothing is clean
      cx->bm_clean_bytes = 0;
      SAH_TRY(ensure_surv(cx, surv_cap, st));
      char* w = (char*)cx->ws.base;
      float* Qd = (float*)(w + L.qd);
      float* qn = (float*)(w + L.qn);
      int32_t* kk = (int32_t*)(w + L.kk);
      PairEntry* pairs = (PairEntry*)(w + L.pairs);
      int32_t* pcount = (int32_t*)(w + L.pcount);
      unsigned long long* survcnt = (unsigned long long*)(w + L.survcnt);
      uint32_t* bitmap = (uint32_t*)(w + L.bitmap);
      int32_t* chunk = (int32_t*)(w + L.chunk);
      int64_t* offsets = (int64_t*)(w + L.offsets);
      unsigned long long* stats = (unsigned long long*)(w + L.stats);
      Survivor* surv = (Survivor*)cx->surv.base;

      // the pinned host block the results are read back into
      const size_t pin_need =
          sizeof(int64_t) * (size_t)(nqb + 1) + sizeof(unsigned long long) * (ST_COUNT + kCtlCounters) + 16;
      if (cx->pin_bytes < pin_need) {
        SAH_CUDA(cudaStreamSynchronize(st));
        if (cx->pin) cudaFreeHost(cx->pin);
        cx->pin = nullptr;
        cx->pin_bytes = 0;
        ++cx->alloc_epoch;
        SAH_CUDA(cudaMallocHost(&cx->pin, pin_need));
        cx->pin_bytes = pin_need;
      }
      // the same layout as the control block: stats, survivor counts, list length, offsets
      unsigned long long* st_h = (unsigned long long*)cx->pin;
      unsigned long long* ns2 = st_h + ST_COUNT;
      int64_t* ob = (int64_t*)(st_h + ST_COUNT + kCtlCounters);
      int* timeout_h = (int*)(ob + nqb + 1);
      // every device operation of the attempt, the readback of its results included
      auto enqueue = [&]() -> sah_status {
        tm.begin(0);
        // with the tensor-core user pass the preparation also writes the split BF16 queries
        const bool tc_pass = ix->nb > 0 && ix->dk > 0 && ix->prm.tc_user_pass && ix->m_nz > 0;
        // the counters of the control block (stats, survivor counts, answer-list length),
        // through the tile flags when the tensor-core user pass reads them
        SAH_CUDA(cudaMemsetAsync(stats, 0,
                                 tc_pass ? L.tneed_end - L.stats
                                         : sizeof(unsigned long long) * (ST_COUNT + kCtlCounters),
                                 st));
        prep_queries_kernel<<<grid_for(nqb, 8), 256, 0, st>>>(Q_dev + (int64_t)q0 * ix->d, nqb, ix->d, ix->dp, Qd, qn,
                                                               ks_dev + q0, kk, modes_q, stats,
                                                               tc_pass ? (uint16_t*)(w + L.qb) : nullptr, ix->dk,
                                                               tc_pass ? (uint64_t*)(w + L.qh) : nullptr,
                                                               ix->inject_collide);
        SAH_CUDA(cudaGetLastError());
        tm.end(0, 1);
        if (ix->nb > 0) {
          tm.begin(1);
          const int mask_words = (nqb + 31) / 32;
          uint32_t* kmask = (uint32_t*)(w + L.kmask);
          int bf_launches = 1;
          if (tc_pass) {
            // the distinct query vectors first: the block bound is taken once per vector
            SAH_TRY(prepare_user_pass_tc(ix, Qd, qn, (const uint64_t*)(w + L.qh), w + L.coltab, kk, modes_q, nqb,
                                         st, &bf_launches));
            SAH_TRY(block_filter_tc(ix, w + L.coltab, nqb, kmask, mask_words, (uint8_t*)(w + L.tneed), stats,
                                    ST_PAIRS_KEPT, ST_KEPT_USERS, ST_USERS_SCORED, ST_BF_COLPAIRS, st));
          } else {
            block_filter_kernel<<<ix->nb, 128, sizeof(float) * ix->dp, st>>>(
                ix->bcent, ix->bcos, ix->bsin, ix->LB, ix->nb, ix->kmax, ix->n, ix->dp, Qd, qn, kk, nqb,
                ix->cone_slack, pairs, pcount, stats, nullptr, mask_words, ix->bstart, 0);
            SAH_CUDA(cudaGetLastError());
          }
          tm.end(1, bf_launches);
          // ---- A4: register-tiled kernel for d <= 128, the shared-memory one otherwise
          const int threads = std::max(32, ((ix->prm.leaf_size + 31) / 32) * 32);
          const int dp4 = ix->dp / 4;
          const int reg_variant = dp4 <= 16 ? 16 : (dp4 <= 32 ? 32 : 0);
          tm.begin(2);
          int up_launches = 1;
          if (tc_pass) {
            up_launches = 0;
            SAH_TRY(run_user_pass_tc(ix, Qd, (uint16_t*)(w + L.qb), w + L.coltab, qn, kk, nqb, kmask,
                                     mask_words, (uint8_t*)(w + L.tneed), bitmap, words, surv + 2 * surv_cap,
                                     survcnt + 2, surv + 3 * surv_cap, survcnt + 3, surv, survcnt, surv_cap, stats,
                                     ST_YES_EARLY, ST_FP64, ST_TC_SCORES, ST_TC_ROWS, ST_CAND_BLOCKS, st,
                                     &up_launches, tm.slot(6)));
          } else if (reg_variant) {
            const size_t smem = (size_t)16 * kQChunk * dp4 + sizeof(PairInfo) * kQChunk + sizeof(float) * 64 * threads;
            auto fn = reg_variant == 16 ? user_scan_reg_kernel<16> : user_scan_reg_kernel<32>;
            if (smem > 48 * 1024)
              SAH_TRY(raise_smem_limit((const void*)fn, (size_t)((int)smem)));
            fn<<<ix->nb, threads, smem, st>>>(
                ix->Ut, ix->unorm, ix->ucos, ix->usin, ix->uid, ix->bstart, ix->Lt, ix->Eu, ix->pnorm, ix->n,
                ix->m_nz, ix->kmax, ix->l_exact ? 1 : 0, ix->dp, Qd, qn, kk, nqb, pairs, pcount, ix->gamma,
                ix->cone_slack, bitmap, words, surv, survcnt, surv_cap, stats, modes_q, ix->T64, ix->d);
          } else {
            size_t smem = (size_t)16 * threads * ((ix->dp / 4) | 1);
            const int stage = smem <= 160 * 1024 ? 1 : 0;
            if (!stage) smem = 0;
            smem += sizeof(PairInfo) * kPairChunk;
            if (smem > 48 * 1024)
              SAH_TRY(raise_smem_limit((const void*)user_scan_kernel, (size_t)((int)smem)));
            user_scan_kernel<<<ix->nb, threads, smem, st>>>(
                ix->Ut, ix->unorm, ix->ucos, ix->usin, ix->uid, ix->bstart, ix->Lt, ix->Eu, ix->pnorm, ix->n,
                ix->m_nz, ix->kmax, ix->l_exact ? 1 : 0, ix->dp, Qd, qn, kk, nqb, pairs, pcount, ix->gamma,
                ix->cone_slack, bitmap, words, surv, survcnt, surv_cap, stats, stage, modes_q, ix->T64, ix->d);
          }
          SAH_CUDA(cudaGetLastError());
          tm.end(2, up_launches);
          // ---- A5/A6 on the survivors (their number stays on the device)
          tm.begin(3);
          int nl = 0;
          if (ix->dk > 0) {
            SAH_TRY(run_verify_tc(ix, cx, surv, survcnt, surv_cap, Qd, qn, kk, bitmap, words, stats, ST_FP64, ST_ITEMS,
                                  st, &nl, tm.slot(7)));
          } else {
            const size_t vsmem = (size_t)16 * kVerifyWarps * (ix->dp / 4);
            if (vsmem > 48 * 1024)
              SAH_TRY(raise_smem_limit((const void*)verify_exact_kernel, (size_t)((int)vsmem)));
            verify_exact_kernel<<<sms * 8, kVerifyWarps * 32, vsmem, st>>>(
                surv, survcnt, surv_cap, ix->Ut, ix->unorm, ix->uid, ix->Ps, ix->pnorm, ix->n, ix->d, ix->dp, Qd, qn,
                kk, ix->gamma, bitmap, words, stats);
            SAH_CUDA(cudaGetLastError());
            nl = 1;
          }
          tm.end(3, nl);
          if (modes_q) {
            int nsa = 0;
            tm.begin(5);
            SAH_TRY(run_saalsh(ix, surv + surv_cap, survcnt + 1, surv_cap, Qd, qn, kk, bitmap, words, stats, ST_ITEMS,
                               st, &nsa));
            tm.end(5, nsa);
          }
        }
        tm.begin(4);
        int n_compact = 3;
        if (ix->nzero > 0) {
          zero_users_kernel<<<grid_for(ix->nzero * nqb, 256), 256, 0, st>>>(ix->zero_uid, ix->nzero, nqb, bitmap,
                                                                             words);
          ++n_compact;
        }
        // after the per-word counts: the per-query counts, the list of words with answers
        // and its length, the heavy rows and theirs
        int32_t* qcnt = chunk + (int64_t)nqb * nsw;
        int32_t* alist = qcnt + nqb;
        int32_t* heavy = alist + (int64_t)nqb * nsw;
        unsigned int* alist_n = (unsigned int*)(w + L.alist_n);
        unsigned int* heavy_n = (unsigned int*)(w + L.heavy_n);
        answer_count_light_kernel<<<(nqb + kAnswerWarps - 1) / kAnswerWarps, kAnswerWarps * 32, 0, st>>>(
            bitmap, words, kk, ix->n, chunk, alist, alist_n, qcnt, heavy, heavy_n, nqb);
        answer_count_heavy_kernel<<<(unsigned)std::max(1, std::min(nqb, sms * 2)), kHeavyThreads, 0, st>>>(
            bitmap, words, kk, ix->n, ix->m, chunk, alist, alist_n, qcnt, heavy, heavy_n, nqb,
            direct ? 0 : res_total, offsets, direct ? offsets_dev : nullptr, (unsigned int*)(w + L.ticket));
        int32_t* dst;
        int64_t dst_cap;
        if (direct) {
          dst = out_dev;
          dst_cap = out_cap;
        } else {
          dst = (int32_t*)cx->res.base;
          dst_cap = (int64_t)(cx->res.bytes / sizeof(int32_t));
        }
        if (dst) {
          answer_emit_kernel<<<emit_grid, 256, 0, st>>>(bitmap, words, kk, ix->n, ix->m, chunk, alist, alist_n,
                                                        offsets, nqb, dst, dst_cap, &stats[ST_EMIT_OVERFLOW]);
        } else {
          SAH_CUDA(cudaMemsetAsync(&stats[ST_EMIT_OVERFLOW], 0xff, sizeof(unsigned long long), st));
        }
        SAH_CUDA(cudaGetLastError());
        tm.end(4, n_compact);
        // ---- the one synchronisation of the sub-batch: offsets, counters, survivor counts
        *timeout_h = 0;
        SAH_CUDA(cudaMemcpyAsync(st_h, stats,
                                 sizeof(unsigned long long) * (ST_COUNT + kCtlCounters) + sizeof(int64_t) * (nqb + 1),
                                 cudaMemcpyDeviceToHost, st));
        if (ix->dev_timeout)
          SAH_CUDA(cudaMemcpyAsync(timeout_h, ix->dev_timeout, sizeof(int), cudaMemcpyDeviceToHost, st));
        return SAH_OK;
      };
      if (tm.on || !ix->use_graphs || !cx->graphs_allowed || ix->inject_site || ix->inject_collide) {
        SAH_TRY(enqueue());
      } else {
        // the same shapes and buffers as an earlier call: replay its captured graph
        const std::vector<uint64_t> key = {(uint64_t)Q_dev, (uint64_t)ks_dev, (uint64_t)modes_dev,
                                           (uint64_t)out_dev, (uint64_t)out_cap, (uint64_t)offsets_dev,
                                           (uint64_t)nqb, (uint64_t)q0, (uint64_t)surv_cap, (uint64_t)res_total,
                                           (uint64_t)direct, (uint64_t)cx->ws.base, (uint64_t)cx->surv.base,
                                           (uint64_t)cx->res.base, (uint64_t)cx->res.bytes, (uint64_t)cx->tcws.base,
                                           (uint64_t)cx->tcws.bytes, (uint64_t)cx->pin, cx->alloc_epoch};
        SAH_TRY(run_captured(cx, key, enqueue, st));
      }
      SAH_CUDA(cudaStreamSynchronize(st));
      tm.collect();
      if (*timeout_h) {
        SAH_CUDA(cudaMemsetAsync(ix->dev_timeout, 0, sizeof(int), st));
        SAH_CUDA(cudaStreamSynchronize(st));
        set_error("a bounded device-side wait of a tensor-core pass ran out");
        return SAH_ERR_DEVICE_TIMEOUT;
      }
      if (st_h[ST_BAD_Q]) {
        set_error("a query vector holds a non-finite value");
        return SAH_ERR_ARG;
      }
      if (st_h[ST_BAD_K]) {
        set_error("k must be >= 1 and the mode SAH_EXACT or SAH_SAALSH");
        return SAH_ERR_ARG;
      }
      const int64_t nsmax = (int64_t)std::max(std::max(ns2[0], ns2[1]), std::max(ns2[2], ns2[3]));
      if (nsmax > surv_cap) {
        // a survivor list overflowed: grow it and run this sub-batch again
        if (attempt > 4) {
          set_error("survivor list kept overflowing");
          return SAH_ERR_OOM;
        }
        surv_cap = (nsmax * 5 / 4 + 1024 + 15) & ~int64_t(15);
        continue;
      }
      const int64_t new_total = ob[nqb];
      if (st_h[ST_EMIT_OVERFLOW]) {
        if (direct) {
          // the caller's buffer is too small: report the sizes, nothing was written
          for (int j = 0; j <= nqb; ++j) offs[q0 + j] = ob[j];
          agg.results = new_total;
          cx->stats = agg;
          std::memcpy(offsets_host, offs.data(), sizeof(int64_t) * (nq + 1));
          set_error("result buffer too small: " + std::to_string(new_total) + " ids needed");
          return SAH_ERR_BUFFER_TOO_SMALL;
        }
        // internal buffer too small: grow it (keeping earlier sub-batches) and emit again
        Workspace nr;
        SAH_TRY(ensure_buf(&nr, std::max(sizeof(int32_t) * (size_t)new_total, 2 * cx->res.bytes), st));
        if (res_total)
          SAH_CUDA(cudaMemcpyAsync(nr.base, cx->res.base, sizeof(int32_t) * res_total, cudaMemcpyDeviceToDevice, st));
        SAH_CUDA(cudaStreamSynchronize(st));
        if (cx->res.base) cudaFree(cx->res.base);
        cx->res = nr;
        ++cx->alloc_epoch;
        SAH_CUDA(cudaMemsetAsync(&stats[ST_EMIT_OVERFLOW], 0, sizeof(unsigned long long), st));
        {
          int32_t* qcnt = (int32_t*)(w + L.chunk) + (int64_t)nqb * nsw;
          int32_t* alist = qcnt + nqb;
          const unsigned int* alist_n = (const unsigned int*)(w + L.alist_n);
          answer_emit_kernel<<<emit_grid, 256, 0, st>>>(bitmap, words, kk, ix->n, ix->m, chunk, alist, alist_n,
                                                        offsets, nqb, (int32_t*)cx->res.base,
                                                        (int64_t)(cx->res.bytes / sizeof(int32_t)),
                                                        &stats[ST_EMIT_OVERFLOW]);
        }
        SAH_CUDA(cudaGetLastError());
        SAH_CUDA(cudaStreamSynchronize(st));
      }
      // the emit pass has read and cleared every answer of the sub-batch
      cx->bm_clean_base = cx->ws.base;
      cx->bm_clean_bytes = bm_bytes;
      agg.survivors += (int64_t)(ns2[0] + ns2[1]);
      agg.pairs_rescored += (int64_t)ns2[2];
      agg.tc_scores += (int64_t)st_h[ST_TC_SCORES];
      agg.block_col_pairs += (int64_t)st_h[ST_BF_COLPAIRS];
      agg.tc_rows += (int64_t)st_h[ST_TC_ROWS];
      agg.cand_blocks += (int64_t)st_h[ST_CAND_BLOCKS];
      // the next call starts from the largest list of this call's sub-batches (twice it)
      surv_call_max = std::max(surv_call_max, nsmax);
      cx->surv_hint = std::max<int64_t>(1 << 16, 2 * surv_call_max);
      agg.block_pairs_total += (int64_t)ix->nb * nqb;
      agg.block_pairs_kept += (int64_t)st_h[ST_PAIRS_KEPT];
      agg.users_scored += (int64_t)st_h[ST_USERS_SCORED];
      agg.users_yes_early += (int64_t)st_h[ST_YES_EARLY];
      agg.fp64_rescored += (int64_t)st_h[ST_FP64];
      agg.users_in_kept_blocks += (int64_t)st_h[ST_KEPT_USERS];
      agg.items_scanned += (int64_t)st_h[ST_ITEMS];
      for (int j = 0; j < nqb; ++j) offs[q0 + j] = ob[j];
      res_total = new_total;
      break;
    }
  }
  offs[nq] = res_total;
  *wrote_out = direct;
  agg.results = res_total;
  agg.n_items = ix->n;
  agg.n_users = ix->m;
  agg.n_blocks = ix->nb;
  agg.n_partitions = ix->sa_parts;
  agg.device_bytes = (int64_t)(ix->bytes + ctx_bytes(cx));
  for (int i = 0; i < StageTimer::kStages; ++i) {
    agg.stage_ms[i] = tm.ms[i];
    agg.stage_launches[i] = tm.launches[i];
  }
  cx->stats = agg;
  std::memcpy(offsets_host, offs.data(), sizeof(int64_t) * (nq + 1));
  return SAH_OK;
}

}  // namespace sah
