// Internal declarations of libsah: the device-resident index, the per-call workspace,
// small device helpers and the launchers each .cu file exports to the C-ABI layer.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sah.h"

namespace sah {

constexpr int kMaxKmax = 64;     // lower-bound arrays per user (two slots per lane of a warp)
constexpr int kMaxLeaf = 256;    // one thread per user of a Cone-Tree leaf
constexpr int kMaxDim = 1024;

// ------------------------------------------------------------------ error plumbing
void set_error(const std::string& msg);
sah_status cuda_status(cudaError_t e, const char* what);
#define SAH_CUDA(call)                                              \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return ::sah::cuda_status(e_, #call);    \
  } while (0)
#define SAH_TRY(call)                                               \
  do {                                                              \
    sah_status s_ = (call);                                         \
    if (s_ != SAH_OK) return s_;                                    \
  } while (0)

// A user sent to the per-user kMIPS decision (Alg. 2 / exact count) for one query.
struct Survivor {
  int32_t upos;   // user position (leaf order)
  int32_t j;      // query within the sub-batch
  float sq;       // FP32 <u,q>
};

// ------------------------------------------------------------------ index layout in HBM
// Items are stored in descending norm order (Alg. 1, Alg. 4), users in Cone-Tree leaf
// order (Alg. 3) so that every block is a contiguous range.  FP32 rows are padded to
// dp = roundup(d, 4) floats (16-byte rows for vector loads); padding is zero.
struct Workspace {
  void* base = nullptr;
  size_t bytes = 0;
};

// Everything one query call needs besides the index: a caller (the C-ABI's blocking
// calls, or one worker of the serving loop) owns one of these, so calls with different
// contexts can run concurrently on different streams.
// A sub-batch's launch sequence captured as a CUDA graph, for one set of shapes and
// buffers (the key); captured the second time the key is seen, replayed after that.
struct GraphEntry {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec = nullptr;
  bool bad = false;          // capture failed: run this key directly
  uint64_t last_use = 0;
};

struct CallCtx {
  Workspace ws;      // queries, pair lists, bitmaps, counters
  Workspace surv;    // survivor lists, grown on demand
  Workspace res;     // ids of the last call, before they go to the caller
  Workspace tcws;    // tensor-core kMIPS decision: sorted rows, statuses, band lists
  int64_t surv_hint = 1 << 16;   // survivor-list capacity for the next call
  sah_stats stats{};
  void* pin = nullptr;           // pinned host memory for the per-call readback
  size_t pin_bytes = 0;
  std::vector<GraphEntry> graphs;
  uint64_t graph_clock = 0;
  // bumped whenever a buffer of this context is (re)allocated: part of every graph's key, so
  // that no graph captured against a freed buffer (device or pinned host) is replayed
  uint64_t alloc_epoch = 0;
  bool graphs_allowed = false;   // set for the index's own context and for each server worker's
  // the answer bitmaps sit at the start of ws; this many bytes of it are known to be zero
  // (the emit pass clears what it reads), valid while ws.base equals bm_clean_base
  void* bm_clean_base = nullptr;
  size_t bm_clean_bytes = 0;
};

void free_ctx(CallCtx* cx);
size_t ctx_bytes(const CallCtx* cx);

// Test hook sites of sah_index_inject_stall: the pipeline whose MMA thread stops after its
// first accumulator tile in the next query call.
constexpr int SAH_INJECT_USER_PASS = 1;   // the tensor-core user pass (A4/A8)
constexpr int SAH_INJECT_VERIFY = 2;      // the tensor-core kMIPS decision (A5)

struct Index {
  int device = 0;
  int64_t n = 0, m = 0, m_nz = 0;
  int32_t d = 0, dp = 0;
  sah_params prm{};
  int32_t kmax = 0, pp = 0;
  bool l_exact = false;       // p_prime >= n: the lower bounds are the exact thresholds
  float gamma = 0.f;          // FP32 dot-product error factor: |fl(<a,b>) - <a,b>| <= gamma ||a|| ||b||
  float cone_slack = 0.f;     // additive slack (relative to ||q||) of the cone bounds
  float mmax = 0.f;           // largest item norm

  // items, descending norm order
  float* Ps = nullptr;        // n x dp
  float* pnorm = nullptr;     // n, descending
  int32_t* pid = nullptr;     // n, caller's item id of each row

  // users with a nonzero norm, Cone-Tree leaf order
  float* Ut = nullptr;        // m_nz x dp (the caller's values, bit for bit)
  float* unorm = nullptr;     // m_nz
  int32_t* uid = nullptr;     // m_nz, caller's user id of each row
  float* ucos = nullptr;      // cos theta_u to the leaf centre (Lemma 3)
  float* usin = nullptr;      // sin theta_u
  int32_t* ublock = nullptr;  // m_nz: leaf of each user position
  int32_t* zero_uid = nullptr;
  int64_t nzero = 0;

  // Cone-Tree leaves = blocks (Alg. 4)
  int32_t nb = 0;
  int32_t* bstart = nullptr;  // nb + 1
  float* bcent = nullptr;     // nb x dp unit centre directions
  float* bcos = nullptr;      // cos omega (-2 marks a zero centre: no cone bound)
  float* bsin = nullptr;      // sin omega
  float* LB = nullptr;        // [kmax][nb]: L^k(B) for unit users, rounded down
  float* tile_lb = nullptr;   // [kmax][ceil(m_nz / 128)]: the same minimum over each 128-user tile

  // lower-bound arrays (Alg. 4): Lt[k-1][u] = k-th largest FP32 score of u over P'
  float* Lt = nullptr;        // [kmax][m_nz]
  float* Eu = nullptr;        // m_nz: bound on |Lt - exact| (and on any FP32 item score's error)
  double* T64 = nullptr;      // [kmax][m_nz] when |P'| = n: the exact double-precision k-th largest
                              // score (NaN where it could not be certified)

  // BF16 copies for the tensor-core kMIPS decision (precision SAH_BF16), K padded to dk
  int32_t dk = 0;             // roundup(d, 64); 0 when the tensor-core path is off
  uint16_t* Ub = nullptr;     // m_nz x dk, leaf order: bf16(u)
  uint16_t* Ulo = nullptr;    // m_nz x dk: bf16(u - bf16(u)), the low part (user pass, verify)
  uint16_t* Pb = nullptr;     // n x dk, descending norm order
  uint16_t* Plo = nullptr;    // n x dk: bf16(p - bf16(p)), the low part for the verify pass
  CUtensorMap tmap_P{};       // TMA map of Pb: box 64 x 256, 128-byte swizzle
  CUtensorMap tmap_Pv{};      // Pb and Plo in the verify pass's tiles: box 64 x 128
  CUtensorMap tmap_Plo{};
  CUtensorMap tmap_U{};       // TMA map of Ub: box 64 x 128, 128-byte swizzle
  CUtensorMap tmap_Ulo{};     // the same for Ulo
  // FP8 user pass (tc_user_pass 2): the users in E4M3 (128 bytes a row, leaf order) with
  // their per-row scales, and the TMA map of the rows (box 128 x 128 bytes, 128-byte swizzle)
  uint8_t* U8 = nullptr;
  float* usc = nullptr;
  CUtensorMap tmap_U8{};
  int* dev_timeout = nullptr; // set by a kernel whose bounded wait ran out
  int inject_site = 0;        // test hook for the next query call (SAH_INJECT_*), 0: none
  int inject_collide = 0;     // test hook for the next query call: every row hashes alike

  // SA-ALSH over the items behind P' (Alg. 1): norm partitions S_j (descending M_j), their
  // centroids and radii, SRP codes of the SAT-transformed items (Eq. 6, Eq. 9) sorted
  // into buckets per (partition, table), and the users' codes (Eq. 7, Eq. 9).
  int32_t sa_parts = 0;
  int32_t sa_K = 0, sa_bits = 0, sa_d1p = 0, sa_nprobes = 0;
  std::vector<int32_t> sa_start_h;   // t + 1 item positions
  int32_t* sa_start = nullptr;
  float* sa_M = nullptr;             // t: M_j
  float* sa_R = nullptr;             // t: R_j
  float* sa_cent = nullptr;          // t x dp: c_j
  float* sa_A = nullptr;             // (K * bits) x d1p SRP projection vectors
  uint16_t* sa_ucode = nullptr;      // m_nz x K user codes (leaf order)
  int32_t* sa_boff = nullptr;        // t * K + 1 bucket-array offsets
  int32_t* sa_rbin = nullptr;        // per (partition, table): sa_nbin + 1 offsets (relative to the
                                     // segment) of the codes by their top bits: a radix index
  int32_t sa_nbin = 0, sa_rshift = 0;
  uint16_t* sa_bcode = nullptr;      // codes, sorted within each (partition, table)
  int32_t* sa_bitem = nullptr;       // matching item positions
  uint32_t* sa_probes = nullptr;     // XOR masks with popcount <= probe_radius

  double build_gemm_ms = 0.0;         // index-time tensor-core GEMM (|P'| = n, BF16)
  int64_t build_overflow_rows = 0;    // users whose candidate list overflowed (scanned in full)

  std::vector<void*> allocs;
  size_t bytes = 0;
  CallCtx main_ctx;           // context of the blocking C-ABI calls
  bool timing = false;
  bool use_graphs = true;     // replay a call's launch sequence as a CUDA graph when shapes repeat
};

sah_status dev_alloc(Index* ix, void** p, size_t bytes);
// Raises (never lowers) a kernel's dynamic shared-memory limit; thread-safe.
sah_status raise_smem_limit(const void* fn, size_t bytes);

// ------------------------------------------------------------------ device helpers
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Unsigned key with the same order as the float it encodes (finite floats).
__device__ inline uint32_t float_order_key(float x) {
  uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ inline float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// A device-side count (a list's length) that the whole block needs, capped at cap: one
// thread reads it and shares it.  Read by every warp of a large grid, the one word made its
// L2 line a hot spot.  Every thread of the block must call it (it synchronises the block).
__device__ inline int64_t block_count(const unsigned long long* c, int64_t cap) {
  __shared__ long long v;
  if (threadIdx.x == 0) v = (long long)min((unsigned long long)cap, *c);
  __syncthreads();
  return v;
}

// Answer bitmaps.  Per query one row of answer_stride(m) 32-bit words: w = ceil(m / 32)
// rounded up to a multiple of 1024 words whose bit (id & 31) of word (id >> 5) marks user
// id, then w / 32 summary words whose bit i marks a nonzero word i, then w / 1024 top words
// whose bit i marks a nonzero summary word i, so that counting and emitting visit only the
// words that hold answers.
__host__ __device__ inline int64_t answer_stride(int64_t m) {
  const int64_t w = ((m + 31) / 32 + 1023) / 1024 * 1024;
  return w + w / 32 + w / 1024;
}
__host__ __device__ inline int64_t answer_words(int64_t stride) {
  return (int64_t)((uint64_t)stride / 1057 * 1024);
}

// The three ORs are reductions the thread does not wait for.
__device__ __forceinline__ void set_answer(uint32_t* bitmap, int64_t stride, int j, int32_t id) {
  uint32_t* row = bitmap + (int64_t)j * stride;
  const int64_t w = answer_words(stride);
  const int wi = id >> 5;
  atomicOr(&row[wi], 1u << (id & 31));
  atomicOr(&row[w + (wi >> 5)], 1u << (wi & 31));
  atomicOr(&row[w + (w >> 5) + (wi >> 10)], 1u << ((wi >> 5) & 31));
}

// A float widened to double by rewriting its fields (IEEE 754 binary32 -> binary64, exact
// for every value): the sign stays, a normal number's exponent is re-biased (+1023 - 127)
// and its 23-bit fraction moves to the top of the 52-bit one; a subnormal m * 2^-149 is
// normalised around its leading bit p; zeros, infinities and NaNs keep their class.  On
// GPUs whose double-precision pipe is narrow this keeps the conversions on the integer
// units, leaving the double pipe to the multiply-adds.  sah_selftest_f2d checks it
// against the hardware conversion over every float.
__device__ __forceinline__ double f2d_bits(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint64_t sgn = (uint64_t)(b >> 31) << 63;
  const uint32_t e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  uint64_t r;
  if (e - 1u < 254u) {
    r = sgn | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
  } else if (e == 0u) {
    if (m == 0u) {
      r = sgn;
    } else {
      const int p = 31 - __clz(m);   // m = 2^p (1 + f), value 2^(p - 149) (1 + f)
      r = sgn | ((uint64_t)(p + 874) << 52) | (((uint64_t)m << (52 - p)) & 0xFFFFFFFFFFFFFull);
    }
  } else {
    r = sgn | (0x7FFull << 52) | ((uint64_t)m << 29);
  }
  return __longlong_as_double((long long)r);
}

// Sequential double-precision inner product in the order i = 0..d-1.  The product of
// two floats is exact in double, so this equals the double-precision definition of the
// count rule bit for bit, whatever the compiler does with the multiply-add.
__device__ inline double dot64_seq(const float* __restrict__ a, const float* __restrict__ b,
                                   int d) {
  double s = 0.0;
#pragma unroll 2
  for (int i = 0; i < d; ++i) s = __fma_rn(f2d_bits(a[i]), f2d_bits(b[i]), s);
  return s;
}

// ------------------------------------------------------------------ launchers
// index_build.cu
sah_status build_index_device(Index* ix, const float* U_dev, const float* P_dev,
                              cudaStream_t st);
// saalsh.cu
sah_status build_saalsh(Index* ix, const float* srp_host, cudaStream_t st);
// Alg. 2 for every SA-ALSH survivor; sets the answer bits of the "yes" ones.
// (the number of survivors is read on the device from *count_dev, at most cap)
// Standalone kMIPS through the SimHash tables (sah_kmips): Q_dev nq x d on the device,
// out_ids / out_scores (may be null) nq x k on the device.
sah_status run_kmips(Index* ix, const float* Q_dev, int32_t nq, int32_t k, int32_t* out_ids, float* out_scores,
                     cudaStream_t st);
sah_status run_saalsh(Index* ix, const Survivor* surv, const unsigned long long* count_dev, int64_t cap,
                      const float* Qd, const float* qn, const int32_t* kk, uint32_t* bitmap, int64_t words,
                      unsigned long long* stats, int stat_items, cudaStream_t st, int* launches);
// user_pass_tc.cu: the user pass on tcgen05 over every user tile and the distinct query
// vectors of the sub-batch (nq <= kTcMaxRows rows).
//  prepare_user_pass_tc: the column table (distinct vectors, their rows) into scratch
//    (user_pass_tc_scratch_bytes); the split hi / lo BF16 queries (2 nq dk entries) and
//    qh, a 64-bit hash of each padded query row's bits, are written by the query
//    preparation.
//  block_filter_tc: A3 per (leaf, column), the rows' decisions into kept_mask
//    ([nb][mask_words]), a 1 into tile_need (one byte per 128-user tile, zero on entry) for
//    every tile holding a user of a leaf with a kept row, and the counters stats[st_pairs],
//    stats[st_users], stats[st_scored].
//  run_user_pass_tc: the GEMM and its epilogue over the tiles tile_need marks;
//    the pairs its band leaves open go to resc and are re-scored in FP32.
size_t user_pass_tc_scratch_bytes(int nq, int dp);
sah_status prepare_user_pass_tc(Index* ix, const float* Qd, const float* qn, const uint64_t* qh, void* scratch,
                                const int32_t* kk, const int32_t* modes, int nq, cudaStream_t st, int* launches);
sah_status block_filter_tc(Index* ix, void* scratch, int nq, uint32_t* kept_mask, int mask_words, uint8_t* tile_need,
                           unsigned long long* stats, int st_pairs, int st_users, int st_scored, int st_colpairs,
                           cudaStream_t st);
// Rows of one sub-batch the tensor-core user pass's column table takes.
constexpr int kTcMaxRows = 16384;

sah_status run_user_pass_tc(Index* ix, const float* Qd, uint16_t* Qsplit, void* scratch, const float* qn,
                            const int32_t* kk, int nq, const uint32_t* kept_mask, int mask_words, uint8_t* tile_need,
                            uint32_t* bitmap, int64_t words, Survivor* resc, unsigned long long* resc_count,
                            Survivor* cand, unsigned long long* cand_count,
                            Survivor* surv, unsigned long long* surv_count, int64_t surv_cap,
                            unsigned long long* stats, int st_yes, int st_fp64, int st_scores, int st_rows, int st_cand,
                            cudaStream_t st,
                            int* launches, const cudaEvent_t* ev = nullptr);   // ev: begin / end of the GEMM kernel
// topk_tc.cu: the 64 largest FP32 scores of every user over all items, through tcgen05
sah_status topk_full_tc(Index* ix, float* vlast, int32_t* ids64, cudaStream_t st, double* gemm_ms);
// verify_tc.cu
sah_status build_bf16_copies(Index* ix, cudaStream_t st);
// E4M3 rows with a per-row scale (the FP8 user pass): row r of X (rows x dp, the first d
// used, d <= 128) times 448 / max|x_i| rounded to E4M3 with finite saturation, padded to 128
// bytes with zeros; scale[r] = max|x_i| / 448 (0 for a zero row).  One warp per row.
void launch_e4m3_rows(const float* X, int64_t rows, int dp, int d, uint8_t* out, float* scale, cudaStream_t st);
// The users' E4M3 rows, scales and TMA map (tc_user_pass 2).
sah_status build_fp8_users(Index* ix, cudaStream_t st);
// Decides every survivor with the tcgen05 kernel and sets the answer bits; the counters
// of double-precision decisions and scanned items go to stats[stat_fp64], stats[stat_items].
// codes_tc.cu
// SA-ALSH user codes ([m_nz][K], bits per table) on the tensor cores from the BF16 user
// copies; A_host is the SRP matrix (K * bits rows of stride a_stride, the first d
// coordinates used).  Synchronous with respect to the host matrix (copied before return).
sah_status user_codes_tc(Index* ix, const float* A_host, int a_stride, int K, int bits, uint16_t* codes,
                         cudaStream_t st);
// The same for the items from `first` on ([n - first][K]), transformed for their
// partitions (part_of[i - first], the partition centres and radii of the index), d < 128.
sah_status item_codes_tc(Index* ix, int64_t first, const int32_t* part_of, const float* A_host, int a_stride, int K,
                         int bits, uint16_t* codes, cudaStream_t st);
// FP8 E4M3 codes (precision SAH_FP8): the rows X[first, n) of stride dp, as users
// (part_of null, d coordinates) or as items transformed for their partitions (d + 1).
sah_status codes_f8(Index* ix, const float* X, int64_t first, int64_t n, const int32_t* part_of, const float* A_host,
                    int a_stride, int K, int bits, uint16_t* codes, cudaStream_t st);
// rescore.cu
// FP32 (and, with exact thresholds, double-precision) re-score of the pairs listed in
// pairs[0, *count) (at most cap): "yes" pairs set their answer bit, open ones go to surv.
// With kept_mask ([leaf][mask_words] bits of the rows the node-level bound kept), pairs of
// a pruned (leaf, row) are dropped first.
sah_status launch_pair_rescore(Index* ix, const Survivor* pairs, const unsigned long long* count, int64_t cap,
                               const float* Qd, const float* qn, const int32_t* kk, uint32_t* bitmap, int64_t words,
                               Survivor* surv, unsigned long long* surv_count, unsigned long long* stats, int st_yes,
                               int st_fp64, int nq, int sms, cudaStream_t st, const uint32_t* kept_mask = nullptr,
                               int mask_words = 0);
sah_status run_verify_tc(Index* ix, CallCtx* cx, const Survivor* surv, const unsigned long long* surv_count_dev,
                         int64_t surv_cap, const float* Qd, const float* qn, const int32_t* kk, uint32_t* bitmap,
                         int64_t words, unsigned long long* stats, int stat_fp64, int stat_items,
                         cudaStream_t st, int* launches, const cudaEvent_t* ev = nullptr);
// query.cu
// Alg. 5 for nq queries (Q, ks, modes on the device), with one stream synchronisation
// per sub-batch.  When out_dev is given and the call fits one sub-batch, the ascending
// ids go straight to out_dev (only if they fit in out_cap; SAH_ERR_BUFFER_TOO_SMALL with
// the offsets filled otherwise) and the offsets also to offsets_dev; *wrote_out tells.
// Otherwise the ids sit in cx->res (query j at [offsets_host[j], offsets_host[j+1])).
sah_status run_batch(Index* ix, CallCtx* cx, const float* Q_dev, int32_t nq, const int32_t* ks_dev,
                     const int32_t* modes_dev, int32_t* out_dev, int64_t out_cap, int64_t* offsets_dev,
                     int64_t* offsets_host, bool* wrote_out, cudaStream_t st);
// Device bytes a call with nq queries needs in its workspace (pair lists, bitmaps).
size_t batch_workspace_bytes(const Index* ix, int32_t nq);

}  // namespace sah
