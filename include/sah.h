/*
 * libsah: Reverse k-Maximum Inner Product Search (RkMIPS) with SAH on one GB300.
 *
 * SAH (Shifting-aware Asymmetric Hashing, arXiv 2211.12751): a Cone-Tree over the
 * user vectors prunes users block by block (Lemma 2) and one by one (Lemma 3); per-user
 * lower-bound arrays from the largest-norm items answer "no" early (Alg. 4, Alg. 5);
 * the remaining users run a per-user kMIPS decision, either exact or through SA-ALSH
 * (Alg. 1, Alg. 2).
 *
 * Problem (Def. 1): for a query item q, an integer k >= 1, items P (n x d) and users
 * U (m x d), return every user u such that q is among the k largest inner products of
 * u over P u {q}.  Ties keep q: u is returned iff #{p in P : <u,p> > <u,q>} < k (Alg. 2
 * answers "no" only when <u,q> < phi; Alg. 5 prunes only when <u,q> < L and answers
 * "yes" when ||p_k|| <= <u,q>).
 *
 * Conventions shared by every call:
 *  - Vectors are float32, row-major, rows of exactly d floats (no padding).
 *  - Result ids are row indices of the caller's U, sorted ascending.
 *  - Errors are returned as sah_status; nothing throws across the ABI.  The text of
 *    the last error of the calling thread is available from sah_last_error().
 *  - An index is not thread-safe: calls on one index must not overlap, except through
 *    the server API, which serialises them itself.
 *  - cuda_stream is a cudaStream_t (NULL = the legacy default stream).  Calls that
 *    return results to the host synchronise that stream before they return.
 *  - The exact mode returns, for every user, the decision of the count rule evaluated
 *    in double precision with the sum taken over i = 0..d-1 in order: scores are first
 *    computed in the index's working precision with a rigorous a-priori error bound,
 *    and every decision the bound leaves open is recomputed in that double-precision
 *    order on the GPU.
 */
#ifndef SAH_H_
#define SAH_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sah_index sah_index;   /* opaque; owns every device buffer it uses */
typedef struct sah_server sah_server; /* opaque continuous-batching server */

typedef enum {
  SAH_OK = 0,
  SAH_ERR_ARG = 1,              /* invalid argument (null pointer, k < 1, bad sizes, non-finite input) */
  SAH_ERR_OOM = 2,              /* a device allocation failed; the index stays usable */
  SAH_ERR_CUDA = 3,             /* a CUDA call failed; see sah_last_error() */
  SAH_ERR_BUFFER_TOO_SMALL = 4, /* result buffer too small: required size reported, nothing written */
  SAH_ERR_DEVICE_TIMEOUT = 5,   /* a bounded device-side wait ran out; results are not valid */
  SAH_ERR_BUSY = 6,             /* server: the request has not finished yet */
  SAH_ERR_UNSUPPORTED = 7       /* the parameters ask for something this build does not do */
} sah_status;

typedef enum { SAH_EXACT = 0, SAH_SAALSH = 1 } sah_mode;

/* Working precision of the user x query and user x item scores.  Every mode is exact
 * in SAH_EXACT: a lower precision only widens the error band that is re-scored.
 * SAH_FP8: the scores as with SAH_BF16, and the SA-ALSH projections (item and user codes)
 * in FP8 E4M3 on the tensor cores, every vector scaled by its own max |x| / 448 (a code
 * bit can differ from the exact sign only near zero); d <= 127. */
typedef enum { SAH_FP32 = 0, SAH_BF16 = 1, SAH_FP8 = 2 } sah_precision;

typedef struct {
  int32_t k_max;        /* length of the lower-bound arrays L_u^1..k_max (Alg. 4); 1..64; paper: 50 */
  int32_t leaf_size;    /* N_0, the Cone-Tree's maximum leaf size (Alg. 3); 1..256; paper: 20 */
  float b;              /* SA-ALSH interval ratio in (0,1) (Alg. 1); paper: 0.5 */
  int32_t n_tables;     /* K, SimHash tables per SA-ALSH partition (Alg. 1); paper: 128 */
  int32_t code_bits;    /* SRP bits concatenated into one table's code, 1..16 */
  int32_t p_prime;      /* |P'|: items behind the lower bounds (Alg. 4); <= 0 means 4 * k_max;
                           >= n makes the lower bounds the exact k-th largest scores */
  int32_t precision;    /* sah_precision */
  int32_t probe_radius; /* SA-ALSH: Hamming radius probed around the user's code, 0..code_bits */
  uint64_t seed;        /* Cone-Tree random points (Alg. 3) and, when srp is NULL, the SRP matrix */
  const float* srp;     /* optional host matrix (n_tables * code_bits) x (d + 1) of SRP projection
                           vectors (Eq. 1); NULL draws it from seed.  Copied at build time. */
  int32_t tc_user_pass; /* with SAH_BF16 or SAH_FP8 and d <= 128: 1 (default) runs the user pass
                           as one tcgen05 GEMM U Q^T per sub-batch over its distinct query
                           vectors (BF16 operands, FP32 accumulation) whose epilogue applies the
                           bound tests of Alg. 5 to the pairs of the leaves Lemma 2 kept, with a
                           score band of about 2^-7 ||u|| ||q||; 2 runs the same GEMM on E4M3
                           operands with a scale per user and per query vector (kind::f8f6f4,
                           band about 0.13 ||u|| ||q||); 0 runs Lemma 3 and FP32 dot products on
                           the CUDA cores.  Pairs inside the band are re-scored in FP32, then
                           FP64: results are identical; only the speed differs. */
  int32_t blocking;     /* sah_blocking: how users are grouped into blocks.  SAH_BLOCK_CONE (0,
                           default): Cone-Tree leaves (Alg. 3) with the cone bounds of Lemma 2
                           and Lemma 3.  SAH_BLOCK_NORM (1): Simpfer's norm-based blocking, the
                           ablation the paper calls SA-Simpfer (Experiments, ablation study):
                           users in descending norm order cut into runs of leaf_size, each
                           block and user bounded by Cauchy-Schwarz alone (||q|| for a unit
                           user).  Results are identical; only the pruning differs. */
  int32_t transform;    /* sah_transform: the asymmetric transformation behind the SimHash codes.
                           SAH_SAT (0, default): SA-ALSH's shifting-invariant transformation
                           (Eq. 6, Eq. 7), items shifted by their partition's centroid c_j and
                           padded to its radius R_j.  SAH_QNF (1): H2-ALSH's query-normalized-
                           first transformation (Eq. 3, Eq. 4), items unshifted and padded to
                           their partition's largest norm M_j (c_j = 0, R_j = M_j); the
                           paper's H2-ALSH comparison.  Exact mode does not depend on it. */
} sah_params;

typedef enum { SAH_BLOCK_CONE = 0, SAH_BLOCK_NORM = 1 } sah_blocking;
typedef enum { SAH_SAT = 0, SAH_QNF = 1 } sah_transform;

/* Fills *p with the paper's parameters (k_max 50, N_0 20, b 0.5, K 128) and the build's
 * defaults for the rest (code_bits 16, p_prime 4 * k_max, FP32, probe radius 0, seed 0,
 * tensor-core user pass on when the precision is SAH_BF16). */
void sah_default_params(sah_params* p);

/* Alg. 4 (SAH Indexing): item norms and descending-norm order, lower-bound arrays over
 * the first |P'| items, the SA-ALSH index on the other items (Alg. 1), the Cone-Tree over
 * the users (Alg. 3) with its leaves as blocks, and the per-block lower bounds.
 *  U: m x d users, P: n x d items; host pointers unless inputs_on_device != 0, in which
 *  case both are device pointers on the current device.  The index copies them; the
 *  caller may free its arrays once the call returns.  *out receives the index (NULL on
 *  error).  Errors: SAH_ERR_ARG for m < 1, n < 1, d < 1, d > 1024, parameters out of
 *  range or a non-finite input; SAH_ERR_OOM; SAH_ERR_CUDA. */
sah_status sah_build_index(const float* U, int64_t m, const float* P, int64_t n, int32_t d,
                           int32_t inputs_on_device, const sah_params* params,
                           void* cuda_stream, sah_index** out);

/* Alg. 5 (SAH query) for one query: q has d floats (host pointer), k >= 1, mode is a
 * sah_mode.  Writes the ascending user ids to out_ids (host, cap entries) and their
 * number to *out_count.  k > n returns every user.  If cap is too small, *out_count is
 * set to the required size, nothing is written and SAH_ERR_BUFFER_TOO_SMALL returned. */
sah_status sah_rkmips(sah_index* index, const float* q, int32_t k, int32_t mode,
                      int32_t* out_ids, int64_t cap, int64_t* out_count, void* cuda_stream);

/* Alg. 5 for nq queries in one pass (mixed k and modes).  Q: nq x d; ks, modes: nq each;
 * out_offsets: nq + 1 entries, query j's ids are out_ids[out_offsets[j] .. out_offsets[j+1]).
 * If buffers_on_device != 0, Q, ks, modes, out_ids and out_offsets are device pointers
 * (the call still synchronises the stream once, to size the output); otherwise host
 * pointers.  Host buffers that are all pinned and mapped into the device's address space
 * (cudaHostAlloc, cudaMallocHost, cudaHostRegister with mapping; cap > 0) are read and
 * written in place by the kernels, with one synchronisation and no staging copy; other
 * host buffers are copied to and from the device inside the call.  modes may be NULL
 * (all exact).  If the total exceeds cap, out_offsets[nq] is set to the required total
 * (and, for host buffers, out_offsets[0..nq] are filled), no id is written and
 * SAH_ERR_BUFFER_TOO_SMALL is returned. */
sah_status sah_rkmips_batch(sah_index* index, const float* Q, int32_t nq, const int32_t* ks,
                            const int32_t* modes, int32_t buffers_on_device, int32_t* out_ids,
                            int64_t cap, int64_t* out_offsets, void* cuda_stream);

/* kMIPS over the items by the index's SimHash tables (the paper's SA-ALSH vs H2-ALSH
 * comparison, Experiments, kMIPS; with SAH_QNF the tables are H2-ALSH's): for each of the
 * nq query vectors u (rows of Q, nq x d), Alg. 2's candidate loop without a query item.
 * C starts as P' (the index's |P'| largest-norm items, scored exactly); then partition by
 * partition (descending M_j) it stops once phi, the k-th largest FP32 score in C, exceeds
 * mu_j = M_j ||u|| (rounded up), else adds the partition's items whose code lies within
 * probe_radius of u's in some table (codes of [u; 0], Eq. 4 / Eq. 7, in FP32).  Writes u's k
 * best items of C, best first (equal scores: the earlier-found first), to out_ids[j * k ..]
 * (the caller's item ids; -1 past the items C holds) and, if out_scores is not NULL, their
 * FP32 scores (-inf past the end).  1 <= k <= 64.  If buffers_on_device != 0, Q, out_ids and
 * out_scores are device pointers, otherwise host pointers (copied inside the call).
 * With |P'| = n there are no partitions and C holds every item: the exact kMIPS.
 * Errors: SAH_ERR_ARG (k out of range, nq < 0, NULL buffers, a non-finite query value),
 * SAH_ERR_OOM, SAH_ERR_CUDA. */
sah_status sah_kmips(sah_index* index, const float* Q, int32_t nq, int32_t k, int32_t buffers_on_device,
                     int32_t* out_ids, float* out_scores, void* cuda_stream);

/* ---- Serving: continuous batching over one index -------------------------------------
 * A server owns `workers` host threads, each with its own CUDA stream, workspace and
 * pinned staging buffers.  Requests are queued by sah_server_submit (any thread); every
 * free worker takes all queued requests up to max_batch as one batch, answers them with
 * one pass of the query path and publishes each request's ids and latency (submit to
 * completion).  Requests arriving while batches run are taken by the next free worker,
 * so batches overlap on the device.  A batch is admitted only if its workspace (the part
 * that grows with the batch size) fits the worker's share of hbm_budget_bytes (0: 8 GiB)
 * and half the device's free memory; otherwise it is halved until it fits.  A worker
 * replays a captured CUDA graph for a batch shape it has seen twice (captures are taken
 * one at a time per process).  Results are identical to sah_rkmips for the same request.
 * The index must outlive the server and must not be used through the blocking calls
 * while the server runs. */

/* Starts a server.  max_slots bounds requests held at once (queued, running or finished
 * but not yet polled); 1 <= workers <= 8.  Errors: SAH_ERR_ARG, SAH_ERR_OOM. */
sah_status sah_server_start(sah_index* index, int32_t max_slots, int32_t max_batch, int32_t workers,
                            int64_t hbm_budget_bytes, sah_server** out);

/* Queues one request (q: d floats, host; copied).  *ticket identifies it.  Returns
 * SAH_ERR_BUSY when max_slots requests are held (poll finished ones first), SAH_ERR_ARG
 * for k < 1, an unknown mode or a non-finite q. */
sah_status sah_server_submit(sah_server* server, const float* q, int32_t k, int32_t mode, uint64_t* ticket);

/* Collects a finished request: ids (ascending) to out_ids (host, cap entries), their
 * number to *out_count, its latency in seconds to *latency_s (may be NULL).  Returns
 * SAH_ERR_BUSY while it is queued or running, SAH_ERR_BUFFER_TOO_SMALL (with *out_count
 * set; the result is kept) when cap is too small, SAH_ERR_ARG for an unknown ticket, or
 * the error of its batch.  A collected ticket is forgotten. */
sah_status sah_server_poll(sah_server* server, uint64_t ticket, int32_t* out_ids, int64_t cap,
                           int64_t* out_count, double* latency_s);

/* Batches run so far, requests they held, the largest batch, and admissions that had to
 * halve a batch to fit the memory budget.  Any pointer may be NULL. */
sah_status sah_server_info(sah_server* server, int64_t* batches, int64_t* batched_requests,
                           int64_t* max_batch_seen, int64_t* split_ticks);

/* Finishes every queued request, stops the workers and frees the server.  NULL is ignored. */
sah_status sah_server_stop(sah_server* server);

/* Per-stage counters of the last query call on this index (summed over its queries). */
typedef struct {
  int64_t n_items, n_users, n_blocks, n_partitions, device_bytes;
  int64_t queries;              /* queries in the last call */
  int64_t block_pairs_total;    /* (block, query) pairs examined */
  int64_t block_pairs_kept;     /* pairs that survived the node-level bound (Lemma 2) */
  int64_t users_scored;         /* (user, query) pairs whose <u,q> the user pass used: after the
                                   vector bound (Lemma 3) on the CUDA cores, every pair of a
                                   kept leaf on the tensor cores */
  int64_t users_yes_early;      /* "yes" without a kMIPS (lower/upper-bound tests) */
  int64_t survivors;            /* users sent to the per-user kMIPS decision */
  int64_t fp64_rescored;        /* survivors decided in double precision */
  int64_t results;              /* ids returned */
  int64_t users_in_kept_blocks; /* users of leaves that had at least one surviving pair */
  int64_t items_scanned;        /* (survivor, item) scores computed by the kMIPS decisions */
  /* With timing enabled: CUDA-event time (ms) and kernel launches per stage of the last
   * call: [0] query preparation, [1] block pass (A3), [2] user pass (A4), [3] kMIPS
   * decision (A5/A6), [4] answer compaction (A7), [5] SA-ALSH hashing; [6] the tensor-core
   * user pass's GEMM kernel alone (within [2]); [7] the tensor-core kMIPS decision's GEMM
   * kernel alone (within [3]). */
  double stage_ms[8];
  int64_t stage_launches[8];
  double build_gemm_ms;         /* index build, |P'| = n with SAH_BF16: the tcgen05 GEMM's time */
  int64_t build_overflow_rows;  /* users of that GEMM whose candidate list overflowed */
  int64_t pairs_rescored;       /* pairs the tensor-core user pass left to the FP32 re-score */
  int64_t tc_scores;            /* (user, distinct query vector) scores the tensor-core user pass computed */
  int64_t block_col_pairs;      /* (leaf, distinct query vector) pairs of the tensor-core block filter */
  int64_t tc_rows;              /* user rows the tensor-core user pass streamed (each column set streams
                                   the tiles that need one of its columns) */
  int64_t cand_blocks;          /* candidate blocks (one user's scores of 32 columns) the tensor-core
                                   user pass left to its resolve kernel (exact thresholds) */
} sah_stats;

sah_status sah_index_stats(const sah_index* index, sah_stats* out);

/* Copies the index's Cone-Tree blocks (the leaves of Alg. 3, Alg. 4) to host arrays:
 * ids[m_nz] the caller ids of the users with a nonzero norm in leaf order, starts[nb + 1]
 * the first position of every leaf, cos_theta[m_nz] each user's cos(theta_u) to its
 * leaf centre, cos_omega[nb] each leaf's cos(omega) (-2 for a zero centre; with
 * SAH_BLOCK_NORM the blocks are norm runs: cos_theta 0 and cos_omega -1).  *m_nz and
 * *nb receive the sizes; any array pointer may be NULL (to query the sizes first). */
sah_status sah_index_blocks(const sah_index* index, int64_t* m_nz, int32_t* nb, int32_t* ids,
                            int32_t* starts, float* cos_theta, float* cos_omega);

/* Turns per-stage CUDA-event timing of the query calls on (enable != 0) or off.  Events
 * are recorded on the call's stream around each stage; the times appear in
 * sah_stats.stage_ms after the call. */
sah_status sah_index_set_timing(sah_index* index, int32_t enable);

/* Test hook for the failure path of the bounded device-side waits (the paper has no
 * counterpart; Alg. 5's steps run unchanged).  Every wait inside a tensor-core kernel is
 * bounded; this hook makes one run out without faulting or hanging the GPU.  site 1: in the
 * next query call on this index (sah_rkmips or sah_rkmips_batch), the thread that issues the
 * tensor-core user pass's MMAs (precision SAH_BF16 with tc_user_pass) stops after its first
 * accumulator tile, as a lost pipeline partner would; site 2: the same in the tensor-core
 * kMIPS decision (SAH_BF16, |P'| < n, survivors present).  The waiting epilogue gives up
 * after its bounded spin (about a second), raises the index's device flag, every CTA waits
 * for its own TMA loads and MMAs, frees its tensor memory and returns, and the call returns
 * SAH_ERR_DEVICE_TIMEOUT with no valid result.  If the pass does not run (or finishes its
 * work within one tile) the call succeeds as usual.  The hook applies to one call, which
 * runs its launch sequence directly (never a replayed CUDA graph), then clears itself; the
 * index stays usable.  site 0 clears it.  Not for use with a running server.
 * Errors: SAH_ERR_ARG (NULL index, site outside 0..2). */
sah_status sah_index_inject_stall(sah_index* index, int32_t site);

/* Test hook (the paper has no counterpart): with enable != 0, the next query call on this
 * index gives every row the same 64-bit hash of its vector, so that with the tensor-core
 * user pass every two different vectors of a sub-batch collide in the column table: the
 * bitwise check finds them and the table is built again comparing whole vectors.  The
 * answers are those of a call without the hook.  The hook applies to one call, which runs
 * its launch sequence directly (never a replayed CUDA graph), then clears itself; enable 0
 * clears it.  Not for use with a running server.
 * Errors: SAH_ERR_ARG (NULL index). */
sah_status sah_index_inject_hash_collision(sah_index* index, int32_t enable);

/* Exact RkMIPS for one query without allocating any memory (the paper has no
 * counterpart; it exists for callers that may not allocate).
 *
 * Some callers cannot call cudaMalloc on their request path: a plugin inside a host
 * application whose memory policy forbids allocations by third-party code, a process
 * whose free device memory already belongs to another caching allocator, or a
 * latency-bound loop that cannot absorb the synchronisation an allocation may cause.
 * This call needs no index and makes no allocation: U (m x d), P (n x d), q (d) are the
 * caller's device arrays (float32, row-major), out_ids a device array of cap int32 and
 * out_count a device int64.  It writes the number of answering users to *out_count and,
 * when that number is <= cap, their ids in ascending order to out_ids (nothing when it
 * is larger).  The answer is the exact-mode answer of sah_rkmips (FP32 scores with a
 * rigorous bound; undecided items re-scored in double precision).  All work is queued on
 * cuda_stream; the call does not synchronise it.
 *
 * Its only scratch is a fixed device array of 2^22 bits (512 KiB) compiled into the
 * library, so m must be <= 4,194,304 (larger m: SAH_ERR_ARG, nothing queued).  Every GPU
 * that loads the library holds that array until the process exits.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture begins.  All calls share the array: calls whose
 * work overlaps on the GPU (other streams, other threads) race and must be serialised by
 * the caller.  Each call clears the part of the array it uses before using it.
 * Errors: SAH_ERR_ARG (null pointer, k < 1, n < 1, d outside 1..1024, m outside
 * 1..4,194,304), SAH_ERR_CUDA. */
sah_status sah_rkmips_bruteforce_noalloc(const float* U, int64_t m, const float* P, int64_t n,
                                         int32_t d, const float* q, int32_t k, int32_t* out_ids,
                                         int64_t cap, int64_t* out_count, void* cuda_stream);

/* Self-check of the exact float -> double widening that every double-precision inner
 * product of the count rule (Definition 1, the exact mode above) uses on the GPU: the library's
 * own conversion (field by field, IEEE 754 binary32 -> binary64) is compared bit for bit
 * with the GPU's conversion for all 2^32 float bit patterns on the current device (two
 * NaNs count as equal).  *mismatches receives the number that differ (0 expected).
 * Synchronous, about 4.3e9 conversions; needs no index.
 * Errors: SAH_ERR_ARG (mismatches NULL), SAH_ERR_CUDA. */
sah_status sah_selftest_f2d(uint64_t* mismatches);

/* Frees the index and every device buffer it owns.  NULL is ignored. */
void sah_free_index(sah_index* index);

const char* sah_status_string(sah_status s);

/* Text of the last error reported on the calling thread ("" if none). */
const char* sah_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SAH_H_ */
