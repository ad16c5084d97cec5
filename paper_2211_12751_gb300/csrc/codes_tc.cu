// SA-ALSH codes on tcgen05 (Eq. 7, Eq. 9): the code of a vector x in table t packs the
// signs of <a_r, x> for the code_bits rows r of t.  Users: x = U(u) = (u, 0), so only the
// first d coordinates of every SRP row take part.  Items: x = (p - c_j, sqrt(R_j^2 -
// ||p - c_j||^2)) for the item's partition j (Eq. 6), all d + 1 coordinates.  The
// projections of 128 vectors against a tile of tables are one UMMA (M = 128, N = the
// tile's rows padded to 16, K = 64 or 128) with
// split BF16 operands (hi.hi + hi.lo + lo.hi, as in the user pass: a sign can differ from
// the exact one only when |<a_r, u>| <= about 1e-4 ||a_r|| ||u||), accumulated in TMEM;
// the epilogue turns the 32-column TMEM reads into sign masks and packs each table's
// bits into its 16-bit code.
//
// With SAH_FP8 the projections run in FP8 E4M3 instead (kind::f8f6f4, one product, K =
// 128): every vector and every SRP row is scaled by its own max |x| / 448 before the
// rounding to E4M3.  A positive scale does not change the sign of a projection, so the
// scales are not applied back; the sign differs from the exact one only when the
// projection is within the E4M3 rounding of the two vectors (about 2^-4 of |a| |x|).
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

constexpr int kCRows = 128;      // users per CTA (UMMA M)
constexpr int kCThreads = 128;   // thread 0 loads and issues; all four warps read TMEM
constexpr int kCMaxN = 256;      // projection rows per tile (UMMA N, padded to 16)

struct CodeParams {
  int64_t m;          // vectors
  int K, bits;        // tables, bits per table
  int tpt, NT;        // tables per tile, rows per tile (padded)
  uint16_t* codes;    // [m][K]
  int* timeout;
};

template <int KB>
constexpr size_t code_smem_bytes() {
  return 1024 + 2 * (size_t)KB * kCRows * 128 + 2 * (size_t)KB * kCMaxN * 128 + (size_t)kCThreads * 8 * 4;
}

template <int KB>
__global__ void __launch_bounds__(kCThreads, 2)
codes_tc_kernel(const __grid_constant__ CUtensorMap tmUhi, const __grid_constant__ CUtensorMap tmUlo,
                const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
                CodeParams prm) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t load_bar, mma_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int ok_sh;
  constexpr uint32_t kABytes = kCRows * 128;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;                                      // [hi | lo][KB]
  uint8_t* sB = base + 2 * KB * kABytes;                   // [hi | lo][KB], NT rows each
  uint32_t* masks = reinterpret_cast<uint32_t*>(sB + 2 * KB * kCMaxN * 128);   // [thread][8]
  const uint32_t kBBytes = (uint32_t)prm.NT * 128;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * kCRows;
  const int tile = blockIdx.y;

  if (threadIdx.x == 0) {
    tc::mbar_init(&load_bar, 1);
    // the MMAs' commit and thread 0's own arrival, which publishes ok_sh
    tc::mbar_init(&mma_bar, 2);
    ok_sh = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_sh, kCMaxN);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_base_sh;

  if (threadIdx.x == 0) {
    tc::mbar_arrive_expect_tx(&load_bar, 2 * KB * (kABytes + kBBytes));
    for (int kb = 0; kb < KB; ++kb) {
      tc::tma_load_2d(sA + kb * kABytes, &tmUhi, &load_bar, kb * 64, (int32_t)r0);
      tc::tma_load_2d(sA + (KB + kb) * kABytes, &tmUlo, &load_bar, kb * 64, (int32_t)r0);
      tc::tma_load_2d(sB + kb * kBBytes, &tmBhi, &load_bar, kb * 64, tile * prm.NT);
      tc::tma_load_2d(sB + (KB + kb) * kBBytes, &tmBlo, &load_bar, kb * 64, tile * prm.NT);
    }
    if (tc::mbar_wait(&load_bar, 0, prm.timeout, nullptr)) {
      tc::tc_fence_after();
      const uint32_t idesc = tc::idesc_bf16_f32(kCRows, (uint32_t)prm.NT);
      const uint32_t a_addr = tc::smem_addr(sA), b_addr = tc::smem_addr(sB);
#pragma unroll
      for (int kb = 0; kb < KB; ++kb)
#pragma unroll
        for (int k16 = 0; k16 < 4; ++k16) {
          const uint64_t ah = tc::sw128_kmajor_desc(a_addr + kb * kABytes + k16 * 32);
          const uint64_t al = tc::sw128_kmajor_desc(a_addr + (KB + kb) * kABytes + k16 * 32);
          const uint64_t bh = tc::sw128_kmajor_desc(b_addr + kb * kBBytes + k16 * 32);
          const uint64_t bl = tc::sw128_kmajor_desc(b_addr + (KB + kb) * kBBytes + k16 * 32);
          tc::umma_bf16(tbase, ah, bh, idesc, (kb | k16) ? 1u : 0u);
          tc::umma_bf16(tbase, ah, bl, idesc, 1u);
          tc::umma_bf16(tbase, al, bh, idesc, 1u);
        }
      tc::umma_commit(&mma_bar);
      ok_sh = 1;
      tc::mbar_arrive(&mma_bar);
    } else {
      // the loads did not arrive in time: no MMA was issued; the loads themselves are
      // waited for before the CTA can exit
      tc::mbar_wait_drain(&load_bar, 0);
      tc::mbar_arrive(&mma_bar);
      tc::mbar_arrive(&mma_bar);
    }
  }
  __syncwarp();
  // every thread: its TMEM lane (= its user), the tile's projections as sign masks
  const bool done = tc::mbar_wait(&mma_bar, 0, prm.timeout, nullptr);
  tc::tc_fence_after();
  const int64_t row = r0 + warp * 32 + lane;
  uint32_t* mk = masks + threadIdx.x * 8;
  if (done && ok_sh) {
    for (int c = 0; c < prm.NT; c += 32) {
      float v[32];
      tc::tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + c, v);
      tc::tmem_ld_wait();
      uint32_t m = 0;
#pragma unroll
      for (int i = 0; i < 32; ++i) m |= (v[i] >= 0.f ? 1u : 0u) << i;
      mk[c >> 5] = m;
    }
    if (row < prm.m) {
      const int t0 = tile * prm.tpt, nt = min(prm.tpt, prm.K - t0);
      for (int tt = 0; tt < nt; ++tt) {
        const int s = tt * prm.bits, w = s >> 5, off = s & 31;
        uint64_t x = (uint64_t)mk[w] >> off;
        if (off + prm.bits > 32) x |= (uint64_t)mk[w + 1] << (32 - off);
        prm.codes[row * prm.K + t0 + tt] = (uint16_t)(x & ((1u << prm.bits) - 1u));
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    // the MMAs complete before TMEM is freed, also when a thread's wait gave up early
    if (lane == 0) tc::mbar_wait_drain(&mma_bar, 0);
    __syncwarp();
    tc::tc_fence_after();
    tc::tmem_dealloc(tbase, kCMaxN);
  }
}

// Items from `first` on, transformed for their partitions and split: X_hi, X_lo ([ni][dkx]).
__global__ void item_transform_kernel(const float* __restrict__ Ps, int d, int dp, int64_t first, int64_t n,
                                      const int32_t* __restrict__ part_of, const float* __restrict__ cent,
                                      const float* __restrict__ R, int dkx, uint16_t* __restrict__ Xhi,
                                      uint16_t* __restrict__ Xlo) {
  const int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (it >= n - first) return;
  const int j = part_of[it];
  const float* p = Ps + (first + it) * dp;
  const float* c = cent + (int64_t)j * dp;
  float r2 = 0.f;
  for (int e = lane; e < d; e += 32) {
    const float x = p[e] - c[e];
    r2 = fmaf(x, x, r2);
  }
  for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  const float Rj = R[j];
  const float last = sqrtf(fmaxf(0.f, Rj * Rj - r2));
  for (int e = lane; e < dkx; e += 32) {
    const float x = e < d ? p[e] - c[e] : (e == d ? last : 0.f);
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    Xhi[it * dkx + e] = __bfloat16_as_ushort(h);
    Xlo[it * dkx + e] = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
  }
}

// Rows of E4M3 codes (128 bytes each, zero-padded): user rows x = u (first d coordinates)
// when part_of is null, else transformed item rows x = (p - c_j, sqrt(R_j^2 - ||p -
// c_j||^2)) for the items from `first` on; every row scaled by max |x| / 448 first.  One
// warp per row, four coordinates per lane.
__global__ void fp8_rows_kernel(const float* __restrict__ X, int d, int dp, int64_t first, int64_t n,
                                const int32_t* __restrict__ part_of, const float* __restrict__ cent,
                                const float* __restrict__ R, uint8_t* __restrict__ out) {
  const int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (it >= n - first) return;
  const float* p = X + (first + it) * dp;
  float x[4];
  if (part_of) {
    const int j = part_of[it];
    const float* c = cent + (int64_t)j * dp;
    float r2 = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = lane * 4 + q;
      x[q] = e < d ? p[e] - c[e] : 0.f;
      r2 = fmaf(x[q], x[q], r2);
    }
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    const float last = sqrtf(fmaxf(0.f, R[j] * R[j] - r2));
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (lane * 4 + q == d) x[q] = last;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = lane * 4 + q;
      x[q] = e < d ? p[e] : 0.f;
    }
  }
  float mx = fmaxf(fmaxf(fabsf(x[0]), fabsf(x[1])), fmaxf(fabsf(x[2]), fabsf(x[3])));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float inv = mx > 0.f ? 448.f / mx : 1.f;
  uint32_t packed = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_fp8_e4m3 v(x[q] * inv);
    packed |= (uint32_t)v.__x << (8 * q);
  }
  reinterpret_cast<uint32_t*>(out + it * 128)[lane] = packed;
}

// The FP8 form of codes_tc_kernel: A = 128 rows of 128 E4M3 values, B = NT SRP rows.
__global__ void __launch_bounds__(kCThreads, 2)
codes_f8_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB, CodeParams prm) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t load_bar, mma_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int ok_sh;
  constexpr uint32_t kABytes = kCRows * 128;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + kABytes;
  uint32_t* masks = reinterpret_cast<uint32_t*>(sB + kCMaxN * 128);   // [thread][8]
  const uint32_t kBBytes = (uint32_t)prm.NT * 128;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * kCRows;
  const int tile = blockIdx.y;
  if (threadIdx.x == 0) {
    tc::mbar_init(&load_bar, 1);
    tc::mbar_init(&mma_bar, 2);   // the MMAs' commit and thread 0's own arrival (publishes ok_sh)
    ok_sh = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_sh, kCMaxN);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_base_sh;
  if (threadIdx.x == 0) {
    tc::mbar_arrive_expect_tx(&load_bar, kABytes + kBBytes);
    tc::tma_load_2d(sA, &tmX, &load_bar, 0, (int32_t)r0);
    tc::tma_load_2d(sB, &tmB, &load_bar, 0, tile * prm.NT);
    if (tc::mbar_wait(&load_bar, 0, prm.timeout, nullptr)) {
      tc::tc_fence_after();
      const uint32_t idesc = tc::idesc_e4m3_f32(kCRows, (uint32_t)prm.NT);
      const uint32_t a_addr = tc::smem_addr(sA), b_addr = tc::smem_addr(sB);
#pragma unroll
      for (int k32 = 0; k32 < 4; ++k32)
        tc::umma_e4m3(tbase, tc::sw128_kmajor_desc(a_addr + k32 * 32), tc::sw128_kmajor_desc(b_addr + k32 * 32),
                      idesc, k32 ? 1u : 0u);
      tc::umma_commit(&mma_bar);
      ok_sh = 1;
      tc::mbar_arrive(&mma_bar);
    } else {
      tc::mbar_wait_drain(&load_bar, 0);   // the loads, before the CTA can exit
      tc::mbar_arrive(&mma_bar);
      tc::mbar_arrive(&mma_bar);
    }
  }
  __syncwarp();
  const bool done = tc::mbar_wait(&mma_bar, 0, prm.timeout, nullptr);
  tc::tc_fence_after();
  const int64_t row = r0 + warp * 32 + lane;
  uint32_t* mk = masks + threadIdx.x * 8;
  if (done && ok_sh) {
    for (int c = 0; c < prm.NT; c += 32) {
      float v[32];
      tc::tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + c, v);
      tc::tmem_ld_wait();
      uint32_t m = 0;
#pragma unroll
      for (int i = 0; i < 32; ++i) m |= (v[i] >= 0.f ? 1u : 0u) << i;
      mk[c >> 5] = m;
    }
    if (row < prm.m) {
      const int t0 = tile * prm.tpt, nt = min(prm.tpt, prm.K - t0);
      for (int tt = 0; tt < nt; ++tt) {
        const int s = tt * prm.bits, w = s >> 5, off = s & 31;
        uint64_t x = (uint64_t)mk[w] >> off;
        if (off + prm.bits > 32) x |= (uint64_t)mk[w + 1] << (32 - off);
        prm.codes[row * prm.K + t0 + tt] = (uint16_t)(x & ((1u << prm.bits) - 1u));
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    // the MMAs complete before TMEM is freed, also when a thread's wait gave up early
    if (lane == 0) tc::mbar_wait_drain(&mma_bar, 0);
    __syncwarp();
    tc::tc_fence_after();
    tc::tmem_dealloc(tbase, kCMaxN);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
float bf16_value(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

}  // namespace

// Codes of `rows` vectors given as split BF16 rows (TMA maps tmXhi / tmXlo, box 64 x 128,
// row width dkx = 64 or 128) against the SRP matrix A (K * bits rows of stride a_stride,
// the first ncoord coordinates used), into codes[rows][K].
sah_status codes_tc(Index* ix, const CUtensorMap& tmXhi, const CUtensorMap& tmXlo, int64_t rows, int dkx,
                    const float* A_host, int a_stride, int ncoord, int K, int bits, uint16_t* codes,
                    cudaStream_t st) {
  if (rows == 0) return SAH_OK;
  if (dkx != 64 && dkx != 128) {
    set_error("tensor-core codes: rows must be 64 or 128 BF16 wide");
    return SAH_ERR_UNSUPPORTED;
  }
  const int tpt = std::min(K, std::max(1, kCMaxN / bits));
  const int NT = (tpt * bits + 15) / 16 * 16;
  const int ntile = (K + tpt - 1) / tpt;
  // the SRP rows of every tile (zero rows up to NT), split into BF16 high and low parts
  std::vector<uint16_t> hi((size_t)ntile * NT * dkx, 0), lo((size_t)ntile * NT * dkx, 0);
  for (int tl = 0; tl < ntile; ++tl)
    for (int tt = 0; tt < tpt && tl * tpt + tt < K; ++tt)
      for (int b = 0; b < bits; ++b) {
        const float* a = A_host + (size_t)((tl * tpt + tt) * bits + b) * a_stride;
        const size_t o = ((size_t)tl * NT + (size_t)tt * bits + b) * dkx;
        for (int e = 0; e < ncoord && e < dkx; ++e) {
          const uint16_t h = bf16_bits(a[e]);
          hi[o + e] = h;
          lo[o + e] = bf16_bits(a[e] - bf16_value(h));
        }
      }
  uint16_t *dhi = nullptr, *dlo = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&dhi, sizeof(uint16_t) * hi.size(), st));
  SAH_CUDA(cudaMallocAsync((void**)&dlo, sizeof(uint16_t) * lo.size(), st));
  SAH_CUDA(cudaMemcpyAsync(dhi, hi.data(), sizeof(uint16_t) * hi.size(), cudaMemcpyHostToDevice, st));
  SAH_CUDA(cudaMemcpyAsync(dlo, lo.data(), sizeof(uint16_t) * lo.size(), cudaMemcpyHostToDevice, st));
  auto encode = encode_fn();
  CUresult r = CUDA_ERROR_NOT_SUPPORTED;
  CUtensorMap tbhi, tblo;
  if (encode) {
    cuuint64_t dims[2] = {(cuuint64_t)dkx, (cuuint64_t)ntile * NT};
    cuuint64_t strides[1] = {(cuuint64_t)dkx * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)NT};
    cuuint32_t estr[2] = {1, 1};
    r = encode(&tbhi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, dhi, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
      r = encode(&tblo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, dlo, dims, strides, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) {
    cudaFreeAsync(dhi, st);
    cudaFreeAsync(dlo, st);
    set_error("cuTensorMapEncodeTiled (SRP tiles) failed with code " + std::to_string((int)r));
    return SAH_ERR_CUDA;
  }
  CodeParams prm;
  prm.m = rows;
  prm.K = K;
  prm.bits = bits;
  prm.tpt = tpt;
  prm.NT = NT;
  prm.codes = codes;
  prm.timeout = ix->dev_timeout;
  const dim3 grid((unsigned)((rows + kCRows - 1) / kCRows), (unsigned)ntile);
  if (dkx == 64) {
    constexpr size_t smem = code_smem_bytes<1>();
    SAH_TRY(raise_smem_limit((const void*)codes_tc_kernel<1>, smem));
    codes_tc_kernel<1><<<grid, kCThreads, smem, st>>>(tmXhi, tmXlo, tbhi, tblo, prm);
  } else {
    constexpr size_t smem = code_smem_bytes<2>();
    SAH_TRY(raise_smem_limit((const void*)codes_tc_kernel<2>, smem));
    codes_tc_kernel<2><<<grid, kCThreads, smem, st>>>(tmXhi, tmXlo, tbhi, tblo, prm);
  }
  SAH_CUDA(cudaGetLastError());
  cudaFreeAsync(dhi, st);
  cudaFreeAsync(dlo, st);
  return SAH_OK;
}

sah_status user_codes_tc(Index* ix, const float* A_host, int a_stride, int K, int bits, uint16_t* codes,
                         cudaStream_t st) {
  if (ix->m_nz == 0) return SAH_OK;
  if (ix->dk != 64 && ix->dk != 128) {
    set_error("tensor-core user codes need the BF16 user copies");
    return SAH_ERR_UNSUPPORTED;
  }
  return codes_tc(ix, ix->tmap_U, ix->tmap_Ulo, ix->m_nz, ix->dk, A_host, a_stride, ix->d, K, bits, codes, st);
}

sah_status item_codes_tc(Index* ix, int64_t first, const int32_t* part_of, const float* A_host, int a_stride, int K,
                         int bits, uint16_t* codes, cudaStream_t st) {
  const int64_t ni = ix->n - first;
  if (ni <= 0) return SAH_OK;
  const int dkx = ix->d + 1 <= 64 ? 64 : 128;
  if (ix->d + 1 > 128) {
    set_error("tensor-core item codes: d + 1 > 128");
    return SAH_ERR_UNSUPPORTED;
  }
  uint16_t *xhi = nullptr, *xlo = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&xhi, sizeof(uint16_t) * (size_t)ni * dkx, st));
  SAH_CUDA(cudaMallocAsync((void**)&xlo, sizeof(uint16_t) * (size_t)ni * dkx, st));
  item_transform_kernel<<<(unsigned)((ni * 32 + 255) / 256), 256, 0, st>>>(ix->Ps, ix->d, ix->dp, first, ix->n, part_of,
                                                                           ix->sa_cent, ix->sa_R, dkx, xhi, xlo);
  SAH_CUDA(cudaGetLastError());
  auto encode = encode_fn();
  CUresult r = CUDA_ERROR_NOT_SUPPORTED;
  CUtensorMap thi, tlo;
  if (encode) {
    cuuint64_t dims[2] = {(cuuint64_t)dkx, (cuuint64_t)ni};
    cuuint64_t strides[1] = {(cuuint64_t)dkx * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)kCRows};
    cuuint32_t estr[2] = {1, 1};
    r = encode(&thi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, xhi, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
      r = encode(&tlo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, xlo, dims, strides, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  sah_status s2 = SAH_OK;
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (item rows) failed with code " + std::to_string((int)r));
    s2 = SAH_ERR_CUDA;
  } else {
    s2 = codes_tc(ix, thi, tlo, ni, dkx, A_host, a_stride, ix->d + 1, K, bits, codes, st);
  }
  cudaFreeAsync(xhi, st);
  cudaFreeAsync(xlo, st);
  return s2;
}

// FP8 E4M3 codes of user rows (part_of null) or transformed item rows from `first` on.
sah_status codes_f8(Index* ix, const float* X, int64_t first, int64_t n, const int32_t* part_of, const float* A_host,
                    int a_stride, int K, int bits, uint16_t* codes, cudaStream_t st) {
  const int64_t rows = n - first;
  if (rows <= 0) return SAH_OK;
  const int ncoord = part_of ? ix->d + 1 : ix->d;
  if (ncoord > 128) {
    set_error("FP8 codes: at most 128 coordinates");
    return SAH_ERR_UNSUPPORTED;
  }
  const int tpt = std::min(K, std::max(1, kCMaxN / bits));
  const int NT = (tpt * bits + 15) / 16 * 16;
  const int ntile = (K + tpt - 1) / tpt;
  // SRP rows of every tile in E4M3, each scaled by its own max |a| / 448
  std::vector<uint8_t> b8((size_t)ntile * NT * 128, 0);
  for (int tl = 0; tl < ntile; ++tl)
    for (int tt = 0; tt < tpt && tl * tpt + tt < K; ++tt)
      for (int b = 0; b < bits; ++b) {
        const float* a = A_host + (size_t)((tl * tpt + tt) * bits + b) * a_stride;
        float mx = 0.f;
        for (int e = 0; e < ncoord; ++e) mx = std::max(mx, std::fabs(a[e]));
        const float inv = mx > 0.f ? 448.f / mx : 1.f;
        const size_t o = ((size_t)tl * NT + (size_t)tt * bits + b) * 128;
        for (int e = 0; e < ncoord; ++e) b8[o + e] = __nv_fp8_e4m3(a[e] * inv).__x;
      }
  uint8_t *db = nullptr, *dx = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&db, b8.size(), st));
  SAH_CUDA(cudaMallocAsync((void**)&dx, (size_t)rows * 128, st));
  SAH_CUDA(cudaMemcpyAsync(db, b8.data(), b8.size(), cudaMemcpyHostToDevice, st));
  fp8_rows_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(X, ix->d, ix->dp, first, n, part_of, ix->sa_cent,
                                                                       ix->sa_R, dx);
  SAH_CUDA(cudaGetLastError());
  auto encode = encode_fn();
  CUresult r = CUDA_ERROR_NOT_SUPPORTED;
  CUtensorMap tx, tb;
  if (encode) {
    cuuint64_t xd[2] = {128, (cuuint64_t)rows}, bd[2] = {128, (cuuint64_t)ntile * NT};
    cuuint64_t strides[1] = {128};
    cuuint32_t xbox[2] = {128, (cuuint32_t)kCRows}, bbox[2] = {128, (cuuint32_t)NT};
    cuuint32_t estr[2] = {1, 1};
    r = encode(&tx, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, dx, xd, strides, xbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
      r = encode(&tb, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, db, bd, strides, bbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  sah_status res = SAH_OK;
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (FP8 rows) failed with code " + std::to_string((int)r));
    res = SAH_ERR_CUDA;
  } else {
    CodeParams prm;
    prm.m = rows;
    prm.K = K;
    prm.bits = bits;
    prm.tpt = tpt;
    prm.NT = NT;
    prm.codes = codes;
    prm.timeout = ix->dev_timeout;
    const size_t smem = 1024 + (size_t)kCRows * 128 + (size_t)kCMaxN * 128 + (size_t)kCThreads * 8 * 4;
    res = raise_smem_limit((const void*)codes_f8_kernel, smem);
    if (res == SAH_OK) {
      const dim3 grid((unsigned)((rows + kCRows - 1) / kCRows), (unsigned)ntile);
      codes_f8_kernel<<<grid, kCThreads, smem, st>>>(tx, tb, prm);
      if (cudaGetLastError() != cudaSuccess) {
        set_error("FP8 codes kernel launch failed");
        res = SAH_ERR_CUDA;
      }
    }
  }
  cudaFreeAsync(db, st);
  cudaFreeAsync(dx, st);
  return res;
}

}  // namespace sah
