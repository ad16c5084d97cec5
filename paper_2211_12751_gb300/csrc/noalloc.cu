// An exact RkMIPS entry point that allocates no memory.
//
// Who needs it: code that may not call cudaMalloc on its request path.  Examples are a
// plugin inside a host application whose memory policy forbids allocations by
// third-party code, a process whose device memory has been handed in full to another
// caching allocator (a new cudaMalloc would fail or fragment that pool), and a
// latency-bound loop that cannot afford the device synchronisation cudaMalloc/cudaFree
// can cause.  Such callers already own their inputs and outputs; the only extra memory
// this path needs is a bitmap over the users, and it lives in a fixed array inside the
// library instead of a fresh allocation.
//
// The computation is the brute-force form of the exact decision that the index-based
// path makes: for every user, items are scored in FP32 with a rigorous error bound
// (|fl(<u,p>) - <u,p>| <= gamma_d * sum |u_i p_i|, the absolute sum accumulated beside the
// score); items the bound cannot separate from <u,q> are re-scored in double precision,
// summed i = 0..d-1; the user answers "yes" iff fewer than k items score strictly above
// <u,q>.  The answers are collected in the bitmap and written in ascending id order.
#include <cmath>
#include <mutex>
#include <string>

#include "sah_internal.cuh"

namespace sah {
namespace {

// The fixed scratch array: one bit per user, for at most kNoAllocMaxUsers users (512 KiB).
// Every GPU that loads the library holds it until the process exits.
constexpr int64_t kNoAllocMaxUsers = int64_t(1) << 22;
constexpr int64_t kNoAllocWords = kNoAllocMaxUsers / 32;
static __device__ __align__(256) uint32_t g_noalloc_bitmap[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
uint32_t* g_noalloc_ptr[kMaxDevices] = {};

// The device address of the array on the current device.  In host code the array's
// name is only a host-side stand-in, so it must never be passed to a kernel directly.
sah_status noalloc_scratch(uint32_t** out) {
  int dev = 0;
  SAH_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("sah_rkmips_bruteforce_noalloc: device ordinal out of range");
    return SAH_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_bitmap);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      set_error(std::string("sah_rkmips_bruteforce_noalloc: cudaGetSymbolAddress failed: ") +
                cudaGetErrorString(e));
      return SAH_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return SAH_OK;
}

__global__ void na_clear_kernel(uint32_t* __restrict__ bm, int64_t words) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
       w += (int64_t)gridDim.x * blockDim.x)
    bm[w] = 0u;
}

// One thread per user: count items certainly above <u,q>, settle the undecided ones in
// double precision, stop at k.
__global__ void na_decide_kernel(const float* __restrict__ U, int64_t m, const float* __restrict__ P,
                                 int64_t n, int d, const float* __restrict__ q, int k, float gamma,
                                 uint32_t* __restrict__ bm) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= m) return;
  const float* ur = U + u * d;
  float sq = 0.f, aq = 0.f;
  for (int i = 0; i < d; ++i) {
    float pr = ur[i] * q[i];
    sq += pr;
    aq += fabsf(pr);
  }
  float eq = __fmul_ru(__fmul_ru(gamma, aq), 1.f + 2.f * gamma) + 1e-30f;
  float hi = __fadd_ru(sq, eq), lo = __fsub_rd(sq, eq);
  bool have64 = false;
  double s64q = 0.0;
  int count = 0;
  for (int64_t p = 0; p < n && count < k; ++p) {
    const float* pr = P + p * d;
    float s = 0.f, a = 0.f;
    for (int i = 0; i < d; ++i) {
      float t = ur[i] * pr[i];
      s += t;
      a += fabsf(t);
    }
    float ep = __fmul_ru(__fmul_ru(gamma, a), 1.f + 2.f * gamma) + 1e-30f;
    if (__fsub_rd(s, ep) > hi) {
      ++count;
    } else if (__fadd_ru(s, ep) > lo) {
      if (!have64) {
        s64q = dot64_seq(ur, q, d);
        have64 = true;
      }
      if (dot64_seq(ur, pr, d) > s64q) ++count;
    }
  }
  if (count < k) atomicOr(&bm[u >> 5], 1u << (u & 31));
}

// One CTA: popcounts of contiguous word ranges, a block scan, then the ids in order.
// The ids are written only when they fit in cap; *out_count always gets the total.
__global__ void na_emit_kernel(const uint32_t* __restrict__ bm, int64_t m, int32_t* __restrict__ out,
                               int64_t cap, int64_t* __restrict__ out_count) {
  __shared__ long long warp_tot[32];
  int64_t words = (m + 31) / 32;
  int64_t per = (words + blockDim.x - 1) / blockDim.x;
  int64_t w0 = (int64_t)threadIdx.x * per;
  int64_t w1 = w0 + per < words ? w0 + per : words;
  long long mine = 0;
  for (int64_t w = w0; w < w1; ++w) mine += __popc(bm[w]);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = mine;
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  long long before = 0, total = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    if (w < warp) before += warp_tot[w];
    total += warp_tot[w];
  }
  before += x - mine;
  if (threadIdx.x == 0) *out_count = total;
  if (total > cap) return;
  int64_t dst = before;
  for (int64_t w = w0; w < w1; ++w) {
    uint32_t v = bm[w];
    while (v) {
      int b = __ffs(v) - 1;
      out[dst++] = (int32_t)(w * 32 + b);
      v &= v - 1;
    }
  }
}

}  // namespace
}  // namespace sah

extern "C" sah_status sah_rkmips_bruteforce_noalloc(const float* U, int64_t m, const float* P, int64_t n,
                                                    int32_t d, const float* q, int32_t k, int32_t* out_ids,
                                                    int64_t cap, int64_t* out_count, void* cuda_stream) {
  if (!U || !P || !q || !out_count || (cap > 0 && !out_ids) || cap < 0 || n < 1 || d < 1 ||
      d > sah::kMaxDim || k < 1 || m < 1) {
    sah::set_error("sah_rkmips_bruteforce_noalloc: invalid argument");
    return SAH_ERR_ARG;
  }
  if (m > sah::kNoAllocMaxUsers) {
    sah::set_error("sah_rkmips_bruteforce_noalloc: m = " + std::to_string(m) +
                   " users exceeds the fixed scratch limit of " + std::to_string(sah::kNoAllocMaxUsers));
    return SAH_ERR_ARG;
  }
  uint32_t* bm = nullptr;
  SAH_TRY(sah::noalloc_scratch(&bm));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t words = (m + 31) / 32;
  // the array keeps the previous call's bits: clear the part this call uses
  sah::na_clear_kernel<<<(unsigned)((words + 255) / 256), 256, 0, st>>>(bm, words);
  double u = std::ldexp(1.0, -24);
  float gamma = (float)(1.01 * (d + 2) * u / (1.0 - (d + 2) * u));
  sah::na_decide_kernel<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(U, m, P, n, d, q, k, gamma, bm);
  sah::na_emit_kernel<<<1, 1024, 0, st>>>(bm, m, out_ids, cap, out_count);
  SAH_CUDA(cudaGetLastError());
  return SAH_OK;
}
