// The C-ABI of libsah: argument checks, index lifetime, host <-> device staging.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <string>
#include <vector>

#include "sah_internal.cuh"

namespace sah {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

// Kernels whose dynamic shared memory depends on the call may be launched from several
// threads at once (the server's workers): the limit only ever rises, so a launch never
// finds it lowered under its feet by another thread.
sah_status raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> limit;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[fn];
  if (bytes <= cur) return SAH_OK;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    return SAH_ERR_CUDA;
  }
  cur = bytes;
  return SAH_OK;
}

namespace {
// Every float bit pattern x = base + i: f2d_bits(x) against the hardware conversion, bit
// for bit (two NaNs count as equal).
__global__ void selftest_f2d_kernel(uint64_t base, uint64_t count, unsigned long long* bad) {
  unsigned long long local = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
    const float x = __uint_as_float((uint32_t)(base + i));
    const double a = f2d_bits(x), h = (double)x;
    const bool same = (a != a && h != h) || __double_as_longlong(a) == __double_as_longlong(h);
    local += same ? 0ull : 1ull;
  }
  if (local) atomicAdd(bad, local);
}
}  // namespace

sah_status cuda_status(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();   // clear a non-sticky error so the index stays usable
  return e == cudaErrorMemoryAllocation ? SAH_ERR_OOM : SAH_ERR_CUDA;
}

sah_status dev_alloc(Index* ix, void** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of " + std::to_string(bytes) + " bytes failed");
    return SAH_ERR_OOM;
  }
  ix->allocs.push_back(*p);
  ix->bytes += bytes;
  return SAH_OK;
}

namespace {

// gamma_d = d u / (1 - d u), u = 2^-24, bounds the error of any FP32 evaluation order of
// a d-term inner product relative to sum |a_i b_i| <= ||a|| ||b||; the factor 1.01 covers
// the rounding of the FP32 norms it is multiplied by.
float fp32_dot_gamma(int d) {
  double u = std::ldexp(1.0, -24);
  double g = (d + 2) * u / (1.0 - (d + 2) * u);
  return (float)(1.01 * g);
}

bool all_finite(const float* x, int64_t cnt) {
  for (int64_t i = 0; i < cnt; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}

}  // namespace
}  // namespace sah

using sah::Index;

struct sah_index {
  Index impl;
};

namespace sah {
Index* index_impl(sah_index* h) { return &h->impl; }
}  // namespace sah

static void destroy_index(sah_index* h) {
  if (!h) return;
  Index* ix = &h->impl;
  for (void* p : ix->allocs) cudaFree(p);
  sah::free_ctx(&ix->main_ctx);
  delete h;
}

extern "C" {

void sah_default_params(sah_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->k_max = 50;
  p->leaf_size = 20;
  p->b = 0.5f;
  p->n_tables = 128;
  p->code_bits = 16;
  p->p_prime = 0;
  p->precision = SAH_FP32;
  p->probe_radius = 0;
  p->seed = 0;
  p->srp = nullptr;
  p->tc_user_pass = 1;
  p->blocking = SAH_BLOCK_CONE;
  p->transform = SAH_SAT;
}

const char* sah_status_string(sah_status s) {
  switch (s) {
    case SAH_OK: return "ok";
    case SAH_ERR_ARG: return "invalid argument";
    case SAH_ERR_OOM: return "out of device memory";
    case SAH_ERR_CUDA: return "CUDA error";
    case SAH_ERR_BUFFER_TOO_SMALL: return "result buffer too small";
    case SAH_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case SAH_ERR_BUSY: return "busy";
    case SAH_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* sah_last_error(void) { return sah::g_last_error.c_str(); }

sah_status sah_build_index(const float* U, int64_t m, const float* P, int64_t n, int32_t d,
                           int32_t inputs_on_device, const sah_params* params, void* cuda_stream,
                           sah_index** out) {
  if (!out) {
    sah::set_error("sah_build_index: out is NULL");
    return SAH_ERR_ARG;
  }
  *out = nullptr;
  sah_params prm;
  if (params) prm = *params;
  else sah_default_params(&prm);
  if (!U || !P || m < 1 || n < 1 || d < 1 || d > sah::kMaxDim || m > INT32_MAX || n > INT32_MAX) {
    sah::set_error("sah_build_index: need non-null U, P and 1 <= m, n < 2^31, 1 <= d <= 1024");
    return SAH_ERR_ARG;
  }
  if (prm.k_max < 1 || prm.k_max > sah::kMaxKmax || prm.leaf_size < 1 || prm.leaf_size > sah::kMaxLeaf ||
      !(prm.b > 0.f && prm.b < 1.f) || prm.n_tables < 1 || prm.code_bits < 1 || prm.code_bits > 16 ||
      prm.probe_radius < 0 || prm.probe_radius > prm.code_bits ||
      (prm.blocking != SAH_BLOCK_CONE && prm.blocking != SAH_BLOCK_NORM) ||
      (prm.transform != SAH_SAT && prm.transform != SAH_QNF) || prm.tc_user_pass < 0 || prm.tc_user_pass > 2) {
    sah::set_error("sah_build_index: parameter out of range");
    return SAH_ERR_ARG;
  }
  if (prm.precision != SAH_FP32 && prm.precision != SAH_BF16 && prm.precision != SAH_FP8) {
    sah::set_error("sah_build_index: precision must be SAH_FP32, SAH_BF16 or SAH_FP8");
    return SAH_ERR_ARG;
  }
  if (prm.precision == SAH_BF16 && d > 128) {
    sah::set_error("sah_build_index: the BF16 tensor-core path supports d <= 128");
    return SAH_ERR_UNSUPPORTED;
  }
  if (prm.precision == SAH_FP8 && d > 127) {
    sah::set_error("sah_build_index: SAH_FP8 supports d <= 127 (item codes use d + 1 coordinates)");
    return SAH_ERR_UNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!inputs_on_device) {
    if (!sah::all_finite(U, m * d) || !sah::all_finite(P, n * d)) {
      sah::set_error("sah_build_index: U or P holds a non-finite value");
      return SAH_ERR_ARG;
    }
  }
  sah_index* h = new sah_index();
  Index* ix = &h->impl;
  ix->main_ctx.graphs_allowed = true;   // the blocking calls replay repeated shapes as CUDA graphs
  cudaGetDevice(&ix->device);
  ix->n = n;
  ix->m = m;
  ix->d = d;
  ix->dp = (d + 3) / 4 * 4;
  ix->prm = prm;
  ix->prm.srp = nullptr;
  ix->kmax = prm.k_max;
  int64_t pp = prm.p_prime <= 0 ? 4 * (int64_t)prm.k_max : prm.p_prime;
  ix->pp = (int32_t)std::min<int64_t>(pp, n);
  ix->l_exact = ix->pp >= n;
  ix->gamma = sah::fp32_dot_gamma(d);
  ix->cone_slack = 8.f * ix->gamma + 1e-6f;

  const float* Ud = U;
  const float* Pd = P;
  float* tmpU = nullptr;
  float* tmpP = nullptr;
  sah_status s = SAH_OK;
  if (!inputs_on_device) {
    cudaError_t e1 = cudaMalloc((void**)&tmpU, sizeof(float) * m * d);
    cudaError_t e2 = cudaMalloc((void**)&tmpP, sizeof(float) * n * d);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      cudaGetLastError();
      if (tmpU) cudaFree(tmpU);
      if (tmpP) cudaFree(tmpP);
      destroy_index(h);
      sah::set_error("sah_build_index: staging allocation failed");
      return SAH_ERR_OOM;
    }
    cudaMemcpyAsync(tmpU, U, sizeof(float) * m * d, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(tmpP, P, sizeof(float) * n * d, cudaMemcpyHostToDevice, st);
    Ud = tmpU;
    Pd = tmpP;
  }
  s = sah::build_index_device(ix, Ud, Pd, st);
  if (s == SAH_OK) s = sah::build_saalsh(ix, params ? params->srp : nullptr, st);
  cudaStreamSynchronize(st);
  if (tmpU) cudaFree(tmpU);
  if (tmpP) cudaFree(tmpP);
  if (s != SAH_OK) {
    destroy_index(h);
    return s;
  }
  *out = h;
  return SAH_OK;
}

// The address under which the current device reaches host memory p: pinned memory mapped
// into the device's address space (as pinned memory is under unified addressing).
static bool device_view(const void* p, const void** out) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return false;
  *out = a.devicePointer;
  return true;
}

static sah_status batch_impl(sah_index* index, const float* Q, int32_t nq, const int32_t* ks,
                             const int32_t* modes, int32_t on_dev, int32_t* out_ids, int64_t cap,
                             int64_t* out_offsets, cudaStream_t st) {
  Index* ix = &index->impl;
  if (nq == 0) {
    if (out_offsets) {
      if (on_dev) {
        SAH_CUDA(cudaMemsetAsync(out_offsets, 0, sizeof(int64_t), st));
        SAH_CUDA(cudaStreamSynchronize(st));
      } else {
        out_offsets[0] = 0;
      }
    }
    return SAH_OK;
  }
  // Host buffers that the GPU addresses directly: the kernels read the requests and write
  // the answers in place, so the call makes no staging copy and synchronises once; k, the
  // modes and the vectors are then checked on the device, as for device buffers.
  bool mapped = false;
  int64_t* host_offsets = out_offsets;
  if (!on_dev && cap > 0) {
    const void *q2 = nullptr, *k2 = nullptr, *m2 = nullptr, *o2 = nullptr, *f2 = nullptr;
    if (device_view(Q, &q2) && device_view(ks, &k2) && (!modes || device_view(modes, &m2)) &&
        device_view(out_ids, &o2) && device_view(out_offsets, &f2)) {
      Q = (const float*)q2;
      ks = (const int32_t*)k2;
      modes = (const int32_t*)m2;
      out_ids = (int32_t*)o2;
      out_offsets = (int64_t*)f2;
      on_dev = 1;
      mapped = true;
    }
  }
  // other host buffers are checked here; device buffers (k, mode, finiteness) on the device
  if (!on_dev) {
    for (int j = 0; j < nq; ++j) {
      if (ks[j] < 1) {
        sah::set_error("k must be >= 1");
        return SAH_ERR_ARG;
      }
      if (modes && modes[j] != SAH_EXACT && modes[j] != SAH_SAALSH) {
        sah::set_error("unknown mode");
        return SAH_ERR_ARG;
      }
    }
    if (!sah::all_finite(Q, (int64_t)nq * ix->d)) {
      sah::set_error("a query vector holds a non-finite value");
      return SAH_ERR_ARG;
    }
  }
  sah::CallCtx* cx = &ix->main_ctx;
  const float* Qd = Q;
  const int32_t* kd = ks;
  const int32_t* md = modes;
  float* tq = nullptr;
  int32_t* tk = nullptr;
  if (!on_dev) {
    SAH_CUDA(cudaMallocAsync((void**)&tq, sizeof(float) * (size_t)nq * ix->d, st));
    SAH_CUDA(cudaMallocAsync((void**)&tk, sizeof(int32_t) * nq * 2, st));
    SAH_CUDA(cudaMemcpyAsync(tq, Q, sizeof(float) * (size_t)nq * ix->d, cudaMemcpyHostToDevice, st));
    SAH_CUDA(cudaMemcpyAsync(tk, ks, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st));
    if (modes) SAH_CUDA(cudaMemcpyAsync(tk + nq, modes, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st));
    Qd = tq;
    kd = tk;
    md = modes ? tk + nq : nullptr;
  }
  std::vector<int64_t> offs(nq + 1);
  bool wrote = false;
  sah_status s = sah::run_batch(ix, cx, Qd, nq, kd, md, on_dev ? out_ids : nullptr, cap,
                                on_dev ? out_offsets : nullptr, offs.data(), &wrote, st);
  if (tq) cudaFreeAsync(tq, st);
  if (tk) cudaFreeAsync(tk, st);
  const int64_t total = offs[nq];
  if (s == SAH_ERR_BUFFER_TOO_SMALL || (s == SAH_OK && total > cap)) {
    if (out_offsets) {
      if (on_dev && !mapped) {
        cudaMemcpyAsync(out_offsets + nq, &total, sizeof(int64_t), cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
      } else {
        std::memcpy(host_offsets, offs.data(), sizeof(int64_t) * (nq + 1));
      }
    }
    sah::set_error("result buffer too small: " + std::to_string(total) + " ids needed");
    return SAH_ERR_BUFFER_TOO_SMALL;
  }
  if (s != SAH_OK) return s;
  if (!wrote) {
    if (total > 0)
      SAH_CUDA(cudaMemcpyAsync(out_ids, cx->res.base, sizeof(int32_t) * total,
                               mapped ? cudaMemcpyDefault
                                      : (on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost), st));
    if (on_dev && !mapped)
      SAH_CUDA(cudaMemcpyAsync(out_offsets, offs.data(), sizeof(int64_t) * (nq + 1), cudaMemcpyHostToDevice, st));
    SAH_CUDA(cudaStreamSynchronize(st));
  }
  if (!on_dev || mapped) std::memcpy(host_offsets, offs.data(), sizeof(int64_t) * (nq + 1));
  return SAH_OK;
}

sah_status sah_rkmips_batch(sah_index* index, const float* Q, int32_t nq, const int32_t* ks,
                            const int32_t* modes, int32_t buffers_on_device, int32_t* out_ids, int64_t cap,
                            int64_t* out_offsets, void* cuda_stream) {
  if (!index || nq < 0 || (nq > 0 && (!Q || !ks || !out_offsets)) || cap < 0 || (cap > 0 && !out_ids)) {
    sah::set_error("sah_rkmips_batch: invalid argument");
    return SAH_ERR_ARG;
  }
  const sah_status s = batch_impl(index, Q, nq, ks, modes, buffers_on_device, out_ids, cap, out_offsets,
                                  (cudaStream_t)cuda_stream);
  index->impl.inject_site = 0;   // the test hooks apply to one call
  index->impl.inject_collide = 0;
  return s;
}

sah_status sah_rkmips(sah_index* index, const float* q, int32_t k, int32_t mode, int32_t* out_ids,
                      int64_t cap, int64_t* out_count, void* cuda_stream) {
  if (!index || !q || !out_count || k < 1 || cap < 0 || (cap > 0 && !out_ids)) {
    sah::set_error("sah_rkmips: invalid argument");
    return SAH_ERR_ARG;
  }
  int64_t offs[2] = {0, 0};
  sah_status s = batch_impl(index, q, 1, &k, &mode, 0, out_ids, cap, offs, (cudaStream_t)cuda_stream);
  index->impl.inject_site = 0;   // the test hooks apply to one call
  index->impl.inject_collide = 0;
  *out_count = offs[1];
  return s;
}

sah_status sah_kmips(sah_index* index, const float* Q, int32_t nq, int32_t k, int32_t buffers_on_device,
                     int32_t* out_ids, float* out_scores, void* cuda_stream) {
  if (!index || nq < 0 || k < 1 || k > 64 || (nq > 0 && (!Q || !out_ids))) {
    sah::set_error("sah_kmips: need an index, nq >= 0, 1 <= k <= 64, Q and out_ids");
    return SAH_ERR_ARG;
  }
  Index* ix = &index->impl;
  cudaSetDevice(ix->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (nq == 0) return SAH_OK;
  if (buffers_on_device) return sah::run_kmips(ix, Q, nq, k, out_ids, out_scores, st);
  // host buffers: staged through the device
  const size_t bq = sizeof(float) * (size_t)nq * ix->d, bo = (size_t)nq * k;
  char* buf = nullptr;
  SAH_CUDA(cudaMallocAsync((void**)&buf, bq + bo * (sizeof(int32_t) + sizeof(float)) + 512, st));
  float* Qd = (float*)buf;
  int32_t* ids_d = (int32_t*)(buf + ((bq + 255) & ~(size_t)255));
  float* sc_d = (float*)((char*)ids_d + ((bo * sizeof(int32_t) + 255) & ~(size_t)255));
  sah_status s = SAH_OK;
  if (cudaMemcpyAsync(Qd, Q, bq, cudaMemcpyHostToDevice, st) != cudaSuccess) s = SAH_ERR_CUDA;
  if (s == SAH_OK) s = sah::run_kmips(ix, Qd, nq, k, ids_d, out_scores ? sc_d : nullptr, st);
  if (s == SAH_OK &&
      (cudaMemcpyAsync(out_ids, ids_d, sizeof(int32_t) * bo, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       (out_scores && cudaMemcpyAsync(out_scores, sc_d, sizeof(float) * bo, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
       cudaStreamSynchronize(st) != cudaSuccess)) {
    s = SAH_ERR_CUDA;
    sah::set_error(std::string("sah_kmips: ") + cudaGetErrorString(cudaGetLastError()));
  }
  cudaFreeAsync(buf, st);
  return s;
}

sah_status sah_index_stats(const sah_index* index, sah_stats* out) {
  if (!index || !out) {
    sah::set_error("sah_index_stats: invalid argument");
    return SAH_ERR_ARG;
  }
  const Index* ix = &index->impl;
  *out = ix->main_ctx.stats;
  out->n_items = ix->n;
  out->n_users = ix->m;
  out->n_blocks = ix->nb;
  out->n_partitions = ix->sa_parts;
  out->device_bytes = (int64_t)(ix->bytes + sah::ctx_bytes(&ix->main_ctx));
  out->build_gemm_ms = ix->build_gemm_ms;
  out->build_overflow_rows = ix->build_overflow_rows;
  return SAH_OK;
}

void sah_free_index(sah_index* index) { destroy_index(index); }

sah_status sah_selftest_f2d(uint64_t* mismatches) {
  if (!mismatches) {
    sah::set_error("sah_selftest_f2d: mismatches is NULL");
    return SAH_ERR_ARG;
  }
  unsigned long long* bad = nullptr;
  SAH_CUDA(cudaMalloc((void**)&bad, sizeof(unsigned long long)));
  cudaError_t e = cudaMemset(bad, 0, sizeof(unsigned long long));
  // four launches of 2^30 patterns each
  for (uint64_t b = 0; e == cudaSuccess && b < (1ull << 32); b += (1ull << 30)) {
    sah::selftest_f2d_kernel<<<4096, 256>>>(b, 1ull << 30, bad);
    e = cudaGetLastError();
  }
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, bad, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(bad);
  if (e != cudaSuccess) return sah::cuda_status(e, "sah_selftest_f2d");
  *mismatches = (uint64_t)h;
  return SAH_OK;
}

sah_status sah_index_blocks(const sah_index* index, int64_t* m_nz, int32_t* nb, int32_t* ids, int32_t* starts,
                            float* cos_theta, float* cos_omega) {
  if (!index || !m_nz || !nb) {
    sah::set_error("sah_index_blocks: invalid argument");
    return SAH_ERR_ARG;
  }
  const Index* ix = &index->impl;
  *m_nz = ix->m_nz;
  *nb = ix->nb;
  if (ids && ix->m_nz) SAH_CUDA(cudaMemcpy(ids, ix->uid, sizeof(int32_t) * ix->m_nz, cudaMemcpyDeviceToHost));
  if (starts) SAH_CUDA(cudaMemcpy(starts, ix->bstart, sizeof(int32_t) * (ix->nb + 1), cudaMemcpyDeviceToHost));
  if (cos_theta && ix->m_nz)
    SAH_CUDA(cudaMemcpy(cos_theta, ix->ucos, sizeof(float) * ix->m_nz, cudaMemcpyDeviceToHost));
  if (cos_omega && ix->nb) SAH_CUDA(cudaMemcpy(cos_omega, ix->bcos, sizeof(float) * ix->nb, cudaMemcpyDeviceToHost));
  return SAH_OK;
}

sah_status sah_index_inject_stall(sah_index* index, int32_t site) {
  if (!index || site < 0 || site > sah::SAH_INJECT_VERIFY) {
    sah::set_error("sah_index_inject_stall: NULL index or site outside 0..2");
    return SAH_ERR_ARG;
  }
  index->impl.inject_site = site;
  return SAH_OK;
}

sah_status sah_index_inject_hash_collision(sah_index* index, int32_t enable) {
  if (!index) {
    sah::set_error("sah_index_inject_hash_collision: index is NULL");
    return SAH_ERR_ARG;
  }
  index->impl.inject_collide = enable != 0 ? 1 : 0;
  return SAH_OK;
}

sah_status sah_index_set_timing(sah_index* index, int32_t enable) {
  if (!index) {
    sah::set_error("sah_index_set_timing: index is NULL");
    return SAH_ERR_ARG;
  }
  index->impl.timing = enable != 0;
  return SAH_OK;
}

}  // extern "C"
