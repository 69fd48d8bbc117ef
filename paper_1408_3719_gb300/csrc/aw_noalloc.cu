// Allocation-free variant of the ready-set computation (the update
// criterion of the LTS sweep), for callers that must not allocate device
// memory.  Its only scratch is a fixed file-scope device array.
#include <mutex>

#include "../../include/aleweno.h"
#include "aw_internal.h"

namespace {

constexpr int kBlockNA = 256;
constexpr int kMaxBlocksNA = 4096;  // elements per call: at most 4096 * 256 = 1,048,576

// Per-block counts of ready elements, overwritten by their exclusive prefix
// sums.  One copy per device, kept for the life of the process (16 KB).
static __device__ __align__(256) unsigned int g_ready_scratch[kMaxBlocksNA];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned int* g_scratch_ptr[kMaxDevices] = {};

__device__ __forceinline__ bool ready_criterion(const aw::Dev& d, long long T, int i) {
  const long long ti = d.t[i];
  if (ti >= T) return false;
  const long long tn = ti + d.dt[i];
  for (int p = d.sw_ptr[i], pe = d.sw_ptr[i + 1]; p < pe; ++p) {
    const int j = d.sw[p];
    const long long tj = d.t[j];
    if (tj > tn || tn > tj + d.dt[j]) return false;
  }
  return true;
}

__global__ void __launch_bounds__(kBlockNA) k_na_count(aw::Dev d, long long T, unsigned int* scratch) {
  const int i = blockIdx.x * kBlockNA + threadIdx.x;
  const bool r = i < d.ne && ready_criterion(d, T, i);
  const int c = __syncthreads_count(r);
  if (threadIdx.x == 0) scratch[blockIdx.x] = (unsigned int)c;
}

// one block of 1024 threads turns the nb <= 4096 counts into exclusive offsets
__global__ void __launch_bounds__(1024) k_na_scan(unsigned int* scratch, int nb, long long* n_out) {
  __shared__ unsigned int s[1024];
  const int t = threadIdx.x;
  unsigned int v[4], sum = 0;
  for (int k = 0; k < 4; ++k) {
    const int idx = 4 * t + k;
    v[k] = idx < nb ? scratch[idx] : 0u;
    sum += v[k];
  }
  s[t] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const unsigned int add = t >= off ? s[t - off] : 0u;
    __syncthreads();
    s[t] += add;
    __syncthreads();
  }
  unsigned int run = s[t] - sum;
  for (int k = 0; k < 4; ++k) {
    const int idx = 4 * t + k;
    if (idx < nb) scratch[idx] = run;
    run += v[k];
  }
  if (t == 1023) *n_out = (long long)s[1023];
}

__global__ void __launch_bounds__(kBlockNA) k_na_write(aw::Dev d, long long T, const unsigned int* scratch,
                                                      int* out) {
  __shared__ int warp_count[kBlockNA / 32];
  const int i = blockIdx.x * kBlockNA + threadIdx.x;
  const bool r = i < d.ne && ready_criterion(d, T, i);
  const unsigned int m = __ballot_sync(0xffffffffu, r);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_count[warp] = __popc(m);
  __syncthreads();
  int base = (int)scratch[blockIdx.x];
  for (int w = 0; w < warp; ++w) base += warp_count[w];
  if (r) out[base + __popc(m & ((1u << lane) - 1u))] = i;
}

// address of device dev's copy of the scratch array (looked up once per
// device, with that device current)
int scratch_address(int dev, unsigned int** p) {
  if (dev < 0 || dev >= kMaxDevices) return AW_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* a = nullptr;
    if (cudaGetSymbolAddress(&a, g_ready_scratch) != cudaSuccess || !a) return AW_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<unsigned int*>(a);
  }
  *p = g_scratch_ptr[dev];
  return AW_OK;
}

}  // namespace

extern "C" int aw_ready_set_noalloc(aw_ctx* ctx, int32_t* ready_out, int64_t* n_ready_out) {
  if (!ctx || !ready_out || !n_ready_out) return AW_ERR_INVALID_ARG;
  aw::CtxView v;
  if (!aw::ctx_view(ctx, &v)) {
    aw::ctx_error(ctx, "aw_ready_set_noalloc: no valid state loaded");
    return AW_ERR_STATE;
  }
  // the context's device is current from here on (its stream and its copy of
  // the scratch array belong to it); the caller's device is given back
  aw::DeviceGuard guard(v.device);
  cudaGetLastError();  // a launch error left by earlier work is not this call's
  const int ne = v.d->ne;
  const int nb = (ne + kBlockNA - 1) / kBlockNA;
  if (nb > kMaxBlocksNA) {
    aw::ctx_error(ctx, "aw_ready_set_noalloc: more than 1,048,576 elements (the fixed scratch holds 4096 block counts)");
    return AW_ERR_INVALID_ARG;
  }
  unsigned int* scratch = nullptr;
  if (scratch_address(v.device, &scratch) != AW_OK) {
    aw::ctx_error(ctx, "aw_ready_set_noalloc: cudaGetSymbolAddress failed");
    return AW_ERR_CUDA;
  }
  k_na_count<<<nb, kBlockNA, 0, v.stream>>>(*v.d, v.T, scratch);
  if (cudaGetLastError() != cudaSuccess) {
    aw::ctx_error(ctx, "aw_ready_set_noalloc: launch of the counting kernel failed");
    return AW_ERR_CUDA;
  }
  k_na_scan<<<1, 1024, 0, v.stream>>>(scratch, nb, reinterpret_cast<long long*>(n_ready_out));
  if (cudaGetLastError() != cudaSuccess) {
    aw::ctx_error(ctx, "aw_ready_set_noalloc: launch of the scan kernel failed");
    return AW_ERR_CUDA;
  }
  k_na_write<<<nb, kBlockNA, 0, v.stream>>>(*v.d, v.T, scratch, ready_out);
  if (cudaGetLastError() != cudaSuccess) {
    aw::ctx_error(ctx, "aw_ready_set_noalloc: launch of the listing kernel failed");
    return AW_ERR_CUDA;
  }
  return AW_OK;
}
