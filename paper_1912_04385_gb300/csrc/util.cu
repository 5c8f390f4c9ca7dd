// util.cu -- errors, device allocation through the handle's hooks, a
// device-wide exclusive scan, fills and host read-backs.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace mss {

[[noreturn]] void fail(int code, const std::string& msg) { throw Error{code, msg}; }

static std::atomic<long long> g_launches{0};
static thread_local long long* t_capture_count = nullptr;
void count_launch() {
  if (t_capture_count) {
    ++*t_capture_count;
    return;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
}
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void capture_count(long long* c) { t_capture_count = c; }
long long launch_count(bool reset) {
  return reset ? g_launches.exchange(0) : g_launches.load();
}

static cudaEvent_t take_event(Handle* h) {
  if (!h->ev_free.empty()) {
    cudaEvent_t e = h->ev_free.back();
    h->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e;
  MSS_CK(cudaEventCreate(&e));
  return e;
}

// NVTX range names of the trace kinds (host-side ranges for nsys/ncu timelines;
// no cost without an attached tool)
static const char* const kTraceNames[TR_KINDS] = {
    "mss.spmv", "mss.bilu_fwd", "mss.bilu_bwd", "mss.vcycle", "mss.ortho",
    "mss.setup_scale", "mss.setup_amg", "mss.setup_bilu", "mss.apply", "mss.condense",
    "mss.recover"};

TraceScope::TraceScope(Handle* hh, int k) : h(hh), kind(k) {
  if (h->capturing) return;   // no event nodes (and no host ranges) inside a solve graph
  nvtxRangePushA(kTraceNames[k]);
  ranged = true;
  if (!h->trace) return;
  a = take_event(h);
  MSS_CK(cudaEventRecord(a, h->stream));
}

TraceScope::~TraceScope() {
  if (ranged) nvtxRangePop();
  if (!a) return;
  cudaEvent_t b = take_event(h);
  cudaEventRecord(b, h->stream);
  h->ev_pending.push_back({kind, a, b});
}

void trace_drain(Handle* h) {
  if (h->ev_pending.empty()) return;
  MSS_CK(cudaStreamSynchronize(h->stream));
  for (auto& r : h->ev_pending) {
    float ms = 0.f;
    MSS_CK(cudaEventElapsedTime(&ms, r.a, r.b));
    h->trace_ms[r.kind] += ms;
    h->trace_n[r.kind] += 1;
    h->ev_free.push_back(r.a);
    h->ev_free.push_back(r.b);
  }
  h->ev_pending.clear();
}

Handle::~Handle() {
  if (sgraph) cudaGraphExecDestroy(sgraph);
  for (auto& r : ev_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ev_free) cudaEventDestroy(e);
}

void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file,
                line);
  fail(e == cudaErrorMemoryAllocation ? MSS_ERR_OOM : MSS_ERR_CUDA, buf);
}

// Size classes of the pool allocations: eight per octave (at most 12.5 %
// rounding), 256 bytes at least, so that freed blocks fit later requests of
// nearby sizes.
static size_t size_class(size_t b) {
  if (b <= 256) return 256;
  int e = 0;
  while (((size_t)1 << (e + 1)) < b) ++e;          // 2^e < b <= 2^(e+1)
  const size_t step = (size_t)1 << (e >= 3 ? e - 3 : 0);
  return (b + step - 1) / step * step;
}
constexpr size_t kCacheBlockMax = (size_t)64 << 20;   // larger blocks go back to the pool
constexpr size_t kCacheMax = (size_t)256 << 20;       // per handle

BlockCache::~BlockCache() {
  for (auto& kv : blocks)
    for (void* p : kv.second) cudaFreeAsync(p, s);
}

void* dev_alloc(Handle* h, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) return nullptr;
  if (h->alloc) {
    p = h->alloc(bytes, h->ctx);
    if (!p) fail(MSS_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    if (reinterpret_cast<uintptr_t>(p) % 256 != 0)
      fail(MSS_ERR_INVALID_ARG, "allocator returned memory not aligned to 256 bytes");
    return p;
  }
  const size_t cls = size_class(bytes);
  BlockCache& C = h->cache;
  if (!h->capturing && C.s == h->stream) {
    auto it = C.blocks.find(cls);
    if (it != C.blocks.end() && !it->second.empty()) {
      p = it->second.back();
      it->second.pop_back();
      C.bytes -= cls;
      return p;
    }
  }
  cudaError_t e = cudaMallocFromPoolAsync(&p, cls, device_pool(h->device), h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(MSS_ERR_OOM, "pool allocation of " + std::to_string(bytes) + " bytes failed");
  }
  return p;
}

void dev_free(Handle* h, void* p, size_t bytes) {
  if (!p) return;
  if (h->free_fn) {
    h->free_fn(p, h->ctx);
    return;
  }
  const size_t cls = size_class(bytes);
  BlockCache& C = h->cache;
  if (!C.s && C.blocks.empty()) C.s = h->stream;
  if (!h->capturing && C.s == h->stream && cls <= kCacheBlockMax && C.bytes + cls <= kCacheMax) {
    C.blocks[cls].push_back(p);
    C.bytes += cls;
    return;
  }
  cudaFreeAsync(p, h->stream);
}

// One stream-ordered memory pool per device for handles without hooks (and
// for the set-up's worker streams). Freed blocks stay in the pool for reuse
// (release threshold: unlimited) until mss_destroy trims it.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};

cudaMemPool_t device_pool(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (dev < 0 || dev >= 64) fail(MSS_ERR_CUDA, "device index out of range");
  if (!g_pools[dev]) {
    cudaMemPoolProps pr = {};
    pr.allocType = cudaMemAllocationTypePinned;
    pr.location.type = cudaMemLocationTypeDevice;
    pr.location.id = dev;
    MSS_CK(cudaMemPoolCreate(&g_pools[dev], &pr));
    unsigned long long keep = ~0ull;
    MSS_CK(cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
  }
  return g_pools[dev];
}

void trim_pools() {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (auto& pl : g_pools)
    if (pl) cudaMemPoolTrimTo(pl, 0);
}

// ---- exclusive scan (three passes over tiles of SCAN_TILE ints) ------------
namespace {
constexpr int SCAN_T = 512;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_IPT;

__device__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[SCAN_T / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = lane < SCAN_T / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < SCAN_T / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  int warp_prefix = wid > 0 ? warp_sums[wid - 1] : 0;
  *total = warp_sums[SCAN_T / 32 - 1];
  __syncthreads();
  return warp_prefix + x - v;
}

__global__ void k_scan_reduce(const int* __restrict__ in, int n, int* __restrict__ bsum) {
  long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_IPT;
  int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k) {
    long long idx = base + k;
    if (idx < n) s += in[idx];
  }
  int tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: exclusive scan of the tile sums in place
__global__ void k_scan_tiles(int* bsum, int ntiles) {
  int carry = 0;
  for (int base = 0; base < ntiles; base += SCAN_T) {
    int idx = base + threadIdx.x;
    int v = idx < ntiles ? bsum[idx] : 0;
    int tot;
    int ex = block_exclusive_scan(v, &tot);
    if (idx < ntiles) bsum[idx] = carry + ex;
    carry += tot;
    __syncthreads();
  }
}

__global__ void k_scan_apply(const int* __restrict__ in, int* __restrict__ out, int n,
                             const int* __restrict__ bsum) {
  long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_IPT;
  int vals[SCAN_IPT];
  int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k) {
    long long idx = base + k;
    vals[k] = idx < n ? in[idx] : 0;
    s += vals[k];
  }
  int tot;
  int ex = block_exclusive_scan(s, &tot) + bsum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k) {
    long long idx = base + k;
    if (idx < n) out[idx] = ex;
    if (idx == n - 1) out[n] = ex + vals[k];
    ex += vals[k];
  }
}

// one block: the whole scan tile by tile with a running carry (arrays of at
// most kScanOneBlock entries: one launch instead of three)
constexpr int kScanOneBlock = 16 * SCAN_TILE;
__global__ void k_scan_one_block(const int* __restrict__ in, int* __restrict__ out, int n) {
  int carry = 0;
  for (int t0 = 0; t0 < n; t0 += SCAN_TILE) {
    const int base = t0 + threadIdx.x * SCAN_IPT;
    int vals[SCAN_IPT];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
      vals[k] = base + k < n ? in[base + k] : 0;
      s += vals[k];
    }
    int tot;
    int ex = block_exclusive_scan(s, &tot) + carry;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
      if (base + k < n) out[base + k] = ex;
      if (base + k == n - 1) out[n] = ex + vals[k];
      ex += vals[k];
    }
    carry += tot;
  }
}

__global__ void k_fill_int(int* p, int v, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += stride) p[i] = v;
}

__global__ void k_fill_double(double* p, double v, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += stride) p[i] = v;
}
}  // namespace

void exclusive_scan(Handle* h, const int* in, int* out, int n) {
  if (n <= 0) {
    fill_int(h, out, 0, 1);
    return;
  }
  if (n <= kScanOneBlock) {
    k_scan_one_block<<<1, SCAN_T, 0, h->stream>>>(in, out, n);
    MSS_LAUNCH_CK("k_scan_one_block");
    return;
  }
  int ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  DBuf<int> bsum(h, ntiles);
  k_scan_reduce<<<ntiles, SCAN_T, 0, h->stream>>>(in, n, bsum.p);
  MSS_LAUNCH_CK("k_scan_reduce");
  k_scan_tiles<<<1, SCAN_T, 0, h->stream>>>(bsum.p, ntiles);
  MSS_LAUNCH_CK("k_scan_tiles");
  k_scan_apply<<<ntiles, SCAN_T, 0, h->stream>>>(in, out, n, bsum.p);
  MSS_LAUNCH_CK("k_scan_apply");
  // bsum is released here while the kernels may still run: the allocation
  // hooks are stream-ordered (or cudaFree, which synchronises).
}

static void* staging(Handle* h, size_t bytes) {
  if (bytes > kPinnedBytes) fail(MSS_ERR_INVALID_ARG, "read-back larger than the staging word");
  if (!h->pin.p) MSS_CK(cudaMallocHost(&h->pin.p, kPinnedBytes));
  return h->pin.p;
}

void read_back(Handle* h, void* dst, const void* dptr, size_t bytes) {
  void* s = staging(h, bytes);
  MSS_CK(cudaMemcpyAsync(s, dptr, bytes, cudaMemcpyDeviceToHost, h->stream));
  MSS_CK(cudaStreamSynchronize(h->stream));
  std::memcpy(dst, s, bytes);
}

void write_to_device(Handle* h, void* dptr, const void* src, size_t bytes) {
  void* s = staging(h, bytes);
  std::memcpy(s, src, bytes);
  MSS_CK(cudaMemcpyAsync(dptr, s, bytes, cudaMemcpyHostToDevice, h->stream));
  MSS_CK(cudaStreamSynchronize(h->stream));   // the staging word is reused
}

void read_ints(Handle* h, const int* const* dptrs, int* out, int count) {
  int* s = static_cast<int*>(staging(h, sizeof(int) * (size_t)count));
  for (int k = 0; k < count; ++k)
    MSS_CK(cudaMemcpyAsync(s + k, dptrs[k], sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  MSS_CK(cudaStreamSynchronize(h->stream));
  std::memcpy(out, s, sizeof(int) * (size_t)count);
}

int read_int(Handle* h, const int* dptr) {
  int v = 0;
  read_back(h, &v, dptr, sizeof(int));
  return v;
}

double read_double(Handle* h, const double* dptr) {
  double v = 0;
  read_back(h, &v, dptr, sizeof(double));
  return v;
}

void fill_int(Handle* h, int* p, int value, long long n) {
  if (n <= 0) return;
  k_fill_int<<<grid_for(n, 256) > 4096 ? 4096 : grid_for(n, 256), 256, 0, h->stream>>>(p, value, n);
  MSS_LAUNCH_CK("k_fill_int");
}

void fill_double(Handle* h, double* p, double value, long long n) {
  if (n <= 0) return;
  k_fill_double<<<grid_for(n, 256) > 4096 ? 4096 : grid_for(n, 256), 256, 0, h->stream>>>(p, value,
                                                                                          n);
  MSS_LAUNCH_CK("k_fill_double");
}

void copy_dev(Handle* h, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return;
  MSS_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, h->stream));
}

}  // namespace mss
