// noalloc.cu -- the residual check of mss_residual_norm for callers that
// cannot allocate device memory when they make the call: a process whose
// device memory pool is wholly reserved by another framework, code running
// inside a region where an allocation call is not allowed (it would break a
// stream capture or synchronise the device), or a latency-bound loop that
// must not enter the allocator.
//
// The two kernels are the same as mss_residual_norm's; only the scratch
// differs: a file-scope device array of a fixed maximum size instead of
// memory from the handle's allocation hooks. Nothing here calls cudaMalloc,
// cudaFree or any allocating routine.
#include <mutex>

#include "common.cuh"

namespace mss {
namespace {

// Largest number of cells (BSR block rows) the no-allocation call accepts:
// the limit the public header announces.
constexpr int kNoAllocMaxCells = MSS_NOALLOC_MAX_CELLS;

// Per-cell partial sums (2 per cell): 16 MiB that every GPU which loads the
// library keeps until the process exits. All calls share it; it keeps the
// last call's contents.
static __device__ __align__(256) double g_noalloc_scratch[2 * (size_t)kNoAllocMaxCells];

constexpr int kMaxDevices = 128;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the array on device `dev` (the current device). In host
// code the array's name is only a host-side stand-in, so the address is
// looked up once per device and cached.
double* scratch_address(int dev) {
  if (dev < 0 || dev >= kMaxDevices) fail(MSS_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      fail(MSS_ERR_CUDA, std::string("cudaGetSymbolAddress of the no-allocation scratch failed: ") +
                             cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  return g_scratch_addr[dev];
}

}  // namespace

void residual_norm_noalloc(Handle* h, const mss_bsr* J, int nb, const double* b, const double* x,
                           double* norms) {
  check_residual_args(J, nb, b, x, norms);
  if (J->n_rows > kNoAllocMaxCells)
    fail(MSS_ERR_INVALID_ARG, "n_rows = " + std::to_string(J->n_rows) +
                                  " exceeds the no-allocation limit of " +
                                  std::to_string(kNoAllocMaxCells) + " cells");
  int dev = -1;
  MSS_CK(cudaGetDevice(&dev));
  if (dev != h->device)
    fail(MSS_ERR_INVALID_ARG, "the current device is not the handle's device");
  // Both kernels write every scratch entry the reduction reads before it
  // reads it, so no clearing is needed.
  residual_norms(h->stream, J, nb, b, x, scratch_address(dev), norms);
}

}  // namespace mss
