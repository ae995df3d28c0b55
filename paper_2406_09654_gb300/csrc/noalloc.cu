// Allocation-free bucketing entry point: the stable counting sort of cells by GenomeIndex with
// its scratch in a fixed device array that lives as long as the library is loaded.
//
// Some callers cannot call cudaMalloc at the time they need the sort: code running between
// the capture begin and end of a stream they do not own, real-time loops that forbid
// allocator calls (an allocation can synchronise the device or fail under memory pressure),
// and hosts that hand the library a fixed memory budget up front. This entry point lets them
// bucket cells with only the input and output buffers they already own.
#include <mutex>
#include <string>

#include "coral_internal.cuh"

namespace coral {
namespace {

constexpr long long kNoAllocMaxCells = 1LL << 20;          // 1,048,576 cells (e.g. 1024 x 1024)
constexpr int kNoAllocMaxCapacity = 1 << 16;               // genome ids below 65,536: two digit passes
constexpr long long kNoAllocMaxBlocks = kNoAllocMaxCells / 4096;
// three [cells] int32 ping-pong arrays + the [256][blocks] digit histograms + 256 digit
// totals: 12.3 MiB
constexpr long long kNoAllocWords = 3 * kNoAllocMaxCells + 256 * kNoAllocMaxBlocks + 256;

__device__ __align__(256) int32_t g_bucket_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
int32_t* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mutex;
thread_local std::string g_noalloc_err = "no error";

int noalloc_fail(int code, const std::string& msg) {
  g_noalloc_err = msg;
  return code;
}

// Device address of this device's copy of g_bucket_scratch (the host-side symbol is only a
// stand-in). Looked up once per device, with that device current.
int scratch_for_device(int dev, int32_t** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_bucket_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_fail(CORAL_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return CORAL_OK;
}

}  // namespace
}  // namespace coral

using namespace coral;

extern "C" const char* coral_bucket_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

extern "C" int coral_bucket_noalloc(const int32_t* G, int64_t n_cells, int32_t capacity, int32_t* counts,
                                    int32_t* perm, void* cuda_stream) {
  if (!G || !counts || !perm) return noalloc_fail(CORAL_E_INVALID, "NULL pointer");
  if (n_cells < 1 || n_cells > kNoAllocMaxCells)
    return noalloc_fail(CORAL_E_INVALID, "n_cells must be in [1, 1048576] (fixed scratch size of the "
                                         "allocation-free sort)");
  if (capacity < 1 || capacity > kNoAllocMaxCapacity)
    return noalloc_fail(CORAL_E_INVALID, "capacity must be in [1, 65536] for the allocation-free sort");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(CORAL_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(CORAL_E_INVALID, "device ordinal out of range");
  int32_t* scratch = nullptr;
  const int rc = scratch_for_device(dev, &scratch);
  if (rc != CORAL_OK) return rc;
  SortArgs a = {};
  a.keys_in = G;
  a.N = n_cells;
  a.capacity = capacity;
  a.count = counts;
  a.perm = perm;
  a.k0 = scratch;                       // every word the passes read is written first in the
  a.v0 = scratch + n_cells;             // same call, so stale contents of earlier calls are
  a.k1 = scratch + 2 * n_cells;         // never read; counts are zeroed by the launch itself
  a.v1 = nullptr;                       // unused: at most two digit passes
  a.hist = scratch + 3 * kNoAllocMaxCells;
  a.totals = a.hist + 256 * kNoAllocMaxBlocks;
  e = launch_bucket(a, reinterpret_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return noalloc_fail(CORAL_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return CORAL_OK;
}
