// noalloc.cu -- an index-table build that allocates no device memory.
//
// Some callers cannot allocate device memory while they run: a serving loop
// whose memory budget is fixed up front, a process whose framework allocator
// already owns nearly all of the GPU, or a hot path that must never stall on
// an allocator call.  lsh_build_tables_static gives them the per-table sort
// and bucket segmentation of lsh_build_index with its sort scratch in a
// file-scope device array instead of the stream-ordered pool.  The caller
// still passes the keys and the output tables.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "internal.h"

namespace {

// Scratch of the allocation-free build: 24 MiB.  A request needs the
// ping-pong keys (2 x 8 B) and ids (4 B) of its n L (point, table) pairs, at
// most 2^20 of them (20 MiB), plus 1 KiB of digit histogram per 4096-row tile
// and table; build_tables_scratch_bytes adds these up and larger requests are
// refused.  Every GPU that loads this library holds it until the process exits.
constexpr size_t kStaticScratchBytes = size_t(24) << 20;
static __device__ __align__(256) unsigned char g_static_sort_scratch[kStaticScratchBytes];

// Device address of g_static_sort_scratch per device (host code must not use
// the symbol itself: on the host it is only a stand-in for the device array).
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_sort_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

using namespace lsh;

extern "C" lsh_status lsh_build_tables_static(const uint64_t *keys, int64_t n, int32_t L, uint32_t *ids,
                                              uint64_t *ukeys, uint32_t *offsets, int64_t *nbuckets,
                                              void *stream) {
  if (L < 1 || n < 0) return fail(LSH_EINVAL, "lsh_build_tables_static: need n >= 0 and L >= 1");
  if (n > int64_t(UINT32_MAX) - 1) return fail(LSH_EINVAL, "lsh_build_tables_static: n must be < 2^32 - 1");
  if (!nbuckets || !offsets) return fail(LSH_EINVAL, "lsh_build_tables_static: NULL output");
  if (n > 0 && (!keys || !ids || !ukeys)) return fail(LSH_EINVAL, "lsh_build_tables_static: NULL argument");
  if (n * int64_t(L) > LSH_STATIC_MAX_PAIRS)
    return fail(LSH_EINVAL, "lsh_build_tables_static: n * L exceeds LSH_STATIC_MAX_PAIRS (2^20); "
                            "use lsh_build_index for larger batches");
  const size_t need = build_tables_scratch_bytes(n, L);
  if (need > kStaticScratchBytes)
    return fail(LSH_EINVAL, "lsh_build_tables_static: n and L need more than the 24 MiB static scratch");
  void *scratch = nullptr;
  LSH_CUDA_TRY(scratch_address(&scratch));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    LSH_CUDA_TRY(cudaMemsetAsync(nbuckets, 0, sizeof(int64_t) * L, s));
    LSH_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(uint32_t) * L, s));
    return LSH_OK;
  }
  LSH_CUDA_TRY(build_tables_scratch(keys, n, L, ids, ukeys, offsets, nbuckets, scratch, s));
  return LSH_OK;
}
