// hasher.cu -- replayed hashing of uneven batches (lsh_hasher_*).
//
// A stream of batches of different sizes would pay, per batch, for the host
// side of lsh_hash: plan lookup, queue allocation, a memset and two kernel
// launches.  A hasher captures that sequence once per batch-size bucket
// (powers of two from 8,192 rows) into a CUDA graph sized for the bucket's
// largest batch and replays it:
//
//   set_batch   1 thread: writes the batch descriptor {X, n, keys, key_ld}
//   memset      the recheck queue's counter
//   sketch      sketch_dense_kernel over all L tables (the plan autotuned
//               for the shape before the first capture of a large bucket)
//   recheck     sketch_recheck_kernel over the queued bins
//
// (the smallest bucket, up to 8,192 rows, rechecks in place inside the
// sketch kernel: no memset, no recheck node)
//
// The two hashing kernels read X, n and the key buffer from the descriptor,
// so between replays only the parameters of the first node change
// (cudaGraphExecKernelNodeSetParams); the grid, the plan and the queue stay
// those of the bucket.  Keys equal lsh_hash's, bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"

namespace lsh {
namespace {

__global__ void set_batch_kernel(BatchDesc *desc, const void *X, int64_t n, uint64_t *keys, int64_t key_ld) {
  desc->X = X;
  desc->n = n;
  desc->keys = keys;
  desc->key_ld = key_ld;
}

constexpr int kMinBucketLog2 = 13;  // 8,192 rows

struct Bucket {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t set_node = nullptr;
};

}  // namespace
}  // namespace lsh

using namespace lsh;

struct lsh_hasher_s {
  lsh_family_t fam = nullptr;  // borrowed: the family must outlive the hasher
  int32_t dtype = 0;
  int64_t ld = 0, max_rows = 0;
  bool vec = false;            // rows 16-byte aligned: every batch's X must be too
  BatchDesc *d_desc = nullptr;
  void *d_queue = nullptr;     // 16-byte counter + queue for the largest bucket
  int64_t qcap = 0;
  cudaStream_t cap_stream = nullptr;  // graphs are captured here (the caller's stream may be the legacy one)
  std::map<int, Bucket> buckets;
  int64_t captures = 0, replays = 0;
  std::mutex mu;
};

namespace {

int bucket_log2(int64_t n) {
  int b = kMinBucketLog2;
  while ((int64_t(1) << b) < n) ++b;
  return b;
}

void destroy_bucket(Bucket &b) {
  if (b.exec) cudaGraphExecDestroy(b.exec);
  if (b.graph) cudaGraphDestroy(b.graph);
  b = Bucket{};
}

lsh_status capture_bucket(lsh_hasher_s *h, int blog2, const void *X, int64_t n, uint64_t *keys, int64_t key_ld,
                          cudaStream_t stream, Bucket &out) {
  lsh_family_s *f = h->fam;
  SketchLaunch p = family_launch(f);
  p.X = X;
  p.dtype = h->dtype;
  p.ld = h->ld;
  p.n = std::min<int64_t>(int64_t(1) << blog2, std::max<int64_t>(h->max_rows, int64_t(1) << kMinBucketLog2));
  p.keys = keys;
  p.key_ld = key_ld;
  // the smallest bucket rechecks in place, as lsh_hash does below 8,192 rows:
  // no queue, no second kernel
  const bool queued = blog2 > kMinBucketLog2;
  if (queued) {
    p.qcount = static_cast<uint32_t *>(h->d_queue);
    p.queue = reinterpret_cast<int4 *>(static_cast<char *>(h->d_queue) + 16);
    p.qcap = uint32_t(h->qcap);
  }
  p.desc = h->d_desc;
  {
    // the autotuner times on this batch's rows, outside the capture
    SketchLaunch t = p;
    t.n = n;
    t.desc = nullptr;
    sketch_autotune(t, stream);
  }
  Bucket b;
  cudaStream_t cs = h->cap_stream;
  LSH_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  set_batch_kernel<<<1, 1, 0, cs>>>(h->d_desc, X, n, keys, key_ld);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && queued) e = cudaMemsetAsync(h->d_queue, 0, 16, cs);
  if (e == cudaSuccess) e = launch_sketch_dense(p, cs);
  if (e == cudaSuccess && queued) e = launch_sketch_recheck(p, f->d_mlist, f->d_mseg, cs);
  const cudaError_t ee = cudaStreamEndCapture(cs, &b.graph);
  if (e == cudaSuccess) e = ee;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b.exec, b.graph, 0);
  if (e == cudaSuccess) {
    size_t count = 0;
    e = cudaGraphGetNodes(b.graph, nullptr, &count);
    std::vector<cudaGraphNode_t> nodes(count);
    if (e == cudaSuccess && count) e = cudaGraphGetNodes(b.graph, nodes.data(), &count);
    for (size_t i = 0; e == cudaSuccess && i < count && !b.set_node; ++i) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nodes[i], &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
      cudaKernelNodeParams kp;
      if (cudaGraphKernelNodeGetParams(nodes[i], &kp) == cudaSuccess &&
          kp.func == reinterpret_cast<void *>(set_batch_kernel))
        b.set_node = nodes[i];
    }
    if (e == cudaSuccess && !b.set_node) e = cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) {
    destroy_bucket(b);
    cudaGetLastError();
    return cuda_fail(e, "lsh_hasher graph capture");
  }
  out = b;
  return LSH_OK;
}

}  // namespace

extern "C" {

lsh_status lsh_hasher_create(lsh_family_t fam, int32_t dtype, int64_t ld, int64_t max_rows, lsh_hasher_t *out) {
  if (!fam || !out) return fail(LSH_EINVAL, "lsh_hasher_create: NULL argument");
  *out = nullptr;
  const lsh_family_desc &d = fam->host.desc;
  if (kind_is_dense(d.kind))
    return fail(LSH_EUNSUPPORTED, "lsh_hasher: CS/HCS families only (the dense baseline hashes through lsh_hash)");
  if (dtype != LSH_F32 && dtype != LSH_BF16 && dtype != LSH_F16)
    return fail(LSH_EINVAL, "lsh_hasher: rows must be FP32, BF16 or FP16");
  if (ld < d.d) return fail(LSH_EINVAL, "lsh_hasher: ld must be >= d");
  if (max_rows < 1 || max_rows > int64_t(UINT32_MAX) - 1)
    return fail(LSH_EINVAL, "lsh_hasher: need 1 <= max_rows < 2^32 - 1");
  if (!fam->d_mlist) return fail(LSH_EUNSUPPORTED, "lsh_hasher: d too large for the dense-row kernel");
  const SketchPlan sp = plan_sketch_dense(d.d, d.m, d.L, fam->sketch_cap, dtype);
  if (!sp.ok) return fail(LSH_EUNSUPPORTED, "lsh_hasher: rows too long for the dense-row kernel's tile");
  LSH_CUDA_TRY(cudaSetDevice(fam->device));
  lsh_hasher_s *h = new (std::nothrow) lsh_hasher_s();
  if (!h) return fail(LSH_ENOMEM, "host allocation");
  h->fam = fam;
  h->dtype = dtype;
  h->ld = ld;
  h->max_rows = max_rows;
  const int64_t es = dtype == LSH_F32 ? 4 : 2;
  h->vec = (ld * es) % 16 == 0;
  const int64_t top = int64_t(1) << bucket_log2(max_rows);
  h->qcap = sketch_queue_cap(top, d.L, d.m);
  cudaError_t e = cudaMalloc(&h->d_desc, sizeof(BatchDesc));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_queue, size_t(16 + 16 * h->qcap));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    lsh_hasher_destroy(h);
    return cuda_fail(e, "lsh_hasher_create allocation");
  }
  *out = h;
  return LSH_OK;
}

lsh_status lsh_hasher_run(lsh_hasher_t h, const void *X, int64_t n, uint64_t *keys, int64_t key_ld, void *stream_) {
  if (!h) return fail(LSH_EINVAL, "lsh_hasher_run: NULL hasher");
  if (n < 0 || n > h->max_rows) return fail(LSH_EINVAL, "lsh_hasher_run: need 0 <= n <= max_rows");
  if (n == 0) return LSH_OK;
  if (!X || !keys) return fail(LSH_EINVAL, "lsh_hasher_run: NULL X or keys");
  if (key_ld < n) return fail(LSH_EINVAL, "lsh_hasher_run: key_ld must be >= n");
  if (h->vec && reinterpret_cast<uintptr_t>(X) % 16 != 0)
    return fail(LSH_EINVAL, "lsh_hasher_run: X must be 16-byte aligned (the row stride is a multiple of 16 bytes)");
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lock(h->mu);
  const int blog2 = bucket_log2(n);
  auto it = h->buckets.find(blog2);
  if (it == h->buckets.end()) {
    Bucket b;
    const lsh_status st = capture_bucket(h, blog2, X, n, keys, key_ld, stream, b);
    if (st != LSH_OK) return st;
    it = h->buckets.emplace(blog2, b).first;
    ++h->captures;
  }
  Bucket &b = it->second;
  const int kernels = blog2 > kMinBucketLog2 ? 3 : 2;
  BatchDesc *desc = h->d_desc;
  void *args[] = {&desc, &X, &n, &keys, &key_ld};
  cudaKernelNodeParams kp{};
  kp.func = reinterpret_cast<void *>(set_batch_kernel);
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  LSH_CUDA_TRY(cudaGraphExecKernelNodeSetParams(b.exec, b.set_node, &kp));
  LSH_CUDA_TRY(cudaGraphLaunch(b.exec, stream));
  ++h->replays;
  count_launches(kernels);  // set_batch, the sketch kernel and (queued buckets) the recheck kernel
  return LSH_OK;
}

lsh_status lsh_hasher_info(lsh_hasher_t h, int64_t *captures, int64_t *replays) {
  if (!h) return fail(LSH_EINVAL, "lsh_hasher_info: NULL hasher");
  std::lock_guard<std::mutex> lock(h->mu);
  if (captures) *captures = h->captures;
  if (replays) *replays = h->replays;
  return LSH_OK;
}

void lsh_hasher_destroy(lsh_hasher_t h) {
  if (!h) return;
  cudaDeviceSynchronize();  // no replay may still use the graphs, the descriptor or the queue
  for (auto &kv : h->buckets) destroy_bucket(kv.second);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  cudaFree(h->d_desc);
  cudaFree(h->d_queue);
  delete h;
}

}  // extern "C"
