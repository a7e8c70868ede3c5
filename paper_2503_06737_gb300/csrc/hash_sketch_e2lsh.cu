// hash_sketch_e2lsh.cu -- the dense-row sketch kernel and its recheck
// kernel instantiated for the E2LSH kinds (CS-E2LSH, HCS-E2LSH).
#include "sketch_dense_kernel.cuh"

namespace lsh {
namespace sk {

cudaError_t launch_e2lsh(const Args &a, bool full, cudaStream_t stream) {
  return full ? launch_e<false, true>(a, stream) : launch_e<false, false>(a, stream);
}

cudaError_t launch_recheck_e2lsh(const SketchLaunch &p, const uint16_t *mlist, const uint32_t *mseg, int blocks,
                                 cudaStream_t stream) {
  return launch_recheck_dt<false>(p, mlist, mseg, blocks, stream);
}

}  // namespace sk
}  // namespace lsh
