// hash_sketch_srp.cu -- the dense-row sketch kernel and its recheck
// kernel instantiated for the SRP kinds (CS-SRP, HCS-SRP, CSSRP-L).
#include "sketch_dense_kernel.cuh"

namespace lsh {
namespace sk {

cudaError_t launch_srp(const Args &a, bool full, cudaStream_t stream) {
  return full ? launch_e<true, true>(a, stream) : launch_e<true, false>(a, stream);
}

cudaError_t launch_recheck_srp(const SketchLaunch &p, const uint16_t *mlist, const uint32_t *mseg, int blocks,
                                 cudaStream_t stream) {
  return launch_recheck_dt<true>(p, mlist, mseg, blocks, stream);
}

}  // namespace sk
}  // namespace lsh
