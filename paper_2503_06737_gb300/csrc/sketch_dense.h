// sketch_dense.h -- the tile plan of the dense-row CS/HCS hashing kernel
// (sketch_dense_kernel.cuh) and the entry points of its instantiations: one
// translation unit for the E2LSH kinds (hash_sketch_e2lsh.cu), one for the
// SRP kinds (hash_sketch_srp.cu), so that they compile in parallel.  Plans,
// the autotuner and the host launch are in hash_sketch.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace lsh {
namespace sk {

constexpr int kWarp = 32;
constexpr float kU32 = 5.9604644775390625e-08f;  // 2^-24, unit roundoff of FP32
constexpr int kMaxSmem = 232448;                 // 227 KB opt-in per block

struct Plan {
  int Lg, G, RG, WPT, W, smem;
  int RPL;       // rows per lane
  int hw;        // 1: the half-warps split every bin (16 row groups per warp)
  int es;        // entry bytes (2 or 4)
  int cap;       // entry capacity per table (multiple of 4)
  int dp;        // odd word stride of a row inside a group (>= d + 1)
  int off_ent, off_seg, off_cst, off_rng, off_key, off_x, off_xmax, off_bad, off_ctr;
};

struct Args {
  SketchLaunch p;
  Plan pl;
  int ntiles;
  int slots;     // CTAs per table group
  int vec;       // rows are 16-byte aligned: 128-bit tile loads
  float sqrtm_f, invw_f;
};
constexpr int kMaxWpt = 4;  // warps per table at most; a table keeps kMaxWpt + 1 range records

// Threads per CTA at most: 768 (80 registers) for one or two rows per lane,
// 512 for four (their accumulators need more registers).
__host__ __device__ constexpr int max_threads(int rpl) { return rpl == 4 ? 512 : 768; }

// Row groups (lanes with their own rows) per warp: 32, or 16 when the two
// half-warps split every bin between them (HW: half h sums the quads 2k + h
// of the bin for the same 16 row groups, and the halves combine at the end
// of the bin) -- which keeps RPL rows per lane with half the rows per tile.
__host__ __device__ constexpr int groups_per_warp(bool hw) { return hw ? 16 : 32; }

// Launch the sketch kernel of plan a.pl (full: codes, SRP bits, projections
// or counters are requested; otherwise keys only).
cudaError_t launch_e2lsh(const Args &a, bool full, cudaStream_t stream);
cudaError_t launch_srp(const Args &a, bool full, cudaStream_t stream);

// Launch the recheck kernel of the queued bins of p on the given grid.
cudaError_t launch_recheck_e2lsh(const SketchLaunch &p, const uint16_t *mlist, const uint32_t *mseg, int blocks,
                                 cudaStream_t stream);
cudaError_t launch_recheck_srp(const SketchLaunch &p, const uint16_t *mlist, const uint32_t *mseg, int blocks,
                               cudaStream_t stream);

}  // namespace sk
}  // namespace lsh
