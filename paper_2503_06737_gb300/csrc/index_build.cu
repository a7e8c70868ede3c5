// index_build.cu -- the L hash tables of the (m, tau)-amplified LSH scheme
// (Sec. 3.1): every point is stored in the bucket of its key in each table.
//
// Per table the (key, id) pairs are put in (key, id) order by a stable LSD
// radix sort over the 64-bit key, 8 bits per pass (ids start in ascending
// order, so stability gives ascending ids inside a bucket), and the sorted
// keys are cut into buckets: distinct keys ascending and the start offset of
// each bucket.  All L tables are sorted by the same launches (grid.y = table).
//
// One pass = three kernels:
//   histogram  per (table, tile of 4096 keys): digit counts, digit-major;
//   scan       per table: exclusive scan over (digit, tile) -> global offsets;
//   scatter    per (table, tile): stable ranks inside the tile from warp
//              match-any over 32 consecutive keys at a time, warp-ordered
//              prefix, sorted tile staged in shared memory, then written out
//              in order (runs of one digit land contiguously).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace lsh {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;                    // keys per thread
constexpr int kTile = kThreads * kItems;      // 4096 keys per tile
constexpr int kRadix = 256;

__device__ __forceinline__ uint32_t digit_of(uint64_t k, int shift) {
  return uint32_t(k >> shift) & (kRadix - 1);
}

__global__ void __launch_bounds__(kThreads) radix_hist(const uint64_t *__restrict__ keys, int64_t n,
                                                       int shift, int ntiles, uint32_t *__restrict__ hist) {
  __shared__ uint32_t h[kWarps][kRadix];
  const int t = blockIdx.y, tile = blockIdx.x;
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  const uint64_t *k = keys + int64_t(t) * n;
  const int64_t base = int64_t(tile) * kTile;
  // all kItems loads of a thread in flight before the first use
  uint64_t kk[kItems];
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int64_t idx = base + it * kThreads + threadIdx.x;
    kk[it] = idx < n ? __ldg(k + idx) : 0ull;
  }
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int64_t idx = base + it * kThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[warp][digit_of(kk[it], shift)], 1u);
  }
  __syncthreads();
  for (int dgt = threadIdx.x; dgt < kRadix; dgt += kThreads) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += h[w][dgt];
    hist[(int64_t(t) * kRadix + dgt) * ntiles + tile] = s;
  }
}

// Block-wide exclusive scan of one value per thread (blockDim.x = 1024).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_sums, uint32_t &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= o) s += u;
  }
  if (lane == 31) warp_sums[warp] = s;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? warp_sums[lane] : 0u;
    uint32_t ws = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, ws, o);
      if (lane >= o) ws += u;
    }
    if (lane < nw) warp_sums[lane] = ws - w;
    if (lane == 31) warp_sums[32] = ws;
  }
  __syncthreads();
  const uint32_t r = warp_sums[warp] + s - v;
  total = warp_sums[32];
  __syncthreads();
  return r;
}

// Exclusive scan, in place, of cnt[t][0..len) for each table t (grid.x = table).
// Optionally writes the table total to total_out[t].  Each warp owns a
// contiguous segment, read 32 consecutive words at a time (coalesced) with
// eight such loads in flight: a first pass sums the segment, a block scan of
// the warp sums gives each warp its base, and a second pass scans and writes.
constexpr int kScanBatch = 8;
__global__ void __launch_bounds__(1024) scan_rows(uint32_t *__restrict__ cnt, int64_t len,
                                                  int64_t *__restrict__ total_out) {
  __shared__ uint32_t warp_sums[33];
  uint32_t *c = cnt + int64_t(blockIdx.x) * len;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t seg = ((len + nw - 1) / nw + 31) & ~int64_t(31);
  const int64_t beg = int64_t(warp) * seg;
  const int64_t end = beg + seg < len ? beg + seg : len;
  uint32_t s = 0;
  for (int64_t i0 = beg; i0 < end; i0 += 32 * kScanBatch) {
    uint32_t v[kScanBatch];
#pragma unroll
    for (int b = 0; b < kScanBatch; ++b) {
      const int64_t i = i0 + b * 32 + lane;
      v[b] = i < end ? c[i] : 0u;
    }
#pragma unroll
    for (int b = 0; b < kScanBatch; ++b) s += v[b];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  // the warp totals, scanned by the block (one value per warp, in lane 0)
  uint32_t total;
  const uint32_t wbase = block_exclusive_scan(lane == 0 ? s : 0u, warp_sums, total);
  uint32_t run = __shfl_sync(0xffffffffu, wbase, 0);
  for (int64_t i0 = beg; i0 < end; i0 += 32 * kScanBatch) {
    uint32_t v[kScanBatch];
#pragma unroll
    for (int b = 0; b < kScanBatch; ++b) {
      const int64_t i = i0 + b * 32 + lane;
      v[b] = i < end ? c[i] : 0u;
    }
#pragma unroll
    for (int b = 0; b < kScanBatch; ++b) {
      uint32_t x = v[b];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
      }
      const int64_t i = i0 + b * 32 + lane;
      if (i < end) c[i] = run + x - v[b];
      run += __shfl_sync(0xffffffffu, x, 31);
    }
  }
  if (total_out && threadIdx.x == 0) total_out[blockIdx.x] = int64_t(total);
}

__global__ void __launch_bounds__(kThreads) radix_scatter(const uint64_t *__restrict__ kin,
                                                          const uint32_t *__restrict__ iin,
                                                          uint64_t *__restrict__ kout,
                                                          uint32_t *__restrict__ iout, int64_t n, int shift,
                                                          int ntiles, const uint32_t *__restrict__ gscan) {
  extern __shared__ __align__(16) unsigned char sm[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(sm);                       // [kTile]
  uint32_t *si = reinterpret_cast<uint32_t *>(sk + kTile);               // [kTile]
  uint32_t *wc = si + kTile;                                             // [kWarps][kRadix]
  uint32_t *dstart = wc + kWarps * kRadix;                               // [kRadix]
  uint32_t *gbase = dstart + kRadix;                                     // [kRadix]
  uint32_t *wsum = gbase + kRadix;                                       // [33]

  const int t = blockIdx.y, tile = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t *k = kin + int64_t(t) * n;
  const uint32_t *ids = iin ? iin + int64_t(t) * n : nullptr;
  const int64_t base = int64_t(tile) * kTile;
  const int64_t cnt64 = n - base < kTile ? n - base : kTile;
  const int count = int(cnt64);

  for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) wc[i] = 0;
  __syncthreads();

  // warp w owns keys [w*512, (w+1)*512) of the tile, 32 consecutive per round
  uint64_t key[kItems];
  uint32_t id[kItems];
  uint32_t rank[kItems];
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t *mycnt = wc + warp * kRadix;
  // all loads of the tile in flight before the ranking uses them
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int pos = warp * (kItems * 32) + it * 32 + lane;
    const bool act = pos < count;
    key[it] = act ? __ldg(k + base + pos) : ~0ull;
    id[it] = act ? (ids ? __ldg(ids + base + pos) : uint32_t(base + pos)) : 0u;
  }
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int pos = warp * (kItems * 32) + it * 32 + lane;
    const bool act = pos < count;
    const uint32_t dg = act ? digit_of(key[it], shift) : 0xffffffffu;
    const uint32_t peers = __match_any_sync(0xffffffffu, dg);
    uint32_t r = 0;
    if (act) r = mycnt[dg] + __popc(peers & lt);
    __syncwarp();
    if (act && (peers & lt) == 0) mycnt[dg] += __popc(peers);
    __syncwarp();
    rank[it] = r;
  }
  __syncthreads();
  // per digit: prefix over warps; totals; block-local digit starts
  {
    const int dgt = threadIdx.x;  // kThreads == kRadix
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = wc[w * kRadix + dgt];
      wc[w * kRadix + dgt] = run;
      run += c;
    }
    uint32_t tot;
    const uint32_t st = block_exclusive_scan(run, wsum, tot);
    dstart[dgt] = st;
    gbase[dgt] = gscan[(int64_t(t) * kRadix + dgt) * ntiles + tile];
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int pos = warp * (kItems * 32) + it * 32 + lane;
    if (pos < count) {
      const uint32_t dg = digit_of(key[it], shift);
      const uint32_t p = dstart[dg] + wc[warp * kRadix + dg] + rank[it];
      sk[p] = key[it];
      si[p] = id[it];
    }
  }
  __syncthreads();
  uint64_t *ko = kout + int64_t(t) * n;
  uint32_t *io = iout + int64_t(t) * n;
  for (int s = threadIdx.x; s < count; s += kThreads) {
    const uint64_t kk = sk[s];
    const uint32_t dg = digit_of(kk, shift);
    const int64_t g = int64_t(gbase[dg]) + (s - int64_t(dstart[dg]));
    ko[g] = kk;
    io[g] = si[s];
  }
}

// Segmentation: bucket heads of sorted keys.
__global__ void __launch_bounds__(kThreads) seg_count(const uint64_t *__restrict__ sk, int64_t n, int ntiles,
                                                      uint32_t *__restrict__ bcnt) {
  __shared__ uint32_t wsum[33];
  const int t = blockIdx.y, tile = blockIdx.x;
  const uint64_t *k = sk + int64_t(t) * n;
  const int64_t base = int64_t(tile) * kTile;
  uint32_t c = 0;
  for (int i = threadIdx.x; i < kTile; i += kThreads) {
    const int64_t idx = base + i;
    if (idx < n && (idx == 0 || k[idx] != k[idx - 1])) ++c;
  }
  uint32_t tot;
  block_exclusive_scan(c, wsum, tot);
  if (threadIdx.x == 0) bcnt[int64_t(t) * ntiles + tile] = tot;
}

// Bucket heads of one tile, in order: warp w walks keys [w*512, (w+1)*512) of
// the tile 32 at a time (lane = consecutive key: coalesced), counts its heads
// with ballots, and after a block scan over the warps writes them with the
// same ballots (order preserved inside the warp and across warps).
__global__ void __launch_bounds__(kThreads) seg_write(const uint64_t *__restrict__ sk, int64_t n, int ntiles,
                                                      const uint32_t *__restrict__ boffs,
                                                      const int64_t *__restrict__ nb,
                                                      uint64_t *__restrict__ ukeys,
                                                      uint32_t *__restrict__ offsets) {
  __shared__ uint32_t wsum[33];
  const int t = blockIdx.y, tile = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t *k = sk + int64_t(t) * n;
  const int64_t wbase = int64_t(tile) * kTile + int64_t(warp) * (kItems * 32);
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t heads = 0;
#pragma unroll 4
  for (int it = 0; it < kItems; ++it) {
    const int64_t idx = wbase + it * 32 + lane;
    const bool h = idx < n && (idx == 0 || k[idx] != k[idx - 1]);
    heads += __popc(__ballot_sync(0xffffffffu, h));
  }
  // block-exclusive scan of the per-warp head counts (one value per warp, lane 0)
  uint32_t tot;
  const uint32_t wpos = block_exclusive_scan(lane == 0 ? heads : 0u, wsum, tot);
  uint32_t pos = boffs[int64_t(t) * ntiles + tile] + __shfl_sync(0xffffffffu, wpos, 0);
  uint64_t *uk = ukeys + int64_t(t) * n;
  uint32_t *of = offsets + int64_t(t) * (n + 1);
#pragma unroll 4
  for (int it = 0; it < kItems; ++it) {
    const int64_t idx = wbase + it * 32 + lane;
    uint64_t key = 0;
    bool h = false;
    if (idx < n) {
      key = k[idx];
      h = idx == 0 || key != k[idx - 1];
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, h);
    if (h) {
      const uint32_t p = pos + __popc(bal & lt);
      uk[p] = key;
      of[p] = uint32_t(idx);
    }
    pos += __popc(bal);
  }
  if (tile == 0 && threadIdx.x == 0) of[nb[t]] = uint32_t(n);
}

}  // namespace

size_t build_tables_scratch_bytes(int64_t n, int32_t L) {
  if (n <= 0 || L <= 0) return 0;
  const size_t ntiles = size_t((n + kTile - 1) / kTile);
  const size_t nk = size_t(n) * L;
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  return up(nk * 8) + up(nk * 8) + up(nk * 4) + up(size_t(kRadix) * ntiles * L * 4);
}

cudaError_t build_tables_scratch(const uint64_t *keys, int64_t n, int32_t L, uint32_t *ids_out,
                                 uint64_t *ukeys_out, uint32_t *offsets_out, int64_t *nb_out, void *scratch,
                                 cudaStream_t stream) {
  if (L <= 0) return cudaSuccess;
  if (n == 0) return cudaMemsetAsync(nb_out, 0, sizeof(int64_t) * L, stream);
  const int ntiles = int((n + kTile - 1) / kTile);
  const size_t nk = size_t(n) * L;
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  unsigned char *base = static_cast<unsigned char *>(scratch);
  uint64_t *kA = reinterpret_cast<uint64_t *>(base);
  uint64_t *kB = reinterpret_cast<uint64_t *>(base + up(nk * 8));
  uint32_t *iA = reinterpret_cast<uint32_t *>(base + 2 * up(nk * 8));
  uint32_t *hist = reinterpret_cast<uint32_t *>(base + 2 * up(nk * 8) + up(nk * 4));
  const size_t hist_len = size_t(kRadix) * ntiles;
  const int scatter_smem = kTile * 12 + (kWarps * kRadix + 2 * kRadix + 33) * 4;
  cudaError_t e = cudaFuncSetAttribute(radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, scatter_smem);
  const uint64_t *kin = keys;
  const uint32_t *iin = nullptr;
  for (int pass = 0; pass < 8 && e == cudaSuccess; ++pass) {
    uint64_t *kout = (pass % 2 == 0) ? kA : kB;
    uint32_t *iout = (pass % 2 == 0) ? iA : ids_out;
    const dim3 grid((unsigned)ntiles, (unsigned)L);
    radix_hist<<<grid, kThreads, 0, stream>>>(kin, n, pass * 8, ntiles, hist);
    scan_rows<<<L, 1024, 0, stream>>>(hist, int64_t(hist_len), nullptr);
    radix_scatter<<<grid, kThreads, scatter_smem, stream>>>(kin, iin, kout, iout, n, pass * 8, ntiles, hist);
    e = cudaGetLastError();
    count_launches(3);
    kin = kout;
    iin = iout;
  }
  if (e == cudaSuccess) {
    const dim3 grid((unsigned)ntiles, (unsigned)L);
    seg_count<<<grid, kThreads, 0, stream>>>(kB, n, ntiles, hist);
    scan_rows<<<L, 1024, 0, stream>>>(hist, ntiles, nb_out);
    seg_write<<<grid, kThreads, 0, stream>>>(kB, n, ntiles, hist, nb_out, ukeys_out, offsets_out);
    e = cudaGetLastError();
    count_launches(3);
  }
  return e;
}

// The same build with its scratch from the stream-ordered pool.
cudaError_t build_tables(const uint64_t *keys, int64_t n, int32_t L, uint32_t *ids_out, uint64_t *ukeys_out,
                         uint32_t *offsets_out, int64_t *nb_out, cudaStream_t stream) {
  if (L <= 0) return cudaSuccess;
  if (n == 0) return cudaMemsetAsync(nb_out, 0, sizeof(int64_t) * L, stream);
  void *scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, build_tables_scratch_bytes(n, L), stream);
  if (e != cudaSuccess) return e;
  e = build_tables_scratch(keys, n, L, ids_out, ukeys_out, offsets_out, nb_out, scratch, stream);
  const cudaError_t f = cudaFreeAsync(scratch, stream);
  return e != cudaSuccess ? e : f;
}

}  // namespace lsh
