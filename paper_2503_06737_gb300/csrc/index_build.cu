// index_build.cu -- the L hash tables of the (m, tau)-amplified LSH scheme
// (Sec. 3.1): every point is stored in the bucket of its key in each table.
//
// Per table the (key, id) pairs are put in (key, id) order by a stable sort
// (ids start in ascending order, so stability gives ascending ids inside a
// bucket), and the sorted keys are cut into buckets: distinct keys ascending
// and the start offset of each bucket.  All L tables are sorted by the same
// launches (grid.y = table).  Two sorts give the same order: the LSD radix
// sort over the 64-bit key, 8 bits per pass, and the bucket sort below.
//
// One LSD pass = three kernels:
//   histogram  per (table, tile of 4096 keys): digit counts, digit-major;
//   scan       per table: exclusive scan over (digit, tile) -> global offsets;
//   scatter    per (table, tile): stable ranks inside the tile from warp
//              match-any over 32 consecutive keys at a time, warp-ordered
//              prefix, sorted tile staged in shared memory, then written out
//              in order (runs of one digit land contiguously).
//
// Bucket sort (the default for 2,048 to kBucketMaxN keys per table): a
// reduction finds the bits on which a table's keys differ; one pass on the 8
// highest of them cuts the table into 256 buckets (about n / 256 keys each
// for hashed keys), and one CTA per (bucket, table) finishes the stable sort
// -- on chip when the bucket has at most kBCap keys and the counting pass
// on the next 8 bits leaves groups of at most kGroupMax (then comparisons
// inside each group place its keys), else by counting passes on the lower
// digits through global memory in sub-tiles of kBCap, skipping digits on
// which the table's, or the bucket's, keys all agree.  The same (key, id) order as the eight global passes, at one global
// pass plus one read and one write of every pair.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

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

// spread[t] = {OR of the keys, OR of their complements}: their AND is the set
// of bits on which two keys of table t differ.  The bucket pass takes the 8
// highest of those bits (digit shift msd_shift), so its 256 digits are all in
// use even when the keys leave their high bits zero (SRP codes of m < 64).
__device__ __forceinline__ uint64_t varying_bits(const unsigned long long *spread, int t) {
  return uint64_t(spread[2 * t]) & uint64_t(spread[2 * t + 1]);
}
__device__ __forceinline__ int msd_shift(uint64_t v) {
  const int hi = v ? 63 - __clzll((long long)v) : 0;
  return hi >= 8 ? hi - 7 : 0;
}

__global__ void __launch_bounds__(kThreads) key_spread(const uint64_t *__restrict__ keys, int64_t n,
                                                       unsigned long long *__restrict__ spread) {
  __shared__ unsigned long long red[2][kWarps];
  const int t = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t *k = keys + int64_t(t) * n;
  const int64_t base = int64_t(blockIdx.x) * kTile;
  uint64_t kk[kItems];
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int64_t idx = base + it * kThreads + threadIdx.x;
    kk[it] = idx < n ? __ldg(k + idx) : 0ull;
  }
  uint64_t o1 = 0, o0 = 0;
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int64_t idx = base + it * kThreads + threadIdx.x;
    if (idx < n) {
      o1 |= kk[it];
      o0 |= ~kk[it];
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    o1 |= __shfl_xor_sync(0xffffffffu, o1, off);
    o0 |= __shfl_xor_sync(0xffffffffu, o0, off);
  }
  if (lane == 0) {
    red[0][warp] = o1;
    red[1][warp] = o0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t a = 0, c = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      a |= red[0][w];
      c |= red[1][w];
    }
    atomicOr(&spread[2 * t], (unsigned long long)a);
    atomicOr(&spread[2 * t + 1], (unsigned long long)c);
  }
}

// kDevShift: the digit shift is the table's msd_shift (bucket pass), else `shift`.
template <bool kDevShift>
__global__ void __launch_bounds__(kThreads) radix_hist(const uint64_t *__restrict__ keys, int64_t n,
                                                       int shift, int ntiles, uint32_t *__restrict__ hist,
                                                       const unsigned long long *__restrict__ spread) {
  __shared__ uint32_t h[kWarps][kRadix];
  const int t = blockIdx.y, tile = blockIdx.x;
  if (kDevShift) shift = msd_shift(varying_bits(spread, t));
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

template <bool kDevShift>
__global__ void __launch_bounds__(kThreads) radix_scatter(const uint64_t *__restrict__ kin,
                                                          const uint32_t *__restrict__ iin,
                                                          uint64_t *__restrict__ kout,
                                                          uint32_t *__restrict__ iout, int64_t n, int shift,
                                                          int ntiles, const uint32_t *__restrict__ gscan,
                                                          const unsigned long long *__restrict__ spread) {
  if (kDevShift) shift = msd_shift(varying_bits(spread, blockIdx.y));
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

// ---- bucket sort: one CTA per (bucket of the highest varying digit, table) ----
constexpr int kBItems = 20;                     // keys per thread held on chip
constexpr int kBCap = kThreads * kBItems;       // 5120 keys
// the automatic bucket path's limit: 256 buckets of 4,400 keys on average,
// whose largest stays below kBCap for hashed keys
constexpr int64_t kBucketMaxN = 1126400;

struct BucketSmem {
  uint64_t *sk;      // [kBCap] a sub-tile in digit order
  uint32_t *si;      // [kBCap]
  uint32_t *wc;      // [kWarps][kRadix] per-warp digit counts, then their prefix over warps
  uint32_t *dstart;  // [kRadix] where digit d starts in the sorted sub-tile
  uint32_t *dcnt;    // [kRadix] items of digit d in the sub-tile
  uint32_t *doff;    // [kRadix] large buckets: where digit d continues in the bucket
  uint32_t *wsum;    // [33]
  int *flag;
};

__device__ __forceinline__ int bpos(int warp, int it, int lane) { return warp * (kBItems * 32) + it * 32 + lane; }

// One stable counting pass over the cnt (<= kBCap) items the CTA holds, item
// `it` of `lane` in `warp` at position bpos(warp, it, lane), on the digit at
// `shift`.  Returns true when all items have one digit: nothing moves.  Else
// sk/si hold the items in (digit, position) order.  Either way dstart/dcnt
// describe the digits.  wc must be zero on entry and is zero on return.
__device__ __forceinline__ bool tile_pass(const uint64_t (&key)[kBItems], const uint32_t (&id)[kBItems], int cnt,
                                          int shift, const BucketSmem &S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t *mycnt = S.wc + warp * kRadix;
  uint32_t rk[kBItems / 2];  // ranks inside the warp's digit run, two 16-bit halves a word
#pragma unroll
  for (int it = 0; it < kBItems; ++it) {
    const bool act = bpos(warp, it, lane) < cnt;
    const uint32_t dg = act ? digit_of(key[it], shift) : 0xffffffffu;
    const uint32_t peers = __match_any_sync(0xffffffffu, dg);
    uint32_t r = 0;
    if (act) r = mycnt[dg] + __popc(peers & lt);
    __syncwarp();
    if (act && (peers & lt) == 0) mycnt[dg] += __popc(peers);
    __syncwarp();
    if (it & 1) rk[it >> 1] |= r << 16;
    else rk[it >> 1] = r;
  }
  __syncthreads();
  {
    const int dgt = threadIdx.x;  // kThreads == kRadix
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = S.wc[w * kRadix + dgt];
      S.wc[w * kRadix + dgt] = run;
      run += c;
    }
    uint32_t tot;
    S.dstart[dgt] = block_exclusive_scan(run, S.wsum, tot);
    S.dcnt[dgt] = run;
    if (run == uint32_t(cnt)) *S.flag = 1;
  }
  __syncthreads();
  const bool same = *S.flag != 0;
  if (!same) {
#pragma unroll
    for (int it = 0; it < kBItems; ++it) {
      if (bpos(warp, it, lane) < cnt) {
        const uint32_t dg = digit_of(key[it], shift);
        const uint32_t p = S.dstart[dg] + S.wc[warp * kRadix + dg] + ((rk[it >> 1] >> (16 * (it & 1))) & 0xffffu);
        S.sk[p] = key[it];
        S.si[p] = id[it];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int w = 0; w < kWarps; ++w) S.wc[w * kRadix + threadIdx.x] = 0;
  if (threadIdx.x == 0) *S.flag = 0;
  __syncthreads();
  return same;
}

// The bucket a CTA of the bucket-sort kernels owns, and the digits it sorts on.
struct BucketJob {
  int64_t s, sz;     // its range [s, s + sz) in the table
  int msd;           // the table's bucket-digit shift
  uint32_t passes;   // bit p: sort on the digit at 8p (below msd, and some keys of the table differ there)
};

__device__ __forceinline__ BucketJob bucket_job(int t, int b, int64_t n, int ntiles,
                                                const uint32_t *__restrict__ gscan,
                                                const unsigned long long *__restrict__ spread) {
  const uint32_t *g = gscan + int64_t(t) * kRadix * ntiles;
  BucketJob j;
  j.s = g[int64_t(b) * ntiles];
  j.sz = (b + 1 < kRadix ? int64_t(g[int64_t(b + 1) * ntiles]) : n) - j.s;
  const uint64_t v = varying_bits(spread, t);
  j.msd = msd_shift(v);
  j.passes = 0;
  for (int p = 0; 8 * p < j.msd; ++p)
    if ((v >> (8 * p)) & 0xffull) j.passes |= 1u << p;
  return j;
}

__device__ __forceinline__ BucketSmem bucket_smem(unsigned char *sm) {
  BucketSmem S;
  S.sk = reinterpret_cast<uint64_t *>(sm);
  S.si = reinterpret_cast<uint32_t *>(S.sk + kBCap);
  S.wc = S.si + kBCap;
  S.dstart = S.wc + kWarps * kRadix;
  S.dcnt = S.dstart + kRadix;
  S.doff = S.dcnt + kRadix;
  S.wsum = S.doff + kRadix;
  S.flag = reinterpret_cast<int *>(S.wsum + 33);
  for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) S.wc[i] = 0;
  if (threadIdx.x == 0) *S.flag = 0;
  __syncthreads();
  return S;
}
constexpr int kBucketSmem = kBCap * 12 + (kWarps * kRadix + 3 * kRadix + 33 + 1) * 4;
// groups of keys equal on the 8 bits below the bucket digit are finished by
// comparisons up to this size (about 15 keys on average for hashed keys)
constexpr int kGroupMax = 96;

// Grid (kRadix, L): CTA (b, t) sorts bucket b of table t -- the keys whose
// digit at msd_shift is b, contiguous in (kin, iin) after the bucket pass and
// in id order there -- into (kout, iout) when it has at most kBCap keys.  One
// stable counting pass on the 8 bits below the bucket digit cuts it into
// groups; a key's place inside its group is the number of group members with
// a smaller key, or an equal key before it (the pass is stable, so equal keys
// are still in id order).  Buckets of more than kBCap keys, and buckets with
// a group above kGroupMax keys (many repeated keys), are appended to `large`
// for bucket_sort_large.
__global__ void __launch_bounds__(kThreads, 2) bucket_sort(const uint64_t *__restrict__ kin,
                                                           const uint32_t *__restrict__ iin,
                                                           uint64_t *__restrict__ kout,
                                                           uint32_t *__restrict__ iout, int64_t n, int ntiles,
                                                           const uint32_t *__restrict__ gscan,
                                                           const unsigned long long *__restrict__ spread,
                                                           uint32_t *__restrict__ large) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int t = blockIdx.y, b = blockIdx.x;
  const BucketJob J = bucket_job(t, b, n, ntiles, gscan, spread);
  if (J.sz <= 0) return;
  if (J.sz > kBCap) {
    if (threadIdx.x == 0) large[1 + atomicAdd(&large[0], 1u)] = (uint32_t(t) << 8) | uint32_t(b);
    return;
  }
  const BucketSmem S = bucket_smem(sm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cnt = int(J.sz);
  const uint64_t *ka = kin + int64_t(t) * n + J.s;
  const uint32_t *ia = iin + int64_t(t) * n + J.s;
  uint64_t *kb = kout + int64_t(t) * n + J.s;
  uint32_t *ib = iout + int64_t(t) * n + J.s;
  uint64_t key[kBItems];
  uint32_t id[kBItems];
#pragma unroll
  for (int it = 0; it < kBItems; ++it) {
    const int pos = bpos(warp, it, lane);
    key[it] = pos < cnt ? __ldg(ka + pos) : ~0ull;
    id[it] = pos < cnt ? __ldg(ia + pos) : 0u;
  }
  if (J.passes != 0) {
    const int s2 = J.msd >= 8 ? J.msd - 8 : 0;
    if (tile_pass(key, id, cnt, s2, S)) {
      // one group: the keys keep their order
#pragma unroll
      for (int it = 0; it < kBItems; ++it) {
        const int pos = bpos(warp, it, lane);
        if (pos < cnt) {
          S.sk[pos] = key[it];
          S.si[pos] = id[it];
        }
      }
    }
    if (!__syncthreads_or(S.dcnt[threadIdx.x] > uint32_t(kGroupMax))) {
      for (int i = threadIdx.x; i < cnt; i += kThreads) {
        const uint64_t k = S.sk[i];
        const uint32_t d = digit_of(k, s2);
        const int a = int(S.dstart[d]), e = a + int(S.dcnt[d]);
        int r = 0;
        for (int j = a; j < e; ++j) {
          const uint64_t kj = S.sk[j];
          r += int(kj < k) + int(kj == k && j < i);
        }
        kb[a + r] = k;
        ib[a + r] = S.si[i];
      }
      return;
    }
    // a large group (many repeated keys): bucket_sort_large sorts this
    // bucket on every lower digit instead
    if (threadIdx.x == 0) large[1 + atomicAdd(&large[0], 1u)] = (uint32_t(t) << 8) | uint32_t(b);
    return;
  }
#pragma unroll
  for (int it = 0; it < kBItems; ++it) {
    const int pos = bpos(warp, it, lane);
    if (pos < cnt) {
      kb[pos] = key[it];
      ib[pos] = id[it];
    }
  }
}

// The buckets of more than kBCap keys (clustered keys, or more than about
// kBucketMaxN rows) and those with large groups of repeated keys, from the
// list bucket_sort left in `large` (count, then
// (table << 8 | bucket) entries), CTAs taking entries in turn: each digit
// pass through global memory -- the bucket's digit counts, then sub-tiles of
// kBCap keys in order, each sorted on chip and written to its digits' places
// -- alternating between (kin, iin) and (kout, iout) over the bucket's own
// range, ending in (kout, iout).
__global__ void __launch_bounds__(kThreads, 1) bucket_sort_large(uint64_t *kin, uint32_t *iin, uint64_t *kout,
                                                                 uint32_t *iout, int64_t n, int ntiles,
                                                                 const uint32_t *__restrict__ gscan,
                                                                 const unsigned long long *__restrict__ spread,
                                                                 const uint32_t *__restrict__ large) {
  extern __shared__ __align__(16) unsigned char sm[];
  const uint32_t njobs = large[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t w = blockIdx.x; w < njobs; w += gridDim.x) {
    const int t = int(large[1 + w] >> 8), b = int(large[1 + w] & 0xffu);
    const BucketJob J = bucket_job(t, b, n, ntiles, gscan, spread);
    const BucketSmem S = bucket_smem(sm);
    const int64_t sz = J.sz;
    uint64_t *ka = kin + int64_t(t) * n + J.s, *kb = kout + int64_t(t) * n + J.s;
    uint32_t *ia = iin + int64_t(t) * n + J.s, *ib = iout + int64_t(t) * n + J.s;
    uint64_t key[kBItems];
    uint32_t id[kBItems];
    bool in_a = true;  // where the bucket's current order is
    for (int p = 0; p < 7; ++p) {
      if (!((J.passes >> p) & 1u)) continue;
      const int shift = 8 * p;
      const uint64_t *sk_src = in_a ? ka : kb;
      const uint32_t *si_src = in_a ? ia : ib;
      uint64_t *sk_dst = in_a ? kb : ka;
      uint32_t *si_dst = in_a ? ib : ia;
      // digit counts of the whole bucket
      S.doff[threadIdx.x] = 0;
      __syncthreads();
      for (int64_t j0 = 0; j0 < sz; j0 += kThreads) {
        const int64_t j = j0 + threadIdx.x;
        const bool act = j < sz;
        const uint32_t dg = act ? digit_of(sk_src[j], shift) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        if (act && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&S.doff[dg], uint32_t(__popc(peers)));
      }
      __syncthreads();
      const uint32_t c = S.doff[threadIdx.x];
      if (__syncthreads_or(int64_t(c) == sz)) continue;  // one digit: the order stays
      uint32_t tot;
      S.doff[threadIdx.x] = block_exclusive_scan(c, S.wsum, tot);
      __syncthreads();
      for (int64_t j0 = 0; j0 < sz; j0 += kBCap) {
        const int cnt = int(sz - j0 < kBCap ? sz - j0 : kBCap);
#pragma unroll
        for (int it = 0; it < kBItems; ++it) {
          const int pos = bpos(warp, it, lane);
          key[it] = pos < cnt ? sk_src[j0 + pos] : ~0ull;
          id[it] = pos < cnt ? si_src[j0 + pos] : 0u;
        }
        if (tile_pass(key, id, cnt, shift, S)) {
          // one digit in this sub-tile: its items keep their order
#pragma unroll
          for (int it = 0; it < kBItems; ++it) {
            const int pos = bpos(warp, it, lane);
            if (pos < cnt) {
              const int64_t gi = int64_t(S.doff[digit_of(key[it], shift)]) + pos;
              sk_dst[gi] = key[it];
              si_dst[gi] = id[it];
            }
          }
        } else {
          for (int i = threadIdx.x; i < cnt; i += kThreads) {
            const uint64_t kk = S.sk[i];
            const uint32_t dg = digit_of(kk, shift);
            const int64_t gi = int64_t(S.doff[dg]) + (i - int64_t(S.dstart[dg]));
            sk_dst[gi] = kk;
            si_dst[gi] = S.si[i];
          }
        }
        __syncthreads();
        S.doff[threadIdx.x] += S.dcnt[threadIdx.x];
        __syncthreads();
      }
      in_a = !in_a;
    }
    if (in_a) {
      for (int64_t j = threadIdx.x; j < sz; j += kThreads) {
        kb[j] = ka[j];
        ib[j] = ia[j];
      }
    }
    __syncthreads();  // the next job re-initialises shared memory
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
  // + the key-spread words (16 L bytes), then the large-bucket list (count and
  // up to 256 L entries of 4 bytes)
  return up(nk * 8) + up(nk * 8) + up(nk * 4) + up(size_t(kRadix) * ntiles * L * 4) +
         up(size_t(L) * 16 + 4 + size_t(kRadix) * L * 4);
}

namespace {
std::atomic<int> g_sort_mode{0};
}  // namespace

int set_sort_mode(int mode) {
  if (mode < 0 || mode > 2) return -1;
  g_sort_mode.store(mode);
  return 0;
}

bool bucket_sort_used(int64_t n) {
  const int mode = g_sort_mode.load();
  // below 2,048 rows most of the 256 buckets of a table are nearly empty and
  // their CTAs cost more than the global passes over so few keys
  return mode == 2 || (mode == 0 && n >= 2048 && n <= kBucketMaxN);
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
  unsigned long long *spread =
      reinterpret_cast<unsigned long long *>(base + 2 * up(nk * 8) + up(nk * 4) + up(hist_len * L * 4));
  const int scatter_smem = kTile * 12 + (kWarps * kRadix + 2 * kRadix + 33) * 4;
  const dim3 grid((unsigned)ntiles, (unsigned)L);
  cudaError_t e = cudaSuccess;
  if (bucket_sort_used(n)) {
    e = cudaFuncSetAttribute(radix_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, scatter_smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(bucket_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, kBucketSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(bucket_sort_large, cudaFuncAttributeMaxDynamicSharedMemorySize, kBucketSmem);
    uint32_t *large = reinterpret_cast<uint32_t *>(spread + 2 * size_t(L));
    int nsm = 0;
    if (e == cudaSuccess) {
      int dev = 0;
      e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    // the spread words and the large-bucket count start at zero
    if (e == cudaSuccess) e = cudaMemsetAsync(spread, 0, sizeof(unsigned long long) * 2 * size_t(L) + 4, stream);
    if (e == cudaSuccess) {
      key_spread<<<grid, kThreads, 0, stream>>>(keys, n, spread);
      radix_hist<true><<<grid, kThreads, 0, stream>>>(keys, n, 0, ntiles, hist, spread);
      scan_rows<<<L, 1024, 0, stream>>>(hist, int64_t(hist_len), nullptr);
      radix_scatter<true><<<grid, kThreads, scatter_smem, stream>>>(keys, nullptr, kA, iA, n, 0, ntiles, hist,
                                                                     spread);
      bucket_sort<<<dim3(kRadix, (unsigned)L), kThreads, kBucketSmem, stream>>>(kA, iA, kB, ids_out, n, ntiles,
                                                                                hist, spread, large);
      bucket_sort_large<<<nsm, kThreads, kBucketSmem, stream>>>(kA, iA, kB, ids_out, n, ntiles, hist, spread,
                                                                large);
      e = cudaGetLastError();
      count_launches(6);
    }
  } else {
    e = cudaFuncSetAttribute(radix_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, scatter_smem);
    const uint64_t *kin = keys;
    const uint32_t *iin = nullptr;
    for (int pass = 0; pass < 8 && e == cudaSuccess; ++pass) {
      uint64_t *kout = (pass % 2 == 0) ? kA : kB;
      uint32_t *iout = (pass % 2 == 0) ? iA : ids_out;
      radix_hist<false><<<grid, kThreads, 0, stream>>>(kin, n, pass * 8, ntiles, hist, nullptr);
      scan_rows<<<L, 1024, 0, stream>>>(hist, int64_t(hist_len), nullptr);
      radix_scatter<false><<<grid, kThreads, scatter_smem, stream>>>(kin, iin, kout, iout, n, pass * 8, ntiles,
                                                                      hist, nullptr);
      e = cudaGetLastError();
      count_launches(3);
      kin = kout;
      iin = iout;
    }
  }
  if (e == cudaSuccess) {
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
