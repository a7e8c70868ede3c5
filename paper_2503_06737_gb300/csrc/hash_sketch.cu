// hash_sketch.cu -- CS / HCS hashing of dense rows for all L tables in one
// persistent launch (Definitions 4, 5, 12, 19, 25, 31).
//
// Design (sm_103a):
//   * A CTA owns a group of Lg tables and walks row tiles of 32*RG rows.  Its
//     tables are staged once in shared memory as per-table member lists: for
//     each bin, the coordinates j < d with s = +1 (ascending j), then those
//     with s = -1, each half padded to a multiple of four with the offset of
//     the row's zero slot, every entry the byte offset 4j (16-bit while
//     4(d+1) < 2^16, else 32-bit).  HCS lists are derived in the CTA from the
//     per-mode tables h_k, s_k (the sign of j is prod_k s_k(i_k)), so HBM
//     holds only O(N d^(1/N)) words per table.
//   * The row tile is read once from HBM with coalesced loads into a padded
//     row-major tile (row stride d+1 words: lane r reading row r hits bank
//     (r + j) mod 32, conflict free; word d is the zero slot).  The next tile
//     is prefetched into L2 while this one is hashed; the CTAs of the G table
//     groups that share a tile run concurrently, so it leaves HBM once.
//   * Lane = row.  A table is split over WPT warps (bins l = k, k+WPT, ...),
//     which gives the SM enough independent shared-memory loads in flight.
//     Entries are read four at a time as warp-uniform broadcasts; each x read
//     is one conflict-free 32-bit load into one of two accumulators per half.
//     Partial keys of the warps of one table are combined in shared memory:
//     the key fold is a sum mod 2^32 (E2LSH, SRP m > 64) or an OR of bits
//     (SRP m <= 64), so partials combine exactly.  The plan (RG, WPT, Lg) is
//     autotuned per shape on the first large batch (see tuned_plan).
//   * Exactness.  The FP32 sum of the k terms of a bin differs from the exact
//     sum by at most gamma_{k-1} * sum|x_j| <= gamma_{k-1} * k * max|x|
//     (Higham's bound, any summation order; zero padding adds no error), and
//     the FP64 reference by at most gamma64_{k-1} * k * max|x| (covered by a
//     2% widening).  For E2LSH, with y = the FP32 sum, t = fl(fl(fma(sqrt(m),
//     y, b)) * fl(1/w)):
//        |t - t_fp64| <= (sqrt(m)/w) E + 4.1u (sqrt(m)|y| + b)/w + 2.1u(|t|+1)
//                     <= A max|x| + 10.2u |t| + 15.3u,
//     using (sqrt(m)|y| + b)/w <= 1.0001 |t| + 2 (b < w), where u = 2^-24 and
//     A = 1.02 (sqrt(m)/w) gamma_{k-1}(1 + 2 gamma) k; the distance of t to the
//     nearest integer is computed exactly.  A bin whose t lies within that
//     bound of an integer (E2LSH), or whose |y| is within A max|x| of 0 (SRP,
//     A without sqrt(m)/w), gets the canonical value of Definitions 12/19/25/31
//     -- the ascending FP64 sum, one IEEE rounding per operation: large
//     batches queue such bins for sketch_recheck_kernel, which patches codes,
//     bits and keys; small batches (and queue overflow) recheck in place.
//     Either way the value is computed exactly as an int64 sum on the least
//     exponent grid of the bin's terms when that sum is exact in the FP64
//     loop, else by the FP64 loop itself.
#include <algorithm>
#include <cstring>
#include <vector>
#include <mutex>
#include <map>

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace lsh {
namespace {

constexpr int kWarp = 32;
constexpr float kU32 = 5.9604644775390625e-08f;  // 2^-24, unit roundoff of FP32
constexpr int kMaxSmem = 232448;                 // 227 KB opt-in per block
constexpr int kLoadBatch = 16;                   // row-tile loads in flight per lane

struct Plan {
  int Lg, G, RG, WPT, W, smem;
  int cap;       // entry capacity per table (multiple of 4)
  int off_ent, off_seg, off_cst, off_key, off_x, off_xmax, off_bad;
  int x_stride;  // d + 1 words
};

struct Args {
  SketchLaunch p;
  Plan pl;
  int ntiles;
  int slots;     // CTAs per table group
  float sqrtm_f, invw_f;
};

template <int DT>
__device__ __forceinline__ float load_x(const void *X, int64_t idx) {
  if (DT == LSH_F32) return __ldg(reinterpret_cast<const float *>(X) + idx);
  const unsigned short h = __ldg(reinterpret_cast<const unsigned short *>(X) + idx);
  if (DT == LSH_BF16) return __uint_as_float(uint32_t(h) << 16);
  return __half2float(__ushort_as_half(h));
}

// Bin and sign of coordinate j in table t (per-mode tables, first mode fastest).
__device__ __forceinline__ void coord_bin(const SketchLaunch &p, int t, int j, int &bin, uint32_t &neg) {
  const uint16_t *hb = p.bins + int64_t(t) * p.dsum;
  const int8_t *sb = p.signs + int64_t(t) * p.dsum;
  if (p.N == 1) {
    bin = hb[j];
    neg = sb[j] < 0 ? 1u : 0u;
    return;
  }
  int r = j, off = 0, stride = 1;
  bin = 0;
  neg = 0;
  for (int k = 0; k < p.N; ++k) {
    const int ik = r % p.dims[k];
    r /= p.dims[k];
    bin += int(hb[off + ik]) * stride;
    neg ^= sb[off + ik] < 0 ? 1u : 0u;
    stride *= p.mdims[k];
    off += p.dims[k];
  }
}

// Stage table t (one warp): member list (sign-split, quad-padded) and the
// per-bin records seg[l] = {start, quads(+) | quads(-) << 16},
// cst[l] = {b_l (f32 bits), A_l, ka_l, kb_l}.
template <typename EntT>
__device__ void stage_table(const SketchLaunch &p, int t, float a_scale, EntT *ent, uint2 *seg,
                            uint4 *cst, uint32_t *scratch, int lane) {
  const int d = p.d, m = p.m;
  uint32_t *cur = scratch;  // [2m]: counts, then write cursors (key = 2 bin + neg)
  for (int i = lane; i < 2 * m; i += kWarp) cur[i] = 0;
  __syncwarp();
  for (int j = lane; j < d; j += kWarp) {
    int bin;
    uint32_t neg;
    coord_bin(p, t, j, bin, neg);
    atomicAdd(&cur[2 * bin + neg], 1u);
  }
  __syncwarp();
  const uint32_t zslot = uint32_t(d) << 2;
  uint32_t carry = 0;
  for (int base = 0; base < m; base += kWarp) {
    const int l = base + lane;
    uint32_t cp = 0, cn = 0, sz = 0;
    if (l < m) {
      cp = cur[2 * l];
      cn = cur[2 * l + 1];
      sz = ((cp + 3) & ~3u) + ((cn + 3) & ~3u);
    }
    uint32_t s = sz;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    const uint32_t start = carry + s - sz;
    if (l < m) {
      const uint32_t qp = (cp + 3) & ~3u, qn = (cn + 3) & ~3u;
      seg[l] = make_uint2(start, (qp >> 2) | ((qn >> 2) << 16));
      for (uint32_t i = cp; i < qp; ++i) ent[start + i] = EntT(zslot);
      for (uint32_t i = cn; i < qn; ++i) ent[start + qp + i] = EntT(zslot);
      cur[2 * l] = start;
      cur[2 * l + 1] = start + qp;
      const float k = float(cp + cn);
      const float g = fmaxf(k - 1.f, 0.f) * kU32;
      const float A = 1.02f * a_scale * g * (1.f + 2.f * g) * k;
      cst[l] = make_uint4(__float_as_uint(p.b32[int64_t(t) * m + l]), __float_as_uint(A),
                          p.ka[int64_t(t) * m + l], p.kb[int64_t(t) * m + l]);
    }
    carry += __shfl_sync(0xffffffffu, s, kWarp - 1);
  }
  __syncwarp();
  const uint32_t lt = (1u << lane) - 1u;
  for (int base = 0; base < d; base += kWarp) {
    const int j = base + lane;
    const bool act = j < d;
    const uint32_t amask = __ballot_sync(0xffffffffu, act);
    if (act) {
      int bin;
      uint32_t neg;
      coord_bin(p, t, j, bin, neg);
      const uint32_t key = 2u * uint32_t(bin) + neg;
      const uint32_t peers = __match_any_sync(amask, key);
      ent[cur[key] + __popc(peers & lt)] = EntT(uint32_t(j) << 2);
      __syncwarp(amask);
      if ((peers & lt) == 0) cur[key] += __popc(peers);
    }
    __syncwarp();
  }
}

// Explicit shared-space loads with 32-bit addresses (row tile and entries).
__device__ __forceinline__ float lds_at(uint32_t saddr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(saddr));
  return v;
}
__device__ __forceinline__ void load_quad_s(uint32_t qaddr, bool u16, uint32_t (&o)[4]) {
  if (u16) {
    uint32_t x, y;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(x), "=r"(y) : "r"(qaddr));
    o[0] = x & 0xFFFFu;
    o[1] = x >> 16;
    o[2] = y & 0xFFFFu;
    o[3] = y >> 16;
  } else {
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3])
                 : "r"(qaddr));
  }
}

__device__ __forceinline__ float lds_f32(const unsigned char *base, uint32_t off) {
  return *reinterpret_cast<const float *>(base + off);
}

// FP64 recheck of one bin for this lane: merge the two ascending halves back
// into ascending j and sum s(j) x_j with one IEEE rounding per addition.
template <typename EntT>
__device__ __noinline__ double bin_fp64(const EntT *P, int np, const EntT *N, int nn,
                                        const unsigned char *xr, uint32_t zslot) {
  int ip = 0, in = 0;
  double y = 0.0;
  while (true) {
    const uint32_t a = ip < np ? P[ip] : zslot;
    const uint32_t b = in < nn ? N[in] : zslot;
    if (a == zslot && b == zslot) break;
    if (a < b) {
      y = __dadd_rn(y, double(lds_f32(xr, a)));
      ++ip;
    } else {
      y = __dadd_rn(y, -double(lds_f32(xr, b)));
      ++in;
    }
  }
  return y;
}

// The same FP64 value without the sequential loop, when the bin's terms
// allow it: an FP32 value is M 2^E with |M| < 2^24 an integer; with the
// bin's least exponent E0 every term is an integer multiple of 2^E0, and if
// the exponents span at most 29 and the magnitudes sum to less than 2^53
// (in units of 2^E0), every partial sum of the ascending FP64 loop is exact,
// so that loop returns the exact sum -- which int64 addition gets in any
// order.  Returns false (the caller runs the loop) when a condition fails.
__device__ __forceinline__ void fp32_parts(uint32_t v, int &E, uint32_t &M) {
  const int e = int((v >> 23) & 0xFF);
  E = max(e, 1) - 150;
  M = (v & 0x7FFFFFu) | (e ? 0x800000u : 0u);
}
template <typename EntT>
__device__ __noinline__ bool bin_exact(const EntT *P, int np, const EntT *N, int nn,
                                       const unsigned char *xr, double &y) {
  int emin = 1 << 20, emax = -(1 << 20);
  for (int h = 0; h < 2; ++h) {
    const EntT *L = h ? N : P;
    const int k = h ? nn : np;
    for (int i = 0; i < k; ++i) {
      const uint32_t v = __float_as_uint(lds_f32(xr, L[i]));
      if (v & 0x7FFFFFFFu) {
        int E;
        uint32_t M;
        fp32_parts(v, E, M);
        emin = min(emin, E);
        emax = max(emax, E);
      }
    }
  }
  if (emax < emin) {
    y = 0.0;
    return true;
  }
  if (emax - emin > 29) return false;
  constexpr unsigned long long kCap = 1ull << 53;
  unsigned long long sum = 0, mag = 0;  // two's complement sum; saturating magnitude
  for (int h = 0; h < 2; ++h) {
    const EntT *L = h ? N : P;
    const int k = h ? nn : np;
    for (int i = 0; i < k; ++i) {
      const uint32_t v = __float_as_uint(lds_f32(xr, L[i]));
      int E;
      uint32_t M;
      fp32_parts(v, E, M);
      const unsigned long long t = (unsigned long long)M << max(E - emin, 0);  // zero stays zero
      sum += ((v >> 31) ^ uint32_t(h)) ? 0ull - t : t;
      mag = min(mag + t, kCap);
    }
  }
  if (mag >= kCap) return false;
  y = ldexp(double((long long)sum), emin);
  return true;
}

// Append this lane's flagged bin to the recheck queue (warp-aggregated);
// false when there is no queue or it is full (the lane then rechecks in place).
__device__ __forceinline__ bool queue_bin(const SketchLaunch &p, bool flag, int64_t row, int t, int l, int code,
                                          int lane) {
  if (!p.queue) return false;
  const uint32_t bal = __ballot_sync(0xffffffffu, flag);
  const int leader = __ffs(bal) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(p.qcount, uint32_t(__popc(bal)));
  base = __shfl_sync(0xffffffffu, base, leader);
  const uint32_t pos = base + __popc(bal & ((1u << lane) - 1u));
  if (!flag || pos >= p.qcap) return false;
  p.queue[pos] = make_int4(int(row), t, l, code);
  return true;
}

template <bool SRP, int DT, typename EntT>
__global__ void __launch_bounds__(1024, 1) sketch_dense_kernel(const Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SketchLaunch &p = a.p;
  const Plan &pl = a.pl;
  const int lane = threadIdx.x & (kWarp - 1);
  const int warp = threadIdx.x >> 5;
  const int g = blockIdx.x % pl.G;
  const int slot = blockIdx.x / pl.G;
  const int t0 = g * pl.Lg;
  const int Lg = min(pl.Lg, p.L - t0);
  if (Lg <= 0 || slot >= a.slots) return;
  const int d = p.d, m = p.m;
  const int cap = pl.cap;
  const int WPT = pl.WPT;

  EntT *ent = reinterpret_cast<EntT *>(smem + pl.off_ent);
  uint2 *seg = reinterpret_cast<uint2 *>(smem + pl.off_seg);
  uint4 *cst = reinterpret_cast<uint4 *>(smem + pl.off_cst);
  uint2 *kacc = reinterpret_cast<uint2 *>(smem + pl.off_key);  // [R][Lg] partial keys
  float *xs = reinterpret_cast<float *>(smem + pl.off_x);
  float *xmax = reinterpret_cast<float *>(smem + pl.off_xmax);
  int *bad = reinterpret_cast<int *>(smem + pl.off_bad);

  const float sq_w = a.sqrtm_f * a.invw_f;
  {
    uint32_t *scratch = reinterpret_cast<uint32_t *>(xs) + warp * 2 * m;  // aliases the tile
    for (int tl = warp; tl < Lg; tl += pl.W)
      stage_table(p, t0 + tl, SRP ? 1.f : sq_w, ent + tl * cap, seg + tl * m, cst + tl * m, scratch, lane);
  }
  __syncthreads();

  const int R = pl.RG * kWarp;
  const int xst = pl.x_stride;
  const int ntasks = pl.RG * Lg * WPT;
  const uint32_t zslot = uint32_t(d) << 2;
  constexpr int es = DT == LSH_F32 ? 4 : 2;

  for (int tile = slot; tile < a.ntiles; tile += a.slots) {
    const int64_t row0 = int64_t(tile) * R;
    // ---- load the row tile (warp per row, coalesced, kLoadBatch loads in flight) ----
    for (int r = warp; r < R; r += pl.W) {
      const int64_t row = row0 + r;
      float *dst = xs + r * xst;
      float mx = 0.f;
      bool fin = true;
      if (row < p.n) {
        const int64_t base = row * p.ld;
        for (int j0 = lane; j0 < d; j0 += kLoadBatch * kWarp) {
          float v[kLoadBatch];
#pragma unroll
          for (int u = 0; u < kLoadBatch; ++u) {
            const int j = j0 + u * kWarp;
            v[u] = j < d ? load_x<DT>(p.X, base + j) : 0.f;
          }
#pragma unroll
          for (int u = 0; u < kLoadBatch; ++u) {
            const int j = j0 + u * kWarp;
            if (j < d) dst[j] = v[u];
            mx = fmaxf(mx, fabsf(v[u]));
            fin = fin && isfinite(v[u]);
          }
        }
      } else {
        for (int j = lane; j < d; j += kWarp) dst[j] = 0.f;
      }
      if (lane == 0) dst[d] = 0.f;  // the zero slot the padding entries point at
      for (int tl = lane; tl < Lg; tl += kWarp) kacc[r * Lg + tl] = make_uint2(0u, 0u);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const bool allfin = __all_sync(0xffffffffu, fin);
      if (lane == 0) {
        xmax[r] = mx;
        bad[r] = allfin ? 0 : 1;
      }
    }
    __syncthreads();
    // ---- prefetch the next tile into L2 while this one is hashed ----
    if (warp == pl.W - 1) {
      const int64_t nrow0 = int64_t(tile + a.slots) * R;
      const char *X = reinterpret_cast<const char *>(p.X);
      for (int r = 0; r < R; ++r) {
        const int64_t row = nrow0 + r;
        if (row >= p.n) break;
        const char *rp = X + row * p.ld * es;
        for (int off = lane * 128; off < d * es; off += kWarp * 128)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(rp + off));
      }
    }

    // ---- one task = (row group, table, bin subset): lane = row ----
    for (int task = warp; task < ntasks; task += pl.W) {
      const int sub = task % WPT;
      const int rt = task / WPT;
      const int rg = rt / Lg;
      const int tl = rt - rg * Lg;
      const int t = t0 + tl;
      const int r = rg * kWarp + lane;
      const int64_t row = row0 + r;
      const bool valid = row < p.n;
      const bool isbad = bad[r] != 0;
      const float xm = xmax[r];
      const unsigned char *xr = reinterpret_cast<const unsigned char *>(xs + r * xst);
      const EntT *E = ent + tl * cap;
      const uint2 *S = seg + tl * m;
      const uint4 *C = cst + tl * m;
      uint32_t ha = 0, hb = 0;
      uint64_t word = 0;
      int nflag = 0, nchanged = 0, novf = 0;
      for (int l = sub; l < m; l += WPT) {
        const uint2 sg = S[l];
        const int qp = int(sg.y & 0xffffu), qn = int(sg.y >> 16);
        const EntT *Q = E + sg.x;
        // two quads per iteration (eight loads in flight), then the odd quad;
        // two accumulators per half (the FP32 error bound holds in any order)
        constexpr bool kU16 = sizeof(EntT) == 2;
        constexpr uint32_t kQuadBytes = 4 * sizeof(EntT);
        const uint32_t xs_a = static_cast<uint32_t>(__cvta_generic_to_shared(xr));
        uint32_t qa = static_cast<uint32_t>(__cvta_generic_to_shared(Q));
        float p0 = 0.f, p1 = 0.f;
        int q = 0;
#pragma unroll 1
        for (; q + 2 <= qp; q += 2, qa += 2 * kQuadBytes) {
          uint32_t e[4], f[4];
          load_quad_s(qa, kU16, e);
          load_quad_s(qa + kQuadBytes, kU16, f);
          p0 += lds_at(xs_a + e[0]);
          p1 += lds_at(xs_a + e[1]);
          p0 += lds_at(xs_a + e[2]);
          p1 += lds_at(xs_a + e[3]);
          p0 += lds_at(xs_a + f[0]);
          p1 += lds_at(xs_a + f[1]);
          p0 += lds_at(xs_a + f[2]);
          p1 += lds_at(xs_a + f[3]);
        }
        if (q < qp) {
          uint32_t e[4];
          load_quad_s(qa, kU16, e);
          qa += kQuadBytes;
          p0 += lds_at(xs_a + e[0]);
          p1 += lds_at(xs_a + e[1]);
          p0 += lds_at(xs_a + e[2]);
          p1 += lds_at(xs_a + e[3]);
        }
        float n0 = 0.f, n1 = 0.f;
        q = 0;
#pragma unroll 1
        for (; q + 2 <= qn; q += 2, qa += 2 * kQuadBytes) {
          uint32_t e[4], f[4];
          load_quad_s(qa, kU16, e);
          load_quad_s(qa + kQuadBytes, kU16, f);
          n0 += lds_at(xs_a + e[0]);
          n1 += lds_at(xs_a + e[1]);
          n0 += lds_at(xs_a + e[2]);
          n1 += lds_at(xs_a + e[3]);
          n0 += lds_at(xs_a + f[0]);
          n1 += lds_at(xs_a + f[1]);
          n0 += lds_at(xs_a + f[2]);
          n1 += lds_at(xs_a + f[3]);
        }
        if (q < qn) {
          uint32_t e[4];
          load_quad_s(qa, kU16, e);
          n0 += lds_at(xs_a + e[0]);
          n1 += lds_at(xs_a + e[1]);
          n0 += lds_at(xs_a + e[2]);
          n1 += lds_at(xs_a + e[3]);
        }
        const float y = (p0 + p1) - (n0 + n1);
        const uint4 c = C[l];
        const float A = __uint_as_float(c.y);
        if (SRP) {
          // A = 0 when the bin holds at most one term: the FP32 value is then exact
          const bool flag = valid && !isbad && A > 0.f && !(fabsf(y) > A * xm);
          int bit = y > 0.f ? 1 : 0;
          if (__any_sync(0xffffffffu, flag)) {
            if (!queue_bin(p, flag, row, t, l, bit, lane) && flag) {
              const EntT *P = E + sg.x;
              double y64;
              if (!bin_exact(P, 4 * qp, P + 4 * qp, 4 * qn, xr, y64))
                y64 = bin_fp64(P, 4 * qp, P + 4 * qp, 4 * qn, xr, zslot);
              const int b64 = y64 > 0.0 ? 1 : 0;
              ++nflag;
              nchanged += b64 != bit;
              bit = b64;
            }
          }
          if (p.proj && valid) p.proj[(row * p.L + t) * m + l] = y;
          if (m <= 64) {
            word |= uint64_t(bit) << l;
          } else if (bit) {
            ha += c.z;
            hb += c.w;
            if (p.bits && valid)
              atomicOr(reinterpret_cast<unsigned long long *>(p.bits) + (row * p.L + t) * ((m + 63) >> 6) + (l >> 6),
                       1ull << (l & 63));
          }
        } else {
          const float bl = __uint_as_float(c.x);
          const float tf = __fmul_rn(__fmaf_rn(a.sqrtm_f, y, bl), a.invw_f);
          const float dist = fabsf(tf - rintf(tf));  // exact (Sterbenz)
          const float M = fmaf(A, xm, fmaf(10.2f * kU32, fabsf(tf), 15.3f * kU32));
          const bool flag = valid && !isbad && !(dist > M && fabsf(tf) < 4194304.f);
          int code = __float2int_rd(tf);
          if (__any_sync(0xffffffffu, flag)) {
            if (!queue_bin(p, flag, row, t, l, code, lane) && flag) {
              const EntT *P = E + sg.x;
              double y64;
              if (!bin_exact(P, 4 * qp, P + 4 * qp, 4 * qn, xr, y64))
                y64 = bin_fp64(P, 4 * qp, P + 4 * qp, 4 * qn, xr, zslot);
              const double t1 = __dmul_rn(p.sqrtm, y64);
              const double t2 = __dadd_rn(t1, p.b64[int64_t(t) * m + l]);
              const double t3 = __ddiv_rn(t2, p.w);
              const double f = floor(t3);
              int c64;
              if (f >= -2147483648.0 && f <= 2147483647.0) {
                c64 = int(f);
              } else {
                c64 = INT32_MIN;
                ++novf;
              }
              ++nflag;
              nchanged += c64 != code;
              code = c64;
            }
          }
          if (isbad) code = INT32_MIN;
          ha += uint32_t(code) * c.z;
          hb += uint32_t(code) * c.w;
          if (valid) {
            if (p.codes) p.codes[(row * p.L + t) * m + l] = code;
            if (p.proj) p.proj[(row * p.L + t) * m + l] = y;
          }
        }
      }
      // partial key of this warp -> the (row, table) slot
      if (SRP && m <= 64) {
        if (word) {
          atomicOr(&kacc[r * Lg + tl].x, uint32_t(word));
          atomicOr(&kacc[r * Lg + tl].y, uint32_t(word >> 32));
        }
      } else {
        atomicAdd(&kacc[r * Lg + tl].x, ha);
        atomicAdd(&kacc[r * Lg + tl].y, hb);
      }
      if (p.counters) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          nflag += __shfl_xor_sync(0xffffffffu, nflag, o);
          nchanged += __shfl_xor_sync(0xffffffffu, nchanged, o);
          novf += __shfl_xor_sync(0xffffffffu, novf, o);
        }
        if (lane == 0) {
          if (nflag) atomicAdd(p.counters + CNT_FLAGGED, (unsigned long long)nflag);
          if (nchanged) atomicAdd(p.counters + CNT_CHANGED, (unsigned long long)nchanged);
          if (novf) atomicAdd(p.counters + CNT_OVERFLOW, (unsigned long long)novf);
        }
      } else if (__any_sync(0xffffffffu, novf != 0) && lane == 0) {
        atomicOr(p.status, STATUS_OVERFLOW);
      }
    }
    __syncthreads();
    // ---- keys of the tile: consecutive threads write consecutive rows of a table ----
    for (int i = threadIdx.x; i < Lg * R; i += blockDim.x) {
      const int tl = i / R, r = i - tl * R;
      const int64_t row = row0 + r;
      if (row >= p.n) continue;
      const uint2 k2 = kacc[r * Lg + tl];
      uint64_t key;
      if (SRP && m <= 64) {
        key = (uint64_t(k2.y) << 32) | k2.x;
        if (p.bits) p.bits[row * p.L + t0 + tl] = key;
      } else {
        key = (uint64_t(k2.x) << 32) | k2.y;
      }
      if (bad[r]) {
        key = ~0ull;
        if (tl == 0) {
          if (p.counters) atomicAdd(p.counters + CNT_NONFINITE, 1ull);
          atomicOr(p.status, STATUS_NONFINITE);
        }
      }
      if (p.keys) p.keys[int64_t(t0 + tl) * p.key_ld + row] = key;
    }
    __syncthreads();
  }
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

int align16(int v) { return (v + 15) & ~15; }

// Entry width: 16-bit byte offsets while 4 (d + 1) fits, else 32-bit.
int entry_bytes(int d) { return 4 * (d + 1) < 65536 ? 2 : 4; }

// The shared-memory layout of one plan: RG row groups of 32 rows, WPT warps
// per table, table groups of (balanced) size <= Lg.  smem > kMaxSmem when it
// does not fit.
Plan plan_of(int d, int m, int L, int cap, int RG, int WPT, int Lg) {
  const int G = (L + Lg - 1) / Lg;
  const int Lgb = (L + G - 1) / G;  // balanced group size
  Plan pl{};
  pl.Lg = Lgb;
  pl.G = G;
  pl.RG = RG;
  pl.WPT = WPT;
  const int tasks = RG * Lgb * WPT;
  int W = tasks < 32 ? tasks : 32;
  if (tasks > 32) {
    for (int w = 32; w >= 16; --w)
      if (tasks % w == 0) {
        W = w;
        break;
      }
  }
  if (W < 4) W = 4;
  pl.W = W;
  pl.x_stride = d + 1;
  pl.cap = cap;
  const int R = RG * kWarp;
  int off = 0;
  pl.off_ent = off;
  off = align16(off + Lgb * cap * entry_bytes(d));
  pl.off_seg = off;
  off = align16(off + Lgb * m * 8);
  pl.off_cst = off;
  off = align16(off + Lgb * m * 16);
  pl.off_key = off;
  off = align16(off + R * Lgb * 8);
  pl.off_x = off;
  const int xbytes = R * (d + 1) * 4;
  const int scratch = W * 2 * m * 4;
  off = align16(off + (xbytes > scratch ? xbytes : scratch));
  pl.off_xmax = off;
  off = align16(off + R * 4);
  pl.off_bad = off;
  off = align16(off + R * 4);
  pl.smem = off;
  return pl;
}

// The default plan: most rows per tile, then two warps per table, then the
// largest table group that fits.
Plan make_plan(int d, int m, int L, int cap, int64_t n) {
  Plan best{};
  best.smem = -1;
  const int sms = num_sms();
  for (int RG = 4; RG >= 1; RG >>= 1) {
    const int64_t ntiles = (n + RG * kWarp - 1) / (RG * kWarp);
    if (RG > 1 && ntiles < 2 * sms) continue;  // keep every SM busy twice over
    for (int WPT = 2; WPT >= 1; --WPT)
      for (int Lg = (L < 32 ? L : 32); Lg >= 1; --Lg) {
        const Plan pl = plan_of(d, m, L, cap, RG, WPT, Lg);
        if (pl.smem <= kMaxSmem) return pl;
      }
  }
  return best;
}

// Candidate plans for the autotuner: for each row-group count and warps per
// table, the largest fitting table group and the next smaller group count.
std::vector<Plan> plan_candidates(int d, int m, int L, int cap, int64_t n) {
  std::vector<Plan> out;
  const int sms = num_sms();
  for (int RG = 4; RG >= 1; RG >>= 1) {
    const int64_t ntiles = (n + RG * kWarp - 1) / (RG * kWarp);
    if (RG > 1 && ntiles < 2 * sms) continue;
    for (int WPT = 4; WPT >= 1; WPT >>= 1) {
      if (WPT > m) continue;
      int found = 0, lastG = -1;
      for (int Lg = (L < 32 ? L : 32); Lg >= 1 && found < 2; --Lg) {
        const Plan pl = plan_of(d, m, L, cap, RG, WPT, Lg);
        if (pl.smem > kMaxSmem || pl.G == lastG) continue;
        if (pl.RG * pl.Lg * pl.WPT > 1024 / kWarp * 4) continue;
        lastG = pl.G;
        out.push_back(pl);
        ++found;
      }
    }
  }
  return out;
}

template <bool SRP, int DT, typename EntT>
cudaError_t launch_e(const Args &a, cudaStream_t stream) {
  const dim3 grid((unsigned)(a.slots * a.pl.G)), block((unsigned)(a.pl.W * kWarp));
  cudaError_t e = cudaFuncSetAttribute(sketch_dense_kernel<SRP, DT, EntT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, a.pl.smem);
  if (e != cudaSuccess) return e;
  sketch_dense_kernel<SRP, DT, EntT><<<grid, block, a.pl.smem, stream>>>(a);
  return cudaGetLastError();
}

template <bool SRP, int DT>
cudaError_t launch_t(const Args &a, cudaStream_t stream) {
  return entry_bytes(a.p.d) == 2 ? launch_e<SRP, DT, uint16_t>(a, stream) : launch_e<SRP, DT, uint32_t>(a, stream);
}

}  // namespace

SketchPlan plan_sketch_dense(int d, int m, int L, int cap, int dtype) {
  (void)dtype;
  Plan pl = make_plan(d, m, L, cap, int64_t(1) << 40);
  SketchPlan sp{};
  sp.ok = pl.smem > 0;
  if (!sp.ok) return sp;
  sp.tables_per_cta = pl.Lg;
  sp.groups = pl.G;
  sp.row_groups = pl.RG;
  sp.warps = pl.W;
  sp.smem = pl.smem;
  sp.ctas = num_sms();
  return sp;
}

int64_t sketch_queue_cap(int64_t n, int32_t L, int32_t m) {
  // about 16x the flag rate seen on Gaussian-mixture rows; the excess is rechecked in place
  return std::min<int64_t>(n * L * m / 256 + 65536, int64_t(1) << 28);
}

namespace {

template <int DT>
__device__ __forceinline__ uint32_t x_bits(const void *X, int64_t idx) {
  return __float_as_uint(load_x<DT>(X, idx));
}

// One queued bin per thread: the exact FP64 value of the bin (int64 sum on
// the least exponent grid of its terms, else the ascending FP64 loop over the
// merged member lists -- the oracle's order), the oracle's code, and the
// patch of code, bits and key where the fast code was wrong.  E2LSH and
// multi-word SRP keys are sums mod 2^32 in both halves; one-word SRP keys are
// the bits themselves.
template <bool SRP, int DT>
__global__ void __launch_bounds__(256) sketch_recheck_kernel(const SketchLaunch p, const uint16_t *mlist,
                                                             const uint32_t *mseg) {
  const int64_t cnt = min(int64_t(*p.qcount), int64_t(p.qcap));
  int nflag = 0, nchanged = 0, novf = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < cnt; i += int64_t(gridDim.x) * blockDim.x) {
    const int4 r = p.queue[i];
    const int64_t row = r.x;
    const int t = r.y, l = r.z;
    const int64_t tl = int64_t(t) * p.m + l;
    const uint32_t start = mseg[2 * tl], np = mseg[2 * tl + 1] & 0xFFFFu, nn = mseg[2 * tl + 1] >> 16;
    const uint16_t *P = mlist + int64_t(t) * p.d + start;
    const uint16_t *N = P + np;
    const int64_t xb = row * p.ld;
    // exact path
    int emin = 1 << 20, emax = -(1 << 20);
    for (uint32_t k = 0; k < np + nn; ++k) {
      const uint32_t v = x_bits<DT>(p.X, xb + P[k]);
      if (v & 0x7FFFFFFFu) {
        const int e = int((v >> 23) & 0xFF);
        const int E = max(e, 1) - 150;
        emin = min(emin, E);
        emax = max(emax, E);
      }
    }
    double y64 = 0.0;
    bool exact = true;
    if (emax >= emin) {
      exact = emax - emin <= 29;
      if (exact) {
        constexpr unsigned long long kCap = 1ull << 53;
        unsigned long long sum = 0, mag = 0;
        for (uint32_t k = 0; k < np + nn; ++k) {
          const uint32_t v = x_bits<DT>(p.X, xb + P[k]);
          const int e = int((v >> 23) & 0xFF);
          const uint32_t M = (v & 0x7FFFFFu) | (e ? 0x800000u : 0u);
          const unsigned long long tv = (unsigned long long)M << max(max(e, 1) - 150 - emin, 0);
          sum += ((v >> 31) ^ (k >= np ? 1u : 0u)) ? 0ull - tv : tv;
          mag = min(mag + tv, kCap);
        }
        exact = mag < kCap;
        if (exact) y64 = ldexp(double((long long)sum), emin);
      }
    }
    if (!exact) {
      // the sequential loop in ascending j over the merged halves
      uint32_t ip = 0, in = 0;
      y64 = 0.0;
      while (ip < np || in < nn) {
        const uint32_t jp = ip < np ? P[ip] : 0xFFFFFFFFu, jn = in < nn ? N[in] : 0xFFFFFFFFu;
        if (jp < jn) {
          y64 = __dadd_rn(y64, double(__uint_as_float(x_bits<DT>(p.X, xb + jp))));
          ++ip;
        } else {
          y64 = __dadd_rn(y64, -double(__uint_as_float(x_bits<DT>(p.X, xb + jn))));
          ++in;
        }
      }
    }
    int c64;
    if (SRP) {
      c64 = y64 > 0.0 ? 1 : 0;
    } else {
      const double f = floor(__ddiv_rn(__dadd_rn(__dmul_rn(p.sqrtm, y64), p.b64[tl]), p.w));
      if (f >= -2147483648.0 && f <= 2147483647.0) {
        c64 = int(f);
      } else {
        c64 = INT32_MIN;
        ++novf;
      }
    }
    ++nflag;
    if (c64 == r.w) continue;
    ++nchanged;
    uint64_t *key = p.keys ? p.keys + int64_t(t) * p.key_ld + row : nullptr;
    if (SRP) {
      const int words = (p.m + 63) >> 6;
      if (p.bits)
        atomicXor(reinterpret_cast<unsigned long long *>(p.bits + (row * p.L + t) * words + (l >> 6)), 1ull << (l & 63));
      if (key) {
        if (p.m <= 64) {
          atomicXor(reinterpret_cast<unsigned long long *>(key), 1ull << l);
        } else {
          const uint32_t sgn = c64 ? 1u : 0xFFFFFFFFu;  // +1 or -1 mod 2^32
          atomicAdd(reinterpret_cast<unsigned int *>(key) + 1, sgn * p.ka[tl]);
          atomicAdd(reinterpret_cast<unsigned int *>(key), sgn * p.kb[tl]);
        }
      }
    } else {
      if (p.codes) p.codes[(row * p.L + t) * p.m + l] = c64;
      const uint32_t dc = uint32_t(c64) - uint32_t(r.w);
      if (key) {
        atomicAdd(reinterpret_cast<unsigned int *>(key) + 1, dc * p.ka[tl]);
        atomicAdd(reinterpret_cast<unsigned int *>(key), dc * p.kb[tl]);
      }
    }
  }
  if (p.counters) {
    if (nflag) atomicAdd(p.counters + CNT_FLAGGED, (unsigned long long)nflag);
    if (nchanged) atomicAdd(p.counters + CNT_CHANGED, (unsigned long long)nchanged);
    if (novf) atomicAdd(p.counters + CNT_OVERFLOW, (unsigned long long)novf);
  }
  if (novf) atomicOr(p.status, STATUS_OVERFLOW);
}

template <bool SRP, int DT>
cudaError_t launch_recheck_t(const SketchLaunch &p, const uint16_t *mlist, const uint32_t *mseg,
                             cudaStream_t stream) {
  sketch_recheck_kernel<SRP, DT><<<unsigned(num_sms()) * 8, 256, 0, stream>>>(p, mlist, mseg);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sketch_recheck(const SketchLaunch &p, const uint16_t *mlist, const uint32_t *mseg,
                                  cudaStream_t stream) {
  if (p.n <= 0 || !p.queue) return cudaSuccess;
  const bool srp = kind_is_srp(p.kind);
  switch (p.dtype) {
    case LSH_F32: return srp ? launch_recheck_t<true, LSH_F32>(p, mlist, mseg, stream)
                             : launch_recheck_t<false, LSH_F32>(p, mlist, mseg, stream);
    case LSH_BF16: return srp ? launch_recheck_t<true, LSH_BF16>(p, mlist, mseg, stream)
                              : launch_recheck_t<false, LSH_BF16>(p, mlist, mseg, stream);
    case LSH_F16: return srp ? launch_recheck_t<true, LSH_F16>(p, mlist, mseg, stream)
                             : launch_recheck_t<false, LSH_F16>(p, mlist, mseg, stream);
    default: return cudaErrorInvalidValue;
  }
}

namespace {

cudaError_t launch_plan(const SketchLaunch &p, const Plan &pl, cudaStream_t stream) {
  Args a{};
  a.p = p;
  a.pl = pl;
  const int R = pl.RG * kWarp;
  const int64_t ntiles = (p.n + R - 1) / R;
  if (ntiles > INT32_MAX) return cudaErrorInvalidValue;
  a.ntiles = int(ntiles);
  const int64_t cap = int64_t(num_sms()) / pl.G;
  int64_t slots = cap < ntiles ? cap : ntiles;
  if (slots < 1) slots = 1;
  a.slots = int(slots);
  a.sqrtm_f = float(p.sqrtm);
  a.invw_f = float(1.0 / p.w);
  const bool srp = kind_is_srp(p.kind);
  switch (p.dtype) {
    case LSH_F32: return srp ? launch_t<true, LSH_F32>(a, stream) : launch_t<false, LSH_F32>(a, stream);
    case LSH_BF16: return srp ? launch_t<true, LSH_BF16>(a, stream) : launch_t<false, LSH_BF16>(a, stream);
    case LSH_F16: return srp ? launch_t<true, LSH_F16>(a, stream) : launch_t<false, LSH_F16>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

// Autotuner: the first batch of at least kTuneRows rows of a shape (device,
// kind, d, m, L, modes, dtype) times every candidate plan on its first
// kTuneRows rows -- keys only, no recheck queue, into the caller's key buffer,
// which the real launch then overwrites -- and keeps the fastest.  It is
// skipped while the stream is being captured (the default plan is used).
constexpr int64_t kTuneRows = 131072;

struct TuneKey {
  int dev, kind, d, m, L, N, dtype, cap;
  int dims[LSH_MAX_MODES], mdims[LSH_MAX_MODES];
  bool operator<(const TuneKey &o) const { return std::memcmp(this, &o, sizeof(TuneKey)) < 0; }
};
std::mutex g_tune_mu;
std::map<TuneKey, Plan> g_tuned;

Plan tuned_plan(const SketchLaunch &p, cudaStream_t stream) {
  const Plan dflt = make_plan(p.d, p.m, p.L, p.cap, p.n);
  if (p.n < kTuneRows || dflt.smem <= 0) return dflt;
  TuneKey key;
  std::memset(&key, 0, sizeof(key));
  cudaGetDevice(&key.dev);
  key.kind = p.kind;
  key.d = p.d;
  key.m = p.m;
  key.L = p.L;
  key.N = p.N;
  key.dtype = p.dtype;
  key.cap = p.cap;
  for (int k = 0; k < p.N && k < LSH_MAX_MODES; ++k) {
    key.dims[k] = p.dims[k];
    key.mdims[k] = p.mdims[k];
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return dflt;
  SketchLaunch q = p;
  q.n = kTuneRows;
  q.codes = nullptr;
  q.bits = nullptr;
  q.proj = nullptr;
  q.counters = nullptr;
  q.queue = nullptr;
  q.qcount = nullptr;
  q.qcap = 0;
  const std::vector<Plan> cands = plan_candidates(p.d, p.m, p.L, p.cap, kTuneRows);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return dflt;
  }
  Plan best = dflt;
  float best_ms = 1e30f;
  for (const Plan &pl : cands) {
    if (launch_plan(q, pl, stream) != cudaSuccess) continue;  // warm-up (and attribute setting)
    cudaEventRecord(e0, stream);
    bool ok = launch_plan(q, pl, stream) == cudaSuccess;
    cudaEventRecord(e1, stream);
    float ms = 0.f;
    if (!ok || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
    if (ms < best_ms) {
      best_ms = ms;
      best = pl;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();  // a candidate that failed to launch leaves no sticky error
  // tuned on kTuneRows rows: keep the row-group choice valid for the real n
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[key] = best;
  return best;
}

}  // namespace

cudaError_t launch_sketch_dense(const SketchLaunch &p, cudaStream_t stream) {
  if (p.n <= 0) return cudaSuccess;
  const Plan pl = tuned_plan(p, stream);
  if (pl.smem <= 0 || pl.smem > kMaxSmem) return cudaErrorInvalidConfiguration;
  return launch_plan(p, pl, stream);
}


}  // namespace lsh
