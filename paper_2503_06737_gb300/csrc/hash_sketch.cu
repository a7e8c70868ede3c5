// hash_sketch.cu -- CS / HCS hashing of dense rows for all L tables in one
// persistent launch (Definitions 4, 5, 12, 19, 25, 31).
//
// Design (sm_103a):
//   * A CTA owns a group of Lg tables and walks row tiles of 32*RG rows.  Its
//     tables are staged once in shared memory as per-table member lists: the
//     coordinates j < d sorted by (bin, j), each entry the byte offset 4j with
//     the sign of s(j) (count sketch) or of prod_k s_k(i_k) (HCS) in bit 31,
//     plus the bin start offsets.  The HCS lists are derived in the CTA from
//     the per-mode tables h_k, s_k (O(N d^(1/N)) words per table in HBM).
//   * The row tile is read once from HBM with coalesced loads into a padded
//     row-major tile (row stride d+1 words, so lane r reading row r hits bank
//     (r + j) mod 32: conflict free).  The CTAs of the G table groups that
//     share a tile run concurrently, so the tile is fetched from HBM once and
//     from L2 for the other groups.
//   * Lane = row, warp = (row group, table).  Every member-list read is a
//     warp-uniform broadcast; every x read is one conflict-free LDS.32; the
//     bin sum lives in one register and is discretised, margin-checked and
//     folded into the key as soon as the bin ends.  No atomics, no partial
//     bins in memory.
//   * Exactness: the FP32 sum of the k terms of a bin is within
//     E = gamma_{k-1} k max|x| of the exact sum (Higham's bound for any
//     summation order); the FP64 oracle is within gamma64_{k-1} k max|x| of
//     it.  The discretisation adds a few rounding errors, bounded relative to
//     |t|.  An entry whose FP32 value lies within that total bound of an
//     integer (E2LSH) or of 0 (SRP) is recomputed by its lane in FP64 from
//     the same staged tile, in ascending j, with one IEEE rounding per
//     operation -- the canonical value of Definitions 12/19/25/31.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace lsh {
namespace {

constexpr int kWarp = 32;
constexpr float kU32 = 5.9604644775390625e-08f;  // 2^-24, unit roundoff of FP32
constexpr int kMaxSmem = 232448;                 // 227 KB opt-in per block

struct Plan {
  int Lg, G, RG, W, smem;
  int off_ent, off_boff, off_b, off_x, off_xmax, off_bad;
  int x_stride;  // d + 1 words
};

struct Args {
  SketchLaunch p;
  Plan pl;
  int ntiles;
  int slots;     // CTAs per table group
  float sqrtm_f, invw_f;
};

__device__ __forceinline__ float load_x(const void *X, int dtype, int64_t idx) {
  if (dtype == LSH_F32) return __ldg(reinterpret_cast<const float *>(X) + idx);
  const unsigned short h = __ldg(reinterpret_cast<const unsigned short *>(X) + idx);
  if (dtype == LSH_BF16) return __uint_as_float(uint32_t(h) << 16);
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

// Build the member list of table t into ent[0..d) and boff[0..m] (one warp).
__device__ void build_members(const SketchLaunch &p, int t, uint32_t *ent, uint16_t *boff,
                              uint32_t *cnt, int lane) {
  const int d = p.d, m = p.m;
  for (int l = lane; l < m; l += kWarp) cnt[l] = 0;
  __syncwarp();
  for (int j = lane; j < d; j += kWarp) {
    int bin;
    uint32_t neg;
    coord_bin(p, t, j, bin, neg);
    atomicAdd(&cnt[bin], 1u);
  }
  __syncwarp();
  // exclusive scan of cnt -> boff, cnt becomes the write cursor
  uint32_t carry = 0;
  for (int base = 0; base < m; base += kWarp) {
    const int l = base + lane;
    const uint32_t v = l < m ? cnt[l] : 0u;
    uint32_t s = v;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    const uint32_t excl = carry + s - v;
    if (l < m) {
      boff[l] = uint16_t(excl);
      cnt[l] = excl;
    }
    carry += __shfl_sync(0xffffffffu, s, kWarp - 1);
  }
  if (lane == 0) boff[m] = uint16_t(d);
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
      const uint32_t peers = __match_any_sync(amask, bin);
      const uint32_t pos = cnt[bin] + __popc(peers & lt);
      ent[pos] = (uint32_t(j) << 2) | (neg << 31);
      __syncwarp(amask);
      if ((peers & lt) == 0) cnt[bin] += __popc(peers);
    }
    __syncwarp();
  }
}

template <bool SRP>
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

  uint32_t *ent = reinterpret_cast<uint32_t *>(smem + pl.off_ent);
  uint16_t *boff = reinterpret_cast<uint16_t *>(smem + pl.off_boff);
  float *bf = reinterpret_cast<float *>(smem + pl.off_b);
  float *xs = reinterpret_cast<float *>(smem + pl.off_x);
  float *xmax = reinterpret_cast<float *>(smem + pl.off_xmax);
  int *bad = reinterpret_cast<int *>(smem + pl.off_bad);

  // ---- stage this group's tables (once per CTA) ----
  {
    uint32_t *cnt = reinterpret_cast<uint32_t *>(xs) + warp * m;  // scratch aliases the tile
    for (int tl = warp; tl < Lg; tl += pl.W)
      build_members(p, t0 + tl, ent + tl * d, boff + tl * (m + 1), cnt, lane);
    for (int i = threadIdx.x; i < Lg * m; i += blockDim.x) bf[i] = p.b32[int64_t(t0) * m + i];
  }
  __syncthreads();

  const int R = pl.RG * kWarp;
  const int xst = pl.x_stride;
  const int ntasks = pl.RG * Lg;
  const float sq_w = a.sqrtm_f * a.invw_f;

  for (int tile = slot; tile < a.ntiles; tile += a.slots) {
    const int64_t row0 = int64_t(tile) * R;
    // ---- load the row tile (warp per row, coalesced) + max|x| and finiteness ----
    for (int r = warp; r < R; r += pl.W) {
      const int64_t row = row0 + r;
      float *dst = xs + r * xst;
      float mx = 0.f;
      bool fin = true;
      if (row < p.n) {
        const int64_t base = row * p.ld;
        int j = lane;
        for (; j + 3 * kWarp < d; j += 4 * kWarp) {
          const float v0 = load_x(p.X, p.dtype, base + j);
          const float v1 = load_x(p.X, p.dtype, base + j + kWarp);
          const float v2 = load_x(p.X, p.dtype, base + j + 2 * kWarp);
          const float v3 = load_x(p.X, p.dtype, base + j + 3 * kWarp);
          dst[j] = v0;
          dst[j + kWarp] = v1;
          dst[j + 2 * kWarp] = v2;
          dst[j + 3 * kWarp] = v3;
          mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v0), fabsf(v1)), fmaxf(fabsf(v2), fabsf(v3))));
          fin = fin && isfinite(v0) && isfinite(v1) && isfinite(v2) && isfinite(v3);
        }
        for (; j < d; j += kWarp) {
          const float v = load_x(p.X, p.dtype, base + j);
          dst[j] = v;
          mx = fmaxf(mx, fabsf(v));
          fin = fin && isfinite(v);
        }
      } else {
        for (int j = lane; j < d; j += kWarp) dst[j] = 0.f;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const bool allfin = __all_sync(0xffffffffu, fin);
      if (lane == 0) {
        xmax[r] = mx;
        bad[r] = allfin ? 0 : 1;
      }
    }
    __syncthreads();

    // ---- one task = (row group, table): lane = row ----
    for (int task = warp; task < ntasks; task += pl.W) {
      const int rg = task / Lg;
      const int tl = task - rg * Lg;
      const int t = t0 + tl;
      const int r = rg * kWarp + lane;
      const int64_t row = row0 + r;
      const bool valid = row < p.n;
      const bool isbad = bad[r] != 0;
      const float xm = xmax[r];
      const unsigned char *xrow = reinterpret_cast<const unsigned char *>(xs + r * xst);
      const uint32_t *E = ent + tl * d;
      const uint16_t *B = boff + tl * (m + 1);
      const uint32_t *KA = p.ka + int64_t(t) * m;
      const uint32_t *KB = p.kb + int64_t(t) * m;
      uint32_t ha = 0, hb = 0;
      uint64_t word = 0;
      int nflag = 0, nchanged = 0, novf = 0;

      int beg = B[0];
      for (int l = 0; l < m; ++l) {
        const int end = B[l + 1];
        float acc = 0.f;
#pragma unroll 4
        for (int i = beg; i < end; ++i) {
          const uint32_t e = E[i];
          const float v = *reinterpret_cast<const float *>(xrow + (e & 0x7fffffffu));
          acc += __uint_as_float(__float_as_uint(v) ^ (e & 0x80000000u));
        }
        const int k = end - beg;
        // FP32 summation bound: gamma_{k-1} * k * max|x| (gamma_n <= n u (1 + 2 n u)),
        // widened by 2% to cover the FP64 reference's own error and this arithmetic.
        const float gk = float(k > 1 ? k - 1 : 0) * kU32;
        const float E_y = 1.02f * gk * (1.f + 2.f * gk) * float(k) * xm;
        if (SRP) {
          const bool flag = valid && !isbad && k >= 2 && !(fabsf(acc) > E_y);
          int bit = acc > 0.f ? 1 : 0;
          if (__any_sync(0xffffffffu, flag)) {
            if (flag) {
              double y = 0.0;
              for (int i = beg; i < end; ++i) {
                const uint32_t e = E[i];
                const double v = double(*reinterpret_cast<const float *>(xrow + (e & 0x7fffffffu)));
                y = __dadd_rn(y, (e & 0x80000000u) ? -v : v);
              }
              const int b64 = y > 0.0 ? 1 : 0;
              ++nflag;
              nchanged += b64 != bit;
              bit = b64;
            }
          }
          if (p.proj && valid) p.proj[(row * p.L + t) * m + l] = acc;
          if (m <= 64) {
            word |= uint64_t(bit) << l;
          } else {
            word |= uint64_t(bit) << (l & 63);
            if (bit) {
              ha += __ldg(KA + l);
              hb += __ldg(KB + l);
            }
            if ((l & 63) == 63 || l == m - 1) {
              if (p.bits && valid) p.bits[(row * p.L + t) * ((m + 63) >> 6) + (l >> 6)] = word;
              word = 0;
            }
          }
        } else {
          const float bl = bf[tl * m + l];
          const float tf = __fmul_rn(__fmaf_rn(a.sqrtm_f, acc, bl), a.invw_f);
          const float fl = floorf(tf);
          const float fr = tf - fl;
          const float dist = fminf(fr, 1.f - fr);
          const float M = 1.02f * (sq_w * E_y +
                                   5.f * kU32 * ((a.sqrtm_f * fabsf(acc) + bl) * a.invw_f + fabsf(tf) + 1.f));
          const bool flag = valid && !isbad && (!(dist > M) || !(fabsf(tf) < 4194304.f));
          int code = int(fl);
          if (__any_sync(0xffffffffu, flag)) {
            if (flag) {
              double y = 0.0;
              for (int i = beg; i < end; ++i) {
                const uint32_t e = E[i];
                const double v = double(*reinterpret_cast<const float *>(xrow + (e & 0x7fffffffu)));
                y = __dadd_rn(y, (e & 0x80000000u) ? -v : v);
              }
              const double t1 = __dmul_rn(p.sqrtm, y);
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
          ha += uint32_t(code) * __ldg(KA + l);
          hb += uint32_t(code) * __ldg(KB + l);
          if (valid) {
            if (p.codes) p.codes[(row * p.L + t) * m + l] = code;
            if (p.proj) p.proj[(row * p.L + t) * m + l] = acc;
          }
        }
        beg = end;
      }
      if (valid) {
        uint64_t key;
        if (SRP && m <= 64) {
          key = word;
          if (p.bits) p.bits[row * p.L + t] = word;
        } else {
          key = (uint64_t(ha) << 32) | uint64_t(hb);
        }
        if (isbad) key = ~0ull;
        if (p.keys) p.keys[int64_t(t) * p.key_ld + row] = key;
      }
      // counters (one atomic per warp and counter)
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
      if (tl == 0 && valid && isbad) {  // one report per bad row
        if (p.counters) atomicAdd(p.counters + CNT_NONFINITE, 1ull);
        atomicOr(p.status, STATUS_NONFINITE);
      }
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

Plan make_plan(int d, int m, int L, int64_t n) {
  Plan best{};
  best.smem = -1;
  const int sms = num_sms();
  for (int RG = 4; RG >= 1; RG >>= 1) {
    // prefer enough tiles to fill the GPU twice
    const int64_t ntiles = (n + RG * kWarp - 1) / (RG * kWarp);
    if (RG > 1 && ntiles < 2 * sms) continue;
    for (int Lg = (L < 32 ? L : 32); Lg >= 1; --Lg) {
      const int G = (L + Lg - 1) / Lg;
      const int Lgb = (L + G - 1) / G;  // balanced group size
      Plan pl{};
      pl.Lg = Lgb;
      pl.G = G;
      pl.RG = RG;
      const int tasks = RG * Lgb;
      int W = tasks < 32 ? tasks : 32;
      if (tasks > 32) {
        for (int w = 32; w >= 16; --w)
          if (tasks % w == 0) { W = w; break; }
      }
      if (W < 4) W = 4;
      pl.W = W;
      pl.x_stride = d + 1;
      int off = 0;
      pl.off_ent = off;
      off = align16(off + Lgb * d * 4);
      pl.off_boff = off;
      off = align16(off + Lgb * (m + 1) * 2);
      pl.off_b = off;
      off = align16(off + Lgb * m * 4);
      pl.off_x = off;
      const int xbytes = RG * kWarp * (d + 1) * 4;
      const int scratch = W * m * 4;
      off = align16(off + (xbytes > scratch ? xbytes : scratch));
      pl.off_xmax = off;
      off = align16(off + RG * kWarp * 4);
      pl.off_bad = off;
      off = align16(off + RG * kWarp * 4);
      pl.smem = off;
      if (off <= kMaxSmem) return pl;
    }
  }
  return best;
}

}  // namespace

SketchPlan plan_sketch_dense(int d, int m, int L, int dtype) {
  (void)dtype;
  Plan pl = make_plan(d, m, L, int64_t(1) << 40);
  SketchPlan sp{};
  sp.ok = pl.smem > 0;
  if (!sp.ok) return sp;
  sp.tables_per_cta = pl.Lg;
  sp.groups = pl.G;
  sp.row_groups = pl.RG;
  sp.warps = pl.W;
  sp.smem = pl.smem;
  const int per_sm = kMaxSmem / pl.smem;
  sp.ctas = num_sms() * (per_sm > 0 ? per_sm : 1);
  return sp;
}

cudaError_t launch_sketch_dense(const SketchLaunch &p, cudaStream_t stream) {
  if (p.n <= 0) return cudaSuccess;
  Args a{};
  a.p = p;
  a.pl = make_plan(p.d, p.m, p.L, p.n);
  if (a.pl.smem <= 0) return cudaErrorInvalidConfiguration;
  const int R = a.pl.RG * kWarp;
  const int64_t ntiles = (p.n + R - 1) / R;
  if (ntiles > INT32_MAX) return cudaErrorInvalidValue;
  a.ntiles = int(ntiles);
  int per_sm = kMaxSmem / a.pl.smem;
  if (per_sm > 2) per_sm = 2;
  if (per_sm < 1) per_sm = 1;
  const int64_t cap = int64_t(num_sms()) * per_sm / a.pl.G;
  int64_t slots = cap < ntiles ? cap : ntiles;
  if (slots < 1) slots = 1;
  a.slots = int(slots);
  a.sqrtm_f = float(p.sqrtm);
  a.invw_f = float(1.0 / p.w);
  const bool srp = kind_is_srp(p.kind);
  const dim3 grid((unsigned)(a.slots * a.pl.G)), block((unsigned)(a.pl.W * kWarp));
  cudaError_t e;
  if (srp) {
    e = cudaFuncSetAttribute(sketch_dense_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             a.pl.smem);
    if (e != cudaSuccess) return e;
    sketch_dense_kernel<true><<<grid, block, a.pl.smem, stream>>>(a);
  } else {
    e = cudaFuncSetAttribute(sketch_dense_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             a.pl.smem);
    if (e != cudaSuccess) return e;
    sketch_dense_kernel<false><<<grid, block, a.pl.smem, stream>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace lsh
