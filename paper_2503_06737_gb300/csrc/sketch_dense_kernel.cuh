// sketch_dense_kernel.cuh -- CS / HCS hashing of dense rows for all L tables
// in one persistent launch (Definitions 4, 5, 12, 19, 25, 31): the kernel,
// its device helpers and the recheck kernel of queued bins.
//
// Design (sm_103a):
//   * A CTA owns a group of Lg tables and walks row tiles.  Its tables are
//     staged once in shared memory as per-table member lists: for each bin,
//     the coordinates j < d with s = +1 (ascending j), then those with s = -1,
//     each half padded to a multiple of four with the row's zero slot; every
//     entry is the byte offset of x_j from a lane's row base (16-bit while it
//     fits, or 32-bit: one instruction less per term, chosen by the plan).
//     HCS lists are derived in the CTA from the per-mode tables h_k, s_k (the
//     sign of j is prod_k s_k(i_k)), so HBM holds only O(N d^(1/N)) words per
//     table.
//   * Lane = RPL rows (1, 2 or 4).  The row tile keeps rows in groups of RPL:
//     inside a group, x_j of its RPL rows are adjacent words, so one
//     ld.shared.v{1,2,4} fetches the operand of one term for all of a lane's
//     rows, and one entry (and one address add) serves RPL terms.  Groups are
//     RPL * dp words apart with dp odd, which keeps the 32 lanes of a warp on
//     distinct banks.  The tile is read from HBM with 128-bit loads (rows
//     16-byte aligned) and converted to FP32; the next tile is prefetched into
//     L2 while this one is hashed, and the CTAs of the G table groups that
//     share a tile run concurrently, so it leaves HBM once.
//   * A table is split over WPT warps (bins l = k, k+WPT, ...).  Partial keys
//     of the warps of one table combine in shared memory: the key fold is a
//     sum mod 2^32 (E2LSH, SRP m > 64) or an OR of bits (SRP m <= 64).  The
//     keys-only instantiation carries no per-bin output code; the full one
//     also writes codes, SRP bits, projections and counters.  The plan (RPL,
//     row groups, WPT, Lg, entry width) is autotuned per shape on the first
//     large batch (see tuned_plan).
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
//     nearest integer is computed exactly.  When |t| >= 2^22 the bound is above
//     2.5 and every such bin is flagged, as is a non-finite t.  A bin whose t
//     lies within the bound of an integer (E2LSH), or whose |y| is within
//     A max|x| of 0 (SRP, A without sqrt(m)/w), gets the canonical value of
//     Definitions 12/19/25/31 -- the ascending FP64 sum, one IEEE rounding per
//     operation: large batches queue such bins for sketch_recheck_kernel,
//     which patches codes, bits and keys; small batches (and queue overflow)
//     recheck in place.  Either way the value is computed exactly as an int64
//     sum on the least exponent grid of the bin's terms when that sum is exact
//     in the FP64 loop, else by the FP64 loop itself.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

#include "sketch_dense.h"

namespace lsh {
namespace sk {
namespace {

// Flag bits in the first entry of every quad of a member list: the quad
// belongs to the negative half of its bin (kNeg), the quad is the last one of
// its bin (kEnd).  kMask recovers the offset.
template <typename EntT>
struct EntFlags;
template <>
struct EntFlags<uint16_t> {
  static constexpr uint32_t kNeg = 1u << 14, kEnd = 1u << 15, kMask = 0x3fffu;
};
template <>
struct EntFlags<uint32_t> {
  static constexpr uint32_t kNeg = 1u << 30, kEnd = 1u << 31, kMask = 0x3fffffffu;
};

// Bin and sign of entry j of table t: coordinate j (per-mode tables, first
// mode fastest), or for CSSRP-L the incidence j = i l + r (the r-th bin of i).
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

// Stage table t (one warp): member list (sign-split, quad-padded, entries
// j * unit) and the per-bin records seg[l] = {start, quads(+) | quads(-) << 16},
// cst[l] = {b_l (f32 bits), A_l, ka_l, kb_l}.
template <typename EntT>
__device__ void stage_table(const SketchLaunch &p, int t, float a_scale, uint32_t unit, EntT *ent, uint2 *seg,
                            uint4 *cst, uint2 *rng, int wpt, bool pairs, uint32_t *scratch, int lane) {
  const int d = p.d, m = p.m;
  uint32_t *cur = scratch;  // [2m]: counts, then write cursors (key = 2 bin + neg)
  // incidences e = j lc + r: coordinate j's r-th bin (lc = 1 but for CSSRP-L)
  const int lc = p.lc, ne = d * lc;
  for (int i = lane; i < 2 * m; i += kWarp) cur[i] = 0;
  __syncwarp();
  for (int e = lane; e < ne; e += kWarp) {
    int bin;
    uint32_t neg;
    coord_bin(p, t, e, bin, neg);
    atomicAdd(&cur[2 * bin + neg], 1u);
  }
  __syncwarp();
  const uint32_t zslot = uint32_t(d) * unit;
  uint32_t carry = 0;
  for (int base = 0; base < m; base += kWarp) {
    const int l = base + lane;
    uint32_t cp = 0, cn = 0, qp = 0, qn = 0;
    if (l < m) {
      cp = cur[2 * l];
      cn = cur[2 * l + 1];
      qn = (cn + 3) & ~3u;
      qp = cp + cn == 0 ? 4u : (cp + 3) & ~3u;  // an empty bin keeps one quad of zero slots (it carries the end flag)
      if (pairs && ((qp + qn) & 4u)) qn += 4;    // quads come in pairs: one more quad of zero slots
    }
    const uint32_t sz = qp + qn;
    uint32_t s = sz;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    const uint32_t start = carry + s - sz;
    if (l < m) {
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
  for (int base = 0; base < ne; base += kWarp) {
    const int e = base + lane;
    const bool act = e < ne;
    const uint32_t amask = __ballot_sync(0xffffffffu, act);
    if (act) {
      int bin;
      uint32_t neg;
      coord_bin(p, t, e, bin, neg);
      const uint32_t key = 2u * uint32_t(bin) + neg;
      const uint32_t peers = __match_any_sync(amask, key);
      ent[cur[key] + __popc(peers & lt)] = EntT(uint32_t(e / lc) * unit);
      __syncwarp(amask);
      if ((peers & lt) == 0) cur[key] += __popc(peers);
    }
    __syncwarp();
  }
  // flags: negative quads, the last quad of every bin (with paired quads,
  // the last two, which the two half-warps read in the same step)
  for (int l = lane; l < m; l += kWarp) {
    const uint2 sg = seg[l];
    const uint32_t qp = sg.y & 0xffffu, qn = sg.y >> 16;
    for (uint32_t k = 0; k < qn; ++k) ent[sg.x + 4 * (qp + k)] = EntT(ent[sg.x + 4 * (qp + k)] | EntFlags<EntT>::kNeg);
    const uint32_t last = sg.x + 4 * (qp + qn - 1);
    ent[last] = EntT(ent[last] | EntFlags<EntT>::kEnd);
    if (pairs) ent[last - 4] = EntT(ent[last - 4] | EntFlags<EntT>::kEnd);
  }
  __syncwarp();
  // the bin ranges of the table's wpt warps, balanced by quads: rng[r] =
  // {first bin, first quad}, rng[wpt] = {m, total quads}
  const uint32_t total = (seg[m - 1].x >> 2) + (seg[m - 1].y & 0xffffu) + (seg[m - 1].y >> 16);
  if (lane <= wpt) {
    uint32_t lb = 0, qb = 0;
    if (lane == wpt) {
      lb = uint32_t(m);
      qb = total;
    } else if (lane > 0) {
      const uint32_t target = (uint32_t(lane) * total) / uint32_t(wpt);
      uint32_t lo = 0, hi = uint32_t(m);  // first bin whose start quad is >= target
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((seg[mid].x >> 2) < target)
          lo = mid + 1;
        else
          hi = mid;
      }
      lb = lo;
      qb = lo < uint32_t(m) ? (seg[lo].x >> 2) : total;
    }
    rng[lane] = make_uint2(lb, qb);
  }
  __syncwarp();
}

// Explicit shared-space loads with 32-bit addresses.
template <int RPL>
__device__ __forceinline__ void lds_x(uint32_t a, float (&v)[RPL]) {
  if constexpr (RPL == 1) {
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v[0]) : "r"(a));
  } else if constexpr (RPL == 2) {
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v[0]), "=f"(v[1]) : "r"(a));
  } else {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "r"(a));
  }
}
template <int RPL>
__device__ __forceinline__ void sts_x(uint32_t a, const float (&v)[RPL]) {
  if constexpr (RPL == 1) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v[0]));
  } else if constexpr (RPL == 2) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v[0]), "f"(v[1]));
  } else {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]));
  }
}
// Packed FP32 pairs: the x_j of two rows of a lane (adjacent words) and
// their accumulators travel as one 64-bit register pair, so that one
// fma.rn.f32x2 -- two independent IEEE single-precision fmas -- adds a term
// to both rows.
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
template <int NP>
__device__ __forceinline__ void lds_x2(uint32_t a, uint64_t (&v)[NP]) {
  if constexpr (NP == 1) {
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v[0]) : "r"(a));
  } else {
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(v[0]), "=l"(v[1]) : "r"(a));
  }
}

// One quad of entries as stored (two words of 16-bit entries, four of
// 32-bit ones), and its decoding: the four offsets (flags masked off) and the
// raw first word (whose first entry carries the flags).
template <typename EntT>
struct QuadWords;
template <>
struct QuadWords<uint16_t> {
  uint32_t w[2];
};
template <>
struct QuadWords<uint32_t> {
  uint32_t w[4];
};
template <typename EntT>
__device__ __forceinline__ void lds_quad_words(uint32_t qaddr, QuadWords<EntT> &q) {
  if constexpr (sizeof(EntT) == 2) {
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(q.w[0]), "=r"(q.w[1]) : "r"(qaddr));
  } else {
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(q.w[0]), "=r"(q.w[1]), "=r"(q.w[2]), "=r"(q.w[3])
                 : "r"(qaddr));
  }
}
template <typename EntT>
__device__ __forceinline__ void decode_quad(const QuadWords<EntT> &q, uint32_t (&o)[4], uint32_t &w0) {
  w0 = q.w[0];
  if constexpr (sizeof(EntT) == 2) {
    o[0] = q.w[0] & EntFlags<EntT>::kMask;
    o[1] = q.w[0] >> 16;
    o[2] = q.w[1] & 0xFFFFu;
    o[3] = q.w[1] >> 16;
  } else {
    o[0] = q.w[0] & EntFlags<EntT>::kMask;
    o[1] = q.w[1];
    o[2] = q.w[2];
    o[3] = q.w[3];
  }
}

__device__ __forceinline__ float lds_f32(const unsigned char *base, uint32_t off) {
  return *reinterpret_cast<const float *>(base + off);
}

// FP64 recheck of one bin for one row: merge the two ascending halves back
// into ascending j and sum s(j) x_j with one IEEE rounding per addition.
template <typename EntT>
__device__ __noinline__ double bin_fp64(const EntT *P, int np, const EntT *N, int nn,
                                        const unsigned char *xr, uint32_t zslot) {
  int ip = 0, in = 0;
  double y = 0.0;
  constexpr uint32_t kMask = EntFlags<EntT>::kMask;
  while (true) {
    const uint32_t a = ip < np ? P[ip] & kMask : zslot;
    const uint32_t b = in < nn ? N[in] & kMask : zslot;
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
      const uint32_t v = __float_as_uint(lds_f32(xr, L[i] & EntFlags<EntT>::kMask));
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
      const uint32_t v = __float_as_uint(lds_f32(xr, L[i] & EntFlags<EntT>::kMask));
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

// The exact FP64 projection of one bin of one row of the tile.
template <typename EntT>
__device__ __noinline__ double bin_value(const EntT *P, int np4, int nn4, const unsigned char *xr, uint32_t zslot) {
  double y64;
  if (!bin_exact(P, np4, P + np4, nn4, xr, y64)) y64 = bin_fp64(P, np4, P + np4, nn4, xr, zslot);
  return y64;
}

// Append this lane's flagged bin to the recheck queue (warp-aggregated);
// false when there is no queue or it is full (the lane then rechecks in place).
__device__ __forceinline__ bool queue_bin(const SketchLaunch &p, bool flag, int64_t row, int t, int l, int code,
                                          int lane) {
  if (!p.queue) return false;
  const uint32_t bal = __ballot_sync(0xffffffffu, flag);
  if (!bal) return false;
  const int leader = __ffs(bal) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(p.qcount, uint32_t(__popc(bal)));
  base = __shfl_sync(0xffffffffu, base, leader);
  const uint32_t pos = base + __popc(bal & ((1u << lane) - 1u));
  if (!flag || pos >= p.qcap) return false;
  p.queue[pos] = make_int4(int(row), t, l, code);
  return true;
}

// E2LSH code of the exact FP64 projection (Definitions 12, 19; dense:
// Definition 2 with sqrt(m) = 1), one IEEE rounding per operation; an
// out-of-range code is INT32_MIN and counted.
__device__ __forceinline__ int e2lsh_code64(const SketchLaunch &p, double y64, int64_t tl, int &novf) {
  const double t1 = __dmul_rn(p.sqrtm, y64);
  const double t2 = __dadd_rn(t1, p.b64[tl]);
  const double t3 = __ddiv_rn(t2, p.w);
  const double f = floor(t3);
  if (f >= -2147483648.0 && f <= 2147483647.0) return int(f);
  ++novf;
  return INT32_MIN;
}

// The rare path of one bin and row (the whole warp calls it when some lane's
// value lies within the error bound): flagged lanes of valid, finite rows
// queue the bin, or recheck it in place when there is no queue or it is
// full.  Returns the lane's code (SRP: bit) and, in ev, bit 0 = rechecked in
// place, bit 1 = its code changed, bit 2 = the code overflowed int32.
struct ColdOut {
  int code, ev;
};
template <bool SRP, typename EntT>
__device__ __noinline__ ColdOut bin_cold(const SketchLaunch &p, bool flag, int64_t row, int t, int l, int code,
                                         const EntT *P, int qp, int qn, const unsigned char *xr, uint32_t zslot,
                                         int lane) {
  ColdOut o{code, 0};
  if (queue_bin(p, flag, row, t, l, code, lane) || !flag) return o;
  const double y64 = bin_value(P, 4 * qp, 4 * qn, xr, zslot);
  int c64, novf = 0;
  if (SRP)
    c64 = y64 > 0.0 ? 1 : 0;
  else
    c64 = e2lsh_code64(p, y64, int64_t(t) * p.m + l, novf);
  o.ev = 1 | (c64 != code ? 2 : 0) | (novf ? 4 : 0);
  o.code = c64;
  return o;
}

template <int DT>
__device__ __forceinline__ float load_x(const void *X, int64_t idx) {
  if (DT == LSH_F32) return __ldg(reinterpret_cast<const float *>(X) + idx);
  const unsigned short h = __ldg(reinterpret_cast<const unsigned short *>(X) + idx);
  if (DT == LSH_BF16) return __uint_as_float(uint32_t(h) << 16);
  return __half2float(__ushort_as_half(h));
}

template <int DT>
__device__ __forceinline__ float cvt16(uint32_t h) {
  if (DT == LSH_BF16) return __uint_as_float(h << 16);
  return __half2float(__ushort_as_half((unsigned short)h));
}

// 16 bytes of a row (4 FP32 or 8 16-bit values) as FP32.
template <int DT>
__device__ __forceinline__ void unpack_vec(const uint4 q, float (&v)[8]) {
  if (DT == LSH_F32) {
    v[0] = __uint_as_float(q.x);
    v[1] = __uint_as_float(q.y);
    v[2] = __uint_as_float(q.z);
    v[3] = __uint_as_float(q.w);
  } else {
    v[0] = cvt16<DT>(q.x & 0xFFFFu);
    v[1] = cvt16<DT>(q.x >> 16);
    v[2] = cvt16<DT>(q.y & 0xFFFFu);
    v[3] = cvt16<DT>(q.y >> 16);
    v[4] = cvt16<DT>(q.z & 0xFFFFu);
    v[5] = cvt16<DT>(q.z >> 16);
    v[6] = cvt16<DT>(q.w & 0xFFFFu);
    v[7] = cvt16<DT>(q.w >> 16);
  }
}

// Load the R rows of a tile into the grouped layout (group g at word g*S,
// row i of the group's x_j at word g*S + j*RPL + i), one warp per group of
// RPL rows, plus each row's max |x| and finiteness.  With 16-byte aligned
// rows, lane u reads 16-byte chunk u of each row and writes its V values
// rotated by rot(lane), which keeps the shared-memory stores of a warp on
// distinct banks; the remainder (and unaligned rows) go one value at a time.
template <int DT, int RPL>
__device__ void load_tile(const Args &a, const void *X, int64_t n, uint32_t xs_s, int64_t row0, int R, int warp,
                          int lane, float *xmax, int *bad) {
  const SketchLaunch &p = a.p;
  const int d = p.d;
  const int S = RPL * a.pl.dp;
  constexpr int V = DT == LSH_F32 ? 4 : 8;
  const int ngroups = R / RPL;
  for (int g = warp; g < ngroups; g += a.pl.W) {
    const uint32_t gb = xs_s + uint32_t(g * S) * 4u;
    float mx[RPL];
    bool fin[RPL], live[RPL];
    int64_t rb[RPL];
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      const int64_t row = row0 + g * RPL + i;
      live[i] = row < n;
      rb[i] = row * p.ld;
      mx[i] = 0.f;
      fin[i] = true;
    }
    int jdone = 0;
    if (a.vec) {
      // NB chunks per lane in flight: all loads of a batch issue before use
      constexpr int NB = 8 / RPL;
      const int nvec = d / V;
      const int rot = ((lane * V * RPL) >> 5) & (V - 1);
      for (int u0 = lane; u0 < nvec; u0 += NB * kWarp) {
        uint4 q[NB][RPL];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const int u = u0 + b * kWarp;
#pragma unroll
          for (int i = 0; i < RPL; ++i) {
            constexpr int es = DT == LSH_F32 ? 4 : 2;
            q[b][i] = (u < nvec && live[i])
                          ? __ldg(reinterpret_cast<const uint4 *>(static_cast<const char *>(X) +
                                                                  (rb[i] + int64_t(u) * V) * es))
                          : make_uint4(0u, 0u, 0u, 0u);
          }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const int u = u0 + b * kWarp;
          if (u >= nvec) break;
          float v[RPL][8];
#pragma unroll
          for (int i = 0; i < RPL; ++i) {
            unpack_vec<DT>(q[b][i], v[i]);
#pragma unroll
            for (int c = 0; c < V; ++c) {
              mx[i] = fmaxf(mx[i], fabsf(v[i][c]));
              fin[i] = fin[i] && isfinite(v[i][c]);
            }
            // rotate left by rot: position c then holds value (c + rot) mod V
#pragma unroll
            for (int sft = 1; sft < V; sft <<= 1) {
              const bool bsel = (rot & sft) != 0;
              float t[8];
#pragma unroll
              for (int c = 0; c < V; ++c) t[c] = bsel ? v[i][(c + sft) & (V - 1)] : v[i][c];
#pragma unroll
              for (int c = 0; c < V; ++c) v[i][c] = t[c];
            }
          }
#pragma unroll
          for (int c = 0; c < V; ++c) {
            const int j = u * V + ((c + rot) & (V - 1));
            float o[RPL];
#pragma unroll
            for (int i = 0; i < RPL; ++i) o[i] = v[i][c];
            sts_x<RPL>(gb + uint32_t(j * RPL) * 4u, o);
          }
        }
      }
      jdone = nvec * V;
    }
    // the remainder (and unaligned rows): 8 values per lane in flight
    for (int j0 = jdone + lane; j0 < d; j0 += 8 * kWarp) {
      float o[8][RPL];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int j = j0 + b * kWarp;
#pragma unroll
        for (int i = 0; i < RPL; ++i) o[b][i] = (j < d && live[i]) ? load_x<DT>(X, rb[i] + j) : 0.f;
      }
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int j = j0 + b * kWarp;
        if (j >= d) break;
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          mx[i] = fmaxf(mx[i], fabsf(o[b][i]));
          fin[i] = fin[i] && isfinite(o[b][i]);
        }
        sts_x<RPL>(gb + uint32_t(j * RPL) * 4u, o[b]);
      }
    }
    if (lane == 0) {  // the zero slot the padding entries point at
      float z[RPL];
#pragma unroll
      for (int i = 0; i < RPL; ++i) z[i] = 0.f;
      sts_x<RPL>(gb + uint32_t(d * RPL) * 4u, z);
    }
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      float x = mx[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
      const bool allfin = __all_sync(0xffffffffu, fin[i]);
      if (lane == 0) {
        xmax[g * RPL + i] = x;
        bad[g * RPL + i] = allfin ? 0 : 1;
      }
    }
  }
}

// The next task of the tile for this warp (lane 0 takes it from the counter).
__device__ __forceinline__ int claim_task(uint32_t *ctr, int lane) {
  uint32_t t = 0;
  if (lane == 0) t = atomicAdd(ctr, 1u);
  return int(__shfl_sync(0xffffffffu, t, 0));
}

template <bool SRP, typename EntT, int RPL, bool FULL, bool HW>
__global__ void __launch_bounds__(max_threads(RPL), 1) sketch_dense_kernel(const __grid_constant__ Args a) {
  static_assert(!HW || RPL >= 2, "split bins need two or more rows per lane");
  extern __shared__ __align__(16) unsigned char smem[];
  const SketchLaunch &p = a.p;
  const Plan &pl = a.pl;
  // the batch: from the launch, or, in a replayed graph, from the device
  // descriptor (the launch then gives the largest batch it is sized for)
  const void *X = p.X;
  int64_t n = p.n;
  uint64_t *keys = p.keys;
  int64_t key_ld = p.key_ld;
  if (p.desc) {
    X = p.desc->X;
    n = p.desc->n;
    keys = p.desc->keys;
    key_ld = p.desc->key_ld;
  }
  const int lane = threadIdx.x & (kWarp - 1);
  const int warp = threadIdx.x >> 5;
  const int tg = blockIdx.x % pl.G;
  const int slot = blockIdx.x / pl.G;
  const int t0 = tg * pl.Lg;
  const int Lg = min(pl.Lg, p.L - t0);
  constexpr int GPW = groups_per_warp(HW);
  const int R = pl.RG * GPW * RPL;
  const int ntiles = p.desc ? int((n + R - 1) / R) : a.ntiles;
  // CTAs without a tile (a replayed graph sized for a larger batch) skip the table staging too
  if (Lg <= 0 || slot >= a.slots || slot >= ntiles) return;
  const int d = p.d, m = p.m;
  const int cap = pl.cap;
  const int WPT = pl.WPT;
  constexpr uint32_t unit = RPL * 4;
  constexpr int EPR = HW ? RPL / 2 : RPL;  // rows whose bin epilogue a lane runs
  const int h = HW ? lane >> 4 : 0;        // the lane's half-warp
  const int gl = HW ? lane & 15 : lane;    // the lane's row group in the warp

  EntT *ent = reinterpret_cast<EntT *>(smem + pl.off_ent);
  uint2 *seg = reinterpret_cast<uint2 *>(smem + pl.off_seg);
  uint2 *rng = reinterpret_cast<uint2 *>(smem + pl.off_rng);  // [Lg][kMaxWpt + 1] warp ranges
  uint4 *cst = reinterpret_cast<uint4 *>(smem + pl.off_cst);
  uint2 *kacc = reinterpret_cast<uint2 *>(smem + pl.off_key);  // [R][Lg] partial keys
  float *xs = reinterpret_cast<float *>(smem + pl.off_x);
  float *xmax = reinterpret_cast<float *>(smem + pl.off_xmax);
  int *bad = reinterpret_cast<int *>(smem + pl.off_bad);
  uint32_t *task_ctr = reinterpret_cast<uint32_t *>(smem + pl.off_ctr);

  {
    const float sq_w = a.sqrtm_f * a.invw_f;
    uint32_t *scratch = reinterpret_cast<uint32_t *>(xs) + warp * 2 * m;  // aliases the tile
    for (int tl = warp; tl < Lg; tl += pl.W)
      stage_table(p, t0 + tl, SRP ? 1.f : sq_w, unit, ent + tl * cap, seg + tl * m, cst + tl * m,
                  rng + tl * (kMaxWpt + 1), WPT, HW, scratch, lane);
  }
  if (threadIdx.x == 0) *task_ctr = 0u;
  __syncthreads();

  const int S = RPL * pl.dp;
  const int ntasks = pl.RG * Lg * WPT;
  const uint32_t zslot = uint32_t(d) * unit;
  const uint32_t xs_s = static_cast<uint32_t>(__cvta_generic_to_shared(xs));
  const uint32_t ent_s = static_cast<uint32_t>(__cvta_generic_to_shared(ent));
  const int es = p.dtype == LSH_F32 ? 4 : 2;

  for (int tile = slot; tile < ntiles; tile += a.slots) {
    const int64_t row0 = int64_t(tile) * R;
    for (int i = threadIdx.x; i < R * Lg; i += blockDim.x) kacc[i] = make_uint2(0u, 0u);
    if (p.dtype == LSH_F32)
      load_tile<LSH_F32, RPL>(a, X, n, xs_s, row0, R, warp, lane, xmax, bad);
    else if (p.dtype == LSH_BF16)
      load_tile<LSH_BF16, RPL>(a, X, n, xs_s, row0, R, warp, lane, xmax, bad);
    else
      load_tile<LSH_F16, RPL>(a, X, n, xs_s, row0, R, warp, lane, xmax, bad);
    __syncthreads();
    // ---- prefetch the next tile into L2 while this one is hashed ----
    if (warp == pl.W - 1) {
      const int64_t nrow0 = int64_t(tile + a.slots) * R;
      const char *Xc = reinterpret_cast<const char *>(X);
      for (int r = 0; r < R; ++r) {
        const int64_t row = nrow0 + r;
        if (row >= n) break;
        const char *rp = Xc + row * p.ld * es;
        for (int off = lane * 128; off < d * es; off += kWarp * 128)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(rp + off));
      }
    }

    // ---- one task = (row group, table, bin range): lane = RPL rows.  Warps
    // claim tasks from a shared counter, so the ones that finish early take
    // more and the barrier at the end of the tile waits for one task at most ----
    for (int task = claim_task(task_ctr, lane); task < ntasks; task = claim_task(task_ctr, lane)) {
      const int sub = task % WPT;
      const int rt = task / WPT;
      const int rg = rt / Lg;
      const int tl = rt - rg * Lg;
      const int t = t0 + tl;
      const int grp = rg * GPW + gl;  // the lane's row group in the tile
      const int rl0 = grp * RPL;      // its first row in the tile
      const int re0 = rl0 + h * EPR;  // the first row of its bin epilogues
      const uint32_t xb = xs_s + uint32_t(grp * S) * 4u;
      float xm[EPR];
#pragma unroll
      for (int k = 0; k < EPR; ++k) xm[k] = xmax[re0 + k];
      const uint32_t eb = ent_s + uint32_t(tl * cap) * uint32_t(sizeof(EntT));
      const uint2 *Sg = seg + tl * m;
      const uint4 *C = cst + tl * m;
      uint32_t ha[EPR], hb[EPR];
#pragma unroll
      for (int k = 0; k < EPR; ++k) ha[k] = hb[k] = 0u;
      int nflag = 0, nchanged = 0, novf = 0;
      // this warp's bins: a contiguous range, walked as one flat list of
      // quads (or quad pairs); the last quad of every bin ends in that bin's
      // epilogue
      const uint2 rb = rng[tl * (kMaxWpt + 1) + sub], rn = rng[tl * (kMaxWpt + 1) + sub + 1];
      int l = int(rb.x);
      // full outputs: the codes and projections of a row's last four bins,
      // written four at a time (one 16-byte store per row and output) when
      // the bin index reaches a multiple of four, and at the range's ends
      int cq[EPR][4];
      float pq[EPR][4];
      const bool vec_out = (m & 3) == 0 && (reinterpret_cast<uintptr_t>(p.codes) & 15) == 0 &&
                           (reinterpret_cast<uintptr_t>(p.proj) & 15) == 0;
      auto put_out = [&](int k, int64_t row, int code, float y) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          cq[k][j] = cq[k][j + 1];
          pq[k][j] = pq[k][j + 1];
        }
        cq[k][3] = code;
        pq[k][3] = y;
        if ((l & 3) != 3 && l != int(rn.x) - 1) return;
        if (row >= n) return;
        const int64_t o = (row * p.L + t) * m;
        if (vec_out && (l & 3) == 3 && l - 3 >= int(rb.x)) {
          if (p.codes) *reinterpret_cast<int4 *>(p.codes + o + l - 3) = make_int4(cq[k][0], cq[k][1], cq[k][2], cq[k][3]);
          if (p.proj) *reinterpret_cast<float4 *>(p.proj + o + l - 3) = make_float4(pq[k][0], pq[k][1], pq[k][2], pq[k][3]);
          return;
        }
        const int lo = max(l & ~3, int(rb.x));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int bl = l - 3 + j;
          if (bl >= lo) {
            if (p.codes) p.codes[o + bl] = cq[k][j];
            if (p.proj) p.proj[o + bl] = pq[k][j];
          }
        }
      };
      // two accumulators per row: scalars for one row per lane, packed pairs
      // of rows (fma.rn.f32x2) for two or four
      constexpr int NP = RPL >= 2 ? RPL / 2 : 1;
      float a0[RPL], a1[RPL];
      uint64_t p0[NP], p1[NP];
#pragma unroll
      for (int i = 0; i < RPL; ++i) a0[i] = a1[i] = 0.f;
#pragma unroll
      for (int i = 0; i < NP; ++i) p0[i] = p1[i] = 0ull;
      auto finish_bin = [&]() {
        const uint4 c = C[l];
        const float A = __uint_as_float(c.y);
        float ys[RPL];
        if constexpr (RPL >= 2) {
          // p0 * 1 + p1: one rounding per row, the same as the scalar sums
          const uint64_t one2 = pack2(1.f, 1.f);
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            unpack2(ffma2(p0[i], one2, p1[i]), ys[2 * i], ys[2 * i + 1]);
            p0[i] = p1[i] = 0ull;
          }
        } else {
#pragma unroll
          for (int i = 0; i < RPL; ++i) {
            ys[i] = a0[i] + a1[i];
            a0[i] = a1[i] = 0.f;
          }
        }
        if (HW) {
          // half h finishes rows h*EPR.. of its pair: it sends the other
          // half's rows and adds what it receives (FP32 addition commutes,
          // so the sum is the one either half would form)
#pragma unroll
          for (int k = 0; k < EPR; ++k) {
            const float mine = h ? ys[EPR + k] : ys[k];
            const float other = __shfl_xor_sync(0xffffffffu, h ? ys[k] : ys[EPR + k], 16);
            ys[k] = mine + other;
          }
        }
#pragma unroll
        for (int k = 0; k < EPR; ++k) {
          const float y = ys[k];
          const int ri = re0 + k;  // the row in the tile
          const int64_t row = row0 + ri;
          int code;
          bool flag;
          if (SRP) {
            // A = 0 when the bin holds at most one term: the FP32 value is then exact
            flag = A > 0.f && !(fabsf(y) > A * xm[k]);
            code = y > 0.f ? 1 : 0;
          } else {
            const float tf = __fmul_rn(__fmaf_rn(a.sqrtm_f, y, __uint_as_float(c.x)), a.invw_f);
            const float dist = fabsf(tf - rintf(tf));  // exact (Sterbenz)
            const float M = fmaf(A, xm[k], fmaf(10.2f * kU32, fabsf(tf), 15.3f * kU32));
            flag = !(dist > M);
            code = __float2int_rd(tf);
          }
          if (__any_sync(0xffffffffu, flag)) {
            const uint2 sg = Sg[l];
            const ColdOut o = bin_cold<SRP>(p, flag && row < n && !bad[ri], row, t, l, code,
                                            ent + tl * cap + sg.x, int(sg.y & 0xffffu), int(sg.y >> 16),
                                            reinterpret_cast<const unsigned char *>(xs + grp * S + (ri - rl0)),
                                            zslot, lane);
            code = o.code;
            nflag += o.ev & 1;
            nchanged += (o.ev >> 1) & 1;
            novf += (o.ev >> 2) & 1;
          }
          if (SRP) {
            if (FULL && p.proj) put_out(k, row, 0, y);
            if (m <= 64) {
              if (l < 32)
                ha[k] |= uint32_t(code) << l;
              else
                hb[k] |= uint32_t(code) << (l - 32);
            } else if (code) {
              ha[k] += c.z;
              hb[k] += c.w;
              if (FULL && p.bits && row < n)
                atomicOr(reinterpret_cast<unsigned long long *>(p.bits) + (row * p.L + t) * ((m + 63) >> 6) +
                             (l >> 6),
                         1ull << (l & 63));
            }
          } else {
            if (FULL) {
              if (bad[ri]) code = INT32_MIN;
              if (p.codes || p.proj) put_out(k, row, code, y);
            }
            ha[k] += uint32_t(code) * c.z;
            hb[k] += uint32_t(code) * c.w;
          }
        }
        ++l;
      };
      auto step = [&](const QuadWords<EntT> &qw) {
        uint32_t e[4], w0;
        decode_quad<EntT>(qw, e, w0);
        const float sgn = (w0 & EntFlags<EntT>::kNeg) ? -1.f : 1.f;
        // x * (+-1) is exact: each fma is one rounded addition
        if constexpr (RPL >= 2) {
          const uint64_t s2 = pack2(sgn, sgn);
          uint64_t v0[NP], v1[NP], v2[NP], v3[NP];
          lds_x2<NP>(xb + e[0], v0);
          lds_x2<NP>(xb + e[1], v1);
          lds_x2<NP>(xb + e[2], v2);
          lds_x2<NP>(xb + e[3], v3);
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            p0[i] = ffma2(v0[i], s2, p0[i]);
            p1[i] = ffma2(v1[i], s2, p1[i]);
            p0[i] = ffma2(v2[i], s2, p0[i]);
            p1[i] = ffma2(v3[i], s2, p1[i]);
          }
        } else {
          float v0[RPL], v1[RPL], v2[RPL], v3[RPL];
          lds_x<RPL>(xb + e[0], v0);
          lds_x<RPL>(xb + e[1], v1);
          lds_x<RPL>(xb + e[2], v2);
          lds_x<RPL>(xb + e[3], v3);
#pragma unroll
          for (int i = 0; i < RPL; ++i) {
            a0[i] = __fmaf_rn(v0[i], sgn, a0[i]);
            a1[i] = __fmaf_rn(v1[i], sgn, a1[i]);
            a0[i] = __fmaf_rn(v2[i], sgn, a0[i]);
            a1[i] = __fmaf_rn(v3[i], sgn, a1[i]);
          }
        }
        if (w0 & EntFlags<EntT>::kEnd) finish_bin();
      };
      // The flat loop over the range's quads (split bins: half h takes quads
      // 2k + h; bins, and so the ranges, start at even quads and both halves
      // take the same number of steps).  The next quad's entries are loaded
      // one step ahead, so that their shared-memory latency overlaps this
      // step's operand loads.
      {
        constexpr uint32_t kStep = uint32_t(4 * sizeof(EntT)) * (HW ? 2u : 1u);  // bytes per step
        uint32_t qa = eb + (rb.y + uint32_t(h)) * uint32_t(4 * sizeof(EntT));
        const uint32_t qa_end = eb + rn.y * uint32_t(4 * sizeof(EntT));
        if (qa < qa_end) {
          QuadWords<EntT> cur;
          lds_quad_words<EntT>(qa, cur);
#pragma unroll 1
          for (; qa < qa_end; qa += kStep) {
            // one step ahead; past the range's end this reads the next
            // range's quads or the table's two spare quads, never used
            QuadWords<EntT> nxt;
            lds_quad_words<EntT>(qa + kStep, nxt);
            step(cur);
            cur = nxt;
          }
        }
      }
      // partial keys of this warp -> the (row, table) slots
#pragma unroll
      for (int k = 0; k < EPR; ++k) {
        uint2 *ks = &kacc[(re0 + k) * Lg + tl];
        if (WPT == 1) {
          *ks = make_uint2(ha[k], hb[k]);
        } else if (SRP && m <= 64) {
          if (ha[k]) atomicOr(&ks->x, ha[k]);
          if (hb[k]) atomicOr(&ks->y, hb[k]);
        } else {
          atomicAdd(&ks->x, ha[k]);
          atomicAdd(&ks->y, hb[k]);
        }
      }
      if (FULL && p.counters) {
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
      }
      if (__any_sync(0xffffffffu, novf != 0) && lane == 0) atomicOr(p.status, STATUS_OVERFLOW);
    }
    __syncthreads();
    // ---- keys of the tile: consecutive threads write consecutive rows of a table ----
    if (threadIdx.x == 0) *task_ctr = 0u;  // claimed again after the next tile's load barrier
    for (int i = threadIdx.x; i < Lg * R; i += blockDim.x) {
      const int tl = i / R, r = i - tl * R;
      const int64_t row = row0 + r;
      if (row >= n) continue;
      const uint2 k2 = kacc[r * Lg + tl];
      uint64_t key;
      if (SRP && m <= 64) {
        key = (uint64_t(k2.y) << 32) | k2.x;
        if (FULL && p.bits) p.bits[row * p.L + t0 + tl] = key;
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
      if (keys) keys[int64_t(t0 + tl) * key_ld + row] = key;
    }
    __syncthreads();
  }
}

template <bool SRP, typename EntT, int RPL, bool FULL, bool HW>
cudaError_t launch_k(const Args &a, cudaStream_t stream) {
  const dim3 grid((unsigned)(a.slots * a.pl.G)), block((unsigned)(a.pl.W * kWarp));
  cudaError_t e = cudaFuncSetAttribute(sketch_dense_kernel<SRP, EntT, RPL, FULL, HW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, a.pl.smem);
  if (e != cudaSuccess) return e;
  sketch_dense_kernel<SRP, EntT, RPL, FULL, HW><<<grid, block, a.pl.smem, stream>>>(a);
  return cudaGetLastError();
}

template <bool SRP, typename EntT, bool FULL>
cudaError_t launch_r(const Args &a, cudaStream_t stream) {
  if (a.pl.hw) {
    switch (a.pl.RPL) {
      case 2: return launch_k<SRP, EntT, 2, FULL, true>(a, stream);
      case 4: return launch_k<SRP, EntT, 4, FULL, true>(a, stream);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (a.pl.RPL) {
    case 1: return launch_k<SRP, EntT, 1, FULL, false>(a, stream);
    case 2: return launch_k<SRP, EntT, 2, FULL, false>(a, stream);
    case 4: return launch_k<SRP, EntT, 4, FULL, false>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <bool SRP, bool FULL>
cudaError_t launch_e(const Args &a, cudaStream_t stream) {
  return a.pl.es == 2 ? launch_r<SRP, uint16_t, FULL>(a, stream) : launch_r<SRP, uint32_t, FULL>(a, stream);
}

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
  const void *X = p.desc ? p.desc->X : p.X;
  uint64_t *keys = p.desc ? p.desc->keys : p.keys;
  const int64_t key_ld = p.desc ? p.desc->key_ld : p.key_ld;
  int nflag = 0, nchanged = 0, novf = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < cnt; i += int64_t(gridDim.x) * blockDim.x) {
    const int4 r = p.queue[i];
    const int64_t row = int64_t(uint32_t(r.x));
    const int t = r.y, l = r.z;
    const int64_t tl = int64_t(t) * p.m + l;
    const uint32_t start = mseg[2 * tl], np = mseg[2 * tl + 1] & 0xFFFFu, nn = mseg[2 * tl + 1] >> 16;
    const uint16_t *P = mlist + int64_t(t) * p.d * p.lc + start;
    const uint16_t *N = P + np;
    const int64_t xb = row * p.ld;
    // exact path
    int emin = 1 << 20, emax = -(1 << 20);
    for (uint32_t k = 0; k < np + nn; ++k) {
      const uint32_t v = x_bits<DT>(X, xb + P[k]);
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
          const uint32_t v = x_bits<DT>(X, xb + P[k]);
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
          y64 = __dadd_rn(y64, double(__uint_as_float(x_bits<DT>(X, xb + jp))));
          ++ip;
        } else {
          y64 = __dadd_rn(y64, -double(__uint_as_float(x_bits<DT>(X, xb + jn))));
          ++in;
        }
      }
    }
    int c64;
    if (SRP) {
      c64 = y64 > 0.0 ? 1 : 0;
    } else {
      c64 = e2lsh_code64(p, y64, tl, novf);
    }
    ++nflag;
    if (c64 == r.w) continue;
    ++nchanged;
    uint64_t *key = keys ? keys + int64_t(t) * key_ld + row : nullptr;
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
cudaError_t launch_recheck_t(const SketchLaunch &p, const uint16_t *mlist, const uint32_t *mseg, int blocks,
                             cudaStream_t stream) {
  sketch_recheck_kernel<SRP, DT><<<unsigned(blocks), 256, 0, stream>>>(p, mlist, mseg);
  return cudaGetLastError();
}

template <bool SRP>
cudaError_t launch_recheck_dt(const SketchLaunch &p, const uint16_t *mlist, const uint32_t *mseg, int blocks,
                              cudaStream_t stream) {
  switch (p.dtype) {
    case LSH_F32: return launch_recheck_t<SRP, LSH_F32>(p, mlist, mseg, blocks, stream);
    case LSH_BF16: return launch_recheck_t<SRP, LSH_BF16>(p, mlist, mseg, blocks, stream);
    case LSH_F16: return launch_recheck_t<SRP, LSH_F16>(p, mlist, mseg, blocks, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace sk
}  // namespace lsh
