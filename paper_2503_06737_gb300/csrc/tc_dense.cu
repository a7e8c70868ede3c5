// tc_dense.cu -- the dense baselines E2LSH (Definition 2) and SRP (Definition
// 3) on the 5th-generation tensor cores: Y = X G for BF16 rows X [n][d] and a
// family whose Gaussian G is stored in BF16, fused with discretisation, the
// boundary test and the key fold; an exact recheck kernel patches the rare
// entries near a bin edge (or near 0 for SRP).
//
// Main kernel: persistent, one CTA per SM; CTA b owns the 128-row tiles
// b, b + gridDim.x, ... and, for each, walks all 128-column projection tiles.
//   warp 0   TMA loads (128-byte swizzle): the row tile's K slices into 8
//            slots -- once per row tile while they fit (d <= 512 BF16, 1024
//            E4M3: the tile stays resident), else once per use, streamed --
//            and the slices of G^T through a ring of SB stages;
//   warp 1   tcgen05.mma kind::f16 (M = N = 128, K = 16, FP32 accumulate),
//            issued by one elected lane of the converged warp;
//   warps 2-17 drain the accumulators (tcgen05.ld) and run the epilogue.
// K is split into two chunks, each accumulated into its own TMEM region, and
// the accumulators are double buffered (2 x 2 x 128 of the 512 columns), so
// the MMAs of one tile overlap the epilogue of the previous one.
//
// Exactness.  Products of two BF16 values are exact in FP32.  Accumulation
// model for one chunk of s MMA steps: the error is at most 2u * s * (sum of
// |products| of the chunk) -- each step rounds once relative to a partial
// sum no larger than that -- with sum |products| <= ||x_chunk|| ||g_chunk||
// (row chunk norms from a pre-pass, column chunk norms from the host).  The
// two chunk sums are added in FP32.  Entries within that bound (widened 2%)
// of an E2LSH bin edge, or of 0 for SRP, are queued with their fast code; the
// recheck kernel computes their exact FP64 value sum_j x_j G[j][c] in
// ascending j (the oracle's) as an integer sum on a common 2^e grid, derives
// the oracle's code from it and patches code, bits and key where the fast
// code was wrong.  Every mbarrier wait is bounded; a timeout sets an error
// flag, and on that path too the producer waits (bounded) for every TMA load
// it issued and the MMA warp for a final commit of its MMAs, so that no
// asynchronous copy or MMA is in flight when the CTA releases its TMEM and
// exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "internal.h"

namespace lsh {
namespace {

constexpr int BM = 128, BN = 128, KMAX = 8, SB = 5, NCH = 2;
constexpr int BKB = 128;  // bytes of K per tile row: 64 BF16 or 128 E4M3 elements (one 128-byte swizzle row)
constexpr int kEpiWarps = 16, kThreads = 64 + 32 * kEpiWarps;
constexpr int CONST_Q = 5;  // per-column constants staged per epilogue warp: gn0, gn1, b, ka, kb
constexpr int BW = 8;       // epilogue block: columns read from TMEM at a time
// Row records: NCH chunk norms, least exponent, exponent range, FP8 row scale.
// Column records: NCH chunk norms, least exponent, exponent range, sum of
// |G_j| on the column's grid (two words).
constexpr int XNC_LD = 8, GNC_LD = kTcColRecord;
static_assert(NCH <= 2, "the chunk norms share a four-word record with the exponent range");
constexpr int TILE_A = BM * BKB, TILE_B = BN * BKB;
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr float kU = 5.9604644775390625e-08f;

struct TcArgs {
  int64_t n, mtiles, ML;
  int32_t d, m, L, srp, ktiles, ktpc, nch;
  const void *X;             // bf16 rows, or E4M3 codes (fp8) with row_scale
  const float *row_scale;
  int32_t fp8;
  int64_t ld;
  const float *Gt;           // [mL][d] FP32 copy (sequential recheck fallback)
  const int32_t *Gint;       // [mL][d] columns of G as integers on their own grids (exact recheck)
  const float *gnc;          // [mL][NCH] column chunk norms (rounded up)
  const float *xnc;          // [n][NCH] row chunk norms (widened; NaN = row not finite)
  const float *b32;
  const double *b64;
  const uint32_t *ka, *kb;
  double w;
  float invw;
  int32_t *codes;
  uint64_t *bits;
  uint64_t *keys;
  int64_t key_ld;
  float *proj;
  unsigned long long *counters;
  uint32_t *status;
  int4 *queue;        // flagged entries {row, column, fast code, 0} for the recheck kernel
  uint32_t *qcount;   // entries appended (may exceed qcap: the excess is rechecked in place)
  uint32_t qcap;
};

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ uint64_t gtimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
  uint32_t done;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(done) : "r"(su32(b)), "r"(parity) : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_try_sleep(uint64_t *b, uint32_t parity, uint32_t hint_ns) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done) : "r"(su32(b)), "r"(parity), "r"(hint_ns) : "memory");
  return done != 0;
}
// The same wait by a whole warp, with a warp-uniform answer.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *b, uint32_t parity);
// Bounded wait for the phase of the given parity: false after about two
// seconds.  hint_ns > 0 lets the thread sleep between polls (it wakes when the
// phase completes), so that waiting warps leave the issue slots to others.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, uint32_t hint_ns = 0) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtimer_ns();
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (hint_ns ? mbar_try_sleep(b, parity, hint_ns) : mbar_try(b, parity)) return true;
    if ((it & 63) == 63 && gtimer_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *b, uint32_t parity) {
  // the waiting warp sleeps until the phase completes (or 1 us passes) rather
  // than spinning on the issue slots the epilogue warps of its scheduler need
  return __all_sync(0xffffffffu, mbar_wait(b, parity, 1000));
}
// One elected lane of a converged warp arms the barrier with the expected
// bytes and issues the tile load (the predicate stays inside the asm, so the
// warp never diverges around it).
__device__ __forceinline__ void tma_2d_elect(void *dst, const CUtensorMap *map, uint64_t *bar, uint32_t bytes, int x,
                                             int y) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%2], %5;\n"
      " @e cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n}\n"
      ::"r"(su32(dst)), "l"(map), "r"(su32(bar)), "r"(x), "r"(y), "r"(bytes) : "memory");
}
template <bool FP8>
__device__ __forceinline__ void umma_elect(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  if (FP8)
    asm volatile(
        "{\n .reg .pred p, e;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
        " @e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(dt), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n .reg .pred p, e;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(dt), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void commit_elect(uint64_t *bar) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n"
      ::"r"(su32(bar)) : "memory");
}
// UMMA shared-memory descriptor: K-major operand, 128-byte swizzle, 8-row
// atoms 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3 (format 0), both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Element k of a 16-byte chunk: BF16 (eight) or E4M3 (sixteen) as a value
// M 2^E with M an integer (|M| < 256 resp. < 16); the sign separately.
__device__ __forceinline__ void elem_parts(const uint32_t (&w)[4], int k, bool fp8, int &M, int &E, uint32_t &neg) {
  if (!fp8) {
    const uint32_t h = (k & 1) ? (w[k >> 1] >> 16) : (w[k >> 1] & 0xFFFFu);
    const int e = (h >> 7) & 0xFF;
    M = int(h & 0x7F) | (min(e, 1) << 7);
    E = max(e, 1) - 134;
    neg = h >> 15;
  } else {
    const uint32_t h = (w[k >> 2] >> (8 * (k & 3))) & 0xFFu;
    const int e = (h >> 3) & 15;
    M = int(h & 7) | (min(e, 1) << 3);
    E = max(e, 1) - 10;
    neg = h >> 7;
  }
}

// FP64 value of one projection as the oracle computes it: sum_j x_j G[j][c]
// in ascending j, one IEEE rounding per operation; for an FP8 row the sum is
// over its E4M3 values and the row scale multiplies it once at the end.
// Rows are 16-byte aligned and d a multiple of the 16-byte chunk on this path.
__device__ __noinline__ double tc_fp64(const TcArgs &a, int64_t row, int64_t col) {
  const float *g = a.Gt + col * a.d;
  const int per = a.fp8 ? 16 : 8;
  const uint4 *xr = reinterpret_cast<const uint4 *>(static_cast<const char *>(a.X) + row * a.ld * (a.fp8 ? 1 : 2));
  double y = 0.0;
  for (int c = 0; c < a.d / per; ++c) {
    const uint4 xv = xr[c];
    const uint32_t w[4] = {xv.x, xv.y, xv.z, xv.w};
    for (int k = 0; k < per; ++k) {
      int M, E;
      uint32_t neg;
      elem_parts(w, k, a.fp8 != 0, M, E, neg);
      const double x = ldexp(double(neg ? -M : M), E);  // exact
      y = __dadd_rn(y, __dmul_rn(x, double(g[c * per + k])));
    }
  }
  return a.fp8 ? __dmul_rn(double(a.row_scale[row]), y) : y;
}

// The FP64 value of sum_j x_j G[j][c] (ascending j, one rounding per
// operation) computed by a group of G lanes exactly, in 64-bit fixed point.
// A BF16 value is M 2^E with M < 256 an integer; the row (pre-pass) and the
// column (family set-up) carry their least exponent and exponent range.  With
// row range Rx <= 23, column range Rg <= 23 and Rx + Rg <= 37, x_j = X_j 2^ex0
// and G_jc = G_j 2^eg0 with |X_j|, |G_j| < 2^31 and every product X_j G_j
// below 2^53.  Every partial sum of the sequential FP64 loop is then an
// integer multiple of 2^(ex0 + eg0); while each stays below 2^53 in magnitude
// it is exact, so the loop returns the exact sum -- which integer addition
// (associative) gets in any order.  The product magnitudes sum to less than
// 2^(bits of M + Rx) sum_j |G_j| (the column's sum is part of its record):
// when that is below 2^53 one pass suffices; when it is not (but below 2^62,
// so that nothing overflows) a second pass takes the partial sums of the
// ascending loop themselves.  The result is S 2^e (S below 2^53 in magnitude)
// in every lane of a group of G consecutive lanes (gl = lane within the
// group); false (the caller runs the FP64 loop) when a condition fails.  The
// whole warp calls this with the same d (the second pass is warp-uniform).
//
// X_j on the row's grid: for BF16 rows whose least exponent keeps 2^-ex0 a
// normal float, x_j 2^-ex0 is an integer below 2^31 with at most 8
// significant bits, so one multiply and one conversion give it exactly;
// otherwise (FP8 rows, rows with subnormal entries) it is assembled from the
// bit fields.
template <bool FAST>
__device__ __forceinline__ int grid_x(const uint32_t (&w)[4], int k, bool fp8, int ex0, float sx) {
  if (FAST) {
    const uint32_t h = (k & 1) ? (w[k >> 1] & 0xFFFF0000u) : (w[k >> 1] << 16);
    return __float2int_rz(__uint_as_float(h) * sx);
  }
  int M, E;
  uint32_t neg;
  elem_parts(w, k, fp8, M, E, neg);
  const int X = M << max(E - ex0, 0);  // zero stays zero
  return neg ? -X : X;
}
// First pass: the exact sum (two's complement; it wraps harmlessly when a
// condition fails).
template <int G, bool FAST>
__device__ __forceinline__ long long grid_sum(const uint4 *xr, const int4 *gr, int nch, int per, bool fp8, int ex0,
                                              float sx, int gl) {
  long long sum = 0;
#pragma unroll 2
  for (int c = gl; c < nch; c += G) {
    const uint4 xv = __ldg(xr + c);
    const uint32_t w[4] = {xv.x, xv.y, xv.z, xv.w};
    for (int h = 0; h < per; h += 8) {
      const int4 g0 = __ldg(gr + (c * per + h) / 4), g1 = __ldg(gr + (c * per + h) / 4 + 1);
      const int gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
      for (int k = 0; k < 8; ++k) sum += (long long)grid_x<FAST>(w, h + k, fp8, ex0, sx) * gv[k];
    }
  }
  return sum;
}
// Second pass: the largest partial sum of the ascending loop in magnitude.
// The lanes of a group hold consecutive chunks; a chunk's partial sums are its
// own prefix sums offset by the total of all chunks before it (an exclusive
// scan over the group plus the running total of the earlier iterations), so
// their extremes are those of its prefix sums.
template <int G, bool FAST>
__device__ __forceinline__ unsigned long long grid_max_partial(const uint4 *xr, const int4 *gr, int nch, int per,
                                                               bool fp8, int ex0, float sx, int gl, bool active) {
  long long run = 0;
  unsigned long long big = 0;
  for (int c0 = 0; c0 < nch; c0 += G) {
    const int c = c0 + gl;
    long long T = 0, qmax = 0, qmin = 0;
    if (active && c < nch) {
      const uint4 xv = __ldg(xr + c);
      const uint32_t w[4] = {xv.x, xv.y, xv.z, xv.w};
      qmax = LLONG_MIN;
      qmin = LLONG_MAX;
      for (int h = 0; h < per; h += 8) {
        const int4 g0 = __ldg(gr + (c * per + h) / 4), g1 = __ldg(gr + (c * per + h) / 4 + 1);
        const int gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          T += (long long)grid_x<FAST>(w, h + k, fp8, ex0, sx) * gv[k];
          qmax = max(qmax, T);
          qmin = min(qmin, T);
        }
      }
    }
    long long incl = T;
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const long long v = __shfl_up_sync(0xffffffffu, incl, o, G);
      if (gl >= o) incl += v;
    }
    const long long base = run + incl - T;
    if (active && c < nch) {
      const long long hi = base + qmax, lo = base + qmin;
      big = max(big, (unsigned long long)max(hi < 0 ? -hi : hi, lo < 0 ? -lo : lo));
    }
    run += __shfl_sync(0xffffffffu, incl, G - 1, G);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) big = max(big, __shfl_xor_sync(0xffffffffu, big, o));
  return big;
}
template <int G>
__device__ __forceinline__ bool exact_sum_group(const TcArgs &a, int64_t row, int64_t col, int gl, long long &S,
                                                int &e) {
  const int4 xi = __ldg(reinterpret_cast<const int4 *>(a.xnc + row * XNC_LD));
  const int4 gi = __ldg(reinterpret_cast<const int4 *>(a.gnc + col * GNC_LD));
  const uint2 gw = __ldg(reinterpret_cast<const uint2 *>(a.gnc + col * GNC_LD + 4));
  const unsigned long long gabs = (unsigned long long)gw.y << 32 | gw.x;
  const int ex0 = xi.z, rx = xi.w, eg0 = gi.z, rg = gi.w;
  const bool fp8 = a.fp8 != 0;
  const int per = fp8 ? 16 : 8;  // elements per 16-byte chunk
  const int nch = a.d / per;
  const uint4 *xr = reinterpret_cast<const uint4 *>(static_cast<const char *>(a.X) + row * a.ld * (fp8 ? 1 : 2));
  const int4 *gr = reinterpret_cast<const int4 *>(a.Gint + col * a.d);
  const bool fast = !fp8 && ex0 >= -127 && ex0 <= 126;
  const float sx = __int_as_float((127 - ex0) << 23);  // 2^-ex0 (used only when fast)
  long long sum = fast ? grid_sum<G, true>(xr, gr, nch, per, fp8, ex0, sx, gl)
                       : grid_sum<G, false>(xr, gr, nch, per, fp8, ex0, sx, gl);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  S = sum;
  e = ex0 + eg0;
  // every product below 2^53: (M bits) + Rx + (M bits) + Rg <= 53; |X_j| < 2^lx
  const int mbits = fp8 ? 4 : 8;
  const bool shape = rx <= 23 && rg <= 23 && 2 * mbits + rx + rg <= 53;
  const int lx = mbits + min(max(rx, 0), 23);  // <= 31
  const bool one = shape && gabs < (1ull << (53 - lx));
  const bool second = shape && !one && gabs < (1ull << (62 - lx));
  if (!__any_sync(0xffffffffu, second)) return one;
  const unsigned long long big = fast ? grid_max_partial<G, true>(xr, gr, nch, per, fp8, ex0, sx, gl, second)
                                      : grid_max_partial<G, false>(xr, gr, nch, per, fp8, ex0, sx, gl, second);
  return one || (second && big < (1ull << 53));
}

// The oracle's FP64 projection from an exact sum S 2^e: exact, then (FP8 rows)
// one multiply by the row scale.
__device__ __forceinline__ double y_exact(const TcArgs &a, int64_t row, long long S, int e) {
  const double y = ldexp(double(S), e);
  return a.fp8 ? __dmul_rn(double(a.row_scale[row]), y) : y;
}

// The oracle's code from the FP64 projection: SRP the sign, E2LSH
// floor(((y + b) / w)) with one IEEE rounding per operation; INT32_MIN (and
// ++novf) outside the int32 range.
__device__ __forceinline__ int code_from_fp64(const TcArgs &a, double y64, int64_t col, int &novf) {
  if (a.srp) return y64 > 0.0 ? 1 : 0;
  const double f = floor(__ddiv_rn(__dadd_rn(y64, a.b64[col]), a.w));
  if (f >= -2147483648.0 && f <= 2147483647.0) return int(f);
  ++novf;
  return INT32_MIN;
}

// Exact recheck of the flagged entries of one 16-column block, one entry at a
// time by the whole warp; patches code[] of the owning lanes.
template <bool SRP, int W>
__device__ __forceinline__ void recheck_block(const TcArgs &a, int64_t row, int col0, uint32_t fmask, int lane,
                                           int (&code)[W], int &nflag, int &nchanged, int &novf) {
  for (int j = 0; j < W; ++j) {
    uint32_t fm = __ballot_sync(0xffffffffu, (fmask >> j) & 1u);
    while (fm) {
      const int leader = __ffs(fm) - 1;
      fm &= fm - 1;
      const int64_t lrow = __shfl_sync(0xffffffffu, row, leader);
      const int64_t col = col0 + j;
      long long S;
      int e;
      const bool ok = exact_sum_group<32>(a, lrow, col, lane, S, e);
      if (lane == leader) {
        const int c64 = code_from_fp64(a, ok ? y_exact(a, lrow, S, e) : tc_fp64(a, lrow, col), col, novf);
        ++nflag;
#pragma unroll
        for (int k = 0; k < W; ++k)
          if (k == j) {
            nchanged += c64 != code[k];
            code[k] = c64;
          }
      }
    }
  }
}

// Uses of row-tile slot z (z = kt when resident, kt % KMAX when streamed)
// before the load for (local row tile mi, projection tile j, K tile kt):
// resident slots are loaded once per row tile, streamed ones once per use.
__device__ __forceinline__ uint32_t a_use(bool resident, uint32_t mi, int j, int kt, int ntn, int ktiles) {
  if (resident) return mi;
  const int z = kt % KMAX;
  const uint32_t per_tile = uint32_t((ktiles - 1 - z) / KMAX + 1);  // uses of slot z per projection tile
  return (mi * uint32_t(ntn) + uint32_t(j)) * per_tile + uint32_t(kt / KMAX);
}

// Persistent kernel: CTA b walks output tiles b, b + gridDim.x, ... (projection
// tile fastest, so the CTAs running at one time share their X tiles in L2).
// The accumulators are double buffered in TMEM: the MMA warp fills buffer
// i % 2 while the epilogue warps drain the other one.  Epilogue warp e reads
// TMEM lanes 32 (e % 4) .. +31 (the rows it may access) and the 32-column
// slice e / 4; M (the bins per table) is a compile-time power of two.
template <bool SRP, int M, bool FP8>
__global__ void __launch_bounds__(kThreads, 1) tc_dense_kernel(const __grid_constant__ CUtensorMap mapA,
                                                               const __grid_constant__ CUtensorMap mapB,
                                                               const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = smem;                        // the row tile: KMAX K-slices, resident per row tile
  unsigned char *sB = smem + KMAX * TILE_A;        // G^T K-slices: SB-stage ring
  float4 *consts = reinterpret_cast<float4 *>(smem + KMAX * TILE_A + SB * TILE_B);  // [epi warp][CONST_Q][8]
  __shared__ __align__(8) uint64_t afull[KMAX], aempty[KMAX], bfull[SB], bempty[SB], tfull[2], tempty[2], mdone;
  __shared__ uint32_t tmem_base;
  __shared__ uint2 kpart[BM][3];  // M = 64: the odd slices' partial keys; M = 128: slices 1..3
  __shared__ volatile int aborted;  // set on a timed-out wait: later waits are skipped
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int ntn = int(a.ML / BN);
  constexpr int kBKE = FP8 ? BKB : BKB / 2;  // K elements per tile (TMA coordinates are in elements)
  const bool resident = a.ktiles <= KMAX;     // the row tile fits the KMAX slots

  if (threadIdx.x == 0) {
    aborted = 0;
    for (int k = 0; k < KMAX; ++k) {
      mbar_init(&afull[k], 1);
      mbar_init(&aempty[k], 1);
    }
    for (int k = 0; k < SB; ++k) {
      mbar_init(&bfull[k], 1);
      mbar_init(&bempty[k], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);
    }
    mbar_init(&mdone, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  // Every role walks the same sequence: row tiles mt = blockIdx.x, +gridDim.x, ...
  // and, for each, the projection tiles nt = (rot + j) % ntn, j = 0 .. ntn - 1;
  // the rotation spreads the CTAs running at one time over all of G^T in L2.
  const int rot = int(blockIdx.x % ntn);
  if (warp == 0) {
    // producer: the whole warp walks the loop, one elected lane issues
    uint32_t it = 0, mi = 0, s = 0, sph = 0;  // B stage, and the parity of its current fill
    uint32_t aarm = 0, apar = 0;  // A slots loaded at least once, and the parity of each slot's last load
    bool ok = true;
    for (int64_t mt = blockIdx.x; mt < a.mtiles && ok; mt += gridDim.x, ++mi) {
      const int m0 = int(mt) * BM;
      for (int j = 0; j < ntn && ok; ++j) {
        const int n0 = ((rot + j) % ntn) * BN;
        for (int kt = 0; kt < a.ktiles; ++kt, ++it) {
          // the row tile's K slice kt lives in slot z; resident rows load it once
          // per row tile, streamed rows (d too large) for every projection tile
          const int z = resident ? kt : kt % KMAX;
          if (!resident || j == 0) {
            const uint32_t u = a_use(resident, mi, j, kt, ntn, a.ktiles);  // uses of slot z before this one
            // the slot is free once the MMA of its previous use completed
            if (__any_sync(0xffffffffu, aborted != 0) || (u >= 1 && !mbar_wait_warp(&aempty[z], (u - 1) & 1))) {
              ok = false;
              break;
            }
            tma_2d_elect(sA + z * TILE_A, &mapA, &afull[z], TILE_A, kt * kBKE, m0);
            aarm |= 1u << z;
            apar = (apar & ~(1u << z)) | ((u & 1u) << z);
          }
          if (__any_sync(0xffffffffu, aborted != 0) || (it >= SB && !mbar_wait_warp(&bempty[s], sph ^ 1))) {
            ok = false;
            break;
          }
          tma_2d_elect(sB + s * TILE_B, &mapB, &bfull[s], TILE_B, kt * kBKE, n0);
          if (++s == SB) {
            s = 0;
            sph ^= 1;
          }
        }
      }
    }
    if (!ok && lane == 0) {
      atomicOr(a.status, STATUS_TIMEOUT);
      aborted = 1;
    }
    // let every load issued land before the CTA can exit, on the normal and
    // on the aborted path (bounded waits: a load that never lands ends them)
    for (uint32_t k = 0; k < SB && k < it; ++k) {
      const uint32_t jj = it - 1 - k;
      if (!mbar_wait_warp(&bfull[jj % SB], (jj / SB) & 1)) break;
    }
    for (int z = 0; z < KMAX; ++z)
      if ((aarm >> z) & 1u) mbar_wait_warp(&afull[z], (apar >> z) & 1u);
  } else if (warp == 1) {
    // MMA issue: the whole warp walks the loop, one elected lane issues.
    // Descriptors are precomputed and advanced by adding to their address
    // field (shared addresses < 2^18 never carry out of it).
    const uint32_t idesc = FP8 ? idesc_e4m3(BM, BN) : idesc_bf16(BM, BN);
    const uint64_t adesc0 = sdesc(su32(sA)), bdesc0 = sdesc(su32(sB));
    uint32_t i = 0, mi = 0, s = 0, sph = 0;
    bool ok = true;
    for (int64_t mt = blockIdx.x; mt < a.mtiles && ok; mt += gridDim.x, ++mi) {
      for (int j = 0; j < ntn && ok; ++j, ++i) {
        const uint32_t buf = i & 1;
        if (__any_sync(0xffffffffu, aborted != 0) || (i >= 2 && !mbar_wait_warp(&tempty[buf], ((i >> 1) - 1) & 1))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t dt = tmem + buf * (NCH * BN);
        int kc = 0;  // K tile within the current chunk
        for (int kt = 0; kt < a.ktiles; ++kt) {
          const int z = resident ? kt : kt % KMAX;
          const uint32_t u = a_use(resident, mi, j, kt, ntn, a.ktiles);
          if (((!resident || j == 0) && !mbar_wait_warp(&afull[z], u & 1)) || !mbar_wait_warp(&bfull[s], sph)) {
            ok = false;
            break;
          }
          const uint64_t ad = adesc0 + uint64_t(z * (TILE_A >> 4)), bd = bdesc0 + uint64_t(s * (TILE_B >> 4));
          // four MMAs of 32 bytes of K each (K = 16 BF16 or 32 E4M3 elements)
#pragma unroll
          for (int k = 0; k < 4; ++k)
            umma_elect<FP8>(dt, ad + uint64_t(2 * k), bd + uint64_t(2 * k), idesc, (kc == 0 && k == 0) ? 0u : 1u);
          commit_elect(&bempty[s]);
          if (!resident || j == ntn - 1) commit_elect(&aempty[z]);
          if (++s == SB) {
            s = 0;
            sph ^= 1;
          }
          if (++kc == a.ktpc) {
            kc = 0;
            dt += BN;  // the next chunk's accumulator
          }
        }
        if (!ok) break;
        commit_elect(&tfull[buf]);
      }
    }
    if (!ok && lane == 0) {
      atomicOr(a.status, STATUS_TIMEOUT);
      aborted = 1;
    }
    // on the normal and on the aborted path: one more commit tracks every MMA
    // this warp issued; wait for it so that none is in flight at dealloc
    commit_elect(&mdone);
    mbar_wait_warp(&mdone, 0);
  } else {
    const int e = warp - 2;
    const int q = warp % 4;
    const int slice = e / 4;
    // Error bound of an entry: E = xs0 g0 + xs1 g1 with xs_c = kE (steps + 1.01) ||x_c||
    // and g_c = ||g_c|| -- the chunk sums' own rounding (kE steps ||x_c|| ||g_c||)
    // plus that of adding them (kE (|c0| + |c1|) <= kE 1.01 sum_c ||x_c|| ||g_c||).
    // E2LSH folds 1.0001 / w into g_c: the bound on t is then xs0 g0 + xs1 g1
    // + 10.2 u |t| + 15.3 u.
    const float steps = float(a.ktpc * 4);  // MMA steps per K chunk
    const float kE = 2.f * kU * 1.02f;
    const float invw = a.invw, gscale = SRP ? 1.f : a.invw * 1.0001f;
    // per-column constants of this warp's slice: [g0 x8][g1 x8][b x8][ka x8][kb x8] as float4
    float4 *cw = consts + e * (CONST_Q * 8);
    int nflag = 0, nchanged = 0, novf = 0, nbad = 0;
    const int64_t Tend = a.mtiles * ntn;
    auto next_tile = [&](int64_t T) { return T + (((T + 1) % ntn == 0) ? int64_t(gridDim.x - 1) * ntn + 1 : 1); };
    // the next tile's constants are loaded while this one is processed
    float pg0 = 0.f, pg1 = 0.f, pb = 0.f, pka = 0.f, pkb = 0.f, px0 = 0.f, px1 = 0.f, psc = 1.f;
    auto prefetch = [&](int64_t T) {
      if (T >= Tend) return;
      const int col = int((rot + T % ntn) % ntn) * BN + slice * 32 + lane;
      const int64_t prow = (T / ntn) * BM + q * 32 + lane;
      const float4 gq = __ldg(reinterpret_cast<const float4 *>(a.gnc + int64_t(col) * GNC_LD));
      pg0 = gq.x;
      pg1 = gq.y;
      if (!SRP) {
        pb = __ldg(a.b32 + col);
        pka = __uint_as_float(__ldg(a.ka + col));
        pkb = __uint_as_float(__ldg(a.kb + col));
      }
      px0 = px1 = 0.f;
      psc = 1.f;
      if (prow < a.n) {
        const float2 xv = __ldg(reinterpret_cast<const float2 *>(a.xnc + prow * XNC_LD));
        px0 = xv.x;
        px1 = xv.y;
        if (FP8) psc = __ldg(a.xnc + prow * XNC_LD + 4);  // the row scale (NaN-checked by the pre-pass)
      }
    };
    prefetch(int64_t(blockIdx.x) * ntn);
    uint32_t i = 0;
    for (int64_t T = int64_t(blockIdx.x) * ntn; T < Tend; T = next_tile(T), ++i) {
      const uint32_t buf = i & 1;
      const int64_t row = int64_t(T / ntn) * BM + q * 32 + lane;
      const int n0 = int((rot + T % ntn) % ntn) * BN + slice * 32;
      {
        float *cf = reinterpret_cast<float *>(cw);
        __syncwarp();
        cf[0 * 32 + lane] = pg0 * gscale;
        cf[1 * 32 + lane] = pg1 * gscale;
        if (!SRP) {
          cf[2 * 32 + lane] = pb;
          cf[3 * 32 + lane] = pka;
          cf[4 * 32 + lane] = pkb;
        }
        __syncwarp();
      }
      const bool valid = row < a.n;
      const bool bad = valid && !(isfinite(px0) && isfinite(px1));
      // FP8 rows: the accumulator holds q.G, the projection is scale * that
      const float rsc = psc, ars = fabsf(psc);
      const float xs[NCH] = {kE * (steps + 1.01f) * px0 * ars, kE * (steps + 1.01f) * px1 * ars};
      if (bad && n0 == 0) ++nbad;
      prefetch(next_tile(T));
      // on a timeout the warp goes on without waiting (the status reports the
      // failure), so that every epilogue warp reaches the same named barriers
      if (!aborted && !mbar_wait(&tfull[buf], (i >> 1) & 1, 2000)) {
        atomicOr(a.status, STATUS_TIMEOUT);
        aborted = 1;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + buf * (NCH * BN) + slice * 32;
      uint32_t ha = 0, hb = 0, word = 0;
#pragma unroll 1
      for (int blk = 0; blk < 32 / BW; ++blk) {
        float ch[NCH][BW];
        {
          uint32_t r0[BW], r1[BW];
          tmem_ld8_nowait(taddr + blk * BW, r0);
          if (a.nch > 1) tmem_ld8_nowait(taddr + BN + blk * BW, r1);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < BW; ++j) {
            ch[0][j] = __uint_as_float(r0[j]);
            ch[1][j] = a.nch > 1 ? __uint_as_float(r1[j]) : 0.f;
          }
        }
        if (blk == 32 / BW - 1) {
          // every accumulator of this buffer is in registers: hand it back to the MMA warp
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[buf]);
        }
        const int col0 = n0 + blk * BW;
        int code[BW];
        uint32_t fmask = 0;
        // 1. fast codes and the entries within the error bound
#pragma unroll
        for (int g4 = 0; g4 < BW / 4; ++g4) {
          const int q4 = blk * (BW / 4) + g4;  // float4 index within the slice
          const float4 g0 = cw[0 * 8 + q4], g1 = cw[1 * 8 + q4];
          float4 bb = make_float4(0.f, 0.f, 0.f, 0.f);
          if (!SRP) bb = cw[2 * 8 + q4];
          const float gg0[4] = {g0.x, g0.y, g0.z, g0.w}, gg1[4] = {g1.x, g1.y, g1.z, g1.w};
          const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = g4 * 4 + u;
            // FP8: the scale multiply adds one rounding, u |y| (<= u (|t| + 1) w): wider constants
            const float y = FP8 ? __fmul_rn(rsc, ch[0][j] + ch[1][j]) : ch[0][j] + ch[1][j];
            bool flag;
            if (SRP) {
              const float E = fmaf(xs[0], gg0[u], xs[1] * gg1[u]);
              code[j] = y > 0.f ? 1 : 0;
              flag = !((FP8 ? fabsf(y) * (1.f - 2.f * kU) : fabsf(y)) > E);
            } else {
              const float tf = __fmul_rn(y + bv[u], invw);
              const float dist = fabsf(tf - rintf(tf));  // exact
              const float Mb = fmaf(xs[0], gg0[u], fmaf(xs[1], gg1[u], fmaf((FP8 ? 11.3f : 10.2f) * kU, fabsf(tf),
                                                                             (FP8 ? 16.4f : 15.3f) * kU)));
              code[j] = __float2int_rd(tf);
              flag = !(dist > Mb && fabsf(tf) < 4194304.f);
            }
            if (flag) fmask |= 1u << j;
          }
        }
        if (a.proj && valid)
#pragma unroll
          for (int j = 0; j < BW; j += 4)
            *reinterpret_cast<float4 *>(a.proj + row * a.ML + col0 + j) =
                FP8 ? make_float4(__fmul_rn(rsc, ch[0][j] + ch[1][j]), __fmul_rn(rsc, ch[0][j + 1] + ch[1][j + 1]),
                                  __fmul_rn(rsc, ch[0][j + 2] + ch[1][j + 2]), __fmul_rn(rsc, ch[0][j + 3] + ch[1][j + 3]))
                    : make_float4(ch[0][j] + ch[1][j], ch[0][j + 1] + ch[1][j + 1], ch[0][j + 2] + ch[1][j + 2],
                                  ch[0][j + 3] + ch[1][j + 3]);
        if (!valid || bad) fmask = 0;
        // 2. the rare slow path: queue the flagged entries for the recheck
        //    kernel; entries beyond the queue's capacity are rechecked here
        if (__any_sync(0xffffffffu, fmask != 0)) {
          const uint32_t cnt = __popc(fmask);
          uint32_t incl = cnt;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
          }
          uint32_t base = 0;
          if (lane == 31) base = atomicAdd(a.qcount, incl);
          uint32_t pos = __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
          uint32_t over = 0;
#pragma unroll
          for (int j = 0; j < BW; ++j)
            if ((fmask >> j) & 1u) {
              if (pos < a.qcap) a.queue[pos] = make_int4(int(row), col0 + j, code[j], 0);
              else over |= 1u << j;
              ++pos;
            }
          if (__any_sync(0xffffffffu, over != 0))
            recheck_block<SRP, BW>(a, row, col0, over, lane, code, nflag, nchanged, novf);
        }
        // 3. codes out, key fold
        if (!SRP && a.codes && valid) {
          int4 *dst = reinterpret_cast<int4 *>(a.codes + row * a.ML + col0);
#pragma unroll
          for (int j = 0; j < BW; j += 4)
            dst[j / 4] = bad ? make_int4(INT32_MIN, INT32_MIN, INT32_MIN, INT32_MIN)
                             : make_int4(code[j], code[j + 1], code[j + 2], code[j + 3]);
        }
        uint32_t wb = 0;  // SRP bits of this block
#pragma unroll
        for (int g4 = 0; g4 < BW / 4; ++g4) {
          const int q4 = blk * (BW / 4) + g4;
          uint4 kav = make_uint4(0, 0, 0, 0), kbv = make_uint4(0, 0, 0, 0);
          if (!SRP) {
            const float4 fa = cw[3 * 8 + q4], fb = cw[4 * 8 + q4];
            kav = make_uint4(__float_as_uint(fa.x), __float_as_uint(fa.y), __float_as_uint(fa.z), __float_as_uint(fa.w));
            kbv = make_uint4(__float_as_uint(fb.x), __float_as_uint(fb.y), __float_as_uint(fb.z), __float_as_uint(fb.w));
          }
          const uint32_t kav4[4] = {kav.x, kav.y, kav.z, kav.w}, kbv4[4] = {kbv.x, kbv.y, kbv.z, kbv.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = g4 * 4 + u;  // column within the block (static)
            if (SRP) {
              wb |= uint32_t(code[j]) << j;
            } else {
              ha += uint32_t(code[j]) * kav4[u];
              hb += uint32_t(code[j]) * kbv4[u];
            }
            // does a table end at this column?  static for M <= BW, one test per block otherwise
            const bool ends = M <= BW ? (j % M == M - 1) : (j == BW - 1 && ((blk + 1) * BW) % M == 0);
            if (ends && M <= 32) {
              const int jj = blk * BW + j;  // column within the slice
              uint64_t bitsv = 0;
              if (SRP) {
                const uint32_t wfull = word | (wb << (blk * BW));
                bitsv = uint64_t(wfull >> (jj + 1 - M)) & (M == 32 ? 0xFFFFFFFFull : ((1ull << (M & 31)) - 1));
              }
              if (valid) {
                const int t = (n0 + jj) / M;
                if (SRP && a.bits) a.bits[row * a.L + t] = bitsv;
                if (a.keys) a.keys[int64_t(t) * a.key_ld + row] = bad ? ~0ull : (SRP ? bitsv : ((uint64_t(ha) << 32) | hb));
              }
              ha = hb = 0;
            }
          }
        }
        if (SRP) word |= wb << (blk * BW);
      }
      if (M == 64) {
        // a table spans slices (0, 1) or (2, 3): the odd slice hands its partial key to the even one
        const int r = q * 32 + lane;
        if (slice & 1) kpart[r][slice >> 1] = make_uint2(SRP ? word : ha, hb);
        asm volatile("bar.sync 1, %0;" ::"r"(kEpiWarps * 32) : "memory");
        if (!(slice & 1) && valid) {
          const uint2 o = kpart[r][slice >> 1];
          const int t = n0 / 64;
          uint64_t key;
          if (SRP) {
            key = uint64_t(word) | (uint64_t(o.x) << 32);
            if (a.bits) a.bits[row * a.L + t] = key;
          } else {
            key = (uint64_t(ha + o.x) << 32) | (hb + o.y);
          }
          if (bad) key = ~0ull;
          if (a.keys) a.keys[int64_t(t) * a.key_ld + row] = key;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kEpiWarps * 32) : "memory");
      }
      if (M == 128) {
        // E2LSH only: one table spans the four slices; slices 1..3 hand their
        // partial sums to slice 0 (the key is a sum mod 2^32 in each half)
        static_assert(M != 128 || !SRP, "m = 128 on the tensor cores is E2LSH only");
        const int r = q * 32 + lane;
        if (slice != 0) kpart[r][slice - 1] = make_uint2(ha, hb);
        asm volatile("bar.sync 1, %0;" ::"r"(kEpiWarps * 32) : "memory");
        if (slice == 0 && valid && a.keys) {
          const uint2 o1 = kpart[r][0], o2 = kpart[r][1], o3 = kpart[r][2];
          const uint64_t key = (uint64_t(ha + o1.x + o2.x + o3.x) << 32) | (hb + o1.y + o2.y + o3.y);
          a.keys[int64_t(n0 / 128) * a.key_ld + row] = bad ? ~0ull : key;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kEpiWarps * 32) : "memory");
      }
    }
    if (nbad) {
      if (a.counters) atomicAdd(a.counters + CNT_NONFINITE, (unsigned long long)nbad);
      atomicOr(a.status, STATUS_NONFINITE);
    }
    if (a.counters) {
      if (nflag) atomicAdd(a.counters + CNT_FLAGGED, (unsigned long long)nflag);
      if (nchanged) atomicAdd(a.counters + CNT_CHANGED, (unsigned long long)nchanged);
      if (novf) atomicAdd(a.counters + CNT_OVERFLOW, (unsigned long long)novf);
    }
    if (novf) atomicOr(a.status, STATUS_OVERFLOW);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// Grouping of the recheck queue by row (a counting sort): the entries of one
// row end up adjacent, so the recheck warps that take them read the row from
// HBM once and from L1 after that.  Order inside a row is immaterial.
__global__ void __launch_bounds__(256) queue_row_count(const int4 *__restrict__ queue,
                                                       const uint32_t *__restrict__ qcount, uint32_t qcap,
                                                       uint32_t *__restrict__ cnt) {
  const int64_t c = min(int64_t(*qcount), int64_t(qcap));
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < c; i += int64_t(gridDim.x) * blockDim.x)
    atomicAdd(&cnt[uint32_t(queue[i].x)], 1u);
}

// Exclusive scan of cnt[0..n) in place over kScanBlocks blocks of 1024
// threads, in two launches.  Block b owns a contiguous segment; inside it each
// warp owns a contiguous run read 32 words at a time (eight loads in flight).
// scan_row_counts<false> writes each block's total to sums[b];
// scan_row_counts<true> scans the totals of the blocks before it and rewrites
// its segment with exclusive prefixes.
constexpr int kScanBlocks = 128;
template <bool WRITE>
__global__ void __launch_bounds__(1024) scan_row_counts(uint32_t *__restrict__ cnt, int64_t n,
                                                        uint32_t *__restrict__ sums) {
  __shared__ uint32_t ws[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t bseg = (n + kScanBlocks - 1) / kScanBlocks;
  const int64_t b0 = int64_t(blockIdx.x) * bseg, b1 = min(b0 + bseg, n);
  const int64_t seg = ((bseg + 31) / 32 + 31) & ~int64_t(31);
  const int64_t beg = b0 + int64_t(warp) * seg, end = min(beg + seg, b1);
  constexpr int B = 8;
  uint32_t s = 0;
  for (int64_t i0 = beg; i0 < end; i0 += 32 * B) {
    uint32_t v[B];
#pragma unroll
    for (int k = 0; k < B; ++k) v[k] = i0 + k * 32 + lane < end ? cnt[i0 + k * 32 + lane] : 0u;
#pragma unroll
    for (int k = 0; k < B; ++k) s += v[k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) ws[warp] = s;
  __syncthreads();
  if (warp == 0) {
    const uint32_t x = ws[lane];
    uint32_t y = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += u;
    }
    ws[lane] = y - x;  // exclusive prefix of the warps
    if (!WRITE && lane == 31) sums[blockIdx.x] = y;
  }
  if (!WRITE) return;
  // the totals of the blocks before this one (at most kScanBlocks words)
  if (warp == 1) {
    uint32_t t = 0;
    for (int i = lane; i < int(blockIdx.x); i += 32) t += sums[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) ws[32] = t;
  }
  __syncthreads();
  uint32_t run = ws[32] + ws[warp];
  for (int64_t i0 = beg; i0 < end; i0 += 32 * B) {
    uint32_t v[B];
#pragma unroll
    for (int k = 0; k < B; ++k) v[k] = i0 + k * 32 + lane < end ? cnt[i0 + k * 32 + lane] : 0u;
#pragma unroll
    for (int k = 0; k < B; ++k) {
      uint32_t x = v[k];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
      }
      if (i0 + k * 32 + lane < end) cnt[i0 + k * 32 + lane] = run + x - v[k];
      run += __shfl_sync(0xffffffffu, x, 31);
    }
  }
}

__global__ void __launch_bounds__(256) queue_row_scatter(const int4 *__restrict__ queue,
                                                         const uint32_t *__restrict__ qcount, uint32_t qcap,
                                                         uint32_t *__restrict__ off, int4 *__restrict__ out) {
  const int64_t c = min(int64_t(*qcount), int64_t(qcap));
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < c; i += int64_t(gridDim.x) * blockDim.x) {
    const int4 r = queue[i];
    out[atomicAdd(&off[uint32_t(r.x)], 1u)] = r;
  }
}

// The queued entries, 32 to a warp: the whole warp computes the exact sum of
// each entry in turn (lane k keeps entry k's), then every lane converts and
// discretises its own entry -- the FP64 steps run once for 32 entries -- and
// patches, where the fast code was wrong, the code, the SRP bits and the key.
// E2LSH keys are sums mod 2^32 in both halves, so a changed code c -> c' adds
// (c' - c) ka and (c' - c) kb.  Entries whose exactness condition fails take
// the sequential FP64 loop in their own lane.
__global__ void __launch_bounds__(256) tc_recheck_kernel(const TcArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t cnt = min(*a.qcount, a.qcap);
  int nflag = 0, nchanged = 0, novf = 0;
  for (int64_t base = w0 * 32; base < cnt; base += nw * 32) {
    const bool mine = base + lane < cnt;
    const int4 r = mine ? a.queue[base + lane] : make_int4(0, 0, 0, 0);
    const int nb = int(min(int64_t(32), cnt - base));
    long long Sm = 0;
    int em = 0;
    bool okm = false;
    // four entries at a time, eight lanes each: entry 4k + lane / 8
    for (int k = 0; k < (nb + 3) / 4; ++k) {
      const int src = min(4 * k + (lane >> 3), nb - 1);
      const int64_t row = __shfl_sync(0xffffffffu, r.x, src), col = __shfl_sync(0xffffffffu, r.y, src);
      long long S;
      int e;
      const bool ok = exact_sum_group<8>(a, row, col, lane & 7, S, e);
      // lane 4k + g takes the result of group g (held by its lane 8g)
      const int from = (min(max(lane - 4 * k, 0), 3)) * 8;
      const long long Sg = __shfl_sync(0xffffffffu, S, from);
      const int eg = __shfl_sync(0xffffffffu, e, from);
      const bool okg = __shfl_sync(0xffffffffu, ok ? 1 : 0, from) != 0;
      if (lane >= 4 * k && lane < 4 * k + 4) {
        Sm = Sg;
        em = eg;
        okm = okg;
      }
    }
    if (mine) {
      const int64_t row = r.x, col = r.y;
      const int c64 = code_from_fp64(a, okm ? y_exact(a, row, Sm, em) : tc_fp64(a, row, col), col, novf);
      ++nflag;
      if (c64 != r.z) {
        ++nchanged;
        const int t = int(col / a.m), l = int(col - int64_t(t) * a.m);
        uint64_t *key = a.keys ? a.keys + int64_t(t) * a.key_ld + row : nullptr;
        if (a.srp) {
          if (key) atomicXor(reinterpret_cast<unsigned long long *>(key), 1ull << l);
          if (a.bits) atomicXor(reinterpret_cast<unsigned long long *>(a.bits + row * a.L + t), 1ull << l);
        } else {
          if (a.codes) a.codes[row * a.ML + col] = c64;
          const uint32_t dc = uint32_t(c64) - uint32_t(r.z);
          if (key) {
            atomicAdd(reinterpret_cast<unsigned int *>(key) + 1, dc * a.ka[col]);
            atomicAdd(reinterpret_cast<unsigned int *>(key), dc * a.kb[col]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nflag += __shfl_xor_sync(0xffffffffu, nflag, o);
    nchanged += __shfl_xor_sync(0xffffffffu, nchanged, o);
    novf += __shfl_xor_sync(0xffffffffu, novf, o);
  }
  if (lane == 0) {
    if (a.counters) {
      if (nflag) atomicAdd(a.counters + CNT_FLAGGED, (unsigned long long)nflag);
      if (nchanged) atomicAdd(a.counters + CNT_CHANGED, (unsigned long long)nchanged);
      if (novf) atomicAdd(a.counters + CNT_OVERFLOW, (unsigned long long)novf);
    }
    if (novf) atomicOr(a.status, STATUS_OVERFLOW);
  }
}

// Row records: chunk norms ||x_chunk|| widened to an upper bound (NaN when
// the row -- or its FP8 scale -- is not finite), then the least exponent and
// the exponent range of the nonzero coordinates (x = M 2^E, M an integer),
// then the FP8 row scale.  FP8 rows are measured unscaled (the accumulator
// holds q.G).  Warp per row, 16-byte loads (d and the row stride are
// multiples of the 16-byte chunk on this path).
__global__ void __launch_bounds__(256) row_chunk_norms(const void *X, int fp8, const float *row_scale, int64_t n,
                                                       int d, int64_t ld, int chunk_len, float *out) {
  const int64_t row = int64_t(blockIdx.x) * 8 + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (row >= n) return;
  float s[NCH];
#pragma unroll
  for (int cc = 0; cc < NCH; ++cc) s[cc] = 0.f;
  bool fin = true;
  int emin = 1 << 20, emax = -(1 << 20);
  const int per = fp8 ? 16 : 8;
  const uint4 *xr = reinterpret_cast<const uint4 *>(static_cast<const char *>(X) + row * ld * (fp8 ? 1 : 2));
  for (int c = lane; c < d / per; c += 32) {
    const uint4 v4 = xr[c];
    const uint32_t w[4] = {v4.x, v4.y, v4.z, v4.w};
    const int ch = min((c * per) / chunk_len, NCH - 1);
    float acc = 0.f;
    for (int k = 0; k < per; ++k) {
      int M, E;
      uint32_t neg;
      elem_parts(w, k, fp8 != 0, M, E, neg);
      float v;
      if (!fp8) {
        const uint32_t h = (k & 1) ? (w[k >> 1] >> 16) : (w[k >> 1] & 0xFFFFu);
        v = __uint_as_float(h << 16);
      } else {
        const uint32_t h = (w[k >> 2] >> (8 * (k & 3))) & 0xFFu;
        v = ((h & 0x7F) == 0x7F) ? __int_as_float(0x7fc00000) : ldexpf(float(M), E);  // E4M3 NaN code
      }
      fin = fin && isfinite(v);
      acc = fmaf(v, v, acc);
      if (M) {
        emin = min(emin, E);
        emax = max(emax, E);
      }
    }
#pragma unroll
    for (int cc = 0; cc < NCH; ++cc)
      if (cc == ch) s[cc] += acc;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int cc = 0; cc < NCH; ++cc) s[cc] += __shfl_xor_sync(0xffffffffu, s[cc], o);
    emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
    emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  }
  const float sc = fp8 ? row_scale[row] : 1.f;
  const bool allfin = __all_sync(0xffffffffu, fin) && isfinite(sc);
  if (emax < emin) emin = emax = 0;  // an all-zero row
  if (lane < NCH) {
    float v = 0.f;
#pragma unroll
    for (int cc = 0; cc < NCH; ++cc)
      if (cc == lane) v = s[cc];
    // FP32 sum of squares of at most d terms: relative error below (d + 8) u
    const float widen = 1.f + float(d + 8) * kU;
    out[row * XNC_LD + lane] = allfin ? sqrtf(v * widen) * (1.f + 2.f * kU) : __int_as_float(0x7fc00000);
  } else if (lane == 2) {
    out[row * XNC_LD + 2] = __int_as_float(emin);
  } else if (lane == 3) {
    out[row * XNC_LD + 3] = __int_as_float(emax - emin);
  } else if (lane == 4) {
    out[row * XNC_LD + 4] = sc;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Tile map over a row-major [rows][K] matrix of 1- or 2-byte elements: boxes
// of 128 rows x 128 bytes (64 BF16 or 128 E4M3), 128-byte swizzle.
bool make_map(CUtensorMap *map, const void *base, int64_t rows, int K, int64_t row_stride_elems, bool fp8) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const int es = fp8 ? 1 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)row_stride_elems * es};
  cuuint32_t box[2] = {(cuuint32_t)(BKB / es), 128};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base),
             dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int tc_chunk_ktiles(int d, bool fp8) {
  const int bk = fp8 ? BKB : BKB / 2;  // elements per K tile
  const int ktiles = (d + bk - 1) / bk;
  return (ktiles + NCH - 1) / NCH;
}

// Scratch of one call: the row records [n][8] floats, the queue counter, the
// recheck queue (16 bytes an entry, one slot per 256 projections: the flag
// rate of Gaussian rows at w = 4 grows about as d^2 and is 2.3e-3 at d = 960;
// entries beyond it are rechecked inside the main kernel, slowly), and for
// the grouping by row a count per row and a second queue.
static int64_t tc_queue_cap(int64_t n, int64_t ML) {
  return std::min<int64_t>(n * ML / 256 + 65536, int64_t(1) << 28);
}
static int64_t tc_align16(int64_t b) { return (b + 15) & ~int64_t(15); }

size_t tc_dense_scratch_bytes(int64_t n, int64_t ML) {
  return size_t(tc_align16(n * XNC_LD * 4) + 16 + 2 * tc_queue_cap(n, ML) * 16 + tc_align16(n * 4) +
                4 * kScanBlocks);
}

bool tc_dense_supported(const lsh_family_desc &fd, const lsh_matrix *X) {
  const int64_t ML = int64_t(fd.m) * fd.L;
  if (!kind_is_dense(fd.kind) || !X || X->rowptr) return false;
  const bool fp8 = fd.compute == LSH_FP8_E4M3;
  // the row type is the family's operand type (the MMA takes one type for both)
  if (!((fd.compute == LSH_BF16 && X->dtype == LSH_BF16) || (fp8 && X->dtype == LSH_FP8_E4M3 && X->row_scale)))
    return false;
  const int per = fp8 ? 16 : 8;  // elements per 16 bytes (TMA rows and strides)
  if (fd.d % per != 0 || X->ld % per != 0 || (reinterpret_cast<uintptr_t>(X->values) & 15) != 0) return false;
  // a 32-column slice, a pair of them, or (E2LSH, m = 128) the whole 128-column tile holds whole tables
  if (ML % BN != 0 || (64 % fd.m != 0 && !(fd.m == 128 && fd.kind == LSH_E2LSH))) return false;
  if (fp8 && fd.m < 8) return false;
  if (fd.d > 16384) return false;  // larger rows stream their K slices; bounded for the scratch records
  if (X->n > (int64_t(1) << 31) - BM || (X->n + BM - 1) / BM > 2147483647) return false;
  return encode_fn() != nullptr;
}

cudaError_t launch_tc_dense(const SketchLaunch &p, const void *Gtc, const float *Gt, const float *gnc,
                            const int32_t *Gint, void *scratch, cudaStream_t stream) {
  if (p.n <= 0) return cudaSuccess;
  const bool fp8 = p.dtype == LSH_FP8_E4M3;
  const int bk = fp8 ? BKB : BKB / 2;
  const int ktiles = (p.d + bk - 1) / bk;
  const int ktpc = tc_chunk_ktiles(p.d, fp8);
  const int64_t ML = int64_t(p.m) * p.L;
  float *xnc_scratch = static_cast<float *>(scratch);
  uint32_t *qcount = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + tc_align16(p.n * XNC_LD * 4));
  int4 *queue = reinterpret_cast<int4 *>(qcount + 4);
  const int64_t qcap = tc_queue_cap(p.n, int64_t(p.m) * p.L);
  int4 *queue_by_row = queue + qcap;
  uint32_t *row_cnt = reinterpret_cast<uint32_t *>(queue_by_row + qcap);
  uint32_t *scan_sums = row_cnt + tc_align16(p.n * 4) / 4;  // [kScanBlocks]
  cudaError_t e = cudaMemsetAsync(qcount, 0, 16, stream);
  if (e != cudaSuccess) return e;
  row_chunk_norms<<<(unsigned)((p.n + 7) / 8), 256, 0, stream>>>(p.X, fp8 ? 1 : 0, p.row_scale, p.n, p.d, p.ld,
                                                                   ktpc * bk, xnc_scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap mA, mB;
  if (!make_map(&mA, p.X, p.n, p.d, p.ld, fp8) || !make_map(&mB, Gtc, ML, p.d, p.d, fp8))
    return cudaErrorInvalidValue;
  TcArgs a{};
  a.n = p.n;
  a.mtiles = (p.n + BM - 1) / BM;
  a.ML = ML;
  a.d = p.d;
  a.m = p.m;
  a.L = p.L;
  a.srp = kind_is_srp(p.kind) ? 1 : 0;
  a.ktiles = ktiles;
  a.ktpc = ktpc;
  a.nch = (ktiles + ktpc - 1) / ktpc;
  a.X = p.X;
  a.row_scale = p.row_scale;
  a.fp8 = fp8 ? 1 : 0;
  a.ld = p.ld;
  a.Gt = Gt;
  a.Gint = Gint;
  a.gnc = gnc;
  a.xnc = xnc_scratch;
  a.b32 = p.b32;
  a.b64 = p.b64;
  a.ka = p.ka;
  a.kb = p.kb;
  a.w = p.w;
  a.invw = float(1.0 / p.w);
  a.codes = p.codes;
  a.bits = p.bits;
  a.keys = p.keys;
  a.key_ld = p.key_ld;
  a.proj = p.proj;
  a.counters = p.counters;
  a.status = p.status;
  a.queue = queue;
  a.qcount = qcount;
  a.qcap = uint32_t(tc_queue_cap(p.n, ML));
  const int smem = KMAX * TILE_A + SB * TILE_B + 1024 + kEpiWarps * CONST_Q * 8 * 16;
  void (*kern)(const CUtensorMap, const CUtensorMap, const TcArgs) = nullptr;
  if (!fp8) {
    switch (p.m * 2 + a.srp) {
#define LSH_TC_CASE(M)                                        \
  case 2 * M: kern = tc_dense_kernel<false, M, false>; break; \
  case 2 * M + 1: kern = tc_dense_kernel<true, M, false>; break;
      LSH_TC_CASE(1) LSH_TC_CASE(2) LSH_TC_CASE(4) LSH_TC_CASE(8) LSH_TC_CASE(16) LSH_TC_CASE(32) LSH_TC_CASE(64)
#undef LSH_TC_CASE
      case 2 * 128: kern = tc_dense_kernel<false, 128, false>; break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (p.m * 2 + a.srp) {
#define LSH_TC_CASE(M)                                       \
  case 2 * M: kern = tc_dense_kernel<false, M, true>; break; \
  case 2 * M + 1: kern = tc_dense_kernel<true, M, true>; break;
      LSH_TC_CASE(8) LSH_TC_CASE(16) LSH_TC_CASE(32) LSH_TC_CASE(64)
#undef LSH_TC_CASE
      case 2 * 128: kern = tc_dense_kernel<false, 128, true>; break;
      default: return cudaErrorInvalidValue;
    }
  }
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min<int64_t>(a.mtiles, sms);
  kern<<<grid, kThreads, smem, stream>>>(mA, mB, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the queue grouped by row, then the recheck over the grouped copy
  e = cudaMemsetAsync(row_cnt, 0, size_t(p.n) * 4, stream);
  if (e != cudaSuccess) return e;
  queue_row_count<<<unsigned(sms) * 8, 256, 0, stream>>>(queue, qcount, a.qcap, row_cnt);
  scan_row_counts<false><<<kScanBlocks, 1024, 0, stream>>>(row_cnt, p.n, scan_sums);
  scan_row_counts<true><<<kScanBlocks, 1024, 0, stream>>>(row_cnt, p.n, scan_sums);
  queue_row_scatter<<<unsigned(sms) * 8, 256, 0, stream>>>(queue, qcount, a.qcap, row_cnt, queue_by_row);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  a.queue = queue_by_row;
  tc_recheck_kernel<<<unsigned(sms) * 8, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace lsh
