// hash_csr.cu -- CS / HCS hashing of sparse (CSR) rows for all L tables
// (Definitions 4, 5, 12, 19, 25, 31 on a row whose unstored entries are 0).
//
// One warp per row, persistent grid.  The row's nonzeros are read from HBM
// once, into a per-warp shared-memory buffer (up to 256; longer rows read
// the rest from global memory for each table), with a per-nonzero lookup state
// (its column, or for HCS with N <= 2 the offsets of its mode indices in the
// per-mode tables).  Then, TB tables at a time: every lane adds s(j) v_j of
// its nonzeros into the warp's shared-memory bins of the table (one shared
// atomic per term), and lanes own bins (l = lane, lane + 32, ...) for the
// epilogue: discretise, check the error bound, fold the key.  SRP code words
// come from __ballot_sync over 32 consecutive bins.
//
// Bin lookup: count-sketch entries [d][L] = bin | neg << 15, staged in
// shared memory when they fit, else read from global memory (L2); HCS
// per-mode entries [L][sum d_k] = bin_k | neg_k << 15 are staged per CTA
// (O(N d^(1/N)) words per table), or read from the family's tables.
//
// Exactness.  The bins start at -0.0: a bin still holding -0.0 received no
// term other than -0.0 (IEEE addition turns -0 into +0 as soon as any other
// value arrives, and an exact cancellation gives +0), so its exact value is
// 0.  Any other bin of k <= nnz terms has FP32 error at most
// gamma_{k-1} sum_bin |v| <= gamma_{nnz-1} ||v||_1 whatever the order of the
// atomic additions (Higham), widened by 2% for the FP32 evaluation of the
// bound and by nnz 2^-126 for subnormals flushed by the atomics.  Flagged
// bins are recomputed by the whole warp: the terms of the bin are exact
// multiples of 2^E0 (E0 the least exponent among them), so when their
// exponents span at most 29 and their magnitudes sum below 2^53 units, every
// partial sum of the oracle's ascending FP64 loop is exact and that loop
// returns the int64 sum, which the lanes add in any order; otherwise the
// ascending FP64 loop itself runs over the row (unstored terms are zeros, so
// this equals the dense definition).
#include <algorithm>

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace lsh {
namespace {

constexpr int kWarp = 32;
constexpr int kReg = 8;        // nonzeros per lane held in registers
constexpr float kU32 = 5.9604644775390625e-08f;

struct CsrArgs {
  SketchLaunch p;
  const int64_t *rowptr;
  const int32_t *col;
  const float *val;
  const uint16_t *colmajor;        // CS: [d][L] bin | neg << 15 (global)
  const uint32_t *mseg;            // dense rows: [L][m][2] member records (word 1: n(+) | n(-) << 16)
  uint64_t dmagic[LSH_MAX_MODES];  // HCS: ceil(2^64 / d_k) (0 for d_k = 1)
  int stage;                       // entries staged in shared memory
  int tb;                          // tables per pass
  int fast2;                       // HCS, N <= 2, sum d_k < 65536: per-nonzero mode offsets
  int off_nz, off_tab, smem;
  float sqrtm_f, invw_f;
};

// Stage the lookup entries of the CTA (CS: the [d][L] column-major entries;
// HCS: the per-mode entries packed as bin | neg << 15).
__device__ void stage_entries(const CsrArgs &a, uint16_t *tab) {
  const SketchLaunch &p = a.p;
  if (p.kind == LSH_CS_E2LSH || p.kind == LSH_CS_SRP) {
    const int64_t cnt = int64_t(p.d) * p.L;
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) tab[i] = a.colmajor[i];
  } else {
    const int64_t cnt = int64_t(p.L) * p.dsum;
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x)
      tab[i] = uint16_t(p.bins[i] | (p.signs[i] < 0 ? 0x8000u : 0u));
  }
}

// Mode index i_k of column c (first mode fastest): the quotient by d_k is the
// high word of c ceil(2^64 / d_k), exact for every 32-bit c (Lemire, Kaser
// and Kurz, "Faster remainder by direct computation", 2019).
__device__ __forceinline__ uint32_t next_mode(const CsrArgs &a, int k, uint32_t &r) {
  const uint32_t q = a.dmagic[k] ? uint32_t(__umul64hi(a.dmagic[k], uint64_t(r))) : r;
  const uint32_t ik = r - q * uint32_t(a.p.dims[k]);
  r = q;
  return ik;
}

// Per-nonzero lookup state: the column, or (HCS fast path) the offsets of its
// two mode indices in a table's concatenated mode entries.
__device__ __forceinline__ uint32_t prep_state(const CsrArgs &a, int c) {
  if (!a.fast2) return uint32_t(c);
  uint32_t r = uint32_t(c);
  const uint32_t i1 = next_mode(a, 0, r);
  if (a.p.N == 1) return i1;
  const uint32_t i2 = next_mode(a, 1, r);
  return i1 | ((uint32_t(a.p.dims[0]) + i2) << 16);
}

// Packed per-mode entry (bin | neg << 15) at offset o of table t.
__device__ __forceinline__ uint32_t mode_entry(const CsrArgs &a, const uint16_t *tab, int t, uint32_t o) {
  const int64_t i = int64_t(t) * a.p.dsum + o;
  if (tab) return tab[i];
  return uint32_t(a.p.bins[i]) | (a.p.signs[i] < 0 ? 0x8000u : 0u);
}

// bin | neg << 31 of a nonzero in table t.
__device__ __forceinline__ uint32_t lookup(const CsrArgs &a, const uint16_t *tab, int t, uint32_t s) {
  const SketchLaunch &p = a.p;
  if (p.kind == LSH_CS_E2LSH || p.kind == LSH_CS_SRP) {
    const int64_t i = int64_t(s) * p.L + t;
    const uint32_t e = tab ? uint32_t(tab[i]) : uint32_t(__ldg(a.colmajor + i));
    return (e & 0x7fffu) | ((e >> 15) << 31);
  }
  if (a.fast2) {
    const uint32_t e1 = mode_entry(a, tab, t, s & 0xffffu);
    if (p.N == 1) return (e1 & 0x7fffu) | ((e1 >> 15) << 31);
    const uint32_t e2 = mode_entry(a, tab, t, s >> 16);
    return ((e1 & 0x7fffu) + uint32_t(p.mdims[0]) * (e2 & 0x7fffu)) | (((e1 ^ e2) >> 15) << 31);
  }
  uint32_t r = s, bin = 0, neg = 0, off = 0, stride = 1;
  for (int k = 0; k < p.N; ++k) {
    const uint32_t e = mode_entry(a, tab, t, off + next_mode(a, k, r));
    bin += (e & 0x7fffu) * stride;
    neg ^= e >> 15;
    stride *= uint32_t(p.mdims[k]);
    off += uint32_t(p.dims[k]);
  }
  return bin | (neg << 31);
}

// Element e of the row being hashed.  SRC 0: the CSR row (column and value
// of stored entry e); SRC 1 + dtype: a dense row of that element type, whose
// entry e is coordinate e (xrow = row * ld).
template <int SRC>
__device__ __forceinline__ int nz_col(const CsrArgs &a, int64_t e) {
  return SRC == 0 ? __ldg(a.col + e) : int(e);
}
template <int SRC>
__device__ __forceinline__ float nz_val(const CsrArgs &a, int64_t xrow, int64_t e) {
  if (SRC == 0) return __ldg(a.val + e);
  if (SRC == 1 + LSH_F32) return __ldg(reinterpret_cast<const float *>(a.p.X) + xrow + e);
  const unsigned short h = __ldg(reinterpret_cast<const unsigned short *>(a.p.X) + xrow + e);
  if (SRC == 1 + LSH_BF16) return __uint_as_float(uint32_t(h) << 16);
  return __half2float(__ushort_as_half(h));
}

// Error bound of bin l of table t: CSR rows, gamma_{nnz-1} ||v||_1 of the row
// (rbound); dense rows, 1.02 gamma_{k-1} (1 + 2 gamma) k max|x| with k the
// bin's member count (Higham, as for the dense-row kernel).
template <int SRC>
__device__ __forceinline__ float bin_bound(const CsrArgs &a, int t, int l, float rbound, float xmax) {
  if (SRC == 0) return rbound;
  const uint32_t w = __ldg(a.mseg + 2 * (int64_t(t) * a.p.m + l) + 1);
  const float k = float((w & 0xffffu) + (w >> 16));
  const float g = fmaxf(k - 1.f, 0.f) * kU32;
  return 1.02f * g * (1.f + 2.f * g) * k * xmax;
}

// Exact FP64 value of bin l of table t of this warp's row (warp-collective;
// every lane returns the same value).  nz: the warp's staged nonzeros {value
// bits, lookup state}, lane's k-th at nz[32 k + lane] (kn of them), then the
// row's nonzeros from position rs + 32 kReg on are read from global memory.
template <int SRC>
__device__ __noinline__ double exact_bin(const CsrArgs &a, const uint16_t *tab, int t, uint32_t l,
                                         const uint2 *nz, int kn, int64_t rs, int64_t re, int64_t xrow, int lane) {
  const int64_t tail0 = rs + kWarp * kReg;
  int emin = 1 << 20, emax = -(1 << 20);
  for (int k = 0; k < kn; ++k) {
    if ((lookup(a, tab, t, nz[k * kWarp + lane].y) & 0x7fffffffu) == l) {
      const uint32_t u = nz[k * kWarp + lane].x;
      if (u & 0x7fffffffu) {
        const int E = max(int((u >> 23) & 0xff), 1) - 150;
        emin = min(emin, E);
        emax = max(emax, E);
      }
    }
  }
  for (int64_t e = tail0 + lane; e < re; e += kWarp) {
    const uint32_t u = __float_as_uint(nz_val<SRC>(a, xrow, e));
    if ((lookup(a, tab, t, prep_state(a, nz_col<SRC>(a, e))) & 0x7fffffffu) == l && (u & 0x7fffffffu)) {
      const int E = max(int((u >> 23) & 0xff), 1) - 150;
      emin = min(emin, E);
      emax = max(emax, E);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
    emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  }
  if (emax < emin) return 0.0;
  if (emax - emin <= 29) {
    constexpr unsigned long long kCap = 1ull << 53;
    unsigned long long sum = 0, mag = 0;
    auto add = [&](uint32_t u, uint32_t neg) {
      const int e = int((u >> 23) & 0xff);
      const unsigned long long M = (u & 0x7fffffu) | (e ? 0x800000u : 0u);
      const unsigned long long tv = M << max(max(e, 1) - 150 - emin, 0);
      sum += ((u >> 31) ^ neg) ? 0ull - tv : tv;
      mag = min(mag + tv, kCap);
    };
    for (int k = 0; k < kn; ++k) {
      const uint2 z = nz[k * kWarp + lane];
      const uint32_t e = lookup(a, tab, t, z.y);
      if ((e & 0x7fffffffu) == l) add(z.x, e >> 31);
    }
    for (int64_t e = tail0 + lane; e < re; e += kWarp) {
      const uint32_t en = lookup(a, tab, t, prep_state(a, nz_col<SRC>(a, e)));
      if ((en & 0x7fffffffu) == l) add(__float_as_uint(nz_val<SRC>(a, xrow, e)), en >> 31);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sum += __shfl_xor_sync(0xffffffffu, sum, o);
      mag += __shfl_xor_sync(0xffffffffu, mag, o);  // each lane's part <= 2^53: no overflow
    }
    if (mag < kCap) return ldexp(double((long long)sum), emin);
  }
  // the oracle's loop: ascending column order, one IEEE rounding per addition
  double y = 0.0;
  for (int64_t e = rs; e < re; ++e) {
    const uint32_t en = lookup(a, tab, t, prep_state(a, nz_col<SRC>(a, e)));
    if ((en & 0x7fffffffu) == l) {
      const double x = double(nz_val<SRC>(a, xrow, e));
      y = __dadd_rn(y, (en >> 31) ? -x : x);
    }
  }
  return y;
}

// Add the terms of one nonzero (lookup state st, value x) to the bins of the
// tables tb .. tb + nt - 1 (acc: [nt][m]).  vec4: count-sketch entries read
// from global memory four tables per 8-byte load (L and tb multiples of 4).
__device__ __forceinline__ void scatter_one(const CsrArgs &a, const uint16_t *tab, float *acc, int tb, int nt,
                                            bool vec4, uint32_t st, float x) {
  const int m = a.p.m;
  if (vec4) {
    const uint2 *src = reinterpret_cast<const uint2 *>(a.colmajor + int64_t(st) * a.p.L + tb);
    for (int g = 0; g < nt; g += 4) {
      const uint2 q = __ldg(src + (g >> 2));
      const uint32_t e[4] = {q.x & 0xffffu, q.x >> 16, q.y & 0xffffu, q.y >> 16};
#pragma unroll
      for (int i = 0; i < 4; ++i)
        atomicAdd(&acc[(g + i) * m + int(e[i] & 0x7fffu)], (e[i] >> 15) ? -x : x);
    }
    return;
  }
  for (int tt = 0; tt < nt; ++tt) {
    const uint32_t e = lookup(a, tab, tb + tt, st);
    atomicAdd(&acc[tt * m + int(e & 0x7fffffffu)], (e >> 31) ? -x : x);
  }
}

// Epilogue of one table when m is a multiple of 4: lane owns the 4 adjacent
// bins 4 lane + 128 c (c = 0, 1, ...), read and reset with 128-bit shared
// accesses; offsets and key multipliers come in 128-bit loads.  Flagged bins
// are recomputed exactly by the whole warp, one at a time.  E2LSH and SRP
// with m > 64 leave the lane's partial key sums in ha/hb; SRP with m <= 64
// leaves the bit pattern itself (every lane the same).
template <bool SRP, int SRC>
__device__ __forceinline__ void epilogue_vec4(const CsrArgs &a, const uint16_t *tab, float *A, int64_t row, int t,
                                              bool rowok, float Arow, float xmax, int64_t xrow, float sq_w,
                                              uint32_t words, const uint2 *nz,
                                              int kn, int64_t rs, int64_t re, int lane, uint32_t &ha, uint32_t &hb,
                                              int &nflag, int &nchanged, int &novf) {
  const SketchLaunch &p = a.p;
  const int m = p.m, L = p.L;
  const int64_t tm = int64_t(t) * m;
  for (int base = 0; base < m; base += 4 * kWarp) {
    const int l0 = base + 4 * lane;
    const bool inb = l0 < m;
    float4 yq = make_float4(-0.f, -0.f, -0.f, -0.f);
    if (inb) {
      float4 *Ap = reinterpret_cast<float4 *>(A + l0);
      yq = *Ap;
      *Ap = make_float4(-0.f, -0.f, -0.f, -0.f);
    }
    const float y[4] = {yq.x, yq.y, yq.z, yq.w};
    int code[4];
    uint32_t fm = 0;
    if (SRP) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool ez = __float_as_uint(y[k]) == 0x80000000u;  // exactly zero
        const bool flag = rowok && inb && !ez && !(fabsf(y[k]) > bin_bound<SRC>(a, t, l0 + k, Arow, xmax));
        fm |= uint32_t(flag) << k;
        code[k] = y[k] > 0.f ? 1 : 0;
      }
    } else {
      const float4 bq = inb ? __ldg(reinterpret_cast<const float4 *>(p.b32 + tm + l0)) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float b[4] = {bq.x, bq.y, bq.z, bq.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool ez = __float_as_uint(y[k]) == 0x80000000u;
        const float tf = __fmul_rn(__fmaf_rn(a.sqrtm_f, y[k], b[k]), a.invw_f);
        const float dist = fabsf(tf - rintf(tf));  // exact (Sterbenz)
        const float B = inb ? bin_bound<SRC>(a, t, l0 + k, Arow, xmax) : 0.f;
        const float M = fmaf(ez ? 0.f : sq_w, B, fmaf(10.2f * kU32, fabsf(tf), 15.3f * kU32));
        const bool flag = rowok && inb && !(dist > M);
        fm |= uint32_t(flag) << k;
        code[k] = __float2int_rd(tf);
      }
    }
    // exact values of the flagged bins, one bin at a time by the whole warp
    uint32_t lanes = __ballot_sync(0xffffffffu, fm != 0);
    while (lanes) {
      const int src = __ffs(lanes) - 1;
      lanes &= lanes - 1;
      uint32_t sfm = __shfl_sync(0xffffffffu, fm, src);
      while (sfm) {
        const int k = __ffs(sfm) - 1;
        sfm &= sfm - 1;
        const int l = base + 4 * src + k;
        const double y64 = exact_bin<SRC>(a, tab, t, uint32_t(l), nz, kn, rs, re, xrow, lane);
        if (lane == src) {
          int c64;
          if (SRP) {
            c64 = y64 > 0.0 ? 1 : 0;
          } else {
            const double f = floor(__ddiv_rn(__dadd_rn(__dmul_rn(p.sqrtm, y64), p.b64[tm + l]), p.w));
            if (f >= -2147483648.0 && f <= 2147483647.0) {
              c64 = int(f);
            } else {
              c64 = INT32_MIN;
              ++novf;
            }
          }
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            if (kk == k) {
              ++nflag;
              nchanged += c64 != code[kk];
              code[kk] = c64;
            }
        }
      }
    }
    if (p.proj && inb) *reinterpret_cast<float4 *>(p.proj + (row * L + t) * m + l0) = yq;
    if (SRP) {
      const uint32_t nib = uint32_t(code[0]) | uint32_t(code[1]) << 1 | uint32_t(code[2]) << 2 |
                           uint32_t(code[3]) << 3;
      if (p.bits) {  // two lanes' nibbles make one byte of the code words
        const uint32_t hi = __shfl_down_sync(0xffffffffu, nib, 1);
        if (inb && (lane & 1) == 0)
          reinterpret_cast<unsigned char *>(p.bits)[(row * L + t) * int64_t(words) * 8 + (l0 >> 3)] =
              (unsigned char)(nib | ((l0 + 4 < m ? hi : 0u) << 4));
      }
      if (!inb) continue;
      if (m <= 64) {
        if (lane < 8)
          ha |= nib << (4 * lane);
        else
          hb |= nib << (4 * (lane - 8));
      } else {
        const uint4 ka = __ldg(reinterpret_cast<const uint4 *>(p.ka + tm + l0));
        const uint4 kb = __ldg(reinterpret_cast<const uint4 *>(p.kb + tm + l0));
        ha += (code[0] ? ka.x : 0u) + (code[1] ? ka.y : 0u) + (code[2] ? ka.z : 0u) + (code[3] ? ka.w : 0u);
        hb += (code[0] ? kb.x : 0u) + (code[1] ? kb.y : 0u) + (code[2] ? kb.z : 0u) + (code[3] ? kb.w : 0u);
      }
    } else {
      if (!inb) continue;
      const uint4 ka = __ldg(reinterpret_cast<const uint4 *>(p.ka + tm + l0));
      const uint4 kb = __ldg(reinterpret_cast<const uint4 *>(p.kb + tm + l0));
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (!rowok) code[k] = INT32_MIN;
      ha += uint32_t(code[0]) * ka.x + uint32_t(code[1]) * ka.y + uint32_t(code[2]) * ka.z + uint32_t(code[3]) * ka.w;
      hb += uint32_t(code[0]) * kb.x + uint32_t(code[1]) * kb.y + uint32_t(code[2]) * kb.z + uint32_t(code[3]) * kb.w;
      if (p.codes) *reinterpret_cast<int4 *>(p.codes + (row * L + t) * m + l0) = make_int4(code[0], code[1], code[2], code[3]);
    }
  }
  if (SRP && m <= 64) {
    ha = __reduce_or_sync(0xffffffffu, ha);
    hb = __reduce_or_sync(0xffffffffu, hb);
  }
}

template <bool SRP, int SRC>
__global__ void __launch_bounds__(256, 2) sketch_csr_kernel(const __grid_constant__ CsrArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SketchLaunch &p = a.p;
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int m = p.m, L = p.L, TB = a.tb;
  float *acc = reinterpret_cast<float *>(smem) + int64_t(warp) * TB * m;  // [TB][m] bins of this warp
  uint2 *nz = reinterpret_cast<uint2 *>(smem + a.off_nz) + warp * (kWarp * kReg);  // the row's nonzeros
  const uint16_t *tab = nullptr;
  if (a.stage) {
    uint16_t *st = reinterpret_cast<uint16_t *>(smem + a.off_tab);
    stage_entries(a, st);
    tab = st;
  }
  for (int i = lane; i < TB * m; i += kWarp) acc[i] = -0.f;
  __syncthreads();
  const bool cs = p.kind == LSH_CS_E2LSH || p.kind == LSH_CS_SRP;
  const bool vec4 = cs && !a.stage && (L % 4) == 0 && (TB % 4) == 0;
  const bool vec4b = (m % 4) == 0;
  const int64_t nwarps = int64_t(gridDim.x) * nw;
  const float sq_w = a.sqrtm_f * a.invw_f;
  const uint32_t words = uint32_t((m + 63) >> 6);
  for (int64_t row = int64_t(blockIdx.x) * nw + warp; row < p.n; row += nwarps) {
    const int64_t rs = SRC == 0 ? a.rowptr[row] : 0, re = SRC == 0 ? a.rowptr[row + 1] : p.d;
    const int64_t xrow = SRC == 0 ? 0 : row * p.ld;
    const int64_t nnz = re - rs;
    // ---- the row's first 32 kReg nonzeros into this warp's shared buffer
    // (all loads in flight first); validate the row and take ||v||_1 ----
    int cc[kReg];
    float xv[kReg];
#pragma unroll
    for (int k = 0; k < kReg; ++k) {
      const int64_t e = rs + lane + int64_t(k) * kWarp;
      cc[k] = e < re ? nz_col<SRC>(a, e) : 0;
      xv[k] = e < re ? nz_val<SRC>(a, xrow, e) : 0.f;
    }
    int kn = 0;
    bool ok = nnz >= 0;
    float l1 = 0.f, xmax = 0.f;
    int carry = -1;  // the column before this 32-chunk (lane 31 of the previous one)
#pragma unroll
    for (int k = 0; k < kReg; ++k) {
      const int64_t e = rs + lane + int64_t(k) * kWarp;
      int prev = __shfl_up_sync(0xffffffffu, cc[k], 1);
      if (lane == 0) prev = carry;
      carry = __shfl_sync(0xffffffffu, cc[k], kWarp - 1);
      if (e < re) {
        const int c = cc[k];
        ok = ok && c >= 0 && c < p.d && isfinite(xv[k]) && prev < c;
        nz[k * kWarp + lane] = make_uint2(__float_as_uint(xv[k]), (c >= 0 && c < p.d) ? prep_state(a, c) : 0u);
        l1 += fabsf(xv[k]);
        xmax = fmaxf(xmax, fabsf(xv[k]));
        kn = k + 1;
      }
    }
    for (int64_t e = rs + kWarp * kReg + lane; e < re; e += kWarp) {
      const int c = nz_col<SRC>(a, e);
      const float x = nz_val<SRC>(a, xrow, e);
      ok = ok && c >= 0 && c < p.d && isfinite(x) && (SRC != 0 || a.col[e - 1] < c);
      l1 += fabsf(x);
      xmax = fmaxf(xmax, fabsf(x));
    }
    const bool rowok = __all_sync(0xffffffffu, ok);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      l1 += __shfl_xor_sync(0xffffffffu, l1, o);
      xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    }
    const float gk = float(nnz > 1 ? nnz - 1 : 0) * kU32;
    // gamma_{nnz-1} ||v||_1 (2% slack) plus one flushed subnormal per term
    const float Arow = 1.02f * gk * (1.f + 2.f * gk) * l1 + float(nnz) * 1.1754944e-38f * 1.02f;
    int nflag = 0, nchanged = 0, novf = 0;
    for (int tb = 0; tb < L; tb += TB) {
      const int nt = min(TB, L - tb);
      // ---- scatter: one shared atomic per (nonzero, table) ----
      if (rowok && vec4) {
        // count sketch from global memory: the entry loads of all the lane's
        // buffered nonzeros (four tables per 8-byte load) in flight before
        // their atomics
        constexpr int kBatch = kReg / 2;
        for (int g = 0; g < nt; g += 4) {
#pragma unroll
          for (int k0 = 0; k0 < kReg; k0 += kBatch) {
            uint2 q[kBatch];
#pragma unroll
            for (int k = 0; k < kBatch; ++k)
              if (k0 + k < kn)
                q[k] = __ldg(reinterpret_cast<const uint2 *>(a.colmajor + int64_t(nz[(k0 + k) * kWarp + lane].y) * L +
                                                             tb + g));
#pragma unroll
            for (int k = 0; k < kBatch; ++k) {
              if (k0 + k < kn) {
                const float x = __uint_as_float(nz[(k0 + k) * kWarp + lane].x);
                const uint32_t e[4] = {q[k].x & 0xffffu, q[k].x >> 16, q[k].y & 0xffffu, q[k].y >> 16};
#pragma unroll
                for (int i = 0; i < 4; ++i)
                  atomicAdd(&acc[(g + i) * m + int(e[i] & 0x7fffu)], (e[i] >> 15) ? -x : x);
              }
            }
          }
        }
      } else if (rowok) {
#pragma unroll 1
        for (int k = 0; k < kn; ++k) {
          const uint2 z = nz[k * kWarp + lane];
          scatter_one(a, tab, acc, tb, nt, vec4, z.y, __uint_as_float(z.x));
        }
      }
      if (rowok) {
        for (int64_t e = rs + kWarp * kReg + lane; e < re; e += kWarp)
          scatter_one(a, tab, acc, tb, nt, vec4, prep_state(a, nz_col<SRC>(a, e)), nz_val<SRC>(a, xrow, e));
      }
      __syncwarp();
      // ---- epilogue: lanes own bins ----
      for (int tt = 0; tt < nt; ++tt) {
        const int t = tb + tt;
        float *A = acc + tt * m;
        uint32_t ha = 0, hb = 0;
        if (vec4b) {
          epilogue_vec4<SRP, SRC>(a, tab, A, row, t, rowok, Arow, xmax, xrow, sq_w, words, nz, kn, rs, re, lane, ha,
                                  hb, nflag,
                             nchanged, novf);
        } else {
        for (int base = 0; base < m; base += kWarp) {
          const int l = base + lane;
          const bool inb = l < m;
          float y = -0.f;
          if (inb) {
            y = A[l];
            A[l] = -0.f;
          }
          const bool ez = __float_as_uint(y) == 0x80000000u;  // exactly zero
          if (SRP) {
            const bool flag = rowok && inb && !ez && !(fabsf(y) > bin_bound<SRC>(a, t, l, Arow, xmax));
            int bit = y > 0.f ? 1 : 0;
            uint32_t fm = __ballot_sync(0xffffffffu, flag);
            while (fm) {
              const int src = __ffs(fm) - 1;
              fm &= fm - 1;
              const double y64 = exact_bin<SRC>(a, tab, t, uint32_t(base + src), nz, kn, rs, re, xrow, lane);
              if (lane == src) {
                const int b64 = y64 > 0.0 ? 1 : 0;
                ++nflag;
                nchanged += b64 != bit;
                bit = b64;
              }
            }
            if (p.proj && inb) p.proj[(row * L + t) * m + l] = y;
            const uint32_t ball = __ballot_sync(0xffffffffu, inb && bit);
            if (m > 64) {
              if (inb && bit) {
                ha += __ldg(p.ka + int64_t(t) * m + l);
                hb += __ldg(p.kb + int64_t(t) * m + l);
              }
            } else {
              // m <= 64: the key is the bit pattern, assembled below
              ha |= (base == 0) ? ball : 0u;
              hb |= (base == 32) ? ball : 0u;
            }
            if (p.bits && lane == 0) {
              uint32_t *wb = reinterpret_cast<uint32_t *>(p.bits + (row * L + t) * words);
              wb[base >> 5] = ball;
            }
          } else {
            const float bl = inb ? __ldg(p.b32 + int64_t(t) * m + l) : 0.f;
            const float tf = __fmul_rn(__fmaf_rn(a.sqrtm_f, y, bl), a.invw_f);
            const float dist = fabsf(tf - rintf(tf));  // exact (Sterbenz)
            const float B = inb ? bin_bound<SRC>(a, t, l, Arow, xmax) : 0.f;
            const float M = fmaf(ez ? 0.f : sq_w, B, fmaf(10.2f * kU32, fabsf(tf), 15.3f * kU32));
            const bool flag = rowok && inb && !(dist > M);
            int code = __float2int_rd(tf);
            uint32_t fm = __ballot_sync(0xffffffffu, flag);
            while (fm) {
              const int src = __ffs(fm) - 1;
              fm &= fm - 1;
              const double y64 = exact_bin<SRC>(a, tab, t, uint32_t(base + src), nz, kn, rs, re, xrow, lane);
              if (lane == src) {
                const double t1 = __dmul_rn(p.sqrtm, y64);
                const double t2 = __dadd_rn(t1, p.b64[int64_t(t) * m + l]);
                const double f = floor(__ddiv_rn(t2, p.w));
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
            if (!rowok) code = INT32_MIN;
            if (inb) {
              ha += uint32_t(code) * __ldg(p.ka + int64_t(t) * m + l);
              hb += uint32_t(code) * __ldg(p.kb + int64_t(t) * m + l);
              if (p.codes) p.codes[(row * L + t) * m + l] = code;
              if (p.proj) p.proj[(row * L + t) * m + l] = y;
            }
          }
        }
        }
        uint64_t key;
        if (SRP && m <= 64) {
          key = (uint64_t(hb) << 32) | ha;
        } else {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            ha += __shfl_xor_sync(0xffffffffu, ha, o);
            hb += __shfl_xor_sync(0xffffffffu, hb, o);
          }
          key = (uint64_t(ha) << 32) | hb;
        }
        if (!rowok) key = ~0ull;
        if (lane == 0 && p.keys) p.keys[int64_t(t) * p.key_ld + row] = key;
      }
      __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nflag += __shfl_xor_sync(0xffffffffu, nflag, o);
      nchanged += __shfl_xor_sync(0xffffffffu, nchanged, o);
      novf += __shfl_xor_sync(0xffffffffu, novf, o);
    }
    if (lane == 0) {
      if (p.counters) {
        if (nflag) atomicAdd(p.counters + CNT_FLAGGED, (unsigned long long)nflag);
        if (nchanged) atomicAdd(p.counters + CNT_CHANGED, (unsigned long long)nchanged);
        if (novf) atomicAdd(p.counters + CNT_OVERFLOW, (unsigned long long)novf);
        if (!rowok) atomicAdd(p.counters + CNT_NONFINITE, 1ull);
      }
      if (novf) atomicOr(p.status, STATUS_OVERFLOW);
      if (!rowok) atomicOr(p.status, STATUS_NONFINITE);
    }
  }
}

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

template <bool SRP, int SRC>
cudaError_t launch_k(const CsrArgs &a, int grid, int W, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(sketch_csr_kernel<SRP, SRC>, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem);
  if (e != cudaSuccess) return e;
  sketch_csr_kernel<SRP, SRC><<<grid, W * kWarp, a.smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sketch_csr(const SketchLaunch &p, const int64_t *rowptr, const int32_t *col, const float *val,
                              const uint16_t *colmajor, const uint32_t *mseg, cudaStream_t stream) {
  if (p.n <= 0) return cudaSuccess;
  CsrArgs a{};
  a.p = p;
  a.rowptr = rowptr;
  a.col = col;
  a.val = val;
  a.colmajor = colmajor;
  a.mseg = mseg;
  a.sqrtm_f = float(p.sqrtm);
  a.invw_f = float(1.0 / p.w);
  const bool cs = p.kind == LSH_CS_E2LSH || p.kind == LSH_CS_SRP;
  for (int k = 0; k < p.N && k < LSH_MAX_MODES; ++k)
    a.dmagic[k] = p.dims[k] > 1 ? ~0ull / uint64_t(p.dims[k]) + 1 : 0;
  a.fast2 = (!cs && p.N <= 2 && p.dsum < 65536) ? 1 : 0;
  // staged entries: CS [d][L], HCS [L][sum d_k] (2 bytes each), when small
  const int64_t tab_bytes = cs ? int64_t(p.d) * p.L * 2 : int64_t(p.L) * p.dsum * 2;
  const bool stage = tab_bytes <= 64 * 1024;
  // warps per CTA and tables per pass: a warp's bins are tb * m floats.  Count
  // sketches read from global memory take four tables per pass (each
  // nonzero's entries of the four come in one 8-byte load); otherwise two.
  int W = 8;
  int tb = (cs && !stage && p.L % 4 == 0) ? 4 : std::min(p.L, 2);
  const int64_t acc_cap = 160 * 1024;
  while (int64_t(W) * tb * p.m * 4 > acc_cap) {
    if (tb > 1 && !(cs && !stage && p.L % 4 == 0)) {
      tb = 1;
    } else if (W > 1) {
      W >>= 1;
    } else {
      break;
    }
  }
  if (int64_t(W) * tb * p.m * 4 > acc_cap) return cudaErrorInvalidConfiguration;
  a.tb = tb;
  const int acc_bytes = W * tb * p.m * 4;
  a.off_nz = (acc_bytes + 15) & ~15;
  a.off_tab = a.off_nz + W * kWarp * kReg * 8;
  a.stage = stage ? 1 : 0;
  a.smem = a.off_tab + (stage ? int(tab_bytes) : 0);
  if (a.smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  int per_sm = (228 * 1024) / (a.smem + 1024);
  per_sm = std::max(1, std::min(per_sm, 2));  // __launch_bounds__(256, 2): two CTAs' registers per SM
  const int64_t want = int64_t(sm_count()) * per_sm;
  const int64_t need = (p.n + W - 1) / W;
  const int grid = int(want < need ? want : need);
  const int src = rowptr ? 0 : 1 + p.dtype;
  if (!rowptr && (p.dtype < LSH_F32 || p.dtype > LSH_F16)) return cudaErrorInvalidValue;
  const bool srp = kind_is_srp(p.kind);
  switch (src) {
    case 0: return srp ? launch_k<true, 0>(a, grid, W, stream) : launch_k<false, 0>(a, grid, W, stream);
    case 1 + LSH_F32: return srp ? launch_k<true, 1 + LSH_F32>(a, grid, W, stream)
                                 : launch_k<false, 1 + LSH_F32>(a, grid, W, stream);
    case 1 + LSH_BF16: return srp ? launch_k<true, 1 + LSH_BF16>(a, grid, W, stream)
                                  : launch_k<false, 1 + LSH_BF16>(a, grid, W, stream);
    default: return srp ? launch_k<true, 1 + LSH_F16>(a, grid, W, stream)
                        : launch_k<false, 1 + LSH_F16>(a, grid, W, stream);
  }
}

}  // namespace lsh
