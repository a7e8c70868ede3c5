// hash_csr.cu -- CS / HCS hashing of sparse (CSR) rows for all L tables
// (Definitions 4, 5, 12, 19, 25, 31 on a row whose unstored entries are 0).
//
// One warp per row, persistent grid.  For each table the row's nonzeros are
// spread over the lanes; each lane adds s(j) v_j and |v_j| into the warp's
// shared-memory bins of that table (shared atomics), then lanes own bins
// (l = lane, lane + 32, ...) for the epilogue: discretise, check the error
// bound, recompute flagged bins in FP64, fold the key.  SRP code words come
// straight from __ballot_sync over 32 consecutive bins.
//
// Bin lookup: count sketch tables are stored column-major, entry[col][t] =
// bin | neg << 15, so the L entries of one column share an L1 line across the
// table passes; HCS bins are computed from the per-mode tables, staged once
// per CTA in shared memory (O(N d^(1/N)) words per table).
//
// Exactness.  A bin holding k stored terms has FP32 sum error at most
// gamma_{k-1} S with S = sum |v_j| over the bin (any summation order); k is
// bounded by the row's nonzero count, S is accumulated in FP32 (widened by
// 2%).  A bin with S = 0 holds only zeros and is exactly 0.  Flagged bins
// are recomputed in FP64 over the stored entries in ascending column order,
// which equals the dense definition because the unstored terms are zeros.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace lsh {
namespace {

constexpr int kWarp = 32;
constexpr int kWarpsPerCta = 8;
constexpr float kU32 = 5.9604644775390625e-08f;

struct CsrArgs {
  SketchLaunch p;
  const int64_t *rowptr;
  const int32_t *col;
  const float *val;
  const uint16_t *colmajor;   // CS: [d][L] bin | neg << 15
  uint64_t dmagic[LSH_MAX_MODES];  // HCS: ceil(2^64 / d_k) (0 for d_k = 1), see csr_bin
  int stage_modes;            // HCS per-mode tables staged in shared memory
  int off_acc, off_modes, smem;
  float sqrtm_f, invw_f;
};

__device__ __forceinline__ void csr_bin(const CsrArgs &a, int t, int c, const uint16_t *mh, const int8_t *ms,
                                        int &bin, uint32_t &neg) {
  const SketchLaunch &p = a.p;
  if (p.N == 1) {
    const uint32_t e = __ldg(a.colmajor + int64_t(c) * p.L + t);
    bin = int(e & 0x7fffu);
    neg = e >> 15;
    return;
  }
  const uint16_t *hb = mh + int64_t(t) * p.dsum;
  const int8_t *sb = ms + int64_t(t) * p.dsum;
  // mode indices i_k of column c (first mode fastest); the quotient by d_k is
  // the high word of c ceil(2^64 / d_k), exact for every 32-bit c (Lemire,
  // Kaser and Kurz, "Faster remainder by direct computation", 2019)
  uint32_t r = uint32_t(c);
  int off = 0, stride = 1;
  bin = 0;
  neg = 0;
  for (int k = 0; k < p.N; ++k) {
    const uint32_t q = a.dmagic[k] ? uint32_t(__umul64hi(a.dmagic[k], uint64_t(r))) : r;
    const int ik = int(r - q * uint32_t(p.dims[k]));
    r = q;
    bin += int(hb[off + ik]) * stride;
    neg ^= sb[off + ik] < 0 ? 1u : 0u;
    stride *= p.mdims[k];
    off += p.dims[k];
  }
}

template <bool SRP>
__global__ void __launch_bounds__(kWarpsPerCta * kWarp) sketch_csr_kernel(const CsrArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SketchLaunch &p = a.p;
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x >> 5;
  const int m = p.m, L = p.L;
  float *acc = reinterpret_cast<float *>(smem + a.off_acc) + warp * 2 * m;  // [m] sums, [m] |v| sums
  float *sab = acc + m;
  const uint16_t *mh = p.bins;
  const int8_t *ms = p.signs;
  if (a.stage_modes) {
    uint16_t *smh = reinterpret_cast<uint16_t *>(smem + a.off_modes);
    int8_t *sms = reinterpret_cast<int8_t *>(smh + int64_t(L) * p.dsum);
    for (int i = threadIdx.x; i < L * p.dsum; i += blockDim.x) {
      smh[i] = p.bins[i];
      sms[i] = p.signs[i];
    }
    mh = smh;
    ms = sms;
  }
  for (int i = lane; i < 2 * m; i += kWarp) acc[i] = 0.f;
  __syncthreads();
  const int64_t nwarps = int64_t(gridDim.x) * kWarpsPerCta;
  const float sq_w = a.sqrtm_f * a.invw_f;
  const uint32_t words = uint32_t((m + 63) >> 6);
  for (int64_t row = int64_t(blockIdx.x) * kWarpsPerCta + warp; row < p.n; row += nwarps) {
    const int64_t rs = a.rowptr[row], re = a.rowptr[row + 1];
    const int nnz = int(re - rs);
    // validate the row: columns strictly ascending and < d, values finite
    bool ok = nnz >= 0;
    for (int64_t e = rs + lane; e < re; e += kWarp) {
      const int c = a.col[e];
      const float v = a.val[e];
      ok = ok && c >= 0 && c < p.d && isfinite(v) && (e == rs || a.col[e - 1] < c);
    }
    const bool rowok = __all_sync(0xffffffffu, ok);
    const float gk = float(nnz > 1 ? nnz - 1 : 0) * kU32;
    const float gbound = 1.02f * gk * (1.f + 2.f * gk);  // gamma_{k-1}(1+2 gamma), 2% slack
    int nflag = 0, nchanged = 0, novf = 0;
    for (int t = 0; t < L; ++t) {
      if (rowok) {
        for (int64_t e = rs + lane; e < re; e += kWarp) {
          const int c = a.col[e];
          const float v = a.val[e];
          int bin;
          uint32_t neg;
          csr_bin(a, t, c, mh, ms, bin, neg);
          atomicAdd(&acc[bin], neg ? -v : v);
          atomicAdd(&sab[bin], fabsf(v));
        }
      }
      __syncwarp();
      uint32_t ha = 0, hb = 0;
      for (int base = 0; base < m; base += kWarp) {
        const int l = base + lane;
        const bool inb = l < m;
        float y = 0.f, S = 0.f;
        if (inb) {
          y = acc[l];
          S = sab[l];
          acc[l] = 0.f;
          sab[l] = 0.f;
        }
        int code = 0;
        if (SRP) {
          const bool flag = rowok && inb && S > 0.f && !(fabsf(y) > gbound * S);
          int bit = y > 0.f ? 1 : 0;
          if (flag) {
            double y64 = 0.0;
            for (int64_t e = rs; e < re; ++e) {
              const int c = a.col[e];
              int bin;
              uint32_t neg;
              csr_bin(a, t, c, mh, ms, bin, neg);
              if (bin == l) {
                const double v = double(a.val[e]);
                y64 = __dadd_rn(y64, neg ? -v : v);
              }
            }
            const int b64 = y64 > 0.0 ? 1 : 0;
            ++nflag;
            nchanged += b64 != bit;
            bit = b64;
          }
          code = bit;
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
          const float bl = inb ? p.b32[int64_t(t) * m + l] : 0.f;
          const float tf = __fmul_rn(__fmaf_rn(a.sqrtm_f, y, bl), a.invw_f);
          const float fl = floorf(tf);
          const float fr = tf - fl;
          const float dist = fminf(fr, 1.f - fr);
          const float M = fmaf(sq_w * gbound, S, fmaf(10.2f * kU32, fabsf(tf), 15.3f * kU32));
          const bool flag = rowok && inb && !(dist > M && fabsf(tf) < 4194304.f);
          code = int(fl);
          if (flag) {
            double y64 = 0.0;
            for (int64_t e = rs; e < re; ++e) {
              const int c = a.col[e];
              int bin;
              uint32_t neg;
              csr_bin(a, t, c, mh, ms, bin, neg);
              if (bin == l) {
                const double v = double(a.val[e]);
                y64 = __dadd_rn(y64, neg ? -v : v);
              }
            }
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
          if (!rowok) code = INT32_MIN;
          if (inb) {
            ha += uint32_t(code) * __ldg(p.ka + int64_t(t) * m + l);
            hb += uint32_t(code) * __ldg(p.kb + int64_t(t) * m + l);
            if (p.codes) p.codes[(row * L + t) * m + l] = code;
            if (p.proj) p.proj[(row * L + t) * m + l] = y;
          }
        }
      }
      __syncwarp();
      uint64_t key;
      if (SRP && m <= 64) {
        key = (uint64_t(hb) << 32) | ha;
        if (m <= 32) key &= 0xffffffffull;
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

}  // namespace

cudaError_t launch_sketch_csr(const SketchLaunch &p, const int64_t *rowptr, const int32_t *col, const float *val,
                              const uint16_t *colmajor, cudaStream_t stream) {
  if (p.n <= 0) return cudaSuccess;
  CsrArgs a{};
  a.p = p;
  a.rowptr = rowptr;
  a.col = col;
  a.val = val;
  a.colmajor = colmajor;
  a.sqrtm_f = float(p.sqrtm);
  a.invw_f = float(1.0 / p.w);
  for (int k = 0; k < p.N && k < LSH_MAX_MODES; ++k)
    a.dmagic[k] = p.dims[k] > 1 ? ~0ull / uint64_t(p.dims[k]) + 1 : 0;
  const int acc_bytes = kWarpsPerCta * 2 * p.m * 4;
  a.off_acc = 0;
  a.off_modes = (acc_bytes + 15) & ~15;
  const int modes_bytes = p.N > 1 ? p.L * p.dsum * 3 : 0;
  a.stage_modes = (p.N > 1 && a.off_modes + modes_bytes <= 160 * 1024) ? 1 : 0;
  a.smem = a.off_modes + (a.stage_modes ? modes_bytes : 0);
  if (a.smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  const int per_sm = a.smem > 0 ? (200 * 1024) / (a.smem + 1024) : 8;
  const int64_t want = int64_t(sm_count()) * (per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm));
  const int64_t need = (p.n + kWarpsPerCta - 1) / kWarpsPerCta;
  const int grid = int(want < need ? want : need);
  cudaError_t e;
  if (kind_is_srp(p.kind)) {
    e = cudaFuncSetAttribute(sketch_csr_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem);
    if (e != cudaSuccess) return e;
    sketch_csr_kernel<true><<<grid, kWarpsPerCta * kWarp, a.smem, stream>>>(a);
  } else {
    e = cudaFuncSetAttribute(sketch_csr_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem);
    if (e != cudaSuccess) return e;
    sketch_csr_kernel<false><<<grid, kWarpsPerCta * kWarp, a.smem, stream>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace lsh
