// dense_fp32.cu -- the dense baselines E2LSH (Definition 2) and SRP
// (Definition 3) for all L tables: Y = X G with G [d][m L] Gaussian, fused
// with discretisation, the FP64 boundary recheck and the key fold.  FP32
// SIMT tiled GEMM (128 x 128 CTA tile, 8 x 8 outputs per thread, k-tiles of
// 16 staged in shared memory, double-buffered).
//
// Exactness.  Each k-tile of 16 products is summed into a fresh register by
// an FMA chain and then added to the running sum, so for an output
//   |fl(y) - y| <= gamma_16 sum_j |x_j g_j| + u sum_tiles |acc_tile|
//              <= gamma_16 ||x|| ||g_c|| + u * S,
// where S = sum over k-tiles of the largest |acc| this thread holds (one
// register per thread), ||g_c|| is the column norm precomputed on the host
// (rounded up) and ||x|| the row norm accumulated here (widened).  With the
// FP64 reference's own error and the discretisation roundings covered as in
// hash_sketch.cu, an entry within that bound of an E2LSH bin edge (or of 0
// for SRP) is recomputed by its thread in FP64, sum_j x_j G[j][c] in
// ascending j, from the transposed copy Gt [m L][d] -- the oracle's value.
// Keys are folded per (row, table) in shared memory and added to the zeroed
// global keys with one atomic per CTA, since a table may span CTA tiles.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace lsh {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, TM = 8, TN = 8, NT = 256;
constexpr float kU = 5.9604644775390625e-08f;

struct DenseArgs {
  const void *X;
  int32_t dtype;
  int64_t n, ld;
  int32_t d, m, L, srp;
  const float *G;      // [d][mL]
  const float *Gt;     // [mL][d]
  const float *gnorm;  // [mL] column norms, rounded up
  const float *b32;
  const double *b64;
  const uint32_t *ka, *kb;
  double w;
  float invw;
  int32_t *codes;
  uint64_t *bits;
  uint64_t *keys;      // zeroed [L][key_ld]
  int64_t key_ld;
  float *proj;
  unsigned long long *counters;
  uint32_t *status;
};

template <int DT>
__device__ __forceinline__ float ldx(const void *X, int64_t i) {
  if (DT == LSH_F32) return __ldg(reinterpret_cast<const float *>(X) + i);
  const unsigned short h = __ldg(reinterpret_cast<const unsigned short *>(X) + i);
  if (DT == LSH_BF16) return __uint_as_float(uint32_t(h) << 16);
  return __half2float(__ushort_as_half(h));
}

// FP64 value of one projection, sum_j x_j G[j][c] in ascending j with one
// IEEE rounding per operation; eight terms are loaded before their adds.
template <int DT>
__device__ __noinline__ double dense_fp64(const DenseArgs &a, int64_t row, int64_t col) {
  const float *g = a.Gt + col * a.d;
  const int64_t base = row * a.ld;
  double y = 0.0;
  int j = 0;
  for (; j + 8 <= a.d; j += 8) {
    float xv[8], gv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      xv[k] = ldx<DT>(a.X, base + j + k);
      gv[k] = __ldg(g + j + k);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) y = __dadd_rn(y, __dmul_rn(double(xv[k]), double(gv[k])));
  }
  for (; j < a.d; ++j) y = __dadd_rn(y, __dmul_rn(double(ldx<DT>(a.X, base + j)), double(__ldg(g + j))));
  return y;
}

template <int DT>
__global__ void __launch_bounds__(NT) dense_fp32_kernel(const DenseArgs a, int ntab_max) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  extern __shared__ __align__(16) uint32_t kacc_dyn[];  // [BM][2 * ntab_max] partial keys
  __shared__ int badrow[BM];
  const int kst = 2 * ntab_max;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t row0 = int64_t(blockIdx.x) * BM;
  const int64_t col0 = int64_t(blockIdx.y) * BN;
  const int64_t ML = int64_t(a.m) * a.L;
  const int d = a.d;

  float acc[TM][TN];
  float xsq[TM];
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    xsq[i] = 0.f;
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  }
  float S = 0.f;

  // loaders: A tile 128 x 16 -> As[k][row]; B tile 16 x 128 -> Bs[k][col]
  auto load_tiles = [&](int buf, int k0) {
    for (int i = tid; i < BM * BK; i += NT) {
      const int r = i % BM, kk = i / BM;
      const int64_t gr = row0 + r;
      const int gk = k0 + kk;
      As[buf][kk][r] = (gr < a.n && gk < d) ? ldx<DT>(a.X, gr * a.ld + gk) : 0.f;
    }
    for (int i = tid; i < BK * BN; i += NT) {
      const int kk = i / BN, c = i % BN;
      const int gk = k0 + kk;
      const int64_t gc = col0 + c;
      Bs[buf][kk][c] = (gk < d && gc < ML) ? __ldg(a.G + int64_t(gk) * ML + gc) : 0.f;
    }
  };

  const int ktiles = (d + BK - 1) / BK;
  load_tiles(0, 0);
  __syncthreads();
  for (int kt = 0; kt < ktiles; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < ktiles) load_tiles(buf ^ 1, (kt + 1) * BK);
    float p[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) p[i][j] = 0.f;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float av[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) av[i] = As[buf][kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[buf][kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        xsq[i] = fmaf(av[i], av[i], xsq[i]);
#pragma unroll
        for (int j = 0; j < TN; ++j) p[i][j] = fmaf(av[i], bv[j], p[i][j]);
      }
    }
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        acc[i][j] += p[i][j];
        mx = fmaxf(mx, fabsf(acc[i][j]));
      }
    S += mx;
    __syncthreads();
  }

  // ---- epilogue ----
  for (int i = tid; i < BM * kst; i += NT) kacc_dyn[i] = 0u;
  if (tx == 0)
    for (int i = 0; i < TM; ++i) badrow[ty * TM + i] = isfinite(xsq[i]) ? 0 : 1;
  __syncthreads();
  const float g16 = 16.f * kU * (1.f + 32.f * kU);
  const int m = a.m;
  int nflag = 0, nchanged = 0, novf = 0;
#pragma unroll 1
  for (int i = 0; i < TM; ++i) {
    const int rl = ty * TM + i;
    const int64_t row = row0 + rl;
    if (row >= a.n) continue;
    if (!isfinite(xsq[i])) {
      // a row holding NaN/Inf: no hash; its keys become ~0 below
      if (blockIdx.y == 0 && tx == 0) {
        if (a.counters) atomicAdd(a.counters + CNT_NONFINITE, 1ull);
        atomicOr(a.status, STATUS_NONFINITE);
      }
      if (!a.srp && a.codes)
        for (int j = 0; j < TN; ++j)
          if (col0 + tx * TN + j < ML) a.codes[row * ML + col0 + tx * TN + j] = INT32_MIN;
      continue;
    }
    const float xn = sqrtf(xsq[i]) * (1.f + float(d + 2) * kU);
#pragma unroll 1
    for (int j = 0; j < TN; ++j) {
      const int cl = tx * TN + j;
      const int64_t col = col0 + cl;
      if (col >= ML) continue;
      const int t = int(col / m), l = int(col - int64_t(t) * m);
      const float y = acc[i][j];
      const float E = 1.02f * (g16 * xn * __ldg(a.gnorm + col) + kU * S);
      int code;
      if (a.srp) {
        code = y > 0.f ? 1 : 0;
        if (!(fabsf(y) > E)) {
          const double y64 = dense_fp64<DT>(a, row, col);
          const int c64 = y64 > 0.0 ? 1 : 0;
          ++nflag;
          nchanged += c64 != code;
          code = c64;
        }
      } else {
        const float bl = __ldg(a.b32 + col);
        const float tf = __fmul_rn(y + bl, a.invw);
        const float fl = floorf(tf);
        const float fr = tf - fl;
        const float dist = fminf(fr, 1.f - fr);
        const float M = fmaf(E, a.invw * 1.0001f, fmaf(10.2f * kU, fabsf(tf), 15.3f * kU));
        code = int(fl);
        if (!(dist > M && fabsf(tf) < 4194304.f)) {
          const double y64 = dense_fp64<DT>(a, row, col);
          const double t2 = __dadd_rn(y64, a.b64[col]);
          const double t3 = __ddiv_rn(t2, a.w);
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
      if (a.proj) a.proj[row * ML + col] = y;
      if (!a.srp && a.codes) a.codes[row * ML + col] = code;
      // partial key into the (row, table) slot of this CTA
      const int tl = int(t - col0 / m);  // table index relative to the tile's first table
      if (a.srp && m <= 64) {
        if (code) atomicOr(&kacc_dyn[rl * kst + 2 * tl + (l >> 5)], 1u << (l & 31));
      } else {
        const uint32_t cu = uint32_t(code);
        if (!a.srp || code) {
          atomicAdd(&kacc_dyn[rl * kst + 2 * tl], cu * __ldg(a.ka + col));
          atomicAdd(&kacc_dyn[rl * kst + 2 * tl + 1], cu * __ldg(a.kb + col));
        }
        if (a.srp && code && a.bits)
          atomicOr(reinterpret_cast<unsigned long long *>(a.bits) + (row * a.L + t) * ((m + 63) >> 6) + (l >> 6),
                   1ull << (l & 63));
      }
    }
  }
  __syncthreads();
  // one atomic per (row, table) of the tile into the zeroed global keys
  const int t_first = int(col0 / m);
  const int t_last = int(min(ML, col0 + BN) - 1) / m;
  const int ntab = t_last - t_first + 1;
  for (int i = tid; i < BM * ntab; i += NT) {
    const int tl = i / BM, rl = i % BM;
    const int64_t row = row0 + rl;
    if (row >= a.n) continue;
    const int t = t_first + tl;
    if (!a.keys) continue;
    unsigned long long *kp = reinterpret_cast<unsigned long long *>(a.keys) + int64_t(t) * a.key_ld + row;
    if (badrow[rl]) {
      atomicExch(kp, ~0ull);  // every CTA of a bad row skips its adds, so ~0 is final
    } else if (a.srp && m <= 64) {
      const unsigned long long v = (uint64_t(kacc_dyn[rl * kst + 2 * tl + 1]) << 32) | kacc_dyn[rl * kst + 2 * tl];
      if (v) atomicOr(kp, v);
      if (a.bits && v)
        atomicOr(reinterpret_cast<unsigned long long *>(a.bits) + row * a.L + t, v);
    } else {
      // (a * 2^32 + b): add the halves separately so no carry crosses them
      uint32_t *k32 = reinterpret_cast<uint32_t *>(kp);
      atomicAdd(k32 + 1, kacc_dyn[rl * kst + 2 * tl]);
      atomicAdd(k32, kacc_dyn[rl * kst + 2 * tl + 1]);
    }
  }
  if (a.counters || novf) {
    if (a.counters) {
      if (nflag) atomicAdd(a.counters + CNT_FLAGGED, (unsigned long long)nflag);
      if (nchanged) atomicAdd(a.counters + CNT_CHANGED, (unsigned long long)nchanged);
      if (novf) atomicAdd(a.counters + CNT_OVERFLOW, (unsigned long long)novf);
    }
    if (novf) atomicOr(a.status, STATUS_OVERFLOW);
  }
}

}  // namespace

cudaError_t launch_dense_fp32(const SketchLaunch &p, const float *G, const float *Gt, const float *gnorm,
                              cudaStream_t stream) {
  if (p.n <= 0) return cudaSuccess;
  DenseArgs a{};
  a.X = p.X;
  a.dtype = p.dtype;
  a.n = p.n;
  a.ld = p.ld;
  a.d = p.d;
  a.m = p.m;
  a.L = p.L;
  a.srp = kind_is_srp(p.kind) ? 1 : 0;
  a.G = G;
  a.Gt = Gt;
  a.gnorm = gnorm;
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
  const int64_t ML = int64_t(p.m) * p.L;
  const dim3 grid((unsigned)((p.n + BM - 1) / BM), (unsigned)((ML + BN - 1) / BN));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  const int ntab_max = (BN + p.m - 1) / p.m + 1;
  const int dsmem = BM * 2 * ntab_max * 4;
  cudaError_t e = cudaSuccess;
  switch (p.dtype) {
    case LSH_F32:
      e = cudaFuncSetAttribute(dense_fp32_kernel<LSH_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem);
      if (e == cudaSuccess) dense_fp32_kernel<LSH_F32><<<grid, NT, dsmem, stream>>>(a, ntab_max);
      break;
    case LSH_BF16:
      e = cudaFuncSetAttribute(dense_fp32_kernel<LSH_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem);
      if (e == cudaSuccess) dense_fp32_kernel<LSH_BF16><<<grid, NT, dsmem, stream>>>(a, ntab_max);
      break;
    case LSH_F16:
      e = cudaFuncSetAttribute(dense_fp32_kernel<LSH_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem);
      if (e == cudaSuccess) dense_fp32_kernel<LSH_F16><<<grid, NT, dsmem, stream>>>(a, ntab_max);
      break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace lsh
