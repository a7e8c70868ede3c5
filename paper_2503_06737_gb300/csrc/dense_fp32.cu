// dense_fp32.cu -- the dense baselines E2LSH (Definition 2) and SRP
// (Definition 3) for all L tables: Y = X G with G [d][m L] Gaussian, fused
// with discretisation, the boundary check and the key fold.  FP32 SIMT tiled
// GEMM: 128 x 128 CTA tile, 8 x 8 outputs per thread (rows ty*4 + {0..3} and
// 64 + ty*4 + {0..3}, columns likewise), K tiles of 32 staged in shared memory
// (double-buffered, the next tile's 128-bit global loads held in registers
// while the current one is multiplied).  The grid walks column tiles fastest,
// so the CTAs of one row tile run together and X leaves HBM once.
//
// Exactness.  Each K tile of 32 products is summed into a fresh register by
// an FMA chain and then added to the running sum, so for an output
//   |fl(y) - y| <= gamma_32 sum_j |x_j g_j| + u sum_tiles |acc_tile|
//              <= gamma_32 ||x|| ||g_c|| + u * S,
// where S = sum over K tiles of the largest |acc| this thread holds, ||g_c||
// is the column norm precomputed on the host (rounded up) and ||x|| the row
// norm accumulated while the tiles are staged (widened for its own rounding).
// With the FP64 reference's own error and the discretisation roundings
// covered as in hash_sketch.cu, an entry within that bound of an E2LSH bin
// edge (or of 0 for SRP) is queued with its fast code; dense_recheck_kernel
// computes sum_j x_j G[j][c] in ascending j in FP64 (the oracle's value) from
// the transposed copy Gt [m L][d], one entry per thread, and patches codes,
// bits and keys where the fast code was wrong (without a queue, or past its
// end, the thread rechecks in place).  Keys are folded per (row, table) in
// shared memory and added to the zeroed global keys with one atomic per CTA.
#include <algorithm>

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace lsh {
namespace {

constexpr int BM = 128, BN = 128, BK = 32, NT = 256;
constexpr int ASTR = BM + 4;  // As row stride (floats): rows stay 16-byte aligned
constexpr float kU = 5.9604644775390625e-08f;

struct DenseArgs {
  const void *X;
  int32_t dtype;
  int64_t n, ld;
  int32_t d, m, L, srp;
  int32_t vecA, vecB;  // 128-bit tile loads of X rows / G rows are aligned
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
  int4 *queue;         // deferred rechecks {row, col, fast code, 0}
  uint32_t *qcount;
  uint32_t qcap;
};

template <int DT>
__device__ __forceinline__ float ldx(const void *X, int64_t i) {
  if (DT == LSH_F32) return __ldg(reinterpret_cast<const float *>(X) + i);
  const unsigned short h = __ldg(reinterpret_cast<const unsigned short *>(X) + i);
  if (DT == LSH_BF16) return __uint_as_float(uint32_t(h) << 16);
  return __half2float(__ushort_as_half(h));
}

template <int DT>
__device__ __forceinline__ float cvt16(uint32_t h) {
  if (DT == LSH_BF16) return __uint_as_float(h << 16);
  return __half2float(__ushort_as_half((unsigned short)h));
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

// The oracle's code of an exact projection (E2LSH: floor((y + b) / w), one
// rounding per operation; SRP: y > 0).
__device__ __forceinline__ int code_of(const DenseArgs &a, double y64, int64_t col, int &novf) {
  if (a.srp) return y64 > 0.0 ? 1 : 0;
  const double f = floor(__ddiv_rn(__dadd_rn(y64, a.b64[col]), a.w));
  if (f >= -2147483648.0 && f <= 2147483647.0) return int(f);
  ++novf;
  return INT32_MIN;
}

// Staging of one K tile into registers: A (X rows row0 .. row0+127, columns
// k0 .. k0+31) as four chunks per thread, chunk f = tid + 256 v covering row
// f / 8 and columns 4 (f % 8) .. +3 (FP32; 16-bit rows read 8 columns per
// 16-byte chunk, two chunks per thread); B (G rows k0 .. k0+31, columns
// col0 .. col0+127) as four float4 per thread.
template <int DT>
struct Stage {
  float a[4][4];   // [chunk][4 values] (16-bit inputs: [2][8] in the same registers)
  float4 b[4];
};

template <int DT>
__device__ __forceinline__ void load_stage(const DenseArgs &a, Stage<DT> &s, int64_t row0, int64_t col0, int k0,
                                           int tid, int64_t ML) {
  const int d = a.d;
  if (DT == LSH_F32) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int f = tid + NT * v, r = f >> 3, kq = f & 7;
      const int64_t gr = row0 + r;
      const int gk = k0 + kq * 4;
      if (a.vecA && gr < a.n && gk + 4 <= d) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(a.X) + gr * a.ld + gk));
        s.a[v][0] = q.x, s.a[v][1] = q.y, s.a[v][2] = q.z, s.a[v][3] = q.w;
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) s.a[v][c] = (gr < a.n && gk + c < d) ? ldx<DT>(a.X, gr * a.ld + gk + c) : 0.f;
      }
    }
  } else {
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int f = tid + NT * v, r = f >> 2, kq = f & 3;
      const int64_t gr = row0 + r;
      const int gk = k0 + kq * 8;
      // values c = 0..7 of the chunk live in a[2 v + c / 4][c % 4]
      if (a.vecA && gr < a.n && gk + 8 <= d) {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(reinterpret_cast<const unsigned short *>(a.X) +
                                                              gr * a.ld + gk));
        s.a[2 * v][0] = cvt16<DT>(q.x & 0xffffu), s.a[2 * v][1] = cvt16<DT>(q.x >> 16);
        s.a[2 * v][2] = cvt16<DT>(q.y & 0xffffu), s.a[2 * v][3] = cvt16<DT>(q.y >> 16);
        s.a[2 * v + 1][0] = cvt16<DT>(q.z & 0xffffu), s.a[2 * v + 1][1] = cvt16<DT>(q.z >> 16);
        s.a[2 * v + 1][2] = cvt16<DT>(q.w & 0xffffu), s.a[2 * v + 1][3] = cvt16<DT>(q.w >> 16);
      } else {
#pragma unroll
        for (int c = 0; c < 8; ++c)
          s.a[2 * v + c / 4][c % 4] = (gr < a.n && gk + c < d) ? ldx<DT>(a.X, gr * a.ld + gk + c) : 0.f;
      }
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int f = tid + NT * v, kk = f >> 5, cq = f & 31;
    const int gk = k0 + kk;
    const int64_t gc = col0 + cq * 4;
    if (a.vecB && gk < d && gc + 4 <= ML) {
      s.b[v] = __ldg(reinterpret_cast<const float4 *>(a.G + int64_t(gk) * ML + gc));
    } else {
      float t[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) t[c] = (gk < d && gc + c < ML) ? __ldg(a.G + int64_t(gk) * ML + gc + c) : 0.f;
      s.b[v] = make_float4(t[0], t[1], t[2], t[3]);
    }
  }
}

// Registers -> shared tile (A transposed to As[k][row]); the squares of the
// A values go into the thread's per-chunk row-norm partials.
template <int DT>
__device__ __forceinline__ void store_stage(const Stage<DT> &s, float (*As)[ASTR], float (*Bs)[BN], int tid,
                                            float (&xsq)[4]) {
  if (DT == LSH_F32) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int f = tid + NT * v, r = f >> 3, kq = f & 7;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        As[kq * 4 + c][r] = s.a[v][c];
        xsq[v] = fmaf(s.a[v][c], s.a[v][c], xsq[v]);
      }
    }
  } else {
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int f = tid + NT * v, r = f >> 2, kq = f & 3;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float x = s.a[2 * v + c / 4][c % 4];
        As[kq * 8 + c][r] = x;
        xsq[v] = fmaf(x, x, xsq[v]);
      }
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int f = tid + NT * v, kk = f >> 5, cq = f & 31;
    *reinterpret_cast<float4 *>(&Bs[kk][cq * 4]) = s.b[v];
  }
}

// One output tile: grid index = row tile * (column tiles) + column tile.
template <int DT>
__global__ void __launch_bounds__(NT, 1) dense_fp32_kernel(const __grid_constant__ DenseArgs a, int ntab_max,
                                                           int ncolt) {
  extern __shared__ __align__(16) unsigned char smem[];
  float(*As)[BK][ASTR] = reinterpret_cast<float(*)[BK][ASTR]>(smem);                      // [2][BK][ASTR]
  float(*Bs)[BK][BN] = reinterpret_cast<float(*)[BK][BN]>(smem + 2 * BK * ASTR * 4);        // [2][BK][BN]
  uint32_t *kacc = reinterpret_cast<uint32_t *>(smem + 2 * BK * ASTR * 4 + 2 * BK * BN * 4);  // [BM][2 ntab_max]
  float *xn2 = reinterpret_cast<float *>(kacc + BM * 2 * ntab_max);                           // [BM] |x|^2
  const int kst = 2 * ntab_max;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t row0 = int64_t(blockIdx.x / ncolt) * BM;
  const int64_t col0 = int64_t(blockIdx.x % ncolt) * BN;
  const int64_t ML = int64_t(a.m) * a.L;
  const int d = a.d;
  for (int i = tid; i < BM * kst; i += NT) kacc[i] = 0u;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float xsq[4] = {0.f, 0.f, 0.f, 0.f};
  float S = 0.f;
  Stage<DT> st;
  const int ktiles = (d + BK - 1) / BK;
  load_stage<DT>(a, st, row0, col0, 0, tid, ML);
  store_stage<DT>(st, As[0], Bs[0], tid, xsq);
  __syncthreads();
  for (int kt = 0; kt < ktiles; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < ktiles) load_stage<DT>(a, st, row0, col0, (kt + 1) * BK, tid, ML);
    float p[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) p[i][j] = 0.f;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) p[i][j] = fmaf(av[i], bv[j], p[i][j]);
    }
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        acc[i][j] += p[i][j];
        mx = fmaxf(mx, fabsf(acc[i][j]));
      }
    S += mx;
    if (kt + 1 < ktiles) store_stage<DT>(st, As[buf ^ 1], Bs[buf ^ 1], tid, xsq);
    __syncthreads();
  }
  // row norms: the threads that staged one row's chunks add their partials
  if (DT == LSH_F32) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float x = xsq[v];
      x += __shfl_xor_sync(0xffffffffu, x, 1);
      x += __shfl_xor_sync(0xffffffffu, x, 2);
      x += __shfl_xor_sync(0xffffffffu, x, 4);
      if ((tid & 7) == 0) xn2[(tid >> 3) + 32 * v] = x;
    }
  } else {
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      float x = xsq[v];
      x += __shfl_xor_sync(0xffffffffu, x, 1);
      x += __shfl_xor_sync(0xffffffffu, x, 2);
      if ((tid & 3) == 0) xn2[(tid >> 2) + 64 * v] = x;
    }
  }
  __syncthreads();

  // ---- epilogue: the accumulators wait in the (now idle) tile buffers,
  // [output k][thread], so that the loops below index them freely ----
  float *Y = reinterpret_cast<float *>(smem);  // 64 x 256 floats <= 2 (BK ASTR + BK BN)
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) Y[(i * 8 + j) * NT + tid] = acc[i][j];
  const float g32 = 32.f * kU * (1.f + 64.f * kU);
  const int m = a.m;
  const int lane = tid & 31;
  int nflag = 0, nchanged = 0, novf = 0;
#pragma unroll 1
  for (int i = 0; i < 8; ++i) {
    const int rl = i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4);
    const int64_t row = row0 + rl;
    const bool rowin = row < a.n;
    const float q2 = xn2[rl];
    const bool bad = rowin && !isfinite(q2);
    const float xn = sqrtf(q2) * (1.f + float(d + 2) * kU);
    if (bad && col0 == 0 && tx == 0) {
      if (a.counters) atomicAdd(a.counters + CNT_NONFINITE, 1ull);
      atomicOr(a.status, STATUS_NONFINITE);
    }
#pragma unroll 1
    for (int j = 0; j < 8; ++j) {
      const int cl = j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4);
      const int64_t col = col0 + cl;
      const bool live = rowin && col < ML;
      const float y = Y[(i * 8 + j) * NT + tid];
      int code = 0;
      bool flag = false;
      if (live && !bad) {
        const float E = 1.02f * (g32 * xn * __ldg(a.gnorm + col) + kU * S);
        if (a.srp) {
          code = y > 0.f ? 1 : 0;
          flag = !(fabsf(y) > E);
        } else {
          const float tf = __fmul_rn(y + __ldg(a.b32 + col), a.invw);
          const float dist = fabsf(tf - rintf(tf));  // exact (Sterbenz)
          const float M = fmaf(E, a.invw * 1.0001f, fmaf(10.2f * kU, fabsf(tf), 15.3f * kU));
          flag = !(dist > M);  // |tf| >= 2^22 makes M > 2.5: flagged
          code = __float2int_rd(tf);
        }
      }
      // flagged entries: to the queue (warp-aggregated), else rechecked here
      bool inplace = flag;
      if (a.queue && __any_sync(0xffffffffu, flag)) {
        const uint32_t bal = __ballot_sync(0xffffffffu, flag);
        const int leader = __ffs(bal) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(a.qcount, uint32_t(__popc(bal)));
        base = __shfl_sync(0xffffffffu, base, leader);
        const uint32_t pos = base + __popc(bal & ((1u << lane) - 1u));
        if (flag && pos < a.qcap) {
          a.queue[pos] = make_int4(int(uint32_t(row)), int(col), code, 0);
          inplace = false;
        }
      }
      if (inplace) {
        const int c64 = code_of(a, dense_fp64<DT>(a, row, col), col, novf);
        ++nflag;
        nchanged += c64 != code;
        code = c64;
      }
      if (!live) continue;
      if (bad) code = a.srp ? 0 : INT32_MIN;
      if (a.proj) a.proj[row * ML + col] = y;
      if (!a.srp && a.codes) a.codes[row * ML + col] = code;
      if (bad) continue;
      // partial key into the (row, table) slot of this CTA
      const int t = int(col / m), l = int(col - int64_t(t) * m);
      const int tl = int(t - col0 / m);  // table index relative to the tile's first table
      if (a.srp && m <= 64) {
        if (code) atomicOr(&kacc[rl * kst + 2 * tl + (l >> 5)], 1u << (l & 31));
      } else {
        const uint32_t cu = uint32_t(code);
        if (!a.srp || code) {
          atomicAdd(&kacc[rl * kst + 2 * tl], cu * __ldg(a.ka + col));
          atomicAdd(&kacc[rl * kst + 2 * tl + 1], cu * __ldg(a.kb + col));
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
  const int t_last = int((min(ML, col0 + BN) - 1) / m);
  const int ntab = t_last - t_first + 1;
  for (int i = tid; i < BM * ntab; i += NT) {
    const int tl = i / BM, rl = i % BM;
    const int64_t row = row0 + rl;
    if (row >= a.n || !a.keys) continue;
    const int t = t_first + tl;
    unsigned long long *kp = reinterpret_cast<unsigned long long *>(a.keys) + int64_t(t) * a.key_ld + row;
    if (!isfinite(xn2[rl])) {
      atomicExch(kp, ~0ull);  // every CTA of a bad row skips its adds, so ~0 is final
    } else if (a.srp && m <= 64) {
      const unsigned long long v = (uint64_t(kacc[rl * kst + 2 * tl + 1]) << 32) | kacc[rl * kst + 2 * tl];
      if (v) atomicOr(kp, v);
      if (a.bits && v) atomicOr(reinterpret_cast<unsigned long long *>(a.bits) + row * a.L + t, v);
    } else {
      // (a * 2^32 + b): add the halves separately so no carry crosses them
      uint32_t *k32 = reinterpret_cast<uint32_t *>(kp);
      atomicAdd(k32 + 1, kacc[rl * kst + 2 * tl]);
      atomicAdd(k32, kacc[rl * kst + 2 * tl + 1]);
    }
  }
  if (a.counters) {
    if (nflag) atomicAdd(a.counters + CNT_FLAGGED, (unsigned long long)nflag);
    if (nchanged) atomicAdd(a.counters + CNT_CHANGED, (unsigned long long)nchanged);
    if (novf) atomicAdd(a.counters + CNT_OVERFLOW, (unsigned long long)novf);
  }
  if (novf) atomicOr(a.status, STATUS_OVERFLOW);
}

// The queued entries, one per thread: the oracle's FP64 value and code, and
// the patch of code, bits and key where the fast code was wrong (keys are
// sums mod 2^32 in each half, or bit patterns for SRP with m <= 64).
template <int DT>
__global__ void __launch_bounds__(256) dense_recheck_kernel(const __grid_constant__ DenseArgs a) {
  const int64_t cnt = min(int64_t(*a.qcount), int64_t(a.qcap));
  const int64_t ML = int64_t(a.m) * a.L;
  int nflag = 0, nchanged = 0, novf = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < cnt; i += int64_t(gridDim.x) * blockDim.x) {
    const int4 r = a.queue[i];
    const int64_t row = int64_t(uint32_t(r.x)), col = r.y;
    const int c64 = code_of(a, dense_fp64<DT>(a, row, col), col, novf);
    ++nflag;
    if (c64 == r.z) continue;
    ++nchanged;
    const int t = int(col / a.m), l = int(col - int64_t(t) * a.m);
    uint64_t *key = a.keys ? a.keys + int64_t(t) * a.key_ld + row : nullptr;
    if (a.srp) {
      const int words = (a.m + 63) >> 6;
      if (a.bits)
        atomicXor(reinterpret_cast<unsigned long long *>(a.bits + (row * a.L + t) * words + (l >> 6)),
                  1ull << (l & 63));
      if (key) {
        if (a.m <= 64) {
          atomicXor(reinterpret_cast<unsigned long long *>(key), 1ull << l);
        } else {
          const uint32_t sgn = c64 ? 1u : 0xFFFFFFFFu;  // +1 or -1 mod 2^32
          atomicAdd(reinterpret_cast<unsigned int *>(key) + 1, sgn * a.ka[col]);
          atomicAdd(reinterpret_cast<unsigned int *>(key), sgn * a.kb[col]);
        }
      }
    } else {
      if (a.codes) a.codes[row * ML + col] = c64;
      const uint32_t dc = uint32_t(c64) - uint32_t(r.z);
      if (key) {
        atomicAdd(reinterpret_cast<unsigned int *>(key) + 1, dc * a.ka[col]);
        atomicAdd(reinterpret_cast<unsigned int *>(key), dc * a.kb[col]);
      }
    }
  }
  if (a.counters) {
    if (nflag) atomicAdd(a.counters + CNT_FLAGGED, (unsigned long long)nflag);
    if (nchanged) atomicAdd(a.counters + CNT_CHANGED, (unsigned long long)nchanged);
    if (novf) atomicAdd(a.counters + CNT_OVERFLOW, (unsigned long long)novf);
  }
  if (novf) atomicOr(a.status, STATUS_OVERFLOW);
}

template <int DT>
cudaError_t launch_dt(const DenseArgs &a, int64_t nrowt, int ncolt, int ntab_max, cudaStream_t stream) {
  const int dsmem = 2 * BK * ASTR * 4 + 2 * BK * BN * 4 + BM * 2 * ntab_max * 4 + BM * 4;
  cudaError_t e = cudaFuncSetAttribute(dense_fp32_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem);
  if (e != cudaSuccess) return e;
  dense_fp32_kernel<DT><<<unsigned(nrowt * ncolt), NT, dsmem, stream>>>(a, ntab_max, ncolt);
  e = cudaGetLastError();
  if (e != cudaSuccess || !a.queue) return e;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  dense_recheck_kernel<DT><<<unsigned(sms > 0 ? sms * 8 : 1024), 256, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

int64_t dense_queue_cap(int64_t n, int64_t ML) {
  return std::min<int64_t>(n * ML / 256 + 65536, int64_t(1) << 28);
}

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
  const int es = p.dtype == LSH_F32 ? 4 : 2;
  a.vecA = (reinterpret_cast<uintptr_t>(p.X) % 16 == 0 && (p.ld * es) % 16 == 0) ? 1 : 0;
  const int64_t ML = int64_t(p.m) * p.L;
  a.vecB = (reinterpret_cast<uintptr_t>(G) % 16 == 0 && ML % 4 == 0) ? 1 : 0;
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
  a.queue = p.queue;
  a.qcount = p.qcount;
  a.qcap = p.qcap;
  const int64_t nrowt = (p.n + BM - 1) / BM;
  const int ncolt = int((ML + BN - 1) / BN);
  if (nrowt * ncolt > int64_t(INT32_MAX)) return cudaErrorInvalidConfiguration;
  const int ntab_max = (BN + p.m - 1) / p.m + 1;
  switch (p.dtype) {
    case LSH_F32: return launch_dt<LSH_F32>(a, nrowt, ncolt, ntab_max, stream);
    case LSH_BF16: return launch_dt<LSH_BF16>(a, nrowt, ncolt, ntab_max, stream);
    case LSH_F16: return launch_dt<LSH_F16>(a, nrowt, ncolt, ntab_max, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lsh
