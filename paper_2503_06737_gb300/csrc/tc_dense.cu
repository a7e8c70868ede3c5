// tc_dense.cu -- the dense baselines E2LSH (Definition 2) and SRP (Definition
// 3) on the 5th-generation tensor cores: Y = X G for BF16 rows X [n][d] and a
// family whose Gaussian G is stored in BF16, fused with discretisation, the
// boundary recheck and the key fold.
//
// Per CTA one 128 x 128 output tile (rows x projection columns):
//   warp 0   allocates all 512 TMEM columns, then issues TMA loads (128-byte
//            swizzle) of 64-wide K slices of X and of G^T into a 4-stage
//            shared-memory ring guarded by mbarriers;
//   warp 1   (one thread) issues tcgen05.mma kind::f16 (M = N = 128, K = 16,
//            FP32 accumulate), committing each stage back to its producer;
//   warps 2-5 read the accumulators with tcgen05.ld and run the epilogue.
// The K dimension is split into (at most) four chunks, each accumulated into
// its own 128-column TMEM region, so the epilogue sees every chunk sum.
//
// Exactness.  Products of two BF16 values are exact in FP32.  Accumulation
// model for one chunk of s MMA steps: the error is at most 2u * s * (sum of
// |products| of the chunk) -- each step rounds once relative to a partial
// sum no larger than that -- with sum |products| <= ||x_chunk|| ||g_chunk||
// (row chunk norms from a pre-pass, column chunk norms from the host).  The
// four chunk sums are added in FP32 (error <= 2u sum |chunk|).  Entries
// within that bound (widened 2%) of an E2LSH bin edge, or of 0 for SRP, are
// recomputed in FP64 as sum_j x_j G[j][c] in ascending j -- the oracle's
// value.  Every mbarrier wait is bounded; a timeout sets an error flag and
// the kernel still releases its TMEM.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "internal.h"

namespace lsh {
namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4, NCH = 4;
constexpr int TILE_A = BM * BK * 2, TILE_B = BN * BK * 2;
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr float kU = 5.9604644775390625e-08f;

struct TcArgs {
  int64_t n;
  int32_t d, m, L, srp, ktiles, ktpc, nch;
  const unsigned short *X;   // bf16 rows
  int64_t ld;
  const float *Gt;           // [mL][d] FP32 copy (recheck)
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
};

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(su32(b)), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(su32(dst)), "l"(map), "r"(su32(bar)), "r"(x), "r"(y) : "memory");
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __noinline__ double tc_fp64(const TcArgs &a, int64_t row, int64_t col) {
  const float *g = a.Gt + col * a.d;
  const unsigned short *x = a.X + row * a.ld;
  double y = 0.0;
  for (int j = 0; j < a.d; ++j) y = __dadd_rn(y, __dmul_rn(double(__uint_as_float(uint32_t(x[j]) << 16)), double(g[j])));
  return y;
}

__global__ void __launch_bounds__(192, 1) tc_dense_kernel(const __grid_constant__ CUtensorMap mapA,
                                                          const __grid_constant__ CUtensorMap mapB, const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = smem;
  unsigned char *sB = smem + STAGES * TILE_A;
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], accum_full;
  __shared__ uint32_t tmem_base;
  __shared__ float gn_s[BN][NCH];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t m0 = int64_t(blockIdx.x) * BM;
  const int n0 = blockIdx.y * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accum_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < BN * NCH; i += blockDim.x) (&gn_s[0][0])[i] = a.gnc[int64_t(n0) * NCH + i];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    for (int kt = 0; kt < a.ktiles; ++kt) {
      const int s = kt % STAGES;
      if (kt >= STAGES && !mbar_wait(&empty[s], ((kt / STAGES) - 1) & 1)) {
        atomicOr(a.status, STATUS_TIMEOUT);
        break;
      }
      mbar_expect_tx(&full[s], TILE_A + TILE_B);
      tma_2d(sA + s * TILE_A, &mapA, &full[s], kt * BK, int(m0));
      tma_2d(sB + s * TILE_B, &mapB, &full[s], kt * BK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16(BM, BN);
    for (int kt = 0; kt < a.ktiles; ++kt) {
      const int s = kt % STAGES;
      if (!mbar_wait(&full[s], (kt / STAGES) & 1)) {
        atomicOr(a.status, STATUS_TIMEOUT);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int chunk = kt / a.ktpc;
      const bool first = (kt % a.ktpc) == 0;
      const uint32_t dt = tmem + chunk * BN;
      const uint32_t a0 = su32(sA + s * TILE_A), b0 = su32(sB + s * TILE_B);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k) {
        const uint32_t acc = (first && k == 0) ? 0u : 1u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(dt), "l"(sdesc(a0 + k * 32)), "l"(sdesc(b0 + k * 32)), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&empty[s]))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&accum_full))
                 : "memory");
  } else if (warp >= 2) {
    const int q = warp % 4;
    if (!mbar_wait(&accum_full, 0)) {
      atomicOr(a.status, STATUS_TIMEOUT);
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t row = m0 + q * 32 + lane;
      const bool valid = row < a.n;
      float xn[NCH];
#pragma unroll
      for (int c = 0; c < NCH; ++c) xn[c] = valid ? a.xnc[row * NCH + c] : 0.f;
      const bool bad = valid && !(isfinite(xn[0]) && isfinite(xn[1]) && isfinite(xn[2]) && isfinite(xn[3]));
      const int m = a.m;
      const int64_t ML = int64_t(m) * a.L;
      const float steps = float(a.ktpc * (BK / 16));
      uint32_t ha = 0, hb = 0;
      uint64_t word = 0;
      int nflag = 0, nchanged = 0, novf = 0;
      for (int cb = 0; cb < BN; cb += 16) {
        float ch[NCH][16];
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          if (c < a.nch) tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + c * BN + cb, ch[c]);
          else
#pragma unroll
            for (int j = 0; j < 16; ++j) ch[c][j] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int cl = cb + j;
          const int64_t col = n0 + cl;
          const int t = int(col / m), l = int(col - int64_t(t) * m);
          const float y = (ch[0][j] + ch[1][j]) + (ch[2][j] + ch[3][j]);
          float E = 2.f * kU * (fabsf(ch[0][j]) + fabsf(ch[1][j]) + fabsf(ch[2][j]) + fabsf(ch[3][j]));
#pragma unroll
          for (int c = 0; c < NCH; ++c) E = fmaf(2.f * kU * steps * xn[c], gn_s[cl][c], E);
          E *= 1.02f;
          int code;
          if (a.srp) {
            code = y > 0.f ? 1 : 0;
            if (valid && !bad && !(fabsf(y) > E)) {
              const int c64 = tc_fp64(a, row, col) > 0.0 ? 1 : 0;
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
            if (valid && !bad && !(dist > M && fabsf(tf) < 4194304.f)) {
              const double t3 = __ddiv_rn(__dadd_rn(tc_fp64(a, row, col), a.b64[col]), a.w);
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
            if (bad) code = INT32_MIN;
          }
          if (valid) {
            if (a.proj) a.proj[row * ML + col] = y;
            if (!a.srp && a.codes) a.codes[row * ML + col] = code;
          }
          if (a.srp) {
            word |= uint64_t(code) << l;
          } else {
            ha += uint32_t(code) * __ldg(a.ka + col);
            hb += uint32_t(code) * __ldg(a.kb + col);
          }
          if (l == m - 1) {  // the table is complete in this tile (128 % m == 0)
            if (valid) {
              uint64_t key = a.srp ? word : ((uint64_t(ha) << 32) | hb);
              if (a.srp && a.bits) a.bits[row * a.L + t] = word;
              if (bad) key = ~0ull;
              if (a.keys) a.keys[int64_t(t) * a.key_ld + row] = key;
            }
            ha = hb = 0;
            word = 0;
          }
        }
      }
      if (bad && blockIdx.y == 0) {
        if (a.counters) atomicAdd(a.counters + CNT_NONFINITE, 1ull);
        atomicOr(a.status, STATUS_NONFINITE);
      }
      if (a.counters) {
        if (nflag) atomicAdd(a.counters + CNT_FLAGGED, (unsigned long long)nflag);
        if (nchanged) atomicAdd(a.counters + CNT_CHANGED, (unsigned long long)nchanged);
        if (novf) atomicAdd(a.counters + CNT_OVERFLOW, (unsigned long long)novf);
      }
      if (novf) atomicOr(a.status, STATUS_OVERFLOW);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// Row chunk norms ||x_chunk||, widened to an upper bound; NaN when the row is not finite.
__global__ void __launch_bounds__(256) row_chunk_norms(const unsigned short *X, int64_t n, int d, int64_t ld,
                                                       int chunk_len, float *out) {
  const int64_t row = int64_t(blockIdx.x) * 8 + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (row >= n) return;
  float s[NCH] = {0.f, 0.f, 0.f, 0.f};
  bool fin = true;
  for (int j = lane; j < d; j += 32) {
    const float v = __uint_as_float(uint32_t(X[row * ld + j]) << 16);
    fin = fin && isfinite(v);
    const int c = min(j / chunk_len, NCH - 1);
#pragma unroll
    for (int cc = 0; cc < NCH; ++cc)
      if (cc == c) s[cc] = fmaf(v, v, s[cc]);
  }
#pragma unroll
  for (int cc = 0; cc < NCH; ++cc)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[cc] += __shfl_xor_sync(0xffffffffu, s[cc], o);
  const bool allfin = __all_sync(0xffffffffu, fin);
  if (lane < NCH) {
    const float widen = 1.f + float(d + 8) * kU;
    out[row * NCH + lane] = allfin ? sqrtf(s[lane] * widen) * (1.f + 2.f * kU) : __int_as_float(0x7fc00000);
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

bool make_map(CUtensorMap *map, const void *base, int64_t rows, int K, int64_t row_stride_elems) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)row_stride_elems * 2};
  cuuint32_t box[2] = {BK, 128};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int tc_chunk_ktiles(int d) {
  const int ktiles = (d + BK - 1) / BK;
  return (ktiles + NCH - 1) / NCH;
}

bool tc_dense_supported(const lsh_family_desc &fd, const lsh_matrix *X) {
  const int64_t ML = int64_t(fd.m) * fd.L;
  if (!kind_is_dense(fd.kind) || fd.compute != LSH_BF16 || !X || X->rowptr || X->dtype != LSH_BF16) return false;
  if (fd.d % 8 != 0 || X->ld % 8 != 0 || (reinterpret_cast<uintptr_t>(X->values) & 15) != 0) return false;
  if (ML % BN != 0 || BN % fd.m != 0 || (kind_is_srp(fd.kind) && fd.m > 64)) return false;
  if (X->n > (int64_t(1) << 31) - BM || (X->n + BM - 1) / BM > 2147483647) return false;
  return encode_fn() != nullptr;
}

cudaError_t launch_tc_dense(const SketchLaunch &p, const unsigned short *Gt16, const float *Gt, const float *gnc,
                            float *xnc_scratch, cudaStream_t stream) {
  if (p.n <= 0) return cudaSuccess;
  const int ktiles = (p.d + BK - 1) / BK;
  const int ktpc = tc_chunk_ktiles(p.d);
  const int64_t ML = int64_t(p.m) * p.L;
  row_chunk_norms<<<(unsigned)((p.n + 7) / 8), 256, 0, stream>>>(static_cast<const unsigned short *>(p.X), p.n, p.d,
                                                                   p.ld, ktpc * BK, xnc_scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap mA, mB;
  if (!make_map(&mA, p.X, p.n, p.d, p.ld) || !make_map(&mB, Gt16, ML, p.d, p.d)) return cudaErrorInvalidValue;
  TcArgs a{};
  a.n = p.n;
  a.d = p.d;
  a.m = p.m;
  a.L = p.L;
  a.srp = kind_is_srp(p.kind) ? 1 : 0;
  a.ktiles = ktiles;
  a.ktpc = ktpc;
  a.nch = (ktiles + ktpc - 1) / ktpc;
  a.X = static_cast<const unsigned short *>(p.X);
  a.ld = p.ld;
  a.Gt = Gt;
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
  const int smem = STAGES * (TILE_A + TILE_B) + 1024;
  e = cudaFuncSetAttribute(tc_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((p.n + BM - 1) / BM), (unsigned)(ML / BN));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  tc_dense_kernel<<<grid, 192, smem, stream>>>(mA, mB, a);
  return cudaGetLastError();
}

}  // namespace lsh
