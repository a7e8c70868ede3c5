// query.cu -- the query path of the (m, tau)-amplified LSH scheme (Sec. 3.1)
// with the exact rerank of Sec. 6: probe every table with the query's key,
// take the union of those buckets, rank the distinct candidates by exact
// distance and keep the k best by (distance, id).
//
// G CTAs per query (G = 1 for large batches, up to 32 for small ones: each
// takes every G-th chunk, and the last to finish merges the G lists), fused:
//   probe   thread t binary-searches the query's key in the sorted distinct
//           keys of table t -> (start, count) of its bucket;
//   gather  the union, flattened over tables, is processed in chunks of up
//           to kCap ids staged in shared memory;
//   dedup   each chunk's ids go through a shared-memory hash set; its
//           occupied slots are the chunk's distinct ids;
//   rerank  one thread per candidate: FP32 distance from the index's copy of
//           the data row, read with independent 16-byte loads (Euclidean for
//           E2LSH kinds, 1 - cos for SRP kinds);
//   top-k   merged into a running (distance, id) list.  An id that repeats in
//           a later chunk has the same distance: if it is in the list it is
//           skipped, and if it is not, it lost against a list that has only
//           improved since, so it cannot enter -- the union is deduplicated
//           exactly without a global sort.
#include <algorithm>

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace lsh {
namespace {

constexpr int kThreads = 256;
constexpr int kCap = 4096;  // candidate ids per chunk
constexpr int kHashBits = 13, kHash = 1 << kHashBits;  // dedup set: twice the chunk
constexpr int kMaxL = 128;
constexpr int kMaxK = 256;

struct QueryArgs {
  const uint64_t *qkeys;  // [L][q]
  int64_t q;
  int32_t L, k, metric, d;
  const void *Q;
  int32_t q_dtype;
  int64_t q_ld;
  const uint32_t *ids;     // [L][n]
  const uint64_t *ukeys;   // [L][n]
  const uint32_t *offsets; // [L][n+1]
  const int64_t *nb;       // [L]
  int64_t n;
  const void *X;
  int32_t x_dtype;
  int64_t x_ld;
  int32_t vec16;           // rows 16-byte aligned and d a multiple of the elements per 16 bytes
  int32_t *out_ids;
  float *out_dist;
  unsigned long long *counters;  // [4]: candidates, unique, max unique per CTA (atomicMax), queries
  // split queries: G CTAs per query, each a share of the chunks; partial
  // lists pd/pi [q][G][k]; done[q] counts finished CTAs (the last merges and
  // resets it to 0)
  const int64_t *q_live;   // optional device word: rows >= *q_live are padding, skipped
  int32_t G;
  float *pd;
  uint32_t *pi;
  uint32_t *done;
};

__device__ __forceinline__ float ld_elem(const void *p, int dtype, int64_t idx) {
  if (dtype == LSH_F32) return __ldg(reinterpret_cast<const float *>(p) + idx);
  const unsigned short h = __ldg(reinterpret_cast<const unsigned short *>(p) + idx);
  if (dtype == LSH_BF16) return __uint_as_float(uint32_t(h) << 16);
  return __half2float(__ushort_as_half(h));
}

__device__ __forceinline__ bool better(float da, uint32_t ia, float db, uint32_t ib) {
  return da < db || (da == db && ia < ib);
}

__global__ void __launch_bounds__(kThreads) query_kernel(const QueryArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  float *qv = reinterpret_cast<float *>(sm);                       // [d]
  uint32_t *bstart = reinterpret_cast<uint32_t *>(qv + a.d);       // [L]
  uint32_t *pre = bstart + kMaxL;                                  // [L+1]
  uint32_t *cand = pre + kMaxL + 1;                                // [kCap]
  float *cdist = reinterpret_cast<float *>(cand + kCap);           // [kCap]
  float *topd = cdist + kCap;                                      // [k]
  uint32_t *topi = reinterpret_cast<uint32_t *>(topd + kMaxK);     // [k]
  uint32_t *hset = topi + kMaxK;                                   // [kHash]
  __shared__ uint32_t wsum[kThreads / 32 + 1];
  __shared__ float red_d[kThreads / 32];
  __shared__ uint32_t red_i[kThreads / 32];
  __shared__ int red_s[kThreads / 32];
  __shared__ float qnorm2;

  const int64_t qi = blockIdx.x / a.G;
  const int g = int(blockIdx.x % a.G);
  if (a.q_live && qi >= *a.q_live) return;  // a padding row of a fixed-size batch
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int L = a.L, k = a.k, d = a.d;

  // query row in FP32 and its squared norm
  float part = 0.f;
  for (int j = tid; j < d; j += kThreads) {
    const float v = ld_elem(a.Q, a.q_dtype, qi * a.q_ld + j);
    qv[j] = v;
    part += v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) red_d[warp] = part;
  // probe: table t -> bucket (start, count)
  for (int t = tid; t < L; t += kThreads) {
    const uint64_t key = a.qkeys[int64_t(t) * a.q + qi];
    const uint64_t *uk = a.ukeys + int64_t(t) * a.n;
    int64_t lo = 0, hi = a.nb[t];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (uk[mid] < key) lo = mid + 1; else hi = mid;
    }
    uint32_t s = 0, c = 0;
    if (lo < a.nb[t] && uk[lo] == key) {
      const uint32_t *of = a.offsets + int64_t(t) * (a.n + 1);
      s = of[lo];
      c = of[lo + 1] - s;
    }
    bstart[t] = s;
    pre[t + 1] = c;
  }
  for (int r = tid; r < k; r += kThreads) {
    topd[r] = __int_as_float(0x7f800000);
    topi[r] = 0xffffffffu;
  }
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) s += red_d[w];
    qnorm2 = s;
    pre[0] = 0;
    for (int t = 0; t < L; ++t) pre[t + 1] += pre[t];
  }
  __syncthreads();
  const uint32_t C = pre[L];
  uint32_t uniq_total = 0, uniq_max = 0;

  for (uint32_t c0 = uint32_t(g) * kCap; c0 < C; c0 += uint32_t(a.G) * kCap) {
    const uint32_t cc = min(uint32_t(kCap), C - c0);
    // dedup through a shared-memory hash set (open addressing, load <= 1/2):
    // the gather inserts every id of the chunk; the distinct ids are then the
    // occupied slots (their order does not matter to the top-k merge)
    for (uint32_t i = tid; i < kHash; i += kThreads) hset[i] = 0xffffffffu;
    __syncthreads();
    for (uint32_t f = tid; f < cc; f += kThreads) {
      const uint32_t g = c0 + f;
      int lo = 0, hi = L;  // last t with pre[t] <= g
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= g) lo = mid; else hi = mid;
      }
      const uint32_t id = a.ids[int64_t(lo) * a.n + bstart[lo] + (g - pre[lo])];
      uint32_t slot = (id * 2654435761u) >> (32 - kHashBits);
      for (uint32_t probe = 0; probe < kHash; ++probe) {
        const uint32_t old = atomicCAS(&hset[slot], 0xffffffffu, id);
        if (old == 0xffffffffu || old == id) break;
        slot = (slot + 1) & (kHash - 1);
      }
    }
    __syncthreads();
    // compact the occupied slots into cand with a block scan
    const uint32_t per = kHash / kThreads;
    const uint32_t b0 = tid * per, b1 = b0 + per;
    uint32_t cnt = 0;
    for (uint32_t f = b0; f < b1; ++f) cnt += hset[f] != 0xffffffffu ? 1u : 0u;
    uint32_t s = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    if (lane == 31) wsum[warp] = s;
    __syncthreads();
    if (tid == 0) {
      uint32_t run = 0;
      for (int w = 0; w < kThreads / 32; ++w) {
        const uint32_t v = wsum[w];
        wsum[w] = run;
        run += v;
      }
      wsum[kThreads / 32] = run;
    }
    __syncthreads();
    uint32_t pos = wsum[warp] + s - cnt;
    const uint32_t U = wsum[kThreads / 32];
    for (uint32_t f = b0; f < b1; ++f)
      if (hset[f] != 0xffffffffu) cand[pos++] = hset[f];
    __syncthreads();
    uniq_total += U;
    uniq_max = max(uniq_max, U);
    // distances: one thread per candidate, its row read with independent
    // 16-byte loads (many rows in flight per SM), the query from shared memory
    for (uint32_t u = tid; u < U; u += kThreads) {
      const uint32_t id = cand[u];
      const int64_t base = int64_t(id) * a.x_ld;
      float acc = 0.f, xx = 0.f;
      if (a.vec16) {
        // rows are 16-byte aligned: eight 2-byte or four 4-byte elements a load
        const uint4 *xr = reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(a.X) +
                                                          base * (a.x_dtype == LSH_F32 ? 4 : 2));
        const int per = a.x_dtype == LSH_F32 ? 4 : 8;
        const int nv = d / per;
        // four partial sums per candidate (independent FMA chains); the query
        // row read from shared memory as float4 (a broadcast to the warp)
        float acc4[4] = {0.f, 0.f, 0.f, 0.f}, xx4[4] = {0.f, 0.f, 0.f, 0.f};
        const float4 *q4 = reinterpret_cast<const float4 *>(qv);
        for (int v0 = 0; v0 < nv; v0 += 8) {
          uint4 w[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) w[t] = v0 + t < nv ? __ldg(xr + v0 + t) : make_uint4(0, 0, 0, 0);
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            if (v0 + t >= nv) break;
            float x[8];
            const uint32_t ww[4] = {w[t].x, w[t].y, w[t].z, w[t].w};
            if (a.x_dtype == LSH_F32) {
#pragma unroll
              for (int e = 0; e < 4; ++e) x[e] = __uint_as_float(ww[e]);
            } else if (a.x_dtype == LSH_BF16) {
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                x[2 * e] = __uint_as_float(ww[e] << 16);
                x[2 * e + 1] = __uint_as_float(ww[e] & 0xFFFF0000u);
              }
            } else {
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&ww[e]));
                x[2 * e] = f.x;
                x[2 * e + 1] = f.y;
              }
            }
            const int j0 = (v0 + t) * per;  // a multiple of 4
            float qj[8];
            const float4 qa = q4[j0 / 4];
            qj[0] = qa.x; qj[1] = qa.y; qj[2] = qa.z; qj[3] = qa.w;
            if (per == 8) {
              const float4 qb = q4[j0 / 4 + 1];
              qj[4] = qb.x; qj[5] = qb.y; qj[6] = qb.z; qj[7] = qb.w;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              if (e >= per) break;
              if (a.metric == 0) {
                const float df = qj[e] - x[e];
                acc4[e & 3] = fmaf(df, df, acc4[e & 3]);
              } else {
                acc4[e & 3] = fmaf(qj[e], x[e], acc4[e & 3]);
                xx4[e & 3] = fmaf(x[e], x[e], xx4[e & 3]);
              }
            }
          }
        }
        acc = (acc4[0] + acc4[1]) + (acc4[2] + acc4[3]);
        xx = (xx4[0] + xx4[1]) + (xx4[2] + xx4[3]);
      } else {
        for (int j = 0; j < d; ++j) {
          const float x = ld_elem(a.X, a.x_dtype, base + j);
          if (a.metric == 0) {
            const float df = qv[j] - x;
            acc = fmaf(df, df, acc);
          } else {
            acc = fmaf(qv[j], x, acc);
            xx = fmaf(x, x, xx);
          }
        }
      }
      float dist;
      if (a.metric == 0) {
        dist = sqrtf(acc);
      } else {
        dist = (qnorm2 > 0.f && xx > 0.f) ? 1.f - acc / (sqrtf(qnorm2) * sqrtf(xx)) : 1.f;
      }
      cdist[u] = dist;
    }
    __syncthreads();
    // drop candidates already in the top-k list (same id => same distance)
    for (uint32_t u = tid; u < U; u += kThreads) {
      const uint32_t id = cand[u];
      for (int r = 0; r < k; ++r)
        if (topi[r] == id) {
          cdist[u] = __int_as_float(0x7f800000);
          cand[u] = 0xffffffffu;
          break;
        }
    }
    __syncthreads();
    // merge: k rounds of block argmin over (list entries not yet taken) U (chunk)
    // list and chunk entries are tagged by source; the new list is built in place
    // in registers of thread 0 via shared buffers.
    {
      // candidates: list slots r (source 1) and chunk slots u (source 0)
      __shared__ float newd[kMaxK];
      __shared__ uint32_t newi[kMaxK];
      for (int r = 0; r < k; ++r) {
        float bd = __int_as_float(0x7f800000);
        uint32_t bi = 0xffffffffu;
        int bs = -1;  // encoded slot: >= 0 chunk index, < -1 list index (-(r)-2)
        for (uint32_t u = tid; u < U; u += kThreads)
          if (cand[u] != 0xffffffffu && better(cdist[u], cand[u], bd, bi)) {
            bd = cdist[u];
            bi = cand[u];
            bs = int(u);
          }
        for (int rr = tid; rr < k; rr += kThreads)
          if (topi[rr] != 0xffffffffu && better(topd[rr], topi[rr], bd, bi)) {
            bd = topd[rr];
            bi = topi[rr];
            bs = -rr - 2;
          }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float od = __shfl_xor_sync(0xffffffffu, bd, o);
          const uint32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
          const int os = __shfl_xor_sync(0xffffffffu, bs, o);
          if (better(od, oi, bd, bi)) {
            bd = od;
            bi = oi;
            bs = os;
          }
        }
        if (lane == 0) {
          red_d[warp] = bd;
          red_i[warp] = bi;
          red_s[warp] = bs;
        }
        __syncthreads();
        if (tid == 0) {
          float fd = red_d[0];
          uint32_t fi = red_i[0];
          int fs = red_s[0];
          for (int w = 1; w < kThreads / 32; ++w)
            if (better(red_d[w], red_i[w], fd, fi)) {
              fd = red_d[w];
              fi = red_i[w];
              fs = red_s[w];
            }
          newd[r] = fd;
          newi[r] = fi;
          if (fs >= 0) cand[fs] = 0xffffffffu;             // taken from the chunk
          else if (fs <= -2) topi[-fs - 2] = 0xffffffffu;  // taken from the list
        }
        __syncthreads();
      }
      for (int r = tid; r < k; r += kThreads) {
        topd[r] = newd[r];
        topi[r] = newi[r];
      }
      __syncthreads();
    }
  }
  if (tid == 0 && a.counters) {
    if (g == 0) atomicAdd(a.counters + 0, (unsigned long long)C);
    atomicAdd(a.counters + 1, (unsigned long long)uniq_total);
    atomicMax(a.counters + 2, (unsigned long long)uniq_max);
    if (g == 0) atomicAdd(a.counters + 3, 1ull);
  }
  if (a.G > 1) {
    // hand this CTA's list over; the last CTA of the query merges all G lists
    __shared__ int s_last;
    const int64_t pb = (qi * a.G + g) * k;
    for (int r = tid; r < k; r += kThreads) {
      a.pd[pb + r] = topd[r];
      a.pi[pb + r] = topi[r];
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(a.done + qi, 1u) == uint32_t(a.G - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int U = a.G * k;  // <= kCap (launch_query bounds G)
    for (int u = tid; u < U; u += kThreads) {
      cand[u] = __ldcg(a.pi + qi * a.G * k + u);
      cdist[u] = __ldcg(a.pd + qi * a.G * k + u);
    }
    __shared__ uint32_t s_win;
    __syncthreads();
    // k rounds of block argmin over the G lists; an id in several lists has
    // the same distance in each, so every copy of the winner is retired
    for (int r = 0; r < k; ++r) {
      float bd = __int_as_float(0x7f800000);
      uint32_t bi = 0xffffffffu;
      for (int u = tid; u < U; u += kThreads)
        if (cand[u] != 0xffffffffu && better(cdist[u], cand[u], bd, bi)) {
          bd = cdist[u];
          bi = cand[u];
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float od = __shfl_xor_sync(0xffffffffu, bd, o);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (better(od, oi, bd, bi)) {
          bd = od;
          bi = oi;
        }
      }
      if (lane == 0) {
        red_d[warp] = bd;
        red_i[warp] = bi;
      }
      __syncthreads();
      if (tid == 0) {
        float fd = red_d[0];
        uint32_t fi = red_i[0];
        for (int w = 1; w < kThreads / 32; ++w)
          if (better(red_d[w], red_i[w], fd, fi)) {
            fd = red_d[w];
            fi = red_i[w];
          }
        topd[r] = fd;
        topi[r] = fi;
        s_win = fi;
      }
      __syncthreads();
      const uint32_t win = s_win;
      if (win != 0xffffffffu)
        for (int u = tid; u < U; u += kThreads)
          if (cand[u] == win) cand[u] = 0xffffffffu;
      __syncthreads();
    }
    if (tid == 0) a.done[qi] = 0;  // ready for the next launch on this scratch
  }
  for (int r = tid; r < k; r += kThreads) {
    const bool ok = topi[r] != 0xffffffffu;
    a.out_ids[qi * k + r] = ok ? int32_t(topi[r]) : -1;
    a.out_dist[qi * k + r] = ok ? topd[r] : __int_as_float(0x7f800000);
  }
}

}  // namespace

namespace {
int num_sms_q() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}
int64_t align16(int64_t b) { return (b + 15) & ~int64_t(15); }
}  // namespace

int query_split(int64_t q, int32_t k) {
  // enough CTAs for the SMs (four each); at most 32 per query and G k <= kCap
  const int64_t target = int64_t(num_sms_q()) * 4;
  int64_t G = q > 0 ? target / q : 1;
  G = std::max<int64_t>(1, std::min<int64_t>(G, std::min<int64_t>(32, kCap / std::max(k, 1))));
  return int(G);
}

size_t query_scratch_bytes(int64_t q_max, int32_t k) {
  const int64_t lists = std::max<int64_t>(q_max, int64_t(num_sms_q()) * 4 + 32) * k;
  return size_t(align16(q_max * 4) + 2 * align16(lists * 4));
}

cudaError_t launch_query(const uint64_t *qkeys, int64_t q, int32_t L, int32_t k, int32_t metric, int32_t d,
                         const void *Q, int32_t q_dtype, int64_t q_ld, const lsh_index_s *idx, int32_t *out_ids,
                         float *out_dist, unsigned long long *counters, void *scratch, int64_t scratch_q,
                         const int64_t *q_live, cudaStream_t stream) {
  if (q <= 0) return cudaSuccess;
  if (L > kMaxL || k > kMaxK) return cudaErrorInvalidValue;
  QueryArgs a{};
  a.qkeys = qkeys;
  a.q = q;
  a.L = L;
  a.k = k;
  a.metric = metric;
  a.d = d;
  a.Q = Q;
  a.q_dtype = q_dtype;
  a.q_ld = q_ld;
  a.ids = idx->d_ids;
  a.ukeys = idx->d_ukeys;
  a.offsets = idx->d_offsets;
  a.nb = idx->d_nb;
  a.n = idx->n;
  a.X = idx->d_data;
  a.x_dtype = idx->data_dtype;
  a.x_ld = idx->data_ld;
  {
    const int64_t es = idx->data_dtype == LSH_F32 ? 4 : 2;
    a.vec16 = (d % (16 / es) == 0) && (a.x_ld * es) % 16 == 0 && (reinterpret_cast<uintptr_t>(a.X) & 15) == 0;
  }
  a.out_ids = out_ids;
  a.out_dist = out_dist;
  a.counters = counters;
  a.q_live = q_live;
  a.G = scratch && q <= scratch_q ? query_split(q, k) : 1;
  if (a.G > 1) {
    // layout of query_scratch_bytes(scratch_q, k): done[scratch_q], then the two list arrays
    char *sb = static_cast<char *>(scratch);
    const int64_t lists = std::max<int64_t>(scratch_q, int64_t(num_sms_q()) * 4 + 32) * k;
    a.done = reinterpret_cast<uint32_t *>(sb);
    a.pd = reinterpret_cast<float *>(sb + align16(scratch_q * 4));
    a.pi = reinterpret_cast<uint32_t *>(sb + align16(scratch_q * 4) + align16(lists * 4));
    if (q * a.G * k > lists) a.G = 1;
  }
  const int smem = d * 4 + (2 * kMaxL + 1) * 4 + kCap * 8 + kMaxK * 8 + kHash * 4;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(query_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (q * a.G > INT32_MAX) return cudaErrorInvalidValue;
  query_kernel<<<(unsigned)(q * a.G), kThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace lsh
