// lsh_api.cpp -- the C ABI of include/lsh.h: argument validation, handle
// ownership, per-call temporaries and error reporting around the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

namespace lsh {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void count_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_error(const std::string &msg) { g_last_error = msg; }

lsh_status fail(lsh_status st, const std::string &msg) {
  g_last_error = msg;
  return st;
}

lsh_status cuda_fail(cudaError_t e, const char *what) {
  g_last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? LSH_ENOMEM : LSH_ECUDA;
}

namespace {

lsh_status validate_desc(const lsh_family_desc &d) {
  if (d.kind < LSH_E2LSH || d.kind > LSH_CSL_SRP) return fail(LSH_EINVAL, "unknown kind");
  if (d.kind == LSH_CSL_SRP) {
    if (d.nnz_per_col < 0 || d.nnz_per_col > d.m) return fail(LSH_EINVAL, "CSSRP-L needs 1 <= nnz_per_col <= m");
    if (int64_t(d.d) * incidences(d) >= (int64_t(1) << 31)) return fail(LSH_EINVAL, "d * nnz_per_col too large");
  }
  if (d.d < 1) return fail(LSH_EINVAL, "d must be >= 1");
  if (d.m < 1) return fail(LSH_EINVAL, "m must be >= 1");
  if (d.L < 1) return fail(LSH_EINVAL, "L must be >= 1");
  if (!(d.w > 0.0) || !std::isfinite(d.w)) return fail(LSH_EINVAL, "w must be finite and > 0");
  if (kind_is_dense(d.kind)) {
    if (d.compute != LSH_F32 && d.compute != LSH_BF16 && d.compute != LSH_FP8_E4M3)
      return fail(LSH_EUNSUPPORTED, "dense families store G in FP32, BF16 or FP8 E4M3");
    if (int64_t(d.d) * d.m * d.L > (int64_t(1) << 31)) return fail(LSH_EINVAL, "G too large");
    return LSH_OK;
  }
  if (d.N < 1 || d.N > LSH_MAX_MODES) return fail(LSH_EINVAL, "N must be in [1, 8]");
  int64_t D = 1, M = 1;
  for (int k = 0; k < d.N; ++k) {
    if (d.dims[k] < 1 || d.mdims[k] < 1) return fail(LSH_EINVAL, "mode sizes must be >= 1");
    if (d.mdims[k] > 65535) return fail(LSH_EINVAL, "mode sketch size must be < 65536");
    D *= d.dims[k];
    M *= d.mdims[k];
    if (D > (int64_t(1) << 31) || M > (int64_t(1) << 31)) return fail(LSH_EINVAL, "modes too large");
  }
  if (M != d.m) return fail(LSH_EINVAL, "prod(mdims) must equal m");
  if (D < d.d) return fail(LSH_EINVAL, "prod(dims) must be >= d");
  if ((d.kind == LSH_CS_E2LSH || d.kind == LSH_CS_SRP || d.kind == LSH_CSL_SRP) && (d.N != 1 || d.dims[0] != d.d))
    return fail(LSH_EINVAL, "CS kinds take N = 1, dims = {d}, mdims = {m}");
  if (d.m > 65535) return fail(LSH_EINVAL, "m must be < 65536");
  return LSH_OK;
}

template <class T>
cudaError_t upload(T **dst, const T *src, size_t count) {
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), count * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

void free_family(lsh_family_s *f) {
  if (!f) return;
  cudaFree(f->d_bins);
  cudaFree(f->d_signs);
  cudaFree(f->d_b32);
  cudaFree(f->d_b64);
  cudaFree(f->d_ka);
  cudaFree(f->d_kb);
  cudaFree(f->d_G);
  cudaFree(f->d_Gt);
  cudaFree(f->d_gnorm);
  cudaFree(f->d_Gt16);
  cudaFree(f->d_gnc);
  cudaFree(f->d_Gint);
  cudaFree(f->d_Gt8);
  cudaFree(f->d_status);
  cudaFree(f->d_colmajor);
  cudaFree(f->d_mlist);
  cudaFree(f->d_mseg);
  delete f;
}

lsh_status validate_matrix(const lsh_family_s *f, const lsh_matrix *X, bool allow_csr) {
  if (!X) return fail(LSH_EINVAL, "X is NULL");
  if (X->n < 0) return fail(LSH_EINVAL, "n must be >= 0");
  if (X->n > int64_t(UINT32_MAX) - 1) return fail(LSH_EINVAL, "n must be < 2^32 - 1");
  if (X->d != f->host.desc.d) return fail(LSH_EINVAL, "X->d differs from the family's d");
  const bool csr = X->rowptr != nullptr;
  if (csr) {
    if (!allow_csr) return fail(LSH_EINVAL, "CSR input not accepted here");
    if (X->n > 0 && (!X->col || !X->values)) return fail(LSH_EINVAL, "CSR needs col and values");
    if (X->dtype != LSH_F32) return fail(LSH_EINVAL, "CSR values must be FP32");
    return LSH_OK;
  }
  if (X->n > 0 && !X->values) return fail(LSH_EINVAL, "values is NULL");
  if (X->ld < X->d) return fail(LSH_EINVAL, "ld must be >= d");
  if (X->dtype != LSH_F32 && X->dtype != LSH_BF16 && X->dtype != LSH_F16 && X->dtype != LSH_FP8_E4M3)
    return fail(LSH_EINVAL, "unknown dtype");
  if (X->dtype == LSH_FP8_E4M3 && !X->row_scale) return fail(LSH_EINVAL, "FP8 input needs row_scale");
  return LSH_OK;
}

size_t dtype_size(int dt) { return dt == LSH_F32 ? 4 : (dt == LSH_FP8_E4M3 ? 1 : 2); }

}  // namespace

SketchLaunch family_launch(const lsh_family_s *f) {
  const lsh_family_desc &d = f->host.desc;
  SketchLaunch p{};
  p.d = d.d;
  p.kind = d.kind;
  p.m = d.m;
  p.L = d.L;
  p.N = d.N;
  for (int k = 0; k < d.N; ++k) {
    p.dims[k] = d.dims[k];
    p.mdims[k] = d.mdims[k];
  }
  p.dsum = int32_t(f->host.dsum);
  p.lc = incidences(d);
  p.cap = f->sketch_cap;
  p.bins = f->d_bins;
  p.signs = f->d_signs;
  p.b32 = f->d_b32;
  p.b64 = f->d_b64;
  p.ka = f->d_ka;
  p.kb = f->d_kb;
  p.w = d.w;
  p.sqrtm = kind_scaled(d.kind) ? std::sqrt(double(d.m)) : 1.0;
  p.status = f->d_status;
  return p;
}

// Hash into keys [L][key_ld] (and the optional outputs).  Stream-ordered.
lsh_status hash_impl(lsh_family_s *f, const lsh_matrix *X, void *codes, uint64_t *keys, int64_t key_ld,
                     float *proj, unsigned long long *counters, cudaStream_t stream) {
  const lsh_family_desc &d = f->host.desc;
  if (X->n == 0) return LSH_OK;
  if (kind_is_dense(d.kind) && X->rowptr) return fail(LSH_EUNSUPPORTED, "dense E2LSH/SRP takes dense rows");
  if (X->dtype == LSH_FP8_E4M3 && !(f->d_Gt8 && tc_dense_supported(d, X)))
    return fail(LSH_EUNSUPPORTED, "FP8 rows are hashed by dense families with an FP8 G on the tensor cores "
                                  "(d <= 16384 and the row stride multiples of 16, m in 8..64 dividing 64 or E2LSH with m = 128, "
                                  "m*L a multiple of 128)");
  SketchLaunch p = family_launch(f);
  p.X = X->values;
  p.row_scale = X->row_scale;
  p.dtype = X->dtype;
  p.n = X->n;
  p.ld = X->ld;
  if (kind_is_srp(d.kind))
    p.bits = static_cast<uint64_t *>(codes);
  else
    p.codes = static_cast<int32_t *>(codes);
  p.keys = keys;
  p.key_ld = key_ld;
  p.proj = proj;
  p.counters = counters;
  p.status = f->d_status;
  if (kind_is_dense(d.kind) && (f->d_Gt16 || f->d_Gt8) && tc_dense_supported(d, X)) {
    void *scratch = nullptr;
    LSH_CUDA_TRY(cudaMallocAsync(&scratch, tc_dense_scratch_bytes(X->n, int64_t(d.m) * d.L), stream));
    const void *gtc = X->dtype == LSH_FP8_E4M3 ? static_cast<const void *>(f->d_Gt8) : f->d_Gt16;
    const cudaError_t e = launch_tc_dense(p, gtc, f->d_Gt, f->d_gnc, f->d_Gint, scratch, stream);
    cudaFreeAsync(scratch, stream);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core dense hash");
    count_launches(6);  // row records, the tensor-core kernel, the queue grouping (3), the recheck
    return LSH_OK;
  }
  if (kind_is_dense(d.kind)) {
    if (keys) LSH_CUDA_TRY(cudaMemsetAsync(keys, 0, sizeof(uint64_t) * size_t(key_ld) * d.L, stream));
    if (p.bits) LSH_CUDA_TRY(cudaMemsetAsync(p.bits, 0, size_t(X->n) * d.L * ((d.m + 63) / 64) * 8, stream));
    // batches of 8192 rows or more queue their boundary rechecks for a second
    // kernel (queue from the stream-ordered pool); smaller ones recheck in place
    void *qbuf = nullptr;
    if (X->n >= 8192) {
      const int64_t qcap = dense_queue_cap(X->n, int64_t(d.m) * d.L);
      LSH_CUDA_TRY(cudaMallocAsync(&qbuf, size_t(16 + 16 * qcap), stream));
      p.qcount = static_cast<uint32_t *>(qbuf);
      p.queue = reinterpret_cast<int4 *>(static_cast<char *>(qbuf) + 16);
      p.qcap = uint32_t(qcap);
      LSH_CUDA_TRY(cudaMemsetAsync(qbuf, 0, 16, stream));
    }
    const cudaError_t e = launch_dense_fp32(p, f->d_G, f->d_Gt, f->d_gnorm, stream);
    if (qbuf) cudaFreeAsync(qbuf, stream);
    if (e != cudaSuccess) return cuda_fail(e, "dense FP32 hash");
    count_launches(qbuf ? 2 : 1);
    return LSH_OK;
  }
  if (X->rowptr && d.kind == LSH_CSL_SRP) return fail(LSH_EUNSUPPORTED, "CSSRP-L hashes dense rows only");
  if (X->rowptr) {
    if (d.N == 1 && d.m > 32768) return fail(LSH_EUNSUPPORTED, "CSR count-sketch path needs m <= 32768");
    for (int k = 0; k < d.N; ++k)
      if (d.mdims[k] > 32768) return fail(LSH_EUNSUPPORTED, "CSR HCS hashing needs mode sketch sizes <= 32768");
    if (p.bits) LSH_CUDA_TRY(cudaMemsetAsync(p.bits, 0, size_t(X->n) * d.L * ((d.m + 63) / 64) * 8, stream));
    LSH_CUDA_TRY(launch_sketch_csr(p, X->rowptr, X->col, static_cast<const float *>(X->values), f->d_colmajor,
                                   f->d_mseg, stream));
    count_launches(1);
    return LSH_OK;
  }
  SketchPlan sp = plan_sketch_dense(d.d, d.m, d.L, f->sketch_cap, X->dtype);
  if (!sp.ok) {
    // rows too long for the dense-row kernel's shared-memory tile: the warp-per-row
    // kernel reads them in place (per-bin bounds need the member records, d < 65536)
    const bool cs = d.kind == LSH_CS_E2LSH || d.kind == LSH_CS_SRP;
    if (d.kind == LSH_CSL_SRP) return fail(LSH_EUNSUPPORTED, "CSSRP-L rows must fit the dense-row kernel's tile");
    if (!f->d_mseg || (cs && !f->d_colmajor))
      return fail(LSH_EUNSUPPORTED, "d too large for the dense-row kernel (and >= 65536 for the row-wise one)");
    if (!cs)
      for (int k = 0; k < d.N; ++k)
        if (d.mdims[k] > 32768) return fail(LSH_EUNSUPPORTED, "row-wise HCS hashing needs mode sketch sizes <= 32768");
    if (p.bits) LSH_CUDA_TRY(cudaMemsetAsync(p.bits, 0, size_t(X->n) * d.L * ((d.m + 63) / 64) * 8, stream));
    LSH_CUDA_TRY(launch_sketch_csr(p, nullptr, nullptr, nullptr, f->d_colmajor, f->d_mseg, stream));
    count_launches(1);
    return LSH_OK;
  }
  if (!sketch_pin_fits(d.d, d.m, d.L, f->sketch_cap))
    return fail(LSH_EUNSUPPORTED, "the pinned sketch plan (lsh_set_sketch_plan) does not fit this shape");
  if (p.bits && d.m > 64)  // multi-word SRP codes are assembled with atomic ORs
    LSH_CUDA_TRY(cudaMemsetAsync(p.bits, 0, size_t(X->n) * d.L * ((d.m + 63) / 64) * 8, stream));
  // large batches (8192 rows or more) defer their boundary rechecks to a
  // second kernel (queue from the stream-ordered pool); smaller ones (query
  // batches among them) recheck in place and allocate nothing
  void *qbuf = nullptr;
  if (f->d_mlist && X->n >= 8192) {
    const int64_t qcap = sketch_queue_cap(X->n, d.L, d.m);
    LSH_CUDA_TRY(cudaMallocAsync(&qbuf, size_t(16 + 16 * qcap), stream));
    p.qcount = static_cast<uint32_t *>(qbuf);
    p.queue = reinterpret_cast<int4 *>(static_cast<char *>(qbuf) + 16);
    p.qcap = uint32_t(qcap);
    LSH_CUDA_TRY(cudaMemsetAsync(qbuf, 0, 16, stream));
  }
  cudaError_t e = launch_sketch_dense(p, stream);
  if (e == cudaSuccess && qbuf) e = launch_sketch_recheck(p, f->d_mlist, f->d_mseg, stream);
  if (qbuf) cudaFreeAsync(qbuf, stream);
  if (e != cudaSuccess) return cuda_fail(e, "dense-row sketch hash");
  count_launches(qbuf ? 2 : 1);
  return LSH_OK;
}

namespace {

lsh_family_desc normalized(const lsh_family_desc &in) {
  lsh_family_desc d = in;
  if ((d.kind == LSH_CS_E2LSH || d.kind == LSH_CS_SRP || d.kind == LSH_CSL_SRP || kind_is_dense(d.kind)) &&
      d.N == 0) {
    d.N = 1;
    d.dims[0] = d.d;
    d.mdims[0] = d.m;
  }
  return d;
}

// The per-call temporaries (keys, sort buffers, counters) come from the
// device's default stream-ordered pool.  Keep freed blocks in the pool instead
// of returning them to the driver at every synchronisation, so that repeated
// calls reuse them without remapping (done once per device).
void keep_pool_warm() {
  static std::atomic<uint64_t> done_mask{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return;
  const uint64_t bit = uint64_t(1) << dev;
  if (done_mask.load() & bit) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done_mask.fetch_or(bit);
}

// Hash X into temporary keys and sort/segment them into the index's arrays.
lsh_status index_fill(lsh_index_s *idx, const lsh_matrix *X, cudaStream_t stream) {
  const int L = idx->L;
  const int64_t n = idx->n;
  keep_pool_warm();
  uint64_t *keys = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&keys), sizeof(uint64_t) * size_t(n) * L, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync keys");
  lsh_status st = hash_impl(idx->fam, X, nullptr, keys, n, nullptr, nullptr, stream);
  if (st == LSH_OK) {
    e = build_tables(keys, n, L, idx->d_ids, idx->d_ukeys, idx->d_offsets, idx->d_nb, stream);
    if (e != cudaSuccess) st = cuda_fail(e, "build_tables");
  }
  cudaFreeAsync(keys, stream);
  return st;
}

}  // namespace
}  // namespace lsh

using namespace lsh;

extern "C" {

const char *lsh_last_error(void) { return g_last_error.c_str(); }

const char *lsh_version(void) { return "lsh-gb300 0.1 (sm_103a)"; }

uint64_t lsh_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

lsh_status lsh_make_family(const lsh_family_desc *desc, lsh_family_t *out) {
  if (!desc || !out) return fail(LSH_EINVAL, "NULL argument");
  *out = nullptr;
  const lsh_family_desc d = normalized(*desc);
  lsh_status st = validate_desc(d);
  if (st != LSH_OK) return st;
  lsh_family_s *f = new (std::nothrow) lsh_family_s();
  if (!f) return fail(LSH_ENOMEM, "host allocation");
  try {
    sample_family(d, f->host);
  } catch (const std::bad_alloc &) {
    delete f;
    return fail(LSH_ENOMEM, "host allocation");
  }
  cudaGetDevice(&f->device);
  const HostFamily &h = f->host;
  f->sketch_cap = sketch_capacity(h);
  cudaError_t e = cudaSuccess;
  if (!h.bins.empty()) {
    std::vector<uint16_t> b16(h.bins.begin(), h.bins.end());
    e = upload(&f->d_bins, b16.data(), b16.size());
    if (e == cudaSuccess) e = upload(&f->d_signs, h.signs.data(), h.signs.size());
  }
  std::vector<float> b32(h.b.size());
  for (size_t i = 0; i < b32.size(); ++i) b32[i] = float(h.b[i]);
  if (e == cudaSuccess) e = upload(&f->d_b32, b32.data(), b32.size());
  if (e == cudaSuccess) e = upload(&f->d_b64, h.b.data(), h.b.size());
  if (e == cudaSuccess) e = upload(&f->d_ka, h.ka.data(), h.ka.size());
  if (e == cudaSuccess) e = upload(&f->d_kb, h.kb.data(), h.kb.size());
  if (e == cudaSuccess && !h.G.empty()) {
    e = upload(&f->d_G, h.G.data(), h.G.size());
    const size_t ml = size_t(d.m) * d.L;
    std::vector<float> gt(h.G.size()), gn(ml);
    for (size_t c = 0; c < ml; ++c) {
      double s2 = 0.0;
      for (int j = 0; j < d.d; ++j) {
        const float g = h.G[size_t(j) * ml + c];
        gt[c * d.d + j] = g;
        s2 += double(g) * double(g);
      }
      gn[c] = float(std::sqrt(s2) * (1.0 + 1e-6));  // rounded up
    }
    if (e == cudaSuccess) e = upload(&f->d_Gt, gt.data(), gt.size());
    if (e == cudaSuccess) e = upload(&f->d_gnorm, gn.data(), gn.size());
    if (e == cudaSuccess && (d.compute == LSH_BF16 || d.compute == LSH_FP8_E4M3)) {
      // the compact copy of G^T for the tensor cores (bf16 bits or E4M3 codes),
      // its column norms per K chunk, and each column as integers on the grid
      // of its least exponent (a value is M 2^E, M < 256 resp. M < 16)
      const bool fp8 = d.compute == LSH_FP8_E4M3;
      auto parts = [fp8](float v, int32_t &M, int &E) -> bool {  // false for zero
        uint32_t u;
        std::memcpy(&u, &v, 4);
        const uint32_t a = u & 0x7FFFFFFFu;
        if (a == 0) return false;
        const int ef = int(a >> 23) - 127;
        if (!fp8) {  // bf16: 7 stored fraction bits
          const uint32_t ex = a >> 23, fr = (a >> 16) & 0x7F;
          M = int32_t(ex ? (fr | 0x80) : fr);
          E = ex ? int(ex) - 134 : -133;
        } else if (ef >= -6) {  // normal E4M3: 3 fraction bits
          M = int32_t(8 + ((a >> 20) & 7));
          E = ef - 3;
        } else {  // subnormal E4M3: f 2^-9
          M = int32_t(std::ldexp(double(v < 0 ? -v : v), 9));
          E = -9;
        }
        if (u >> 31) M = -M;
        return true;
      };
      std::vector<uint16_t> g16;
      std::vector<uint8_t> g8;
      if (fp8) g8.resize(gt.size());
      else g16.resize(gt.size());
      for (size_t i = 0; i < gt.size(); ++i) {
        uint32_t u;
        std::memcpy(&u, &gt[i], 4);
        if (!fp8) {
          g16[i] = uint16_t(u >> 16);  // exact: the entries are bf16 values
        } else {
          int32_t M = 0;
          int E = 0;
          uint8_t code = 0;
          if (parts(gt[i], M, E)) {
            const uint32_t am = uint32_t(M < 0 ? -M : M);
            code = E == -9 && am < 8 ? uint8_t(am) : uint8_t(((E + 10) << 3) | (am - 8));
          }
          g8[i] = uint8_t(code | ((u >> 24) & 0x80));
        }
      }
      const int clen = tc_chunk_ktiles(d.d, fp8) * (fp8 ? 128 : 64);
      std::vector<float> gnc(ml * kTcColRecord, 0.f);
      std::vector<int32_t> gint(gt.size(), 0);
      for (size_t c = 0; c < ml; ++c) {
        for (int k = 0; k < 2; ++k) {
          double s2 = 0.0;
          for (int j = k * clen; j < std::min(d.d, (k + 1) * clen); ++j) s2 += double(gt[c * d.d + j]) * gt[c * d.d + j];
          gnc[c * kTcColRecord + k] = float(std::sqrt(s2) * (1.0 + 1e-6));
        }
        int emin = 0, emax = 0;
        bool any = false;
        for (int j = 0; j < d.d; ++j) {
          int32_t M;
          int E;
          if (!parts(gt[c * d.d + j], M, E)) continue;
          emin = any ? std::min(emin, E) : E;
          emax = any ? std::max(emax, E) : E;
          any = true;
        }
        const int range = emax - emin;
        uint64_t gabs = 0;  // sum of |G_j| on the column's grid (below 2^45: d <= 16384, |G_j| < 2^31)
        if (range <= 23)
          for (int j = 0; j < d.d; ++j) {
            int32_t M;
            int E;
            if (parts(gt[c * d.d + j], M, E)) {
              gint[c * d.d + j] = M * (int32_t(1) << (E - emin));
              gabs += uint64_t(gint[c * d.d + j] < 0 ? -int64_t(gint[c * d.d + j]) : int64_t(gint[c * d.d + j]));
            }
          }
        int32_t slots[2] = {emin, range};
        std::memcpy(&gnc[c * kTcColRecord + 2], slots, sizeof(slots));
        const uint32_t gw[2] = {uint32_t(gabs), uint32_t(gabs >> 32)};
        std::memcpy(&gnc[c * kTcColRecord + 4], gw, sizeof(gw));
      }
      if (fp8) e = upload(&f->d_Gt8, g8.data(), g8.size());
      else e = upload(&f->d_Gt16, g16.data(), g16.size());
      if (e == cudaSuccess) e = upload(&f->d_gnc, gnc.data(), gnc.size());
      if (e == cudaSuccess) e = upload(&f->d_Gint, gint.data(), gint.size());
    }

  }
  if (e == cudaSuccess && kind_is_sketch(d.kind) && d.kind != LSH_CSL_SRP && d.N == 1 && d.m <= 32768) {
    // column-major copy of the count-sketch tables for the CSR kernel
    std::vector<uint16_t> cm(size_t(d.d) * d.L);
    for (int t = 0; t < d.L; ++t)
      for (int j = 0; j < d.d; ++j) {
        const size_t src = size_t(t) * h.dsum + j;
        cm[size_t(j) * d.L + t] = uint16_t(h.bins[src] | (h.signs[src] < 0 ? 0x8000 : 0));
      }
    e = upload(&f->d_colmajor, cm.data(), cm.size());
  }
  if (e == cudaSuccess && kind_is_sketch(d.kind) && d.d < 65536) {
    // per-table member lists for the deferred recheck: the coordinates of each
    // bin with s = +1 in ascending j, then those with s = -1
    // (CSSRP-L: one entry per (coordinate, bin) incidence, lc per coordinate)
    const int lc = incidences(d);
    const int64_t D = int64_t(d.d) * lc;
    std::vector<uint16_t> ml(size_t(d.L) * D);
    std::vector<uint32_t> ms(size_t(d.L) * d.m * 2);
    std::vector<int> bin(D), neg(D);
    std::vector<uint32_t> cnt(size_t(2) * d.m), cur(size_t(2) * d.m);
    for (int t = 0; t < d.L; ++t) {
      std::fill(cnt.begin(), cnt.end(), 0u);
      for (int64_t e = 0; e < D; ++e) {
        int bn = 0, ng = 0;
        if (d.kind == LSH_CSL_SRP) {
          bn = h.bins[size_t(t) * h.dsum + e];
          ng = h.signs[size_t(t) * h.dsum + e] < 0 ? 1 : 0;
        } else {
          int r = int(e), off = 0, stride = 1;
          for (int k = 0; k < d.N; ++k) {
            const int ik = r % d.dims[k];
            r /= d.dims[k];
            const size_t src = size_t(t) * h.dsum + off + ik;
            bn += h.bins[src] * stride;
            ng ^= h.signs[src] < 0 ? 1 : 0;
            stride *= d.mdims[k];
            off += d.dims[k];
          }
        }
        bin[e] = bn;
        neg[e] = ng;
        ++cnt[size_t(2) * bn + ng];
      }
      uint32_t start = 0;
      for (int l = 0; l < d.m; ++l) {
        ms[(size_t(t) * d.m + l) * 2] = start;
        ms[(size_t(t) * d.m + l) * 2 + 1] = cnt[2 * l] | (cnt[2 * l + 1] << 16);
        cur[2 * l] = start;
        cur[2 * l + 1] = start + cnt[2 * l];
        start += cnt[2 * l] + cnt[2 * l + 1];
      }
      for (int64_t e = 0; e < D; ++e) ml[size_t(t) * D + cur[size_t(2) * bin[e] + neg[e]]++] = uint16_t(e / lc);
    }
    e = upload(&f->d_mlist, ml.data(), ml.size());
    if (e == cudaSuccess) e = upload(&f->d_mseg, ms.data(), ms.size());
  }
  if (e == cudaSuccess) e = cudaMalloc(&f->d_status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(f->d_status, 0, sizeof(uint32_t));
  if (e != cudaSuccess) {
    free_family(f);
    return cuda_fail(e, "lsh_make_family upload");
  }
  *out = f;
  return LSH_OK;
}

lsh_status lsh_sample_family_tables(const lsh_family_desc *desc, int32_t *bins, int8_t *signs, float *G,
                                    double *b, uint32_t *ka, uint32_t *kb) {
  if (!desc) return fail(LSH_EINVAL, "NULL argument");
  const lsh_family_desc d = normalized(*desc);
  lsh_status st = validate_desc(d);
  if (st != LSH_OK) return st;
  HostFamily h;
  try {
    sample_family(d, h);
  } catch (const std::bad_alloc &) {
    return fail(LSH_ENOMEM, "host allocation");
  }
  if (bins && !h.bins.empty()) std::memcpy(bins, h.bins.data(), h.bins.size() * sizeof(int32_t));
  if (signs && !h.signs.empty()) std::memcpy(signs, h.signs.data(), h.signs.size());
  if (G && !h.G.empty()) std::memcpy(G, h.G.data(), h.G.size() * sizeof(float));
  if (b) std::memcpy(b, h.b.data(), h.b.size() * sizeof(double));
  if (ka) std::memcpy(ka, h.ka.data(), h.ka.size() * sizeof(uint32_t));
  if (kb) std::memcpy(kb, h.kb.data(), h.kb.size() * sizeof(uint32_t));
  return LSH_OK;
}

lsh_status lsh_family_describe(lsh_family_t fam, lsh_family_desc *desc) {
  if (!fam || !desc) return fail(LSH_EINVAL, "NULL argument");
  *desc = fam->host.desc;
  return LSH_OK;
}

lsh_status lsh_family_export(lsh_family_t fam, int32_t *bins, int8_t *signs, float *G, double *b, uint32_t *ka,
                             uint32_t *kb) {
  if (!fam) return fail(LSH_EINVAL, "NULL family");
  const HostFamily &h = fam->host;
  if (bins && !h.bins.empty()) std::memcpy(bins, h.bins.data(), h.bins.size() * sizeof(int32_t));
  if (signs && !h.signs.empty()) std::memcpy(signs, h.signs.data(), h.signs.size());
  if (G && !h.G.empty()) std::memcpy(G, h.G.data(), h.G.size() * sizeof(float));
  if (b) std::memcpy(b, h.b.data(), h.b.size() * sizeof(double));
  if (ka) std::memcpy(ka, h.ka.data(), h.ka.size() * sizeof(uint32_t));
  if (kb) std::memcpy(kb, h.kb.data(), h.kb.size() * sizeof(uint32_t));
  return LSH_OK;
}

lsh_status lsh_family_status(lsh_family_t fam, int32_t *status, int32_t clear) {
  if (!fam || !status) return fail(LSH_EINVAL, "NULL argument");
  LSH_CUDA_TRY(cudaDeviceSynchronize());
  uint32_t s = 0;
  LSH_CUDA_TRY(cudaMemcpy(&s, fam->d_status, sizeof(s), cudaMemcpyDeviceToHost));
  if (clear) LSH_CUDA_TRY(cudaMemset(fam->d_status, 0, sizeof(uint32_t)));
  *status = int32_t(s);
  return LSH_OK;
}

void lsh_family_destroy(lsh_family_t fam) { free_family(fam); }

lsh_status lsh_hash(lsh_family_t fam, const lsh_matrix *X, void *codes, uint64_t *keys, float *proj,
                    lsh_hash_stats *stats, void *stream_) {
  if (!fam) return fail(LSH_EINVAL, "NULL family");
  lsh_status st = validate_matrix(fam, X, true);
  if (st != LSH_OK) return st;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const lsh_family_desc &d = fam->host.desc;
  unsigned long long *cnt = nullptr;
  keep_pool_warm();
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    LSH_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&cnt), CNT_NUM * 8, stream));
    cudaError_t e = cudaMemsetAsync(cnt, 0, CNT_NUM * 8, stream);
    if (e != cudaSuccess) {
      cudaFreeAsync(cnt, stream);
      return cuda_fail(e, "cudaMemsetAsync");
    }
  }
  st = hash_impl(fam, X, codes, keys, X->n, proj, cnt, stream);
  if (stats) {
    unsigned long long h[CNT_NUM] = {};
    cudaError_t e = cudaSuccess;
    if (st == LSH_OK) e = cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, stream);
    cudaFreeAsync(cnt, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (st != LSH_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "lsh_hash stats");
    stats->n_entries = X->n * int64_t(d.L) * d.m;
    stats->n_flagged = int64_t(h[CNT_FLAGGED]);
    stats->n_changed = int64_t(h[CNT_CHANGED]);
    stats->n_nonfinite = int64_t(h[CNT_NONFINITE]);
    stats->n_overflow = int64_t(h[CNT_OVERFLOW]);
    if (stats->n_nonfinite) return fail(LSH_ENONFINITE, "input rows hold NaN or Inf");
    if (stats->n_overflow) return fail(LSH_ERANGE, "E2LSH code outside int32");
  }
  return st;
}

lsh_status lsh_set_sort_mode(int32_t mode) {
  if (set_sort_mode(mode) != 0)
    return fail(LSH_EINVAL, "sort mode must be 0 (automatic), 1 (global passes) or 2 (bucket sort)");
  return LSH_OK;
}

lsh_status lsh_set_sketch_plan(int32_t rows_per_lane, int32_t row_groups, int32_t warps_per_table,
                               int32_t tables_per_cta, int32_t entry_bytes, int32_t split_bins) {
  const bool clear = rows_per_lane == 0 && row_groups == 0 && warps_per_table == 0 && tables_per_cta == 0 &&
                     entry_bytes == 0 && split_bins == 0;
  if (!clear) {
    auto in124 = [](int v) { return v == 1 || v == 2 || v == 4; };
    if (split_bins != 0 && split_bins != 1) return fail(LSH_EINVAL, "split_bins must be 0 or 1");
    if (!in124(rows_per_lane) || !in124(row_groups))
      return fail(LSH_EINVAL, "rows_per_lane and row_groups must be 1, 2 or 4");
    if (split_bins ? (rows_per_lane < 2 || rows_per_lane * row_groups > 8) : rows_per_lane * row_groups > 4)
      return fail(LSH_EINVAL, "a tile holds at most 128 rows (split bins: 16 row groups per warp and "
                              "rows_per_lane >= 2)");
    if (!in124(warps_per_table)) return fail(LSH_EINVAL, "warps_per_table must be 1, 2 or 4");
    if (tables_per_cta < 1) return fail(LSH_EINVAL, "tables_per_cta must be >= 1");
    if (entry_bytes != 2 && entry_bytes != 4) return fail(LSH_EINVAL, "entry_bytes must be 2 or 4");
  }
  set_sketch_pin(SketchPin{rows_per_lane, row_groups, warps_per_table, tables_per_cta, entry_bytes, split_bins});
  return LSH_OK;
}

lsh_status lsh_get_sketch_plan(lsh_family_t fam, int32_t dtype, int64_t n, int32_t plan[6]) {
  if (!fam || !plan) return fail(LSH_EINVAL, "lsh_get_sketch_plan: NULL argument");
  const lsh_family_desc &d = fam->host.desc;
  if (kind_is_dense(d.kind)) return fail(LSH_EUNSUPPORTED, "lsh_get_sketch_plan: CS/HCS families only");
  if (dtype != LSH_F32 && dtype != LSH_BF16 && dtype != LSH_F16) return fail(LSH_EINVAL, "unknown dtype");
  if (n < 1) return fail(LSH_EINVAL, "lsh_get_sketch_plan: n must be >= 1");
  SketchLaunch p = family_launch(fam);
  p.dtype = dtype;
  p.n = n;
  p.ld = d.d;
  SketchPin pin;
  if (!sketch_current_plan(p, pin)) return fail(LSH_EUNSUPPORTED, "no sketch plan fits this shape");
  const int32_t v[6] = {pin.rows_per_lane, pin.row_groups, pin.warps_per_table, pin.tables_per_cta,
                        pin.entry_bytes, pin.split_bins};
  for (int i = 0; i < 6; ++i) plan[i] = v[i];
  return LSH_OK;
}

lsh_status lsh_build_index(lsh_family_t fam, const lsh_matrix *X, int32_t keep_data, lsh_index_t *out,
                           void *stream_) {
  if (!fam || !out) return fail(LSH_EINVAL, "NULL argument");
  *out = nullptr;
  lsh_status st = validate_matrix(fam, X, true);
  if (st != LSH_OK) return st;
  if (keep_data && X->rowptr) return fail(LSH_EUNSUPPORTED, "keep_data needs dense rows");
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const int L = fam->host.desc.L;
  const int64_t n = X->n;
  lsh_index_s *idx = new (std::nothrow) lsh_index_s();
  if (!idx) return fail(LSH_ENOMEM, "host allocation");
  idx->fam = fam;
  idx->n = n;
  idx->L = L;
  idx->d = X->d;
  auto cleanup = [&](lsh_status s) {
    lsh_index_destroy(idx);
    return s;
  };
  cudaError_t e = cudaMalloc(&idx->d_nb, sizeof(int64_t) * L);
  if (e == cudaSuccess && n > 0) e = cudaMalloc(&idx->d_ids, sizeof(uint32_t) * size_t(n) * L);
  if (e == cudaSuccess && n > 0) e = cudaMalloc(&idx->d_ukeys, sizeof(uint64_t) * size_t(n) * L);
  if (e == cudaSuccess) e = cudaMalloc(&idx->d_offsets, sizeof(uint32_t) * size_t(n + 1) * L);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "lsh_build_index allocation"));
  if (keep_data && n > 0) {
    const size_t es = dtype_size(X->dtype);
    e = cudaMalloc(&idx->d_data, es * size_t(n) * X->d);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(idx->d_data, es * X->d, X->values, es * X->ld, es * X->d, size_t(n),
                            cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "lsh_build_index data copy"));
    idx->data_dtype = X->dtype;
    idx->data_ld = X->d;
  }
  if (n == 0) {
    e = cudaMemsetAsync(idx->d_nb, 0, sizeof(int64_t) * L, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(idx->d_offsets, 0, sizeof(uint32_t) * L, stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "memset"));
    *out = idx;
    return LSH_OK;
  }
  st = index_fill(idx, X, stream);
  if (st != LSH_OK) return cleanup(st);
  *out = idx;
  return LSH_OK;
}

lsh_status lsh_index_rebuild(lsh_index_t idx, const lsh_matrix *X, void *stream_) {
  if (!idx) return fail(LSH_EINVAL, "NULL index");
  lsh_status st = validate_matrix(idx->fam, X, true);
  if (st != LSH_OK) return st;
  if (X->n != idx->n) return fail(LSH_EINVAL, "rebuild needs the same n as the index");
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (idx->d_data) {
    if (X->rowptr || X->dtype != idx->data_dtype) return fail(LSH_EINVAL, "rebuild data must match the kept data");
    const size_t es = dtype_size(X->dtype);
    if (X->n > 0)
      LSH_CUDA_TRY(cudaMemcpy2DAsync(idx->d_data, es * X->d, X->values, es * X->ld, es * X->d, size_t(X->n),
                                     cudaMemcpyDeviceToDevice, stream));
  }
  if (X->n == 0) return LSH_OK;
  return index_fill(idx, X, stream);
}

lsh_status lsh_index_rebuild_host(lsh_index_t idx, const lsh_matrix *X, int64_t chunk_rows, void *stream_) {
  if (!idx || !X) return fail(LSH_EINVAL, "NULL argument");
  if (X->rowptr) return fail(LSH_EINVAL, "host rebuild takes dense rows");
  lsh_status st = validate_matrix(idx->fam, X, false);
  if (st != LSH_OK) return st;
  if (X->n != idx->n) return fail(LSH_EINVAL, "rebuild needs the same n as the index");
  if (X->dtype == LSH_FP8_E4M3) return fail(LSH_EUNSUPPORTED, "host rebuild of FP8 rows is not supported");
  if (idx->d_data && X->dtype != idx->data_dtype) return fail(LSH_EINVAL, "rebuild data must match the kept data");
  if (chunk_rows < 0) return fail(LSH_EINVAL, "chunk_rows must be >= 0");
  const int64_t n = X->n;
  if (n == 0) return LSH_OK;
  // small chunks keep the hash of the last one, which no copy hides, short;
  // below about 16,384 rows the per-chunk launches cost more than they save
  if (chunk_rows == 0) chunk_rows = std::max<int64_t>(32768, (n + 31) / 32);
  chunk_rows = std::min(chunk_rows, n);
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const int L = idx->L;
  const size_t es = dtype_size(X->dtype), rowb = es * size_t(X->d);
  keep_pool_warm();
  // the rows stream to the device in chunks on a second stream while the
  // previous chunk is hashed; into the index's data copy when it keeps one,
  // else into two staging buffers used alternately
  uint64_t *keys = nullptr;
  void *stage[2] = {nullptr, nullptr};
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_start = nullptr, copied[2] = {nullptr, nullptr}, hashed[2] = {nullptr, nullptr};
  auto release = [&]() {
    if (keys) cudaFreeAsync(keys, stream);
    for (int b = 0; b < 2; ++b)
      if (stage[b]) cudaFreeAsync(stage[b], stream);
    for (cudaEvent_t ev : {ev_start, copied[0], copied[1], hashed[0], hashed[1]})
      if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
  };
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&keys), sizeof(uint64_t) * size_t(n) * L, stream);
  for (int b = 0; b < 2 && e == cudaSuccess && !idx->d_data; ++b) e = cudaMallocAsync(&stage[b], rowb * chunk_rows, stream);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  for (cudaEvent_t *ev : {&ev_start, &copied[0], &copied[1], &hashed[0], &hashed[1]})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  // the copies start once the caller's stream has reached this call (buffers allocated)
  if (e == cudaSuccess) e = cudaEventRecord(ev_start, stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_start, 0);
  int64_t c = 0;
  for (int64_t r0 = 0; r0 < n && e == cudaSuccess && st == LSH_OK; r0 += chunk_rows, ++c) {
    const int64_t rows = std::min(chunk_rows, n - r0);
    const int b = int(c & 1);
    void *dst = idx->d_data ? static_cast<char *>(idx->d_data) + rowb * size_t(r0) : stage[b];
    if (!idx->d_data && c >= 2) e = cudaStreamWaitEvent(cs, hashed[b], 0);  // the buffer's previous chunk is hashed
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(dst, rowb, static_cast<const char *>(X->values) + es * size_t(X->ld) * size_t(r0),
                            es * size_t(X->ld), rowb, size_t(rows), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(copied[b], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, copied[b], 0);
    if (e != cudaSuccess) break;
    lsh_matrix part = *X;
    part.values = dst;
    part.n = rows;
    part.ld = X->d;
    st = hash_impl(idx->fam, &part, nullptr, keys + r0, n, nullptr, nullptr, stream);
    if (st == LSH_OK) e = cudaEventRecord(hashed[b], stream);
  }
  if (e == cudaSuccess && st == LSH_OK) {
    e = build_tables(keys, n, L, idx->d_ids, idx->d_ukeys, idx->d_offsets, idx->d_nb, stream);
  }
  release();
  if (st != LSH_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "lsh_index_rebuild_host");
  return LSH_OK;
}

lsh_status lsh_index_info(lsh_index_t idx, int64_t *n, int64_t *nbuckets) {
  if (!idx) return fail(LSH_EINVAL, "NULL index");
  if (n) *n = idx->n;
  if (nbuckets) {
    LSH_CUDA_TRY(cudaDeviceSynchronize());
    LSH_CUDA_TRY(cudaMemcpy(nbuckets, idx->d_nb, sizeof(int64_t) * idx->L, cudaMemcpyDeviceToHost));
  }
  return LSH_OK;
}

lsh_status lsh_index_export(lsh_index_t idx, uint32_t *ids, uint64_t *ukeys, uint32_t *offsets, int64_t *nb) {
  if (!idx) return fail(LSH_EINVAL, "NULL index");
  LSH_CUDA_TRY(cudaDeviceSynchronize());
  const size_t nL = size_t(idx->n) * idx->L;
  if (ids && nL) LSH_CUDA_TRY(cudaMemcpy(ids, idx->d_ids, nL * 4, cudaMemcpyDeviceToHost));
  if (ukeys && nL) LSH_CUDA_TRY(cudaMemcpy(ukeys, idx->d_ukeys, nL * 8, cudaMemcpyDeviceToHost));
  if (offsets)
    LSH_CUDA_TRY(cudaMemcpy(offsets, idx->d_offsets, size_t(idx->n + 1) * idx->L * 4, cudaMemcpyDeviceToHost));
  if (nb) LSH_CUDA_TRY(cudaMemcpy(nb, idx->d_nb, sizeof(int64_t) * idx->L, cudaMemcpyDeviceToHost));
  return LSH_OK;
}

lsh_status lsh_query(lsh_index_t idx, const lsh_matrix *Q, int32_t k, int32_t *ids, float *dist,
                     lsh_query_stats *stats, void *stream_) {
  if (!idx || !Q) return fail(LSH_EINVAL, "NULL argument");
  lsh_status st = validate_matrix(idx->fam, Q, false);
  if (st != LSH_OK) return st;
  if (k < 1 || k > 256) return fail(LSH_EINVAL, "k must be in [1, 256]");
  if (!idx->d_data && idx->n > 0) return fail(LSH_EINVAL, "the index was built without keep_data");
  if (Q->n > 0 && (!ids || !dist)) return fail(LSH_EINVAL, "NULL output");
  if (Q->dtype == LSH_FP8_E4M3) return fail(LSH_EUNSUPPORTED, "FP8 queries are not supported");
  const lsh_family_desc &d = idx->fam->host.desc;
  if (d.L > 128) return fail(LSH_EUNSUPPORTED, "lsh_query supports L <= 128");
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (stats) std::memset(stats, 0, sizeof(*stats));
  const int64_t q = Q->n;
  if (q == 0) return LSH_OK;
  keep_pool_warm();
  uint64_t *qkeys = nullptr;
  unsigned long long *cnt = nullptr;
  void *qscratch = nullptr;
  LSH_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&qkeys), sizeof(uint64_t) * size_t(q) * d.L, stream));
  cudaError_t e = cudaMallocAsync(&qscratch, query_scratch_bytes(q, k), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(qscratch, 0, size_t(q) * 4, stream);
  if (stats) {
    e = cudaMallocAsync(reinterpret_cast<void **>(&cnt), 4 * sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), stream);
  }
  if (e == cudaSuccess) st = hash_impl(idx->fam, Q, nullptr, qkeys, q, nullptr, nullptr, stream);
  else st = cuda_fail(e, "lsh_query temporaries");
  if (st == LSH_OK && idx->n > 0) {
    e = launch_query(qkeys, q, d.L, k, kind_is_srp(d.kind) ? 1 : 0, d.d, Q->values, Q->dtype, Q->ld, idx, ids,
                     dist, cnt, qscratch, q, nullptr, stream);
    if (e != cudaSuccess) st = cuda_fail(e, "lsh_query launch");
    else count_launches(1);
  } else if (st == LSH_OK) {
    // empty index: no candidates
    std::vector<int32_t> none(size_t(q) * k, -1);
    std::vector<float> inf(size_t(q) * k, INFINITY);
    e = cudaMemcpyAsync(ids, none.data(), none.size() * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dist, inf.data(), inf.size() * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) st = cuda_fail(e, "lsh_query empty index");
  }
  unsigned long long h[4] = {};
  if (stats && cnt && st == LSH_OK) {
    e = cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) st = cuda_fail(e, "lsh_query stats");
  }
  cudaFreeAsync(qkeys, stream);
  if (qscratch) cudaFreeAsync(qscratch, stream);
  if (cnt) cudaFreeAsync(cnt, stream);
  if (stats && st == LSH_OK) {
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "lsh_query sync");
    stats->n_queries = q;
    stats->n_candidates = int64_t(h[0]);
    stats->n_unique = int64_t(h[1]);
    stats->max_unique = int64_t(h[2]);
  }
  return st;
}

void lsh_index_destroy(lsh_index_t idx) {
  if (!idx) return;
  cudaFree(idx->d_ids);
  cudaFree(idx->d_ukeys);
  cudaFree(idx->d_offsets);
  cudaFree(idx->d_nb);
  cudaFree(idx->d_data);
  delete idx;
}

}  // extern "C"
