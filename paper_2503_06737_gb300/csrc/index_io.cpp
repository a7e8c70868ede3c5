// index_io.cpp -- saving and loading the L hash tables of an index (Sec. 3.1),
// and the merge of per-shard top-k lists for an index sharded by rows.
//
// File layout (little-endian, the host's native integer and IEEE layouts):
//   header   magic "LSHGB300", u32 version (1), u32 header bytes,
//            the family description (kind, d, m, L, N, dims[8], mdims[8],
//            w, seed, compute, l of CSSRP-L or 0), i64 n, i64 d,
//            i32 data dtype, i32 has data
//   nb       i64 [L]           buckets per table
//   offsets  u32 [L][n+1]      bucket starts
//   ids      u32 [L][n]        point ids in (key, id) order
//   ukeys    u64 [L][n]        distinct keys (the first nb[t] of table t)
//   data     [n][d] of the data dtype, when the index keeps its rows
// Arrays stream through a bounded host buffer, so saving or loading a large
// index does not need its size in host memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "internal.h"

namespace lsh {
namespace {

constexpr char kMagic[8] = {'L', 'S', 'H', 'G', 'B', '3', '0', '0'};
constexpr uint32_t kVersion = 1;
constexpr size_t kChunk = size_t(64) << 20;  // host staging per transfer

struct FileHeader {
  char magic[8];
  uint32_t version, header_bytes;
  int32_t kind, d, m, L, N;
  int32_t dims[LSH_MAX_MODES], mdims[LSH_MAX_MODES];
  double w;
  uint64_t seed;
  int32_t compute, nnz_per_col;
  int64_t n, dcols;
  int32_t data_dtype, has_data;
};

struct FileCloser {
  void operator()(FILE *f) const {
    if (f) std::fclose(f);
  }
};
using File = std::unique_ptr<FILE, FileCloser>;

size_t elem_size(int dt) { return dt == LSH_F32 ? 4 : (dt == LSH_FP8_E4M3 ? 1 : 2); }

// Device -> file, through the staging buffer.
bool write_device(FILE *f, const void *dev, size_t bytes, std::vector<unsigned char> &buf) {
  const unsigned char *src = static_cast<const unsigned char *>(dev);
  for (size_t off = 0; off < bytes; off += buf.size()) {
    const size_t len = std::min(buf.size(), bytes - off);
    if (cudaMemcpy(buf.data(), src + off, len, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    if (std::fwrite(buf.data(), 1, len, f) != len) return false;
  }
  return true;
}

// File -> device, through the staging buffer.
bool read_device(FILE *f, void *dev, size_t bytes, std::vector<unsigned char> &buf) {
  unsigned char *dst = static_cast<unsigned char *>(dev);
  for (size_t off = 0; off < bytes; off += buf.size()) {
    const size_t len = std::min(buf.size(), bytes - off);
    if (std::fread(buf.data(), 1, len, f) != len) return false;
    if (cudaMemcpy(dst + off, buf.data(), len, cudaMemcpyHostToDevice) != cudaSuccess) return false;
  }
  return true;
}

bool same_family(const lsh_family_desc &a, const FileHeader &h) {
  if (a.kind != h.kind || a.d != h.d || a.m != h.m || a.L != h.L || a.N != h.N || a.seed != h.seed ||
      a.compute != h.compute || !(a.w == h.w))
    return false;
  if (h.nnz_per_col != (a.kind == LSH_CSL_SRP ? incidences(a) : 0)) return false;
  for (int k = 0; k < a.N && k < LSH_MAX_MODES; ++k)
    if (a.dims[k] != h.dims[k] || a.mdims[k] != h.mdims[k]) return false;
  return true;
}

}  // namespace
}  // namespace lsh

using namespace lsh;

extern "C" {

lsh_status lsh_index_save(lsh_index_t idx, const char *path) {
  if (!idx || !path) return fail(LSH_EINVAL, "lsh_index_save: NULL argument");
  LSH_CUDA_TRY(cudaDeviceSynchronize());
  const lsh_family_desc &fd = idx->fam->host.desc;
  FileHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.header_bytes = uint32_t(sizeof(FileHeader));
  h.kind = fd.kind;
  h.d = fd.d;
  h.m = fd.m;
  h.L = fd.L;
  h.N = fd.N;
  for (int k = 0; k < LSH_MAX_MODES; ++k) {
    h.dims[k] = fd.dims[k];
    h.mdims[k] = fd.mdims[k];
  }
  h.w = fd.w;
  h.seed = fd.seed;
  h.compute = fd.compute;
  h.nnz_per_col = fd.kind == LSH_CSL_SRP ? incidences(fd) : 0;
  h.n = idx->n;
  h.dcols = idx->d;
  h.has_data = idx->d_data ? 1 : 0;
  h.data_dtype = idx->d_data ? idx->data_dtype : 0;
  File f(std::fopen(path, "wb"));
  if (!f) return fail(LSH_EIO, std::string("lsh_index_save: cannot open ") + path);
  std::vector<unsigned char> buf;
  try {
    buf.resize(kChunk);
  } catch (const std::bad_alloc &) {
    return fail(LSH_ENOMEM, "lsh_index_save: host staging buffer");
  }
  const size_t nL = size_t(idx->n) * idx->L;
  bool ok = std::fwrite(&h, sizeof(h), 1, f.get()) == 1;
  ok = ok && write_device(f.get(), idx->d_nb, sizeof(int64_t) * idx->L, buf);
  ok = ok && write_device(f.get(), idx->d_offsets, sizeof(uint32_t) * size_t(idx->n + 1) * idx->L, buf);
  if (nL) {
    ok = ok && write_device(f.get(), idx->d_ids, sizeof(uint32_t) * nL, buf);
    ok = ok && write_device(f.get(), idx->d_ukeys, sizeof(uint64_t) * nL, buf);
  }
  if (idx->d_data && idx->n > 0)
    ok = ok && write_device(f.get(), idx->d_data, elem_size(idx->data_dtype) * size_t(idx->n) * idx->d, buf);
  ok = ok && std::fflush(f.get()) == 0;
  if (!ok) return fail(LSH_EIO, std::string("lsh_index_save: write failed: ") + path);
  return LSH_OK;
}

lsh_status lsh_index_load(lsh_family_t fam, const char *path, lsh_index_t *out) {
  if (!fam || !path || !out) return fail(LSH_EINVAL, "lsh_index_load: NULL argument");
  *out = nullptr;
  File f(std::fopen(path, "rb"));
  if (!f) return fail(LSH_EIO, std::string("lsh_index_load: cannot open ") + path);
  FileHeader h;
  if (std::fread(&h, sizeof(h), 1, f.get()) != 1) return fail(LSH_EIO, "lsh_index_load: short header");
  if (std::memcmp(h.magic, kMagic, 8) != 0) return fail(LSH_EINVAL, "lsh_index_load: not an index file");
  if (h.version != kVersion || h.header_bytes != sizeof(FileHeader))
    return fail(LSH_EUNSUPPORTED, "lsh_index_load: unknown file version");
  if (!same_family(fam->host.desc, h))
    return fail(LSH_EINVAL, "lsh_index_load: the file was built with another family (kind, d, m, L, modes, w, "
                            "seed, compute or nnz_per_col differ)");
  if (h.n < 0 || h.n > int64_t(UINT32_MAX) - 1 || h.dcols != h.d)
    return fail(LSH_EINVAL, "lsh_index_load: corrupt header");
  if (h.has_data && (h.data_dtype < LSH_F32 || h.data_dtype > LSH_F16))
    return fail(LSH_EINVAL, "lsh_index_load: corrupt header (data dtype)");
  lsh_index_s *idx = new (std::nothrow) lsh_index_s();
  if (!idx) return fail(LSH_ENOMEM, "host allocation");
  idx->fam = fam;
  idx->n = h.n;
  idx->L = h.L;
  idx->d = h.d;
  auto cleanup = [&](lsh_status s) {
    lsh_index_destroy(idx);
    return s;
  };
  const size_t nL = size_t(h.n) * h.L;
  cudaError_t e = cudaMalloc(&idx->d_nb, sizeof(int64_t) * h.L);
  if (e == cudaSuccess && nL) e = cudaMalloc(&idx->d_ids, sizeof(uint32_t) * nL);
  if (e == cudaSuccess && nL) e = cudaMalloc(&idx->d_ukeys, sizeof(uint64_t) * nL);
  if (e == cudaSuccess) e = cudaMalloc(&idx->d_offsets, sizeof(uint32_t) * size_t(h.n + 1) * h.L);
  if (e == cudaSuccess && h.has_data && h.n > 0) {
    e = cudaMalloc(&idx->d_data, elem_size(h.data_dtype) * size_t(h.n) * h.d);
    idx->data_dtype = h.data_dtype;
    idx->data_ld = h.d;
  }
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "lsh_index_load allocation"));
  std::vector<unsigned char> buf;
  try {
    buf.resize(kChunk);
  } catch (const std::bad_alloc &) {
    return cleanup(fail(LSH_ENOMEM, "lsh_index_load: host staging buffer"));
  }
  bool ok = read_device(f.get(), idx->d_nb, sizeof(int64_t) * h.L, buf);
  ok = ok && read_device(f.get(), idx->d_offsets, sizeof(uint32_t) * size_t(h.n + 1) * h.L, buf);
  if (nL) {
    ok = ok && read_device(f.get(), idx->d_ids, sizeof(uint32_t) * nL, buf);
    ok = ok && read_device(f.get(), idx->d_ukeys, sizeof(uint64_t) * nL, buf);
  }
  if (idx->d_data) ok = ok && read_device(f.get(), idx->d_data, elem_size(h.data_dtype) * size_t(h.n) * h.d, buf);
  if (!ok) return cleanup(fail(LSH_EIO, std::string("lsh_index_load: short or unreadable file: ") + path));
  *out = idx;
  return LSH_OK;
}

lsh_status lsh_merge_topk(int32_t shards, int64_t q, int32_t k, const int32_t *const *ids,
                          const float *const *dist, const int64_t *id_offset, int64_t *out_ids, float *out_dist) {
  if (shards < 1 || q < 0 || k < 1) return fail(LSH_EINVAL, "lsh_merge_topk: need shards >= 1, q >= 0, k >= 1");
  if (q == 0) return LSH_OK;
  if (!ids || !dist || !id_offset || !out_ids || !out_dist) return fail(LSH_EINVAL, "lsh_merge_topk: NULL argument");
  for (int s = 0; s < shards; ++s)
    if (!ids[s] || !dist[s]) return fail(LSH_EINVAL, "lsh_merge_topk: NULL shard list");
  std::vector<int32_t> head(static_cast<size_t>(shards), 0);
  for (int64_t i = 0; i < q; ++i) {
    std::fill(head.begin(), head.end(), 0);
    const int64_t row = i * k;
    for (int r = 0; r < k; ++r) {
      // the smallest (distance, global id) among the shards' next entries
      int best = -1;
      float bd = INFINITY;
      int64_t bid = 0;
      for (int s = 0; s < shards; ++s) {
        const int h = head[size_t(s)];
        if (h >= k) continue;
        const int32_t lid = ids[s][row + h];
        if (lid < 0) continue;  // the shard's list ended
        const float dv = dist[s][row + h];
        const int64_t gid = int64_t(lid) + id_offset[s];
        if (best < 0 || dv < bd || (dv == bd && gid < bid)) {
          best = s;
          bd = dv;
          bid = gid;
        }
      }
      if (best < 0) {
        out_ids[row + r] = -1;
        out_dist[row + r] = INFINITY;
      } else {
        out_ids[row + r] = bid;
        out_dist[row + r] = bd;
        ++head[size_t(best)];
      }
    }
  }
  return LSH_OK;
}

}  // extern "C"
