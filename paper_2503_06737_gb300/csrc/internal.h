// internal.h -- library-internal declarations shared by the host runtime and
// the CUDA kernels of the LSH library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lsh.h"

namespace lsh {

// ---------------------------------------------------------------------------
// Error plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
lsh_status fail(lsh_status st, const std::string &msg);
lsh_status cuda_fail(cudaError_t e, const char *what);

#define LSH_CUDA_TRY(expr)                                         \
  do {                                                             \
    cudaError_t _e = (expr);                                       \
    if (_e != cudaSuccess) return ::lsh::cuda_fail(_e, #expr);     \
  } while (0)

// Kernel launch accounting (lsh_launch_count).
void count_launches(uint64_t k);

// Sticky device status bits (family status word).
enum : uint32_t { STATUS_NONFINITE = 1u, STATUS_OVERFLOW = 2u, STATUS_TIMEOUT = 4u };

// Per-call device counters (order matches lsh_hash_stats after n_entries).
enum { CNT_FLAGGED = 0, CNT_CHANGED = 1, CNT_NONFINITE = 2, CNT_OVERFLOW = 3, CNT_NUM = 8 };

inline bool kind_is_srp(int k) { return k == LSH_SRP || k == LSH_CS_SRP || k == LSH_HCS_SRP || k == LSH_CSL_SRP; }
// Entries of a coordinate in one table: l for CSSRP-L, else 1.
inline int incidences(const lsh_family_desc &d) {
  return d.kind == LSH_CSL_SRP && d.nnz_per_col > 1 ? d.nnz_per_col : 1;
}
inline bool kind_is_dense(int k) { return k == LSH_E2LSH || k == LSH_SRP; }
inline bool kind_is_sketch(int k) { return !kind_is_dense(k); }
inline bool kind_scaled(int k) { return k == LSH_CS_E2LSH || k == LSH_HCS_E2LSH; }

// ---------------------------------------------------------------------------
// Family: host copy of the drawn tables plus the device copies kernels read.
// ---------------------------------------------------------------------------
struct HostFamily {
  lsh_family_desc desc;
  int64_t dsum = 0;               // sum of mode sizes
  std::vector<int32_t> bins;      // [L][dsum] (CSSRP-L: dsum = d l, entry i l + r)
  std::vector<int8_t> signs;      // [L][dsum]
  std::vector<float> G;           // [d][m*L] dense kinds
  std::vector<double> b;          // [L][m]
  std::vector<uint32_t> ka, kb;   // [L][m]
};

// Draw every table of the family from its seed (host, deterministic).
void sample_family(const lsh_family_desc &desc, HostFamily &hf);

// Largest staged member-list length over the tables of a CS/HCS family: per
// bin, the coordinates with s = +1 and with s = -1, each rounded up to a
// multiple of four (the layout of the dense-row hashing kernel).
int sketch_capacity(const HostFamily &hf);

}  // namespace lsh

struct lsh_family_s {
  lsh::HostFamily host;
  // device copies
  uint16_t *d_bins = nullptr;     // [L][dsum] per-mode bins (< 65536)
  int8_t *d_signs = nullptr;      // [L][dsum]
  float *d_b32 = nullptr;         // [L][m] b rounded to FP32
  double *d_b64 = nullptr;        // [L][m]
  uint32_t *d_ka = nullptr;       // [L][m]
  uint32_t *d_kb = nullptr;       // [L][m]
  float *d_G = nullptr;           // [d][m*L] dense kinds
  float *d_Gt = nullptr;          // [m*L][d] transposed copy (FP64 recheck reads columns)
  float *d_gnorm = nullptr;       // [m*L] column norms, rounded up
  uint16_t *d_Gt16 = nullptr;     // [m*L][d] bf16 bits (families with BF16 G)
  uint8_t *d_Gt8 = nullptr;       // [m*L][d] E4M3 codes (families with FP8 G)
  float *d_gnc = nullptr;         // [m*L][kTcColRecord] column norms per K chunk of the tensor-core
                                  // path; slots 2, 3: the column's least exponent and its range (int
                                  // bits); slots 4, 5: sum_j |G_j| on that grid (uint64, low word first)
  int32_t *d_Gint = nullptr;      // [m*L][d] column j of G as integers on its own 2^e grid (exact recheck)
  uint32_t *d_status = nullptr;   // sticky status word
  int device = 0;
  int sketch_cap = 0;             // see lsh::sketch_capacity
  uint16_t *d_colmajor = nullptr; // CS kinds: [d][L] bin | neg << 15 (CSR path)
  uint16_t *d_mlist = nullptr;    // CS/HCS, d < 65536: [L][d lc] coordinates by (bin, sign, j)
  uint32_t *d_mseg = nullptr;     // [L][m][2]: start in the table's list, n(+) | n(-) << 16
};

struct lsh_index_s {
  lsh_family_t fam = nullptr;     // borrowed (the family must outlive the index)
  int64_t n = 0;
  int32_t L = 0;
  uint32_t *d_ids = nullptr;      // [L][n]
  uint64_t *d_ukeys = nullptr;    // [L][n]
  uint32_t *d_offsets = nullptr;  // [L][n+1]
  int64_t *d_nb = nullptr;        // [L]
  void *d_data = nullptr;         // dense copy of X (optional)
  int32_t data_dtype = 0;
  int64_t data_ld = 0;
  int64_t d = 0;
};

namespace lsh {

// ---------------------------------------------------------------------------
// Kernel launchers (each returns cudaSuccess or the launch error).
// ---------------------------------------------------------------------------
// The batch of a replayed hashing graph (lsh_hasher): written on the device
// by the graph's first node, read by the kernels after it.
struct BatchDesc {
  const void *X;
  int64_t n;
  uint64_t *keys;
  int64_t key_ld;
};

struct SketchLaunch {
  // input
  const void *X;
  int32_t dtype;
  int64_t n, ld;
  const float *row_scale;  // FP8 rows: [n] scales (x = scale * q)
  int32_t d;
  // family
  int32_t kind, m, L, N;
  int32_t dims[LSH_MAX_MODES], mdims[LSH_MAX_MODES];
  int32_t dsum;          // entries per table of bins/signs (sum of mode sizes; CSSRP-L: d l)
  int32_t lc;            // entries per coordinate (CSSRP-L: l, else 1)
  int32_t cap;           // staged member-list capacity per table (sketch_capacity)
  const uint16_t *bins;
  const int8_t *signs;
  const float *b32;
  const double *b64;
  const uint32_t *ka, *kb;
  double w, sqrtm;
  // outputs
  int32_t *codes;        // E2LSH [n][L][m]
  uint64_t *bits;        // SRP [n][L][words]
  uint64_t *keys;        // [L][key_ld]
  int64_t key_ld;
  float *proj;           // [n][L][m]
  unsigned long long *counters;  // CNT_NUM or nullptr
  uint32_t *status;
  // deferred recheck (dense-row sketch kernel): flagged bins {row, t, l, fast code}
  int4 *queue = nullptr;
  uint32_t *qcount = nullptr;
  uint32_t qcap = 0;
  // replayed batches (dense-row sketch kernels only): X, n, keys and key_ld
  // come from this device descriptor at run time; the fields above then give
  // the largest batch the launch is sized for
  const BatchDesc *desc = nullptr;
};

// Dense-row CS/HCS hashing (all L tables, one launch).  With p.queue set,
// bins within the error bound are queued instead of rechecked in place;
// launch_sketch_recheck then computes their exact values from the member
// lists and patches codes, bits and keys.
cudaError_t launch_sketch_dense(const SketchLaunch &p, cudaStream_t stream);
cudaError_t launch_sketch_recheck(const SketchLaunch &p, const uint16_t *mlist, const uint32_t *mseg,
                                  cudaStream_t stream);
int64_t sketch_queue_cap(int64_t n, int32_t L, int32_t m);
// Plan of the dense-row kernel for a shape (for reporting / autotuning).
struct SketchPlan { int tables_per_cta, groups, row_groups, warps, smem, ctas; bool ok; };
SketchPlan plan_sketch_dense(int d, int m, int L, int cap, int dtype);
// Process-wide pinned plan of the dense-row kernel (all zeros: autotuned).
struct SketchPin { int rows_per_lane, row_groups, warps_per_table, tables_per_cta, entry_bytes, split_bins; };
void set_sketch_pin(const SketchPin &pin);
// False when a pinned plan does not fit the shape (the call must not launch).
bool sketch_pin_fits(int d, int m, int L, int cap);

// CSR-row CS/HCS hashing (all L tables, one launch).  colmajor: count-sketch
// tables as [d][L] entries bin | neg << 15 (NULL for HCS).  With rowptr NULL
// the rows are the dense rows p.X (p.dtype, p.ld) -- for d too large for the
// dense-row kernel's tile -- bounded per bin with the member counts of mseg.
cudaError_t launch_sketch_csr(const SketchLaunch &p, const int64_t *rowptr, const int32_t *col, const float *val,
                              const uint16_t *colmajor, const uint32_t *mseg, cudaStream_t stream);

// The family fields of a launch (tables, offsets, key multipliers, w).
SketchLaunch family_launch(const lsh_family_s *f);

// Time the dense-row kernel's candidate plans for the shape of p on its first
// rows (once per shape; nothing when a plan is pinned, the shape is cached,
// or p has fewer rows than the tuner needs), so that a later launch -- or a
// stream capture, which cannot time -- finds the tuned plan.
void sketch_autotune(const SketchLaunch &p, cudaStream_t stream);
// The plan a launch of p would use now (pinned, else tuned for the shape,
// else the default); tables_per_cta is the balanced group size.  False when
// no plan fits.
bool sketch_current_plan(const SketchLaunch &p, SketchPin &out);

// Hash the rows of X into keys [L][key_ld] (+ optional codes, proj, counters);
// stream-ordered, allocates nothing when counters is NULL.
lsh_status hash_impl(lsh_family_s *f, const lsh_matrix *X, void *codes, uint64_t *keys, int64_t key_ld,
                     float *proj, unsigned long long *counters, cudaStream_t stream);

// Dense E2LSH / SRP (FP32 SIMT GEMM, fused discretisation; with p.queue
// set, flagged entries are rechecked by a second kernel, else in place).
// keys and multi-word SRP bits must be zeroed by the caller.
cudaError_t launch_dense_fp32(const SketchLaunch &p, const float *G, const float *Gt, const float *gnorm,
                              cudaStream_t stream);
int64_t dense_queue_cap(int64_t n, int64_t ML);

// Dense E2LSH / SRP on the tensor cores (TMA + tcgen05, BF16 x BF16 -> FP32),
// for BF16 rows and a family whose G is stored in BF16.
constexpr int kTcColRecord = 8;  // floats per column record of d_gnc
bool tc_dense_supported(const lsh_family_desc &fd, const lsh_matrix *X);
int tc_chunk_ktiles(int d, bool fp8);
size_t tc_dense_scratch_bytes(int64_t n, int64_t ML);
cudaError_t launch_tc_dense(const SketchLaunch &p, const void *Gtc, const float *Gt, const float *gnc,
                            const int32_t *Gint, void *scratch, cudaStream_t stream);

// Query path: probe + dedup + exact top-k rerank, G CTAs per query
// (query_split: more CTAs per query for small batches) whose lists the last
// CTA merges.  scratch: query_scratch_bytes(scratch_q, k) bytes, its first
// scratch_q words zero (the kernel leaves them zero); NULL means G = 1.
// q_live: optional device word; rows >= *q_live are padding and skipped.
int query_split(int64_t q, int32_t k);
size_t query_scratch_bytes(int64_t q_max, int32_t k);
cudaError_t launch_query(const uint64_t *qkeys, int64_t q, int32_t L, int32_t k, int32_t metric, int32_t d,
                         const void *Q, int32_t q_dtype, int64_t q_ld, const lsh_index_s *idx, int32_t *out_ids,
                         float *out_dist, unsigned long long *counters, void *scratch, int64_t scratch_q,
                         const int64_t *q_live, cudaStream_t stream);

// Stable per-table sort of keys [L][n] with ids, then bucket segmentation:
// the bucket sort (one global pass on the highest varying digit, buckets
// finished on chip) when bucket_sort_used(n), else eight global 8-bit LSD
// radix passes; both give the same arrays.  Allocates its temporaries with
// cudaMallocAsync on `stream`.
cudaError_t build_tables(const uint64_t *keys, int64_t n, int32_t L, uint32_t *ids_out,
                         uint64_t *ukeys_out, uint32_t *offsets_out, int64_t *nb_out,
                         cudaStream_t stream);

// The same table build with caller-provided scratch (no allocation); the
// scratch must hold build_tables_scratch_bytes(n, L) bytes, 256-byte aligned.
size_t build_tables_scratch_bytes(int64_t n, int32_t L);
// Sort mode of the table build: 0 automatic, 1 global LSD passes, 2 bucket
// sort at any n.  Returns -1 for other values.
int set_sort_mode(int mode);
bool bucket_sort_used(int64_t n);
cudaError_t build_tables_scratch(const uint64_t *keys, int64_t n, int32_t L, uint32_t *ids_out,
                                 uint64_t *ukeys_out, uint32_t *offsets_out, int64_t *nb_out, void *scratch,
                                 cudaStream_t stream);

}  // namespace lsh
