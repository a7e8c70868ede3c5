/*
 * lsh.h -- C ABI of the GB300 (sm_103a) CS/HCS LSH hashing and indexing library.
 *
 * Paper: "Faster and Space Efficient Indexing for Locality Sensitive Hashing"
 * (arXiv 2503.06737).  The library computes, for n points and L tables, the
 * m-dimensional hashcodes of
 *   - CS-E2LSH   (Definition 12, Sec. 4.1)  floor((sqrt(m) CS(x)_l + b_l) / w)
 *   - HCS-E2LSH  (Definition 19, Sec. 4.2)  floor((sqrt(m) vec(HCS(x))_l + b_l) / w)
 *   - CS-SRP     (Definition 25, Sec. 5.1)  1[CS(x)_l > 0]
 *   - HCS-SRP    (Definition 31, Sec. 5.2)  1[vec(HCS(x))_l > 0]
 * and of the dense baselines they replace,
 *   - E2LSH      (Definition 2, Sec. 3.1)   floor((<r_l, x> + b_l) / w)
 *   - SRP        (Definition 3, Sec. 3.1)   1[<r_l, x> > 0]
 * where CS is the count sketch of Definition 4 and HCS the higher-order count
 * sketch of Definition 5 (input viewed as a d_1 x ... x d_N tensor, first mode
 * fastest, zero-padded when prod d_k > d, Sec. 6).  It groups the points into
 * the L hash tables of the (m, tau)-amplified LSH scheme of Sec. 3.1 and
 * answers queries by probing the L tables, taking the union of the buckets
 * and ranking it by exact distance (Sec. 6).
 *
 * Integer results (codes, keys, bucket tables) are exact: the FP32 fast path
 * carries a rigorous error bound, and every entry whose FP32 value lies within
 * that bound of an E2LSH bin edge (or of 0 for SRP) is recomputed in FP64 in
 * ascending coordinate order, one IEEE rounding per operation, which is the
 * canonical result.
 *
 * Conventions for every call:
 *   - Pointers named in the argument lists as "device" are CUDA device
 *     pointers owned by the caller; "host" pointers are ordinary memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are stream-ordered and asynchronous unless a stats or export
 *     argument is given, in which case they synchronise `stream` before
 *     returning.
 *   - Every call returns an lsh_status; no C++ exception crosses the ABI.
 *     On failure lsh_last_error() returns a message for the calling thread.
 *   - Handles are immutable after creation except for a sticky device status
 *     word (lsh_family_status); concurrent calls on different streams that use
 *     the same handle are safe.
 */
#ifndef LSH_GB300_H
#define LSH_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LSH_OK = 0,
  LSH_EINVAL = 1,        /* invalid argument (checked on the host before any launch) */
  LSH_ENOMEM = 2,        /* device or host allocation failed */
  LSH_ECUDA = 3,         /* a CUDA runtime call failed */
  LSH_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
  LSH_ENONFINITE = 5,    /* an input row held NaN or Inf: its codes and keys are not defined */
  LSH_EUNSUPPORTED = 6,  /* valid request the library does not implement */
  LSH_ERANGE = 7,        /* an E2LSH code fell outside int32 */
  LSH_EIO = 8            /* a file could not be opened, read or written */
} lsh_status;

/* Hash kinds (numbering fixed: it is part of the ABI). */
typedef enum {
  LSH_E2LSH = 0,      /* dense Gaussian projection, floor       (Definition 2)  */
  LSH_SRP = 1,        /* dense Gaussian projection, sign        (Definition 3)  */
  LSH_CS_E2LSH = 2,   /* count sketch, scaled floor             (Definition 12) */
  LSH_HCS_E2LSH = 3,  /* higher-order count sketch, scaled floor (Definition 19) */
  LSH_CS_SRP = 4,     /* count sketch, sign                     (Definition 25) */
  LSH_HCS_SRP = 5,    /* higher-order count sketch, sign        (Definition 31) */
  LSH_CSL_SRP = 6     /* CSSRP-L: count-sketch matrix with l nonzeros per column, sign (Table 1) */
} lsh_kind;

/* Element types of inputs. */
typedef enum {
  LSH_F32 = 0,
  LSH_BF16 = 1,
  LSH_F16 = 2,
  LSH_FP8_E4M3 = 3   /* OCP E4M3 (finite-only variant) with a per-row FP32 scale */
} lsh_dtype;

#define LSH_MAX_MODES 8

/*
 * Family description.  The family is drawn from `seed` on the host:
 * per table t, SplitMix64 (Steele, Lea & Flood 2014) started at
 * mix64(seed + (t+1) * 0x9E3779B97F4A7C15) gives, in this order,
 *   for each mode k, each i < dims[k]: bin = (hi32(r) * mdims[k]) >> 32,
 *                                      sign = bit31(r) ? -1 : +1;
 *   (dense kinds instead: G[j][t*m + l] for j < d, l < m by Box-Muller on
 *    two draws, stored as FP32);
 *   b_l = w * hi53(r) * 2^-53 for l < m;
 *   key multipliers ka_l = hi32(r) | 1, kb_l = lo32(r) | 1 for l < m.
 *
 *   kind    lsh_kind.
 *   d       input dimension (>= 1).
 *   m       code length per table (bins per table), >= 1; = prod mdims.
 *   L       number of tables, >= 1.
 *   N       number of HCS modes (1 <= N <= LSH_MAX_MODES); CS kinds: 1.
 *   dims    HCS mode sizes, prod dims >= d (zero padding beyond d); CS: {d}.
 *   mdims   HCS sketch sizes per mode, prod = m; CS: {m}.
 *   w       E2LSH bin width (> 0; ignored by SRP kinds, still drawn).
 *   seed    64-bit family seed.
 *   compute element type the dense kinds store G in: LSH_F32 (the FP32
 *           draws), LSH_BF16 (each FP32 draw rounded to the nearest BF16,
 *           ties to even: BF16 rows then run on the tensor cores) or
 *           LSH_FP8_E4M3 (rounded to E4M3, saturating at 448: per-row-scaled
 *           FP8 rows run on the tensor cores).  CS/HCS kinds ignore it.
 *   nnz_per_col  CSSRP-L only: l, the nonzero entries per column of the
 *           m x d sketch matrix (1 <= l <= m; 0 reads as 1): coordinate i
 *           goes to l distinct bins, drawn in order per i as bin = (hi32(r) m)
 *           >> 32, a draw whose bin i already has being drawn again, each with
 *           its own sign bit31(r); the code is the sign of S x as for CS-SRP.
 *           N = 1, dims = {d}, mdims = {m}.  Dense rows only (no CSR).  Other
 *           kinds ignore it.
 */
typedef struct {
  int32_t kind;
  int32_t d;
  int32_t m;
  int32_t L;
  int32_t N;
  int32_t dims[LSH_MAX_MODES];
  int32_t mdims[LSH_MAX_MODES];
  double w;
  uint64_t seed;
  int32_t compute;
  int32_t nnz_per_col;
} lsh_family_desc;

/*
 * A batch of points (device memory, caller-owned, read-only during the call).
 *   dense: values = [n][ld] elements of `dtype` row-major, col = rowptr = NULL.
 *   CSR:   rowptr = [n+1] int64 offsets, col = [nnz] int32 column indices,
 *          strictly ascending within a row and < d; values = [nnz] FP32.
 *   row_scale: FP8 inputs only, [n] FP32, x[i][j] = row_scale[i] * q[i][j].
 */
typedef struct {
  int32_t dtype;
  int64_t n;
  int64_t d;
  int64_t ld;
  const void *values;
  const int32_t *col;
  const int64_t *rowptr;
  const float *row_scale;
} lsh_matrix;

typedef struct lsh_family_s *lsh_family_t;
typedef struct lsh_index_s *lsh_index_t;

/* Counters of one lsh_hash call (filled only when a stats pointer is given). */
typedef struct {
  int64_t n_entries;    /* n * L * m discretised entries */
  int64_t n_flagged;    /* entries within the FP32 error margin, recomputed in FP64 */
  int64_t n_changed;    /* of those, entries whose FP64 code differs from the FP32 one */
  int64_t n_nonfinite;  /* rows holding NaN or Inf */
  int64_t n_overflow;   /* E2LSH codes outside int32 */
} lsh_hash_stats;

typedef struct {
  int64_t n_queries;
  int64_t n_candidates;        /* sum over queries of the bucket-union sizes (with repeats) */
  int64_t n_unique;            /* sum over queries of distinct candidates */
  int64_t max_unique;          /* largest distinct-candidate count of one query */
} lsh_query_stats;

/* Message describing the last failure on the calling thread ("" if none). */
const char *lsh_last_error(void);

/* Library version string. */
const char *lsh_version(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (for accounting of launches inside a timed region). */
uint64_t lsh_launch_count(void);

/*
 * Draw a family (Definitions 2-5) and upload its tables to the current device.
 *   desc  host pointer, validated (LSH_EINVAL on any inconsistency).
 *   out   host pointer receiving the handle; the handle owns device memory
 *         until lsh_family_destroy.
 */
lsh_status lsh_make_family(const lsh_family_desc *desc, lsh_family_t *out);

/*
 * Draw the tables of the family `desc` on the host only (no device use) into
 * host buffers laid out as in lsh_family_export (any may be NULL).  For
 * checking the sampler against an independent implementation without a GPU.
 */
lsh_status lsh_sample_family_tables(const lsh_family_desc *desc, int32_t *bins, int8_t *signs, float *G,
                                    double *b, uint32_t *ka, uint32_t *kb);

/* Copy the description of a family into *desc (host). */
lsh_status lsh_family_describe(lsh_family_t fam, lsh_family_desc *desc);

/*
 * Copy the family's tables to host buffers (any may be NULL):
 *   bins   [L][sum dims] int32   per-mode bucket hashes h_k, modes concatenated
 *                                (CSSRP-L: [L][d l], entry i l + r the r-th bin of i)
 *   signs  [L][sum dims] int8    per-mode signs s_k (CSSRP-L: [L][d l])
 *   G      [d][m*L] float        dense kinds only
 *   b      [L][m] double         E2LSH offsets
 *   ka, kb [L][m] uint32         key multipliers
 * Synchronous.  For parity checks against an independent implementation.
 */
lsh_status lsh_family_export(lsh_family_t fam, int32_t *bins, int8_t *signs, float *G,
                             double *b, uint32_t *ka, uint32_t *kb);

/*
 * Read (and optionally clear) the family's sticky device status: bit 0 set
 * when some row was not finite, bit 1 when some code overflowed int32 in a
 * call made without stats.  Synchronises the device.
 */
lsh_status lsh_family_status(lsh_family_t fam, int32_t *status, int32_t clear);

void lsh_family_destroy(lsh_family_t fam);

/*
 * Hash the rows of X for all L tables in one launch (Definitions 2, 3, 12,
 * 19, 25, 31).
 *   X      host pointer to the batch description; its arrays are device memory;
 *          X->d must equal the family's d.  Dense inputs: f32/bf16/f16 for every
 *          kind; BF16 rows with a BF16 family, and per-row-scaled FP8 E4M3 rows
 *          with an E4M3 family, go to the tensor cores (the projection of an FP8
 *          row is its scale times the projection of its E4M3 values; FP8 rows
 *          need an E4M3 family, d and ld multiples of 16, 8 <= m <= 64 dividing
 *          64 or E2LSH with m = 128, m*L a multiple of 128, d <= 16384).  CSR
 *          inputs: CS/HCS kinds; dense rows too long for the dense-row kernel's
 *          shared-memory tile (d up to 65535) are hashed row by row.
 *   codes  device, optional: E2LSH kinds int32 [n][L][m]; SRP kinds uint64
 *          [n][L][ceil(m/64)] with code l in bit (l % 64) of word l / 64.
 *   keys   device, optional: uint64 [L][n], the bucket key of (point, table):
 *          SRP with m <= 64: the code bits; otherwise
 *          (sum_l code_l ka_l mod 2^32) * 2^32 + (sum_l code_l kb_l mod 2^32).
 *   proj   device, optional: float [n][L][m], the FP32 projection (sqrt(m) not
 *          applied), for error reporting.
 *   stats  host, optional: if given the call synchronises and fills it, and
 *          returns LSH_ENONFINITE / LSH_ERANGE when such rows/codes occurred.
 * Rows that hold NaN/Inf get key 0xFFFFFFFFFFFFFFFF and code INT32_MIN.
 * Stream-ordered and asynchronous, with two exceptions: the first dense-row
 * CS/HCS call of a shape (device, kind, d, m, L, modes, dtype) with at least
 * 524,288 rows times the candidate tile plans of the hashing kernel on its
 * first 524,288 rows and on half as many, and waits for them (once per
 * shape; skipped while the stream is captured); and calls with stats
 * synchronise.  Temporaries come
 * from the device's stream-ordered memory pool: the recheck queue of a
 * dense-row CS/HCS batch of 8,192 rows or more (16 B per 256 entries of
 * n*L*m, plus 1 MiB), and for a tensor-core call 36 B of row records and
 * counts per row plus two queues of 16 B per 256 projections (plus 1 MiB
 * each; the second holds the first grouped by row) -- 1.2 GiB for 4,000,000
 * rows with m*L = 2048.
 */
lsh_status lsh_hash(lsh_family_t fam, const lsh_matrix *X, void *codes, uint64_t *keys,
                    float *proj, lsh_hash_stats *stats, void *stream);

/*
 * Pin the tile plan of the dense-row CS/HCS hashing kernel for every later
 * call in this process (any family, any device), in place of the autotuned
 * one; all six arguments 0 restore the automatic choice.  Every plan
 * computes the same codes and keys; the plan only sets how the work maps to
 * the GPU:
 *   rows_per_lane    1, 2 or 4 rows per thread (one vector shared-memory load
 *                    per term serves them all);
 *   row_groups       1, 2 or 4 row groups per tile: groups of 32 lanes, or
 *                    of 16 with split_bins; a tile holds at most 128 rows;
 *   warps_per_table  1, 2 or 4 warps sharing the bins of one table;
 *   tables_per_cta   >= 1, the largest table group a CTA stages (balanced);
 *   entry_bytes      2 or 4, the width of a member-list entry;
 *   split_bins       0, or 1: the two halves of a warp sum alternate quads
 *                    of every bin for the same 16 lanes' rows and combine
 *                    their sums at the end of the bin (rows_per_lane >= 2),
 *                    which keeps rows_per_lane rows per thread in a tile of
 *                    half the rows.
 * Host only; returns LSH_EINVAL for values outside these sets.  A pinned plan
 * whose shared memory does not fit a shape (or 2-byte entries for
 * d * rows_per_lane * 4 > 16383) makes lsh_hash return LSH_EUNSUPPORTED.
 */
lsh_status lsh_set_sketch_plan(int32_t rows_per_lane, int32_t row_groups, int32_t warps_per_table,
                               int32_t tables_per_cta, int32_t entry_bytes, int32_t split_bins);

/*
 * The tile plan a dense-row CS/HCS hash of n rows of dtype would use now: the
 * pinned plan, else the one the autotuner chose for the shape (after a call
 * of 524,288 rows or more), else the default.  plan[6] receives
 * rows_per_lane, row_groups, warps_per_table, tables_per_cta (the balanced
 * group size actually staged), entry_bytes and split_bins.  Host only (no
 * timing, no device work); LSH_EUNSUPPORTED for dense families or when no
 * plan fits the shape.
 */
lsh_status lsh_get_sketch_plan(lsh_family_t fam, int32_t dtype, int64_t n, int32_t plan[6]);

/*
 * Replayed hashing of uneven batches of dense rows (keys only; the m*L hashes
 * of Definitions 12, 19, 25, 31 and the bucket keys of Sec. 3.1, equal to
 * lsh_hash's bit for bit).  A hasher captures, per batch-size bucket (powers
 * of two from 8,192 rows up to max_rows), one CUDA graph of the hashing --
 * recheck-queue reset, the sketch kernel over all L tables, the exact recheck
 * of the queued bins (batches of up to 8,192 rows recheck in place, in the
 * sketch kernel) -- sized for the bucket's largest batch, and replays it
 * for every batch that falls in the bucket; only a device-side batch
 * descriptor (X, n, keys, key_ld), written by the graph's first node,
 * changes between replays.  The first batch of a bucket captures its graph
 * (after the autotuner has timed the shape on that batch, when it has
 * 524,288 rows or more; a plan pinned with lsh_set_sketch_plan at capture
 * time is kept).
 *   fam       a CS-E2LSH, HCS-E2LSH, CS-SRP, HCS-SRP or CSSRP-L family whose
 *             rows fit the dense-row kernel's tile (borrowed: it must outlive
 *             the hasher); dense families return LSH_EUNSUPPORTED
 *   dtype     LSH_F32, LSH_BF16 or LSH_F16; ld the row stride in elements
 *             (>= d) of every batch
 *   max_rows  the largest batch (1 <= max_rows < 2^32 - 1); the hasher holds
 *             a recheck queue for it (16 B per 256 of max_rows*L*m, rounded up
 *             to a power of two rows, plus 1 MiB)
 * lsh_hasher_run hashes the n rows at device pointer X (16-byte aligned when
 * ld times the element size is a multiple of 16) into keys [L][key_ld]
 * (key_ld >= n), stream-ordered; 0 <= n <= max_rows.  Calls on one hasher
 * must be ordered on one stream (they share the descriptor and the queue).
 * lsh_hasher_info reports the graphs captured and the replays launched.
 * lsh_hasher_destroy waits for the device, then frees the graphs.
 */
typedef struct lsh_hasher_s *lsh_hasher_t;
lsh_status lsh_hasher_create(lsh_family_t fam, int32_t dtype, int64_t ld, int64_t max_rows, lsh_hasher_t *out);
lsh_status lsh_hasher_run(lsh_hasher_t h, const void *X, int64_t n, uint64_t *keys, int64_t key_ld, void *stream);
lsh_status lsh_hasher_info(lsh_hasher_t h, int64_t *captures, int64_t *replays);
void lsh_hasher_destroy(lsh_hasher_t h);

/*
 * The sort behind every table build (lsh_build_index, lsh_index_rebuild,
 * lsh_index_rebuild_host, lsh_build_tables_static), process-wide:
 *   0  automatic (the default): the bucket sort for 2,048 <= n <= 1,126,400
 *      rows, else the global passes;
 *   1  global passes: a stable LSD radix sort, 8 passes of 8 bits over all
 *      of every table's (key, id) pairs;
 *   2  the bucket sort at any n: per table, the bits on which its keys
 *      differ are found, one stable global pass on the 8 highest of them
 *      cuts the table into 256 buckets, and one CTA per bucket finishes it:
 *      a bucket of up to 5,120 keys in shared memory (one counting pass on
 *      the next 8 bits, then each key placed by comparisons inside its group
 *      of equal such bits), larger buckets and buckets with groups of more
 *      than 96 keys by counting passes on every lower digit through global
 *      memory, skipping digits on which the table's or the bucket's keys
 *      agree.
 * All modes give the same tables bit for bit; the mode only moves time
 * (buckets well above 5,120 keys, from more than about 1.1 M rows or from
 * clustered keys, are slower in mode 2).  Returns LSH_EINVAL for any other
 * mode.  Set it between builds: a build reads it when it is enqueued.
 */
lsh_status lsh_set_sort_mode(int32_t mode);

/*
 * Build the L hash tables of Sec. 3.1 over X: hash (keys only), then per
 * table a stable device sort of (key, id) (lsh_set_sort_mode) and the bucket
 * segmentation.
 *   keep_data  nonzero: the index keeps a device copy of X (dense rows) for
 *              lsh_query's exact rerank; zero: it keeps only the tables.
 *   out        host pointer receiving the handle (owns its device memory).
 * Stream-ordered; the caller may free X once `stream` has passed the call.
 */
lsh_status lsh_build_index(lsh_family_t fam, const lsh_matrix *X, int32_t keep_data,
                           lsh_index_t *out, void *stream);

/*
 * Rebuild an existing index over a new batch X with the same n (and d): hash,
 * sort and segment into the index's own arrays; when the index keeps data the
 * copy of X is refreshed too.  Stream-ordered; no device allocation beyond the
 * per-call temporaries of the sort (stream-ordered pool).
 */
lsh_status lsh_index_rebuild(lsh_index_t idx, const lsh_matrix *X, void *stream);

/*
 * The same rebuild from rows in HOST memory (X->values a host pointer, dense
 * f32/bf16/f16 rows; pinned memory for full copy speed): the rows go to the
 * device in chunks of chunk_rows (0: max(32768, n/32)) on a stream of the
 * call's own while the previous chunk is hashed on `stream` -- the transfer
 * and the hashing overlap -- then the tables are sorted on `stream`.  When the
 * index keeps data the rows land in its copy, else in two staging buffers
 * from the stream-ordered pool.  Returns once the work is enqueued; the
 * caller must keep X's rows unchanged until `stream` has passed the call.
 * Not for stream capture (it creates a stream and events).
 */
lsh_status lsh_index_rebuild_host(lsh_index_t idx, const lsh_matrix *X, int64_t chunk_rows, void *stream);

/* n and, for each table, the number of buckets (host, [L]; may be NULL).  Synchronous. */
lsh_status lsh_index_info(lsh_index_t idx, int64_t *n, int64_t *nbuckets);

/*
 * Copy the tables to host buffers (any may be NULL):
 *   ids      [L][n] uint32   point ids ordered by (key, id)
 *   ukeys    [L][n] uint64   distinct keys, ascending (first nbuckets[t] valid)
 *   offsets  [L][n+1] uint32 bucket starts in ids, offsets[t][nbuckets[t]] = n
 *   nbuckets [L] int64
 * Synchronous.
 */
lsh_status lsh_index_export(lsh_index_t idx, uint32_t *ids, uint64_t *ukeys, uint32_t *offsets,
                            int64_t *nbuckets);

/*
 * Answer a batch of queries (Sec. 3.1 probe, Sec. 6 rerank): hash each query,
 * look its key up in every table, take the union of those buckets, rank the
 * distinct candidates by exact distance (Euclidean for E2LSH kinds, cosine
 * distance 1 - cos for SRP kinds; FP32 arithmetic) and return the k best by
 * (distance, id).  Needs an index built with keep_data.
 *   Q     host pointer to a dense batch (device arrays), same dtype as the index data.
 *   k     1 <= k <= 256.
 *   ids   device int32 [q][k], -1 where fewer than k candidates exist.
 *   dist  device float [q][k], +inf there.
 *   stats host, optional (synchronises).
 */
lsh_status lsh_query(lsh_index_t idx, const lsh_matrix *Q, int32_t k, int32_t *ids, float *dist,
                     lsh_query_stats *stats, void *stream);

void lsh_index_destroy(lsh_index_t idx);

/*
 * Save an index's tables (and its kept rows, if any) to a file, and load them
 * back (Sec. 3.1: the L hash tables are the index; the family is redrawn from
 * its description, so the file stores only that description).
 *   lsh_index_save  path: host string.  Synchronises the device; LSH_EIO when
 *                   the file cannot be written.
 *   lsh_index_load  fam must have the description the file was saved with
 *                   (kind, d, m, L, modes, w, seed, compute), else LSH_EINVAL;
 *                   *out receives a new index (owns its device memory).
 *                   LSH_EIO for a missing or short file, LSH_EUNSUPPORTED for
 *                   another file version.
 * The file holds a versioned header, then nb [L] int64, offsets [L][n+1],
 * ids [L][n] uint32, ukeys [L][n] uint64 and the rows [n][d] when kept, in the
 * host's byte order.
 */
lsh_status lsh_index_save(lsh_index_t idx, const char *path);
lsh_status lsh_index_load(lsh_family_t fam, const char *path, lsh_index_t *out);

/*
 * Merge per-shard top-k lists of an index sharded by rows (each shard an
 * index over its own rows, ids local to the shard): the k best of the union
 * by (distance, global id), global id = local id + id_offset[s].  Because a
 * point's keys do not depend on the shard, a query's candidates over the
 * whole database are the union of its candidates in the shards, so merging
 * the shards' lsh_query results gives the unsharded result exactly.
 *   ids[s], dist[s]  host [q][k] lists of shard s, ascending by (distance, id),
 *                    -1 / +inf past their end (as lsh_query writes them).
 *   out_ids          host int64 [q][k], -1 where fewer than k exist.
 *   out_dist         host float [q][k], +inf there.
 * Host only, no device use.
 */
lsh_status lsh_merge_topk(int32_t shards, int64_t q, int32_t k, const int32_t *const *ids,
                          const float *const *dist, const int64_t *id_offset, int64_t *out_ids, float *out_dist);

/*
 * Serving loop (continuous batching) around lsh_query, with the data and the
 * index resident on the device.  Requests are batches of host queries; a
 * scheduler thread admits the oldest waiting request whenever one of `slots`
 * concurrent batch slots is free and the device bytes held by the batches in
 * flight, plus this request's, stay within `mem_budget`; admitted batches run
 * concurrently, each on its own stream: H2D -> hash -> probe / dedup / exact
 * rerank -> D2H.  With use_graphs, each slot captures one CUDA graph per
 * power-of-two batch bucket (>= 16 rows) and replays it for later batches of
 * that bucket, the rows beyond the batch being padding whose results are
 * dropped.  Each query is answered from its own row by its own CTA, so its
 * result does not depend on the other queries of its batch or of concurrent
 * batches.  The index (and its family) must outlive the server.
 */
typedef struct {
  int32_t max_batch;   /* largest batch (queries) a request may hold, 1..65536 */
  int32_t slots;       /* batches in flight at once (streams), 1..64 */
  int32_t k;           /* top-k of every query, 1..256 */
  int32_t use_graphs;  /* nonzero: replay captured graphs per batch-size bucket */
  int64_t mem_budget;  /* device bytes for batches in flight (0: no limit) */
} lsh_server_config;

typedef struct {
  int64_t completed_requests, completed_queries;
  double p50_ms, p99_ms, mean_ms, max_ms;  /* request latency, submit -> results on host */
  double busy_s;                           /* first submit -> last completion (seconds) */
  int64_t admitted_peak;                   /* most batches in flight at once */
  int64_t graph_replays, graph_captures;
} lsh_server_stats;

typedef struct lsh_server_s *lsh_server_t;

/* Start a serving loop on the current device over an index built with keep_data. */
lsh_status lsh_server_create(lsh_index_t idx, const lsh_server_config *cfg, lsh_server_t *out);

/* Queue a batch: queries = host [q][d] of `dtype` (f32 / bf16 / f16), copied
 * before the call returns; 1 <= q <= max_batch.  *ticket identifies it. */
lsh_status lsh_server_submit(lsh_server_t srv, const void *queries, int32_t dtype, int64_t q, int64_t *ticket);

/* Block until the ticket's batch is done; copy ids [q][k] / dist [q][k] to
 * host buffers (either may be NULL) and its latency in milliseconds. */
lsh_status lsh_server_wait(lsh_server_t srv, int64_t ticket, int32_t *ids, float *dist, double *latency_ms);

/* Latency percentiles and counters since creation or the last reset. */
lsh_status lsh_server_stats_get(lsh_server_t srv, lsh_server_stats *stats, int32_t reset);

/* Finish the queued and running batches, then stop. */
void lsh_server_destroy(lsh_server_t srv);

/*
 * Allocation-free table build.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory while they run
 * (a serving loop with a fixed memory budget, a process whose framework
 * allocator already holds nearly all of the GPU, a hot path that must never
 * stall in an allocator).  It does what lsh_build_index does after hashing --
 * per table, a stable sort of (key, id) and the bucket segmentation -- with
 * its sort scratch in a 24 MiB array of static device memory that every GPU
 * loading this library holds until the process exits.  It calls no cudaMalloc
 * or cudaFree.
 *   keys      device uint64 [L][n], e.g. the keys output of lsh_hash.
 *   ids, ukeys, offsets, nbuckets
 *             device outputs laid out as in lsh_index_export ([L][n], [L][n],
 *             [L][n+1], [L]); the caller owns them.
 *   Limits: n * L <= LSH_STATIC_MAX_PAIRS (2^20), and the sort scratch --
 *   keys twice (8 n L bytes each), ids (4 n L), the digit histograms
 *   (1024 ceil(n / 4096) L) and the bucket sort's key-spread words and
 *   bucket list (1040 L + 4), each rounded up to 256 bytes -- at most 24 MiB;
 *   so with few rows and many tables (n = 64, L = 16384, say) a request
 *   within 2^20 pairs can still be refused.  Requests past either limit
 *   return LSH_EINVAL with a message naming the limit.  The first call on a device looks up the
 *   array's device address (cudaGetSymbolAddress) with that device current;
 *   make that first call before any stream capture.  Every call uses the same
 *   array and leaves its contents behind, so calls that overlap on the GPU
 *   (different streams, or different host threads) race; serialise them.
 */
#define LSH_STATIC_MAX_PAIRS (1 << 20)
lsh_status lsh_build_tables_static(const uint64_t *keys, int64_t n, int32_t L, uint32_t *ids, uint64_t *ukeys,
                                   uint32_t *offsets, int64_t *nbuckets, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LSH_GB300_H */
