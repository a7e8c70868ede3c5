/*
 * lsh_oracle.c -- plain, slow, FP64 CPU oracle for the CS/HCS/dense LSH hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity reference for the CUDA
 * library: only the tests, the smoke check and the bench's CPU-baseline leg may
 * load it.  It shares no code, header, table or constant generator with the
 * library; it restates the paper's definitions directly, in FP64, in the most
 * obvious loop order.  It is built with -O2 -ffp-contract=off so that every
 * floating-point operation below is one IEEE-rounded operation, in source order.
 *
 * Paper: "Faster and Space Efficient Indexing for Locality Sensitive Hashing"
 * (arXiv 2503.06737).  Citations below name the paper's numbered items
 * (Definitions 1-31 share one counter with the theorems) and sections.
 *
 *   - Definition 2 (E2LSH, Sec. 3.1): h(p) = floor((<r,p> + b) / w).
 *   - Definition 3 (SRP, Sec. 3.1): bit = 1 iff <r,u> > 0, else 0.
 *   - Definition 4 (Count Sketch, Sec. 3.2): CS(p)_l = sum_{h(i)=l} s(i) p_i.
 *   - Definition 5 (Higher-Order Count Sketch, Sec. 3.2): HCS(p)_{l1..lN} =
 *       sum over (i1..iN) with h_k(i_k) = l_k of s_1(i1)...s_N(iN) p_j,
 *       j = i1 + sum_{k>=2} i_k prod_{t<k} d_t (first mode fastest).
 *   - Definition 12 (CS-E2LSH, Sec. 4.1): g(p)_l = floor((sqrt(m) CS(p)_l + b) / w).
 *   - Definition 19 (HCS-E2LSH, Sec. 4.2): g'(p)_l = floor((sqrt(m) vec(HCS(p))_l + b)/w),
 *       vec index l = l1 + sum_{k>=2} l_k prod_{t<k} m_t (first mode fastest).
 *   - Definition 25 (CS-SRP, Sec. 5.1): xi(u)_l = 1 iff CS(u)_l > 0.
 *   - Definition 31 (HCS-SRP, Sec. 5.2): xi'(u)_l = 1 iff vec(HCS(u))_l > 0.
 *   - Sec. 3.1 (LSH of Definition 1 and the (m, tau) amplification): tau tables,
 *       each storing every point in the bucket of its concatenated m-code.
 *   - Sec. 6 (Experiment): zero padding when d is not a product of the mode sizes;
 *       top-k by exact distance over the retrieved candidates; recall |S n S'|/|S|.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - the 2-wise independent h, s are fully random tables drawn from SplitMix64
 *     (Steele, Lea & Flood 2014) by the draw order documented at orc_family_tables;
 *   - one offset b per (table, bin), b = w * U, U uniform on [0,1) with 53 bits;
 *   - the bucket of a point in table t is its 64-bit key (orc_key);
 *   - the projection is summed in ascending coordinate order j, in FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Random generator: SplitMix64 as published by Steele, Lea and Flood  */
/* ("Fast splittable pseudorandom number generators", OOPSLA 2014).    */
/* ------------------------------------------------------------------ */
static const uint64_t ORC_GOLDEN_GAMMA = 0x9E3779B97F4A7C15ULL;

uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* One generator step: advance the Weyl state by the golden gamma, return its mix. */
uint64_t orc_splitmix_next(uint64_t *state) {
  *state += ORC_GOLDEN_GAMMA;
  return orc_mix64(*state);
}

/* The stream of table t of the family seeded by `seed`. */
uint64_t orc_table_stream(uint64_t seed, int t) {
  return orc_mix64(seed + (uint64_t)(t + 1) * ORC_GOLDEN_GAMMA);
}

/* 53-bit uniform in [0,1). */
static double orc_unit(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }

/* Bucket in [0, k): high 32 bits scaled to k (multiply-shift). */
static int32_t orc_bucket(uint64_t r, int32_t k) {
  return (int32_t)(((r >> 32) * (uint64_t)(uint32_t)k) >> 32);
}

/* Sign +1/-1 from bit 31. */
static int8_t orc_sign(uint64_t r) { return ((r >> 31) & 1ULL) ? (int8_t)-1 : (int8_t)1; }

/*
 * Count-sketch / HCS family tables for all L tables (Definitions 4 and 5).
 * A count sketch is the N = 1 case: dims = {d}, mdims = {m}.
 *
 * Draw order, per table t, from the stream orc_table_stream(seed, t):
 *   for each mode k = 0..N-1, for each i = 0..dims[k]-1: one draw r;
 *       bin_k(i) = (hi32(r) * mdims[k]) >> 32,  sign_k(i) = bit31(r) ? -1 : +1;
 *   then for l = 0..m-1: one draw r; b_l = w * U(r);
 *   then for l = 0..m-1: one draw r; ka_l = hi32(r) | 1, kb_l = lo32(r) | 1.
 *
 * Output layouts: bins/signs [L][sum_k dims[k]] (modes concatenated),
 * b [L][m], ka/kb [L][m], where m = prod mdims.
 */
void orc_family_tables(uint64_t seed, int L, int N, const int32_t *dims,
                       const int32_t *mdims, double w, int32_t *bins,
                       int8_t *signs, double *b, uint32_t *ka, uint32_t *kb) {
  int64_t D = 0, m = 1;
  for (int k = 0; k < N; ++k) { D += dims[k]; m *= mdims[k]; }
  for (int t = 0; t < L; ++t) {
    uint64_t st = orc_table_stream(seed, t);
    int64_t off = 0;
    for (int k = 0; k < N; ++k) {
      for (int32_t i = 0; i < dims[k]; ++i) {
        uint64_t r = orc_splitmix_next(&st);
        bins[t * D + off + i] = orc_bucket(r, mdims[k]);
        signs[t * D + off + i] = orc_sign(r);
      }
      off += dims[k];
    }
    for (int64_t l = 0; l < m; ++l) {
      uint64_t r = orc_splitmix_next(&st);
      b[t * m + l] = w * orc_unit(r);
    }
    for (int64_t l = 0; l < m; ++l) {
      uint64_t r = orc_splitmix_next(&st);
      ka[t * m + l] = (uint32_t)(r >> 32) | 1u;
      kb[t * m + l] = (uint32_t)r | 1u;
    }
  }
}

/*
 * CSSRP-L family (Table 1: a count-sketch projection matrix with l nonzero
 * entries in each column; the paper names it only by that property).
 * Reading: coordinate i goes to l distinct bins h_1(i) .. h_l(i), each with
 * its own random sign.  Draw order, per table t, from orc_table_stream(seed, t):
 *   for i = 0..d-1, for r = 0..l-1: draws until the bin (hi32(r) * m) >> 32 is
 *       not among the bins already chosen for i; the sign is bit31 of that
 *       accepted draw (-1 when set, else +1);
 *   then b_l and ka_l / kb_l exactly as in orc_family_tables.
 * Output: bins/signs [L][d * l] (entry i * l + r), b [L][m], ka/kb [L][m].
 * Needs 1 <= l <= m.
 */
void orc_family_tables_l(uint64_t seed, int L, int d, int m, int l, double w, int32_t *bins,
                         int8_t *signs, double *b, uint32_t *ka, uint32_t *kb) {
  const int64_t D = (int64_t)d * l;
  for (int t = 0; t < L; ++t) {
    uint64_t st = orc_table_stream(seed, t);
    for (int i = 0; i < d; ++i) {
      for (int r = 0; r < l; ++r) {
        for (;;) {
          uint64_t u = orc_splitmix_next(&st);
          int32_t bin = orc_bucket(u, m);
          int seen = 0;
          for (int q = 0; q < r; ++q)
            if (bins[t * D + (int64_t)i * l + q] == bin) seen = 1;
          if (seen) continue;
          bins[t * D + (int64_t)i * l + r] = bin;
          signs[t * D + (int64_t)i * l + r] = orc_sign(u);
          break;
        }
      }
    }
    for (int64_t q = 0; q < m; ++q) {
      uint64_t u = orc_splitmix_next(&st);
      b[t * m + q] = w * orc_unit(u);
    }
    for (int64_t q = 0; q < m; ++q) {
      uint64_t u = orc_splitmix_next(&st);
      ka[t * m + q] = (uint32_t)(u >> 32) | 1u;
      kb[t * m + q] = (uint32_t)u | 1u;
    }
  }
}

/* Round a finite binary32 value to the nearest bfloat16 (8-bit significand),
 * ties to even, and return it as binary32. */
static float orc_round_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  uint32_t lower = u & 0xFFFFu, keep = u & 0xFFFF0000u;
  uint32_t half = 0x8000u;
  if (lower > half || (lower == half && (keep & 0x10000u))) keep += 0x10000u;
  memcpy(&f, &keep, 4);
  return f;
}

/* Round a finite value to the nearest OCP FP8 E4M3 value (3 fraction bits,
 * exponent bias 7, subnormal quantum 2^-9, largest finite 448), ties to
 * even; magnitudes above 448 saturate to 448.  Written from the format's
 * definition: the quantum of |v| in [2^e, 2^(e+1)) is 2^(e-3) for e >= -6. */
double orc_round_e4m3(double v) {
  if (v == 0.0 || v != v) return v;
  double a = fabs(v);
  int e;
  frexp(a, &e);          /* a = f 2^e, f in [0.5, 1): a in [2^(e-1), 2^e) */
  int q = e - 1 - 3;     /* quantum exponent for the normal range */
  if (e - 1 < -6) q = -9;
  double r = nearbyint(ldexp(a, -q));  /* default mode: ties to even */
  double out = ldexp(r, q);
  if (out > 448.0) out = 448.0;
  return v < 0 ? -out : out;
}

/*
 * Dense Gaussian projection family (Definitions 2 and 3: r ~ N(0, I_d)).
 * Per table t: for j = 0..d-1, for l = 0..m-1: two draws r1, r2;
 *   u1 = (hi53(r1) + 1) 2^-53 in (0,1], u2 = hi53(r2) 2^-53 in [0,1);
 *   g = sqrt(-2 ln u1) cos(2 pi u2)                          (Box-Muller);
 *   G[j][t*m + l] = g rounded to FP32 (compute = 0), or that FP32 value rounded
 *   to bfloat16 (compute = 1) or to FP8 E4M3 (compute = 3);
 * then b and ka/kb exactly as in orc_family_tables.
 * G is [d][m*L] row-major.
 */
void orc_dense_family(uint64_t seed, int L, int d, int m, double w, int compute,
                      float *G, double *b, uint32_t *ka, uint32_t *kb) {
  const double two_pi = 6.283185307179586;
  const int64_t ldg = (int64_t)m * L;
  for (int t = 0; t < L; ++t) {
    uint64_t st = orc_table_stream(seed, t);
    for (int j = 0; j < d; ++j) {
      for (int l = 0; l < m; ++l) {
        uint64_t r1 = orc_splitmix_next(&st);
        uint64_t r2 = orc_splitmix_next(&st);
        double u1 = (double)((r1 >> 11) + 1) * 0x1.0p-53;
        double u2 = (double)(r2 >> 11) * 0x1.0p-53;
        double g = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
        float g32 = (float)g;
        G[(int64_t)j * ldg + (int64_t)t * m + l] =
            compute == 1 ? orc_round_bf16(g32) : compute == 3 ? (float)orc_round_e4m3((double)g32) : g32;
      }
    }
    for (int l = 0; l < m; ++l) {
      uint64_t r = orc_splitmix_next(&st);
      b[t * m + l] = w * orc_unit(r);
    }
    for (int l = 0; l < m; ++l) {
      uint64_t r = orc_splitmix_next(&st);
      ka[t * m + l] = (uint32_t)(r >> 32) | 1u;
      kb[t * m + l] = (uint32_t)r | 1u;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Exact widening of stored inputs to FP64.                            */
/* ------------------------------------------------------------------ */
double orc_from_f32(float v) { return (double)v; }

/* bfloat16: the upper 16 bits of an IEEE binary32. */
double orc_from_bf16(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return (double)f;
}

/* IEEE binary16: 1 sign, 5 exponent (bias 15), 10 fraction bits. */
double orc_from_f16(uint16_t h) {
  int s = (h >> 15) & 1, e = (h >> 10) & 31, f = h & 1023;
  double v;
  if (e == 0) v = ldexp((double)f, -24);
  else if (e == 31) v = f ? NAN : INFINITY;
  else v = ldexp((double)(f + 1024), e - 25);
  return s ? -v : v;
}

/* OCP FP8 E4M3 (fn variant): 1 sign, 4 exponent (bias 7), 3 fraction bits,
 * no infinities, S.1111.111 is NaN, max finite 448. */
double orc_from_e4m3(uint8_t q) {
  int s = (q >> 7) & 1, e = (q >> 3) & 15, f = q & 7;
  double v;
  if (e == 15 && f == 7) v = NAN;
  else if (e == 0) v = ldexp((double)f, -9);
  else v = ldexp((double)(f + 8), e - 10);
  return s ? -v : v;
}

/* dtype codes: 0 = f32, 1 = bf16, 2 = f16, 3 = fp8 e4m3 (x = scale[row] * q;
 * the projection of such a row is scale[row] times the projection of its
 * FP8 values q, one FP64 multiply after the sum -- see orc_hash_dense). */
static double orc_load(const void *X, int dtype, int64_t idx) {
  switch (dtype) {
  case 0: return orc_from_f32(((const float *)X)[idx]);
  case 1: return orc_from_bf16(((const uint16_t *)X)[idx]);
  case 2: return orc_from_f16(((const uint16_t *)X)[idx]);
  default: return orc_from_e4m3(((const uint8_t *)X)[idx]);
  }
}

/* Row `i` of X widened to FP64 (d entries; ld = row stride in elements);
 * FP8 rows are returned unscaled. */
void orc_load_row(const void *X, int dtype, const float *row_scale, int64_t ld,
                  int64_t i, int d, double *x) {
  for (int j = 0; j < d; ++j) {
    double v = orc_load(X, dtype, i * ld + j);
    x[j] = v;
  }
}

/* ------------------------------------------------------------------ */
/* Projections (one table).                                            */
/* ------------------------------------------------------------------ */

/* Definition 4: CS(p)_l = sum_{i in [d], h(i) = l} s(i) p_i.  One pass over
 * i in ascending order adds s(i) p_i into bin h(i), so every bin sums its own
 * terms in ascending i.  y has m entries. */
void orc_cs_project(const double *x, int d, const int32_t *h, const int8_t *s,
                    int m, double *y) {
  for (int l = 0; l < m; ++l) y[l] = 0.0;
  for (int i = 0; i < d; ++i) y[h[i]] = y[h[i]] + (double)s[i] * x[i];
}

/* CSSRP-L projection (Table 1): y_b = sum over (i, r) with h_r(i) = b of
 * s_r(i) p_i.  One pass over i in ascending order adds each of its l terms
 * into its bin, so every bin sums its own terms in ascending i. */
void orc_csl_project(const double *x, int d, int l, const int32_t *h, const int8_t *s,
                     int m, double *y) {
  for (int q = 0; q < m; ++q) y[q] = 0.0;
  for (int i = 0; i < d; ++i)
    for (int r = 0; r < l; ++r) {
      const int64_t e = (int64_t)i * l + r;
      y[h[e]] = y[h[e]] + (double)s[e] * x[i];
    }
}

/* Definition 5 with the vec() of Definitions 19/31.  The vector x of length d
 * is viewed as a d_1 x ... x d_N tensor with j = i_1 + i_2 d_1 + i_3 d_1 d_2 + ...
 * (first mode fastest); coordinates j >= d are the zero padding of Sec. 6.
 * Output l = l_1 + l_2 m_1 + l_3 m_1 m_2 + ... (first mode fastest) collects
 * s_1(i_1) ... s_N(i_N) p_j over all tuples with h_k(i_k) = l_k.  One pass over
 * j in ascending order adds each term into its bin, so every bin sums its own
 * terms in ascending j.  hk/sk hold the modes concatenated: mode k occupies
 * [sum_{t<k} d_t, sum_{t<=k} d_t). */
void orc_hcs_project(const double *x, int d, int N, const int32_t *dims,
                     const int32_t *mdims, const int32_t *hk, const int8_t *sk,
                     double *y) {
  int64_t D = 1, m = 1;
  int32_t moff[16];
  int32_t o = 0;
  for (int k = 0; k < N; ++k) { D *= dims[k]; m *= mdims[k]; moff[k] = o; o += dims[k]; }
  for (int64_t l = 0; l < m; ++l) y[l] = 0.0;
  for (int64_t j = 0; j < D; ++j) {
    int64_t r = j, l = 0, stride = 1;
    double sg = 1.0;
    for (int k = 0; k < N; ++k) {
      int32_t ik = (int32_t)(r % dims[k]);
      r /= dims[k];
      l += (int64_t)hk[moff[k] + ik] * stride;
      stride *= mdims[k];
      sg = sg * (double)sk[moff[k] + ik];
    }
    double pj = (j < d) ? x[j] : 0.0; /* zero padding (Sec. 6) */
    y[l] = y[l] + sg * pj;
  }
}

/* Dense projection of Definitions 2/3 for one table: y_l = <G[:, col0 + l], x>,
 * summed in ascending j.  G is [d][ldg] FP32. */
void orc_dense_project(const double *x, int d, const float *G, int64_t ldg,
                       int64_t col0, int m, double *y) {
  for (int l = 0; l < m; ++l) {
    double acc = 0.0;
    for (int j = 0; j < d; ++j)
      acc = acc + x[j] * (double)G[(int64_t)j * ldg + col0 + l];
    y[l] = acc;
  }
}

/* ------------------------------------------------------------------ */
/* Discretisation and keys.                                            */
/* ------------------------------------------------------------------ */

/* Definitions 12/19 (scale = sqrt(m)) and Definition 2 (scale = 1):
 * code = floor(((scale * y) + b) / w), each operation IEEE-rounded in FP64.
 * Sets *err = 1 when the result does not fit int32. */
int32_t orc_e2lsh_code(double y, double scale, double b, double w, int *err) {
  double t1 = scale * y;
  double t2 = t1 + b;
  double t3 = t2 / w;
  double f = floor(t3);
  if (!(f >= -2147483648.0 && f <= 2147483647.0)) { if (err) *err = 1; return INT32_MIN; }
  return (int32_t)f;
}

/* Definitions 3/25/31: 1 iff y > 0 (zero and -0 give 0). */
int orc_srp_bit(double y) { return y > 0.0 ? 1 : 0; }

/* Key of one (point, table) from its m codes (the bucket of Sec. 3.1's
 * amplified scheme).  SRP with m <= 64: the bit pattern itself, bit l = code l.
 * Otherwise: a = sum_l code_l * ka_l mod 2^32, b = sum_l code_l * kb_l mod 2^32,
 * key = a * 2^32 + b (codes taken as 32-bit two's complement words). */
uint64_t orc_key(const int32_t *codes, int m, int is_srp, const uint32_t *ka,
                 const uint32_t *kb) {
  if (is_srp && m <= 64) {
    uint64_t key = 0;
    for (int l = 0; l < m; ++l)
      if (codes[l]) key |= (uint64_t)1 << l;
    return key;
  }
  uint32_t a = 0, b = 0;
  for (int l = 0; l < m; ++l) {
    a += (uint32_t)codes[l] * ka[l];
    b += (uint32_t)codes[l] * kb[l];
  }
  return ((uint64_t)a << 32) | (uint64_t)b;
}

/* ------------------------------------------------------------------ */
/* Whole-batch hashing.                                                */
/* ------------------------------------------------------------------ */

/* kind codes: 0 E2LSH (dense), 1 SRP (dense), 2 CS-E2LSH, 3 HCS-E2LSH,
 *             4 CS-SRP, 5 HCS-SRP, 6 CSSRP-L (N holds l, tables [L][d l]).
 *             A count sketch is an HCS with N = 1. */
typedef struct {
  int kind, d, m, L, N;
  int32_t dims[8], mdims[8];
  double w;
  const int32_t *bins;  /* [L][sum dims] */
  const int8_t *signs;  /* [L][sum dims] */
  const float *G;       /* dense: [d][m*L] */
  const double *b;      /* [L][m] */
  const uint32_t *ka, *kb;
} orc_family;

static int orc_is_srp(int kind) { return kind == 1 || kind == 4 || kind == 5 || kind == 6; }

/* Projection of one point for table t (FP64, ascending j). */
static void orc_project_table(const orc_family *f, const double *x, int t, double *y) {
  int64_t D = 0;
  if (f->kind != 6)
    for (int k = 0; k < f->N; ++k) D += f->dims[k];
  if (f->kind == 0 || f->kind == 1) {
    orc_dense_project(x, f->d, f->G, (int64_t)f->m * f->L, (int64_t)t * f->m, f->m, y);
  } else if (f->kind == 2 || f->kind == 4) {
    orc_cs_project(x, f->d, f->bins + t * D, f->signs + t * D, f->m, y);
  } else if (f->kind == 6) {
    const int64_t Dl = (int64_t)f->d * f->N;
    orc_csl_project(x, f->d, f->N, f->bins + t * Dl, f->signs + t * Dl, f->m, y);
  } else {
    orc_hcs_project(x, f->d, f->N, f->dims, f->mdims, f->bins + t * D, f->signs + t * D, y);
  }
}

/* Hash n dense rows.  Any of y_out [n][L][m], codes [n][L][m] (E2LSH code or
 * SRP bit), keys [L][n] may be NULL.  Returns 0, or 1 if some E2LSH code
 * overflowed int32, or 2 if some input was not finite. */
int orc_hash_dense(const orc_family *f, const void *X, int dtype,
                   const float *row_scale, int64_t n, int64_t ld, double *y_out,
                   int32_t *codes, uint64_t *keys) {
  const int m = f->m, L = f->L, d = f->d;
  const int srp = orc_is_srp(f->kind);
  const double scale = (f->kind == 2 || f->kind == 3) ? sqrt((double)m) : 1.0;
  int status = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : status)
  for (int64_t i = 0; i < n; ++i) {
    double *x = (double *)malloc(sizeof(double) * (size_t)d);
    double *y = (double *)malloc(sizeof(double) * (size_t)m);
    int32_t *c = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    orc_load_row(X, dtype, row_scale, ld, i, d, x);
    for (int j = 0; j < d; ++j)
      if (!isfinite(x[j])) status |= 2;
    const double rs = (dtype == 3 && row_scale) ? (double)row_scale[i] : 1.0;
    if (!isfinite(rs)) status |= 2;
    for (int t = 0; t < L; ++t) {
      orc_project_table(f, x, t, y);
      /* a per-row-scaled FP8 row: y = scale * (projection of q), one rounding */
      if (dtype == 3 && row_scale)
        for (int l = 0; l < m; ++l) y[l] = rs * y[l];
      for (int l = 0; l < m; ++l) {
        int err = 0;
        c[l] = srp ? orc_srp_bit(y[l]) : orc_e2lsh_code(y[l], scale, f->b[t * m + l], f->w, &err);
        if (err) status |= 1;
        if (y_out) y_out[(i * L + t) * m + l] = y[l];
        if (codes) codes[(i * L + t) * m + l] = c[l];
      }
      if (keys) keys[(int64_t)t * n + i] = orc_key(c, m, srp, f->ka + t * m, f->kb + t * m);
    }
    free(x); free(y); free(c);
  }
  return status;
}

/* Hash n CSR rows (rowptr [n+1], cols sorted ascending within a row, values
 * FP32) of width d.  The row is the dense vector holding the stored values and
 * zeros elsewhere; the projection sums the stored entries in ascending column
 * order, which equals the dense sum because the omitted terms are zeros. */
int orc_hash_csr(const orc_family *f, int64_t n, const int64_t *rowptr,
                 const int32_t *cols, const float *vals, double *y_out,
                 int32_t *codes, uint64_t *keys) {
  const int m = f->m, L = f->L, d = f->d;
  const int srp = orc_is_srp(f->kind);
  const double scale = (f->kind == 2 || f->kind == 3) ? sqrt((double)m) : 1.0;
  int status = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : status)
  for (int64_t i = 0; i < n; ++i) {
    double *x = (double *)calloc((size_t)d, sizeof(double));
    double *y = (double *)malloc(sizeof(double) * (size_t)m);
    int32_t *c = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      x[cols[e]] = (double)vals[e];
      if (!isfinite(x[cols[e]])) status |= 2;
    }
    for (int t = 0; t < L; ++t) {
      orc_project_table(f, x, t, y);
      for (int l = 0; l < m; ++l) {
        int err = 0;
        c[l] = srp ? orc_srp_bit(y[l]) : orc_e2lsh_code(y[l], scale, f->b[t * m + l], f->w, &err);
        if (err) status |= 1;
        if (y_out) y_out[(i * L + t) * m + l] = y[l];
        if (codes) codes[(i * L + t) * m + l] = c[l];
      }
      if (keys) keys[(int64_t)t * n + i] = orc_key(c, m, srp, f->ka + t * m, f->kb + t * m);
    }
    free(x); free(y); free(c);
  }
  return status;
}

/* ------------------------------------------------------------------ */
/* Index: the hash tables of Sec. 3.1 (every point stored in the bucket of  */
/* its key, in each of the L tables).                                   */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t key; uint32_t id; } orc_pair;

static int orc_pair_cmp(const void *a, const void *b) {
  const orc_pair *p = (const orc_pair *)a, *q = (const orc_pair *)b;
  if (p->key != q->key) return p->key < q->key ? -1 : 1;
  return p->id < q->id ? -1 : (p->id > q->id ? 1 : 0);
}

/* For each table: ids [L][n] ordered by (key, id); ukeys [L][n] (first nb[t]
 * valid) the distinct keys ascending; offsets [L][n+1] (first nb[t]+1 valid)
 * the start of each bucket in ids, last = n. */
void orc_build_index(const uint64_t *keys, int64_t n, int L, uint32_t *ids,
                     uint64_t *ukeys, uint32_t *offsets, int64_t *nb) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < L; ++t) {
    orc_pair *p = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { p[i].key = keys[(int64_t)t * n + i]; p[i].id = (uint32_t)i; }
    qsort(p, (size_t)n, sizeof(orc_pair), orc_pair_cmp);
    int64_t B = 0;
    for (int64_t i = 0; i < n; ++i) {
      ids[(int64_t)t * n + i] = p[i].id;
      if (i == 0 || p[i].key != p[i - 1].key) {
        ukeys[(int64_t)t * n + B] = p[i].key;
        offsets[(int64_t)t * (n + 1) + B] = (uint32_t)i;
        ++B;
      }
    }
    offsets[(int64_t)t * (n + 1) + B] = (uint32_t)n;
    nb[t] = B;
    free(p);
  }
}

/* ------------------------------------------------------------------ */
/* Query: probe each table with the query's key, union the buckets,    */
/* rank the union by exact distance (Sec. 6), keep the k best.          */
/* ------------------------------------------------------------------ */
typedef struct { double dist; uint32_t id; } orc_cand;

static int orc_cand_cmp(const void *a, const void *b) {
  const orc_cand *p = (const orc_cand *)a, *q = (const orc_cand *)b;
  if (p->dist != q->dist) return p->dist < q->dist ? -1 : 1;
  return p->id < q->id ? -1 : (p->id > q->id ? 1 : 0);
}

static int orc_u32_cmp(const void *a, const void *b) {
  uint32_t p = *(const uint32_t *)a, q = *(const uint32_t *)b;
  return p < q ? -1 : (p > q ? 1 : 0);
}

/* metric 0: Euclidean distance ||q - x||; metric 1: cosine distance
 * 1 - <q,x>/(||q|| ||x||) (1 when either norm is zero). */
double orc_distance(const double *q, const double *x, int d, int metric) {
  if (metric == 0) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) { double e = q[j] - x[j]; s = s + e * e; }
    return sqrt(s);
  }
  double qq = 0.0, xx = 0.0, qx = 0.0;
  for (int j = 0; j < d; ++j) { qq = qq + q[j] * q[j]; xx = xx + x[j] * x[j]; qx = qx + q[j] * x[j]; }
  if (qq == 0.0 || xx == 0.0) return 1.0;
  return 1.0 - qx / (sqrt(qq) * sqrt(xx));
}

/* The candidate set of one query: sorted distinct ids of the union over
 * tables of the bucket whose key equals qkeys[t].  Returns the count; cand
 * must hold up to L*n ids. */
int64_t orc_candidates(const uint32_t *ids, const uint64_t *ukeys,
                       const uint32_t *offsets, const int64_t *nb, int64_t n,
                       int L, const uint64_t *qkey_of_table, uint32_t *cand) {
  int64_t c = 0;
  for (int t = 0; t < L; ++t) {
    const uint64_t *uk = ukeys + (int64_t)t * n;
    int64_t lo = 0, hi = nb[t];
    while (lo < hi) { /* first ukey >= qkey */
      int64_t mid = (lo + hi) / 2;
      if (uk[mid] < qkey_of_table[t]) lo = mid + 1; else hi = mid;
    }
    if (lo < nb[t] && uk[lo] == qkey_of_table[t]) {
      const uint32_t *off = offsets + (int64_t)t * (n + 1);
      for (uint32_t e = off[lo]; e < off[lo + 1]; ++e) cand[c++] = ids[(int64_t)t * n + e];
    }
  }
  qsort(cand, (size_t)c, sizeof(uint32_t), orc_u32_cmp);
  int64_t u = 0;
  for (int64_t i = 0; i < c; ++i)
    if (u == 0 || cand[i] != cand[u - 1]) cand[u++] = cand[i];
  return u;
}

/* Answer q queries: qkeys [L][q]; database X (n rows, dtype, ld) and queries
 * Q (q rows, dtype_q, ldq).  out_ids [q][k] (-1 where fewer than k
 * candidates), out_dist [q][k] (+inf there), ncand [q] (may be NULL). */
void orc_query(const uint32_t *ids, const uint64_t *ukeys, const uint32_t *offsets,
               const int64_t *nb, int64_t n, int L, int d, const void *X, int dtype,
               int64_t ld, const void *Q, int dtype_q, int64_t ldq, int64_t q,
               const uint64_t *qkeys, int k, int metric, int32_t *out_ids,
               double *out_dist, int64_t *ncand) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < q; ++i) {
    uint64_t *qk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)L);
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(L * n + 1));
    double *qv = (double *)malloc(sizeof(double) * (size_t)d);
    double *xv = (double *)malloc(sizeof(double) * (size_t)d);
    for (int t = 0; t < L; ++t) qk[t] = qkeys[(int64_t)t * q + i];
    int64_t c = orc_candidates(ids, ukeys, offsets, nb, n, L, qk, cand);
    if (ncand) ncand[i] = c;
    orc_cand *cd = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)(c > 0 ? c : 1));
    orc_load_row(Q, dtype_q, NULL, ldq, i, d, qv);
    for (int64_t e = 0; e < c; ++e) {
      orc_load_row(X, dtype, NULL, ld, cand[e], d, xv);
      cd[e].dist = orc_distance(qv, xv, d, metric);
      cd[e].id = cand[e];
    }
    qsort(cd, (size_t)c, sizeof(orc_cand), orc_cand_cmp);
    for (int r = 0; r < k; ++r) {
      out_ids[i * k + r] = r < c ? (int32_t)cd[r].id : -1;
      out_dist[i * k + r] = r < c ? cd[r].dist : INFINITY;
    }
    free(qk); free(cand); free(qv); free(xv); free(cd);
  }
}

/* Exact k nearest neighbours over the whole database (the ground truth S of
 * the recall of Sec. 6). */
void orc_bruteforce_knn(int64_t n, int d, const void *X, int dtype, int64_t ld,
                        const void *Q, int dtype_q, int64_t ldq, int64_t q, int k,
                        int metric, int32_t *out_ids, double *out_dist) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < q; ++i) {
    double *qv = (double *)malloc(sizeof(double) * (size_t)d);
    double *xv = (double *)malloc(sizeof(double) * (size_t)d);
    orc_cand *cd = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)(n > 0 ? n : 1));
    orc_load_row(Q, dtype_q, NULL, ldq, i, d, qv);
    for (int64_t e = 0; e < n; ++e) {
      orc_load_row(X, dtype, NULL, ld, e, d, xv);
      cd[e].dist = orc_distance(qv, xv, d, metric);
      cd[e].id = (uint32_t)e;
    }
    qsort(cd, (size_t)n, sizeof(orc_cand), orc_cand_cmp);
    for (int r = 0; r < k; ++r) {
      out_ids[i * k + r] = r < n ? (int32_t)cd[r].id : -1;
      out_dist[i * k + r] = r < n ? cd[r].dist : INFINITY;
    }
    free(qv); free(xv); free(cd);
  }
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
