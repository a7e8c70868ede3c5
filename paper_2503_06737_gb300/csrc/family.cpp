// family.cpp -- host sampler of the LSH family (the random functions of
// Definitions 2-5: per-mode h_k, s_k; dense Gaussian projection; offsets b;
// key multipliers), drawn from a 64-bit seed with SplitMix64 (Steele, Lea &
// Flood, OOPSLA 2014).  Compiled with -ffp-contract=off so the Box-Muller
// arithmetic is one IEEE rounding per operation.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "internal.h"

namespace lsh {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

inline uint64_t finalize(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// A SplitMix64 stream: Weyl state advanced by the golden gamma, output mixed.
class Stream {
 public:
  Stream(uint64_t seed, int table) : state_(finalize(seed + uint64_t(table + 1) * kGamma)) {}
  uint64_t next() {
    state_ += kGamma;
    return finalize(state_);
  }

 private:
  uint64_t state_;
};

inline double unit53(uint64_t r) { return double(r >> 11) * 0x1.0p-53; }

// Round a finite FP32 value to the nearest bfloat16 (ties to even), widened back.
inline float to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  std::memcpy(&f, &u, 4);
  return f;
}

// Round a finite FP32 value to the nearest FP8 E4M3 value (3 fraction bits,
// exponent bias 7, subnormal quantum 2^-9, largest finite 448), ties to even,
// saturating; integer rounding of the FP32 significand, widened back.
inline float to_e4m3(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t sign = u & 0x80000000u, a = u & 0x7FFFFFFFu;
  if (a < 0x00800000u) return sign ? -0.f : 0.f;  // zero or an FP32 subnormal: below 2^-10
  const int e = int(a >> 23) - 127;
  const int shift = e >= -6 ? 20 : 20 + (-6 - e);  // significand bits below the E4M3 quantum
  if (shift > 24) return sign ? -0.f : 0.f;
  const uint32_t mant = (a & 0x7FFFFFu) | 0x800000u;
  uint32_t keep = mant >> shift;
  const uint32_t rem = mant & ((1u << shift) - 1u), half = 1u << (shift - 1);
  if (rem > half || (rem == half && (keep & 1u))) ++keep;
  double v = std::ldexp(double(keep), e - 23 + shift);
  if (v > 448.0) v = 448.0;
  return float(sign ? -v : v);
}

void draw_offsets_and_keys(Stream &s, const lsh_family_desc &d, int t, HostFamily &hf) {
  const int m = d.m;
  for (int l = 0; l < m; ++l) hf.b[size_t(t) * m + l] = d.w * unit53(s.next());
  for (int l = 0; l < m; ++l) {
    uint64_t r = s.next();
    hf.ka[size_t(t) * m + l] = uint32_t(r >> 32) | 1u;
    hf.kb[size_t(t) * m + l] = uint32_t(r) | 1u;
  }
}

}  // namespace

void sample_family(const lsh_family_desc &d, HostFamily &hf) {
  hf.desc = d;
  const int L = d.L, m = d.m;
  hf.b.assign(size_t(L) * m, 0.0);
  hf.ka.assign(size_t(L) * m, 0u);
  hf.kb.assign(size_t(L) * m, 0u);
  if (kind_is_dense(d.kind)) {
    hf.dsum = 0;
    const size_t ldg = size_t(m) * L;
    hf.G.assign(size_t(d.d) * ldg, 0.f);
    const double two_pi = 6.283185307179586;
    for (int t = 0; t < L; ++t) {
      Stream s(d.seed, t);
      for (int j = 0; j < d.d; ++j)
        for (int l = 0; l < m; ++l) {
          const uint64_t r1 = s.next(), r2 = s.next();
          const double u1 = double((r1 >> 11) + 1) * 0x1.0p-53;  // (0, 1]
          const double u2 = double(r2 >> 11) * 0x1.0p-53;        // [0, 1)
          const double radius = std::sqrt(-2.0 * std::log(u1));
          const double g = radius * std::cos(two_pi * u2);
          const float g32 = float(g);
          hf.G[size_t(j) * ldg + size_t(t) * m + l] =
              d.compute == LSH_BF16 ? to_bf16(g32) : d.compute == LSH_FP8_E4M3 ? to_e4m3(g32) : g32;
        }
      draw_offsets_and_keys(s, d, t, hf);
    }
    return;
  }
  if (d.kind == LSH_CSL_SRP) {
    // CSSRP-L: per coordinate i, l distinct bins in draw order (a draw whose
    // bin i already has is drawn again), each with the sign of its draw
    const int lc = incidences(d);
    const int64_t dsum = int64_t(d.d) * lc;
    hf.dsum = dsum;
    hf.bins.assign(size_t(L) * dsum, 0);
    hf.signs.assign(size_t(L) * dsum, 1);
    for (int t = 0; t < L; ++t) {
      Stream s(d.seed, t);
      const int64_t base = int64_t(t) * dsum;
      for (int i = 0; i < d.d; ++i)
        for (int r = 0; r < lc; ++r) {
          for (;;) {
            const uint64_t u = s.next();
            const int32_t bin = int32_t(((u >> 32) * uint64_t(uint32_t(m))) >> 32);
            bool seen = false;
            for (int q = 0; q < r; ++q) seen = seen || hf.bins[base + int64_t(i) * lc + q] == bin;
            if (seen) continue;
            hf.bins[base + int64_t(i) * lc + r] = bin;
            hf.signs[base + int64_t(i) * lc + r] = (u & (1ULL << 31)) ? int8_t(-1) : int8_t(1);
            break;
          }
        }
      draw_offsets_and_keys(s, d, t, hf);
    }
    return;
  }
  int64_t dsum = 0;
  for (int k = 0; k < d.N; ++k) dsum += d.dims[k];
  hf.dsum = dsum;
  hf.bins.assign(size_t(L) * dsum, 0);
  hf.signs.assign(size_t(L) * dsum, 1);
  for (int t = 0; t < L; ++t) {
    Stream s(d.seed, t);
    int64_t base = int64_t(t) * dsum;
    for (int k = 0; k < d.N; ++k) {
      const uint64_t mk = uint32_t(d.mdims[k]);
      for (int i = 0; i < d.dims[k]; ++i, ++base) {
        const uint64_t r = s.next();
        hf.bins[base] = int32_t(((r >> 32) * mk) >> 32);
        hf.signs[base] = (r & (1ULL << 31)) ? int8_t(-1) : int8_t(1);
      }
    }
    draw_offsets_and_keys(s, d, t, hf);
  }
}

int sketch_capacity(const HostFamily &hf) {
  const lsh_family_desc &d = hf.desc;
  if (kind_is_dense(d.kind)) return 0;
  int best = 0;
  std::vector<uint32_t> cnt(size_t(2) * d.m);
  for (int t = 0; t < d.L; ++t) {
    std::fill(cnt.begin(), cnt.end(), 0u);
    const int32_t *hb = hf.bins.data() + size_t(t) * hf.dsum;
    const int8_t *sb = hf.signs.data() + size_t(t) * hf.dsum;
    if (d.kind == LSH_CSL_SRP) {
      for (int64_t e = 0; e < hf.dsum; ++e) ++cnt[size_t(2) * hb[e] + (sb[e] < 0 ? 1 : 0)];
    } else {
      for (int j = 0; j < d.d; ++j) {
        int r = j, off = 0, stride = 1, bin = 0, neg = 0;
        for (int k = 0; k < d.N; ++k) {
          const int ik = r % d.dims[k];
          r /= d.dims[k];
          bin += hb[off + ik] * stride;
          neg ^= sb[off + ik] < 0 ? 1 : 0;
          stride *= d.mdims[k];
          off += d.dims[k];
        }
        ++cnt[size_t(2) * bin + neg];
      }
    }
    int total = 0;
    for (int l = 0; l < d.m; ++l) {
      const uint32_t cp = cnt[size_t(2) * l], cn = cnt[size_t(2) * l + 1];
      total += cp + cn == 0 ? 4 : int(((cp + 3) & ~3u) + ((cn + 3) & ~3u));  // an empty bin keeps one quad
    }
    best = std::max(best, total);
  }
  return best;
}

}  // namespace lsh
