// hash_sketch.cu -- host side of the CS / HCS hashing of dense rows
// (Definitions 4, 5, 12, 19, 25, 31): the tile plans of the kernel in
// sketch_dense_kernel.cuh, their autotuner, plan pins, and the launches.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>
#include <stdint.h>

#include "sketch_dense.h"

namespace lsh {

using namespace sk;

namespace {

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

int align16(int v) { return (v + 15) & ~15; }

// Odd word stride of a row inside a row group (>= d + 1: word d is the zero slot).
int odd_stride(int d) { return (d + 1) | 1; }

// 16-bit entries hold offsets up to the zero slot d * RPL * 4 in 14 bits
// (bits 14 and 15 of a quad's first entry are its flags).
bool entry16_ok(int d, int RPL) { return int64_t(d) * RPL * 4 <= 0x3fff; }

// Rows of one tile of a plan.
int tile_rows(const Plan &pl) { return pl.RG * groups_per_warp(pl.hw != 0) * pl.RPL; }

// The shared-memory layout of one plan: RPL rows per lane, RG row groups of
// 32 lanes (16 with split bins, hw), WPT warps per table, table groups of
// (balanced) size <= Lg, es-byte entries.  Split bins pad every bin to an
// even number of quads: at most one more quad per bin.  smem > kMaxSmem when
// it does not fit.
Plan plan_of(int d, int m, int L, int cap, int RPL, int RG, int WPT, int Lg, int es, int hw) {
  const int G = (L + Lg - 1) / Lg;
  const int Lgb = (L + G - 1) / G;  // balanced group size
  Plan pl{};
  pl.Lg = Lgb;
  pl.G = G;
  pl.RG = RG;
  pl.WPT = WPT;
  pl.RPL = RPL;
  pl.hw = hw;
  pl.es = es;
  // warps claim tasks dynamically, so every warp the registers allow (one
  // CTA per SM) helps hide shared-memory latency
  const int maxW = max_threads(RPL) / kWarp;
  const int tasks = RG * Lgb * WPT;
  int W = tasks < maxW ? tasks : maxW;
  if (W < 4) W = 4;
  pl.W = W;
  pl.dp = odd_stride(d);
  pl.cap = (hw ? cap + 4 * m : cap) + 8;  // + two spare quads the loop's look-ahead may read
  const int R = tile_rows(pl);
  int off = 0;
  pl.off_ent = off;
  off = align16(off + Lgb * pl.cap * es);
  pl.off_seg = off;
  off = align16(off + Lgb * m * 8);
  pl.off_cst = off;
  off = align16(off + Lgb * m * 16);
  pl.off_rng = off;
  off = align16(off + Lgb * (kMaxWpt + 1) * 8);
  pl.off_key = off;
  off = align16(off + R * Lgb * 8);
  pl.off_x = off;
  const int64_t xbytes = int64_t(R) * pl.dp * 4;
  const int64_t scratch = int64_t(W) * 2 * m * 4;
  const int64_t big = std::max(xbytes, scratch);
  if (big > kMaxSmem) {
    pl.smem = kMaxSmem + 1;
    return pl;
  }
  off = align16(off + int(big));
  pl.off_xmax = off;
  off = align16(off + R * 4);
  pl.off_bad = off;
  off = align16(off + R * 4);
  pl.off_ctr = off;
  off = align16(off + 4);
  pl.smem = off;
  return pl;
}

// Tile shapes {rows per lane, row groups, split bins}, most rows per lane first.
constexpr int kShapes[9][3] = {{4, 1, 0}, {4, 1, 1}, {2, 1, 0}, {2, 1, 1}, {4, 2, 1},
                               {2, 2, 1}, {1, 4, 0}, {1, 2, 0}, {1, 1, 0}};

// The default plan (no timing): the first tile shape that fits, two warps
// per table, 16-bit entries where they fit, and the largest table group that
// fits.  Tiles larger than 32 rows only while every SM gets at least two.
Plan make_plan(int d, int m, int L, int cap, int64_t n) {
  Plan best{};
  best.smem = -1;
  const int sms = num_sms();
  for (const auto &sh : kShapes) {
    const int RPL = sh[0], RG = sh[1], hw = sh[2];
    const int R = RPL * RG * groups_per_warp(hw != 0);
    const int64_t ntiles = (n + R - 1) / R;
    if (R > kWarp && ntiles < 2 * sms) continue;
    for (int es = entry16_ok(d, RPL) ? 2 : 4; es <= 4; es += 2)
      for (int WPT = (m >= 2 ? 2 : 1); WPT >= 1; --WPT)
        for (int Lg = (L < 32 ? L : 32); Lg >= 1; --Lg) {
          const Plan pl = plan_of(d, m, L, cap, RPL, RG, WPT, Lg, es, hw);
          if (pl.smem <= kMaxSmem) return pl;
        }
  }
  return best;
}

// Candidate plans for the autotuner: for each tile shape, entry width and
// warps per table, the largest fitting table group and the next smaller
// group count.
std::vector<Plan> plan_candidates(int d, int m, int L, int cap, int64_t n) {
  std::vector<Plan> out;
  const int sms = num_sms();
  for (const auto &sh : kShapes) {
    const int RPL = sh[0], RG = sh[1], hw = sh[2];
    const int R = RPL * RG * groups_per_warp(hw != 0);
    const int64_t ntiles = (n + R - 1) / R;
    if (R > kWarp && ntiles < 2 * sms) continue;
    for (int es = entry16_ok(d, RPL) ? 2 : 4; es <= 4; es += 2)
      for (int WPT = 4; WPT >= 1; WPT >>= 1) {
        if (WPT > m) continue;
        int found = 0, lastG = -1;
        for (int Lg = (L < 32 ? L : 32); Lg >= 1 && found < 2; --Lg) {
          const Plan pl = plan_of(d, m, L, cap, RPL, RG, WPT, Lg, es, hw);
          if (pl.smem > kMaxSmem || pl.G == lastG) continue;
          if (pl.RG * pl.Lg * pl.WPT > 128) continue;
          lastG = pl.G;
          out.push_back(pl);
          ++found;
        }
      }
  }
  return out;
}

}  // namespace

SketchPlan plan_sketch_dense(int d, int m, int L, int cap, int dtype) {
  (void)dtype;
  Plan pl = make_plan(d, m, L, cap, 1);
  SketchPlan sp{};
  sp.ok = pl.smem > 0;
  if (!sp.ok) return sp;
  sp.tables_per_cta = pl.Lg;
  sp.groups = pl.G;
  sp.row_groups = pl.RG;
  sp.warps = pl.W;
  sp.smem = pl.smem;
  sp.ctas = num_sms();
  return sp;
}

int64_t sketch_queue_cap(int64_t n, int32_t L, int32_t m) {
  // about 16x the flag rate seen on Gaussian-mixture rows; the excess is rechecked in place
  return std::min<int64_t>(n * L * m / 256 + 65536, int64_t(1) << 28);
}

cudaError_t launch_sketch_recheck(const SketchLaunch &p, const uint16_t *mlist, const uint32_t *mseg,
                                  cudaStream_t stream) {
  if (p.n <= 0 || !p.queue) return cudaSuccess;
  const int blocks = num_sms() * 8;
  return kind_is_srp(p.kind) ? launch_recheck_srp(p, mlist, mseg, blocks, stream)
                             : launch_recheck_e2lsh(p, mlist, mseg, blocks, stream);
}

namespace {

cudaError_t launch_plan(const SketchLaunch &p, const Plan &pl, cudaStream_t stream) {
  if (p.dtype != LSH_F32 && p.dtype != LSH_BF16 && p.dtype != LSH_F16) return cudaErrorInvalidValue;
  Args a{};
  a.p = p;
  a.pl = pl;
  const int R = tile_rows(pl);
  const int64_t ntiles = (p.n + R - 1) / R;
  if (ntiles > INT32_MAX) return cudaErrorInvalidValue;
  a.ntiles = int(ntiles);
  const int64_t cap = int64_t(num_sms()) / pl.G;
  int64_t slots = cap < ntiles ? cap : ntiles;
  if (slots < 1) slots = 1;
  a.slots = int(slots);
  const int es = p.dtype == LSH_F32 ? 4 : 2;
  a.vec = (reinterpret_cast<uintptr_t>(p.X) % 16 == 0) && ((p.ld * es) % 16 == 0) ? 1 : 0;
  a.sqrtm_f = float(p.sqrtm);
  a.invw_f = float(1.0 / p.w);
  const bool srp = kind_is_srp(p.kind);
  const bool full = p.codes || p.bits || p.proj || p.counters;
  return srp ? launch_srp(a, full, stream) : launch_e2lsh(a, full, stream);
}

// Autotuner: the first batch of at least kTuneRows rows of a shape (device,
// kind, d, m, L, modes, dtype) times every candidate plan (three launches
// after a warm-up) on its first kTuneRows rows and on half as many -- keys
// only, no recheck queue, into the caller's key buffer, which the real
// launch then overwrites -- and keeps the plan whose fixed cost plus cost
// per row predicts the least time for the batch; later batches of the shape
// with at least two of its tiles per SM use it too.  The timing is skipped
// while the stream is being captured (the default plan is used).  Every plan
// computes the same codes, and a plan fits any row count.
constexpr int64_t kTuneRows = 524288;

struct TuneKey {
  int dev, kind, d, m, L, N, dtype, cap;
  int dims[LSH_MAX_MODES], mdims[LSH_MAX_MODES];
  bool operator<(const TuneKey &o) const { return std::memcmp(this, &o, sizeof(TuneKey)) < 0; }
};
std::mutex g_tune_mu;
std::map<TuneKey, Plan> g_tuned;

Plan tuned_plan(const SketchLaunch &p, cudaStream_t stream, bool may_time = true) {
  const Plan dflt = make_plan(p.d, p.m, p.L, p.cap, p.n);
  if (dflt.smem <= 0) return dflt;
  TuneKey key;
  std::memset(&key, 0, sizeof(key));
  cudaGetDevice(&key.dev);
  key.kind = p.kind;
  key.d = p.d;
  key.m = p.m;
  key.L = p.L;
  key.N = p.N;
  key.dtype = p.dtype;
  key.cap = p.cap;
  for (int k = 0; k < p.N && k < LSH_MAX_MODES; ++k) {
    key.dims[k] = p.dims[k];
    key.mdims[k] = p.mdims[k];
  }
  {
    // a shape tuned before serves any batch that gives every SM two tiles of
    // the tuned plan (smaller ones keep the default, sized for them)
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      const int64_t tiles = (p.n + tile_rows(it->second) - 1) / tile_rows(it->second);
      return tiles >= 2 * int64_t(num_sms()) ? it->second : dflt;
    }
  }
  if (p.n < kTuneRows) return dflt;
  if (!may_time) return dflt;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return dflt;
  SketchLaunch q = p;
  q.n = kTuneRows;
  q.codes = nullptr;
  q.bits = nullptr;
  q.proj = nullptr;
  q.counters = nullptr;
  q.queue = nullptr;
  q.qcount = nullptr;
  q.qcap = 0;
  const std::vector<Plan> cands = plan_candidates(p.d, p.m, p.L, p.cap, kTuneRows);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return dflt;
  }
  // each candidate on kTuneRows and on half as many rows: the difference is
  // its cost per row, the rest a fixed cost (table staging, the last wave);
  // the plan with the least predicted time for the caller's row count wins
  auto timed = [&](const Plan &pl, int64_t rows, float &ms) {
    q.n = rows;
    cudaEventRecord(e0, stream);
    bool ok = true;
    for (int r = 0; r < 3 && ok; ++r) ok = launch_plan(q, pl, stream) == cudaSuccess;  // three: less noise
    cudaEventRecord(e1, stream);
    return ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  };
  Plan best = dflt;
  double best_pred = 1e300;
  for (const Plan &pl : cands) {
    q.n = kTuneRows;
    if (launch_plan(q, pl, stream) != cudaSuccess) continue;  // warm-up (and attribute setting)
    float full = 0.f, half = 0.f;
    if (!timed(pl, kTuneRows, full) || !timed(pl, kTuneRows / 2, half)) continue;
    const double per_row = std::max(0.0, double(full - half) / double(kTuneRows / 2));
    const double fixed = std::max(0.0, double(full) - per_row * double(kTuneRows));
    const double pred = fixed + per_row * double(p.n);
    if (pred < best_pred) {
      best_pred = pred;
      best = pl;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();  // a candidate that failed to launch leaves no sticky error
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[key] = best;
  return best;
}

std::mutex g_pin_mu;
SketchPin g_pin{0, 0, 0, 0, 0, 0};

bool pinned(SketchPin &pin) {
  std::lock_guard<std::mutex> lock(g_pin_mu);
  pin = g_pin;
  return pin.rows_per_lane != 0;
}

Plan pinned_plan(const SketchPin &pin, int d, int m, int L, int cap) {
  if (pin.entry_bytes == 2 && !entry16_ok(d, pin.rows_per_lane)) {
    Plan bad{};
    bad.smem = -1;
    return bad;
  }
  return plan_of(d, m, L, cap, pin.rows_per_lane, pin.row_groups, pin.warps_per_table,
                 std::min(pin.tables_per_cta, L), pin.entry_bytes, pin.split_bins);
}

}  // namespace

void set_sketch_pin(const SketchPin &pin) {
  std::lock_guard<std::mutex> lock(g_pin_mu);
  g_pin = pin;
}

bool sketch_pin_fits(int d, int m, int L, int cap) {
  SketchPin pin;
  if (!pinned(pin)) return true;
  const Plan pl = pinned_plan(pin, d, m, L, cap);
  return pl.smem > 0 && pl.smem <= kMaxSmem;
}

void sketch_autotune(const SketchLaunch &p, cudaStream_t stream) {
  SketchPin pin;
  if (p.n <= 0 || pinned(pin)) return;
  (void)tuned_plan(p, stream);
}

bool sketch_current_plan(const SketchLaunch &p, SketchPin &out) {
  SketchPin pin;
  const Plan pl = pinned(pin) ? pinned_plan(pin, p.d, p.m, p.L, p.cap) : tuned_plan(p, nullptr, false);
  if (pl.smem <= 0 || pl.smem > kMaxSmem) return false;
  out = SketchPin{pl.RPL, pl.RG, pl.WPT, pl.Lg, pl.es, pl.hw};
  return true;
}

cudaError_t launch_sketch_dense(const SketchLaunch &p, cudaStream_t stream) {
  if (p.n <= 0) return cudaSuccess;
  SketchPin pin;
  const Plan pl = pinned(pin) ? pinned_plan(pin, p.d, p.m, p.L, p.cap) : tuned_plan(p, stream);
  if (pl.smem <= 0 || pl.smem > kMaxSmem) return cudaErrorInvalidConfiguration;
  return launch_plan(p, pl, stream);
}

}  // namespace lsh
