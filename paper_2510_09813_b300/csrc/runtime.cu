// Host runtime and C ABI of the B300 state-vector Rydberg library (include/rsv.h).
//
//   - device memory arena with an admission cap (footprint accounting as in
//     arXiv 2510.09813 Sec. III.A.1),
//   - host preparation: FP64 pair energies (Eq. (3)), midpoint pulse
//     parameters (Sec. III), bit-position tables for the kernels,
//   - the Lanczos time-step driver (Sec. III.A, Eq. (6)) over the streaming
//     tile kernels and the device-side Krylov control kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <future>
#include <thread>
#include <tuple>
#include <deque>
#include <condition_variable>
#include <memory>
#include <set>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rsv.h"
#include "kernels.h"
#include "rsv_common.cuh"

using namespace rsv;

namespace {

thread_local std::string g_last_error;

rsv_status fail(rsv_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define RSV_CUDA(call)                                                                                  \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return fail(RSV_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define RSV_TRY(expr)                \
  do {                               \
    rsv_status s_ = (expr);          \
    if (s_ != RSV_OK) return s_;     \
  } while (0)

constexpr int kTileBitsC64 = kTileBitsF;
constexpr int kTileBitsC128 = kTileBitsD;
constexpr int kMinSegmentBits = 4;   // contiguous amplitude bits of the strided pass
constexpr int kMaxSingleGBits = 2;   // bits above the tile resolved in the single pass
constexpr int kMaxGBits = 12;        // partner bits through L2 a pass can take
constexpr int kFirstPassGBits = 0;   // two-pass: partner bits the contiguous pass takes (first_pass_gbits)

int64_t amp_bytes(int precision) { return precision == RSV_C64 ? 8 : 16; }

int* err_ptr(KState* ks) { return reinterpret_cast<int*>(reinterpret_cast<char*>(ks) + offsetof(KState, error)); }

// ---------------------------------------------------------------------------
// Device arena: first-fit free list with coalescing over one allocation, or
// plain cudaMalloc with byte accounting when no cap is given.
// ---------------------------------------------------------------------------
class Arena {
 public:
  rsv_status init(size_t cap) {
    cap_ = cap;
    if (cap_ > 0) {
      cudaError_t e = cudaMalloc(&base_, cap_);
      if (e != cudaSuccess) return fail(RSV_ERR_OUT_OF_MEMORY, std::string("arena cudaMalloc: ") + cudaGetErrorString(e));
      free_[0] = cap_;
    }
    return RSV_OK;
  }
  ~Arena() {
    if (base_) cudaFree(base_);
    for (auto& kv : direct_) cudaFree(kv.first);
  }
  rsv_status alloc(size_t bytes, void** out) {
    std::lock_guard<std::mutex> lk(mu_);
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    if (cap_ == 0) {
      void* p = nullptr;
      cudaError_t e = cudaMalloc(&p, bytes);
      if (e != cudaSuccess) return fail(RSV_ERR_OUT_OF_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
      direct_[p] = bytes;
      used_ += bytes;
      *out = p;
      return RSV_OK;
    }
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, sz = it->second;
        free_.erase(it);
        if (sz > bytes) free_[off + bytes] = sz - bytes;
        used_map_[off] = bytes;
        used_ += bytes;
        *out = static_cast<char*>(base_) + off;
        return RSV_OK;
      }
    }
    return fail(RSV_ERR_OUT_OF_MEMORY, "arena exhausted: " + std::to_string(bytes) + " bytes requested, " +
                                           std::to_string(cap_ - used_) + " free (fragmented or full)");
  }
  void release(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    if (cap_ == 0) {
      auto it = direct_.find(p);
      if (it != direct_.end()) {
        used_ -= it->second;
        cudaFree(p);
        direct_.erase(it);
      }
      return;
    }
    const size_t off = static_cast<char*>(p) - static_cast<char*>(base_);
    auto it = used_map_.find(off);
    if (it == used_map_.end()) return;
    size_t sz = it->second;
    used_ -= sz;
    used_map_.erase(it);
    size_t start = off;
    auto nx = free_.lower_bound(off);
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {
        start = pv->first;
        sz += pv->second;
        free_.erase(pv);
      }
    }
    nx = free_.lower_bound(start);
    if (nx != free_.end() && start + sz == nx->first) {
      sz += nx->second;
      free_.erase(nx);
    }
    free_[start] = sz;
  }
  size_t used() const { return used_; }
  size_t cap() const { return cap_; }

 private:
  std::mutex mu_;
  void* base_ = nullptr;
  size_t cap_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;      // offset -> size
  std::map<size_t, size_t> used_map_;  // offset -> size
  std::map<void*, size_t> direct_;
};

}  // namespace

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct rsv_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  Arena arena;
  // scratch for operator-level calls
  StepParams* d_sp = nullptr;
  double* d_vmat = nullptr;
  void* d_qtab = nullptr;
  KState* d_ks = nullptr;
  double* d_part = nullptr;  // partial sums (large enough for any grid)
  double* d_occ = nullptr;
  KState* h_ks = nullptr;    // pinned
  std::mutex mu;
  // open objects, freed by rsv_destroy if the caller did not free them first
  std::set<rsv_solver*> solvers;
  std::set<rsv_result*> results;
  std::set<rsv_batch*> batches;
  std::set<rsv_server*> servers;
  std::set<rsv_hamiltonian*> hamiltonians;
  // autotuned contiguous-segment bits of the strided pass, per (n_atoms, complex64)
  std::map<std::pair<int, int>, int> tuned_segment;
};

namespace {

size_t partials_doubles(int num_sms) { return (size_t)std::max(4 * num_sms, 2048) * (kMaxAtoms + 1); }

struct Plan {
  TileArgs a{}, b{};   // geometry of the passes
  bool two_pass = false;
  int grid_a = 1, grid_b = 1;
  int grid_c = 1;      // combine/observe grid
  int L_a = 0;         // tile bits of the first pass (Q table size)
};

// L2 partner bits of a two-pass matvec taken by the contiguous first pass
// (amplitude bits [L, L + g)) instead of the strided second pass, whose L2
// traffic (8 bytes per amplitude per partner bit) is what bounds it.
int first_pass_gbits() {
  const char* e = std::getenv("RSV_FIRST_GBITS");
  if (!e) return kFirstPassGBits;
  const int v = std::atoi(e);
  return (v >= 0 && v <= 4) ? v : kFirstPassGBits;
}

// Strided-pass shape: segment bits c, tile-order bits f1_fast and the tile
// kind (x-only 64 KiB tiles, or 32 KiB x and z tiles), packed into one int.
constexpr int kShapeXOnly = 256;
int pack_shape(int seg, int f1f, bool x_only) { return seg * 16 + f1f + (x_only ? kShapeXOnly : 0); }
int shape_seg(int shape) { return (shape & 255) / 16; }
int shape_f1(int shape) { return shape % 16; }
bool shape_x_only(int shape) { return (shape & kShapeXOnly) != 0; }

Plan make_plan(int n, bool c64, int num_sms, int seg_bits = kMinSegmentBits, int f1_fast = 0, bool x_only = false) {
  Plan p;
  const int lt = c64 ? kTileBitsC64 : kTileBitsC128;
  const int lx = c64 ? kStridedTileBitsF : kStridedTileBitsD;
  const int v = c64 ? 1 : 0;
  auto geom = [&](TileArgs& t, int L, int c, int a, int nG) {
    t.n = n;
    t.L = L;
    t.c = c;
    t.a = a;
    t.f2 = a + (L - c);
    t.nF2 = n - t.f2;
    t.nG = nG;
    t.kt = std::min(9, L - v);
    t.num_tiles = int64_t(1) << (n - L);
  };
  if (n <= lt) {
    geom(p.a, n, n, n, 0);
  } else if (n - lt <= kMaxSingleGBits) {
    geom(p.a, lt, lt, lt, n - lt);
  } else {
    const int ga = std::min(first_pass_gbits(), n - lt - 1);
    geom(p.a, lt, lt, lt, ga);
    if (x_only && n - lt - ga >= lx - seg_bits) {
      // x-only 64 KiB tiles: all lx - c strided bits fit above the first pass's
      geom(p.b, lx, seg_bits, lt + ga, 0);
    } else {
      const int h = std::min(n - lt - ga, lt - seg_bits);
      const int c = lt - h;
      geom(p.b, lt, c, lt + ga, 0);
    }
    p.b.split_h = (p.b.L - p.b.c) > 8;
    p.b.f1_fast = std::min(f1_fast, p.b.a - p.b.c);
    p.b.nG = p.b.nF2;  // callers check nG <= kMaxGBits
    p.two_pass = true;
  }
  p.L_a = p.a.L;
  const int resident = num_sms;  // persistent: one CTA per SM
  p.grid_a = (int)std::min<int64_t>(p.a.num_tiles, resident);
  p.grid_b = p.two_pass ? (int)std::min<int64_t>(p.b.num_tiles, resident) : 0;
  const int T = std::min(n, v + 8 + 4);
  const int64_t chunks = int64_t(1) << (n - T);
  p.grid_c = (int)std::min<int64_t>(chunks, 4 * num_sms);
  return p;
}

// Q[t] = sum_{q<r<L} V_qr t_q t_r over tile-local bit patterns t (bit positions).
template <typename Real>
std::vector<Real> q_table(const std::vector<double>& vbit, int L) {
  std::vector<double> q(size_t(1) << L, 0.0);
  for (size_t t = 1; t < q.size(); ++t) {
    int top = 63 - __builtin_clzll((unsigned long long)t);
    const size_t rest = t ^ (size_t(1) << top);
    double s = q[rest];
    for (int r = 0; r < top; ++r)
      if ((rest >> r) & 1) s += vbit[top * kMaxAtoms + r];
    q[t] = s;
  }
  return std::vector<Real>(q.begin(), q.end());
}

// Pair energies by atom (Eq. (3)).
rsv_status pair_energies(int n, int dim, const double* pos, double c6, std::vector<double>& v) {
  v.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      double d2 = 0.0;
      for (int k = 0; k < dim; ++k) {
        const double d = pos[i * dim + k] - pos[j * dim + k];
        d2 += d * d;
      }
      if (d2 == 0.0)
        return fail(RSV_ERR_COINCIDENT_ATOMS, "atoms " + std::to_string(i) + " and " + std::to_string(j) + " coincide");
      v[(size_t)i * n + j] = c6 / (d2 * d2 * d2);
    }
  return RSV_OK;
}

// Atom-ordered [n][n] -> bit-position [kMaxAtoms][kMaxAtoms].
std::vector<double> to_bit_matrix(int n, const double* v_atoms) {
  std::vector<double> vb((size_t)kMaxAtoms * kMaxAtoms, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) vb[(size_t)(n - 1 - i) * kMaxAtoms + (n - 1 - j)] = v_atoms[(size_t)i * n + j];
  return vb;
}

int num_steps(int t_ns, int dt_ns) { return (t_ns + dt_ns - 1) / dt_ns; }

double midpoint(const double* row, int t_ns, int start, int len) {
  const int twice_m = 2 * start + len;
  const int lo = std::min(twice_m / 2, t_ns - 1);
  const int hi = std::min((twice_m + 1) / 2, t_ns - 1);
  return 0.5 * (row[lo] + row[hi]);
}

rsv_status validate_problem(const rsv_problem* p) {
  if (!p) return fail(RSV_ERR_INVALID_ARG, "problem is NULL");
  if (p->n_atoms < 1 || p->n_atoms > 31) return fail(RSV_ERR_INVALID_ARG, "n_atoms out of range");
  if (p->dim != 2 && p->dim != 3) return fail(RSV_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (!p->positions_um) return fail(RSV_ERR_INVALID_ARG, "positions_um is NULL");
  if (p->t_ns < 1) return fail(RSV_ERR_INVALID_ARG, "t_ns must be >= 1");
  auto rows_ok = [&](int r, bool allow0) { return r == 1 || r == p->n_atoms || (allow0 && r == 0); };
  if (!p->omega || !rows_ok(p->omega_rows, false)) return fail(RSV_ERR_INVALID_ARG, "omega rows must be 1 or n_atoms");
  if (!p->delta || !rows_ok(p->delta_rows, false)) return fail(RSV_ERR_INVALID_ARG, "delta rows must be 1 or n_atoms");
  if (!rows_ok(p->phi_rows, true) || (p->phi_rows > 0 && !p->phi))
    return fail(RSV_ERR_INVALID_ARG, "phi rows must be 0, 1 or n_atoms (phi non-NULL when rows > 0)");
  return RSV_OK;
}

// Per-step StepParams (bit positions) and step lengths.
rsv_status step_params(const rsv_problem* p, int dt_ns, std::vector<StepParams>& out) {
  const int n = p->n_atoms, K = num_steps(p->t_ns, dt_ns);
  out.assign(K, StepParams{});
  int start = 0;
  for (int k = 0; k < K; ++k) {
    const int len = std::min(dt_ns, p->t_ns - start);
    StepParams& s = out[k];
    std::memset(&s, 0, sizeof(s));
    s.tau = len / 1000.0;
    s.has_phi = p->phi_rows > 0;
    for (int i = 0; i < n; ++i) {
      const int q = n - 1 - i;
      const double* orow = p->omega + (size_t)(p->omega_rows == 1 ? 0 : i) * p->t_ns;
      const double* drow = p->delta + (size_t)(p->delta_rows == 1 ? 0 : i) * p->t_ns;
      s.half_omega[q] = 0.5 * midpoint(orow, p->t_ns, start, len);
      s.delta[q] = midpoint(drow, p->t_ns, start, len);
      if (p->phi_rows > 0) {
        const double* prow = p->phi + (size_t)(p->phi_rows == 1 ? 0 : i) * p->t_ns;
        s.phi[q] = midpoint(prow, p->t_ns, start, len);
      }
    }
    start += len;
  }
  return RSV_OK;
}

// Device bytes a solver of this problem holds: rsv_footprint_bytes plus what
// depends on the sequence (per-step parameters, recorded occupation rows).
size_t solver_bytes(const rsv_problem* p, const rsv_config& cfg) {
  const size_t steps = (size_t)num_steps(p->t_ns, cfg.dt_ns);
  const size_t rows = (cfg.obs_stride > 0 ? steps / cfg.obs_stride : 0) + 2;
  auto round = [](size_t b) { return (b + 255) & ~size_t(255); };
  return rsv_footprint_bytes(p->n_atoms, cfg.precision, cfg.m_max) + round(sizeof(StepParams) * steps) +
         round(sizeof(double) * p->n_atoms * rows);
}

bool any_phi(const std::vector<StepParams>& sp, int n) {
  for (const auto& s : sp)
    for (int q = 0; q < n; ++q)
      if (s.phi[q] != 0.0) return true;
  return false;
}

// Strided-pass shape autotuner. The contiguous segment of the strided tile
// (2^c amplitudes) trades DRAM segment length against partner bits read through
// L2, and the tile order (f1_fast segment-index bits varied fastest) trades DRAM
// row locality against the L2 reuse distance of those partners. Candidates
// c in {4, 5} x f1_fast in {0, 2, 4} are timed on the caller's buffers (the pass
// only reads x and read-modify-writes z, whose contents do not matter here) and
// the fastest is cached per (n_atoms, precision). RSV_SEGMENT_BITS fixes c,
// and with it RSV_TILE_ORDER_BITS fixes f1_fast (default 0): a plan override
// that skips the tuner (tests force every candidate shape this way).
int segment_override() {
  const char* e = std::getenv("RSV_SEGMENT_BITS");
  if (!e) return 0;
  const int v = std::atoi(e);
  return (v >= 2 && v <= 8) ? v : 0;
}

int tile_order_override() {
  const char* e = std::getenv("RSV_TILE_ORDER_BITS");
  if (!e) return 0;
  const int v = std::atoi(e);
  return (v >= 0 && v <= 8) ? v : 0;
}

int x_only_override() {
  const char* e = std::getenv("RSV_STRIDED_X_ONLY");
  return e ? (std::atoi(e) != 0) : 0;
}

Plan plan_for(int n, bool c64, int num_sms, int shape) {
  return make_plan(n, c64, num_sms, shape_seg(shape), shape_f1(shape), shape_x_only(shape));
}

// A strided-pass shape the kernels accept for this register (an x-only shape
// must get its 64 KiB tile: make_plan falls back to the staged-z tile when
// the register has too few high bits).
bool shape_valid(int n, bool c64, int num_sms, int shape) {
  const Plan p = plan_for(n, c64, num_sms, shape);
  if (!p.two_pass) return true;
  const int lx = c64 ? kStridedTileBitsF : kStridedTileBitsD;
  if (shape_x_only(shape) && p.b.L != lx) return false;
  return p.b.nG <= kMaxGBits && p.b.c >= (c64 ? 1 : 0);
}

// The overridden shape, or 0 when none is set or the one set does not fit
// this register. RSV_STRIDED_X_ONLY=1 selects the x-only tiles.
int shape_override(int n, bool c64, int num_sms) {
  const int o = segment_override();
  if (!o) return 0;
  const int shape = pack_shape(o, tile_order_override(), x_only_override());
  return shape_valid(n, c64, num_sms, shape) ? shape : 0;
}

// Tuned shape (pack_shape) of this register size and precision.
// Tuned shapes are a property of the device and the register size, not of a
// context: every context of the process on the same device shares them, so a
// new context does not time the candidates again.
std::mutex g_tuned_mu;
std::map<std::tuple<int, int, int>, int> g_tuned;  // (device, n_atoms, complex64) -> shape

bool tuned_lookup(rsv_ctx* ctx, int n, bool c64, int* shape) {
  const auto key = std::make_pair(n, c64 ? 1 : 0);
  auto it = ctx->tuned_segment.find(key);
  if (it != ctx->tuned_segment.end()) {
    *shape = it->second;
    return true;
  }
  std::lock_guard<std::mutex> lk(g_tuned_mu);
  auto g = g_tuned.find(std::make_tuple(ctx->device, n, c64 ? 1 : 0));
  if (g == g_tuned.end()) return false;
  ctx->tuned_segment[key] = *shape = g->second;
  return true;
}

int shape_for(rsv_ctx* ctx, int n, bool c64) {
  if (const int o = shape_override(n, c64, ctx->num_sms)) return o;
  int shape = 0;
  return tuned_lookup(ctx, n, c64, &shape) ? shape : pack_shape(kMinSegmentBits, 0, false);
}

// Candidates the tuner times: staged-z tiles with c in {4, 5} x f1_fast in
// {0, 2, 4}, and x-only tiles with c in {2, 3, 4, 5}, each with tile orders
// that put the 256-byte run of its segments (and one step beyond) side by side.
std::vector<int> tune_candidates() {
  std::vector<int> out;
  for (int seg : {4, 5})
    for (int f1f : {0, 2, 4}) out.push_back(pack_shape(seg, f1f, false));
  for (int seg : {2, 3, 4, 5}) {
    const int run = std::max(0, 5 - seg);  // segments per 256 bytes of complex64
    for (int f1f : {0, run, run + 1}) {
      const int sh = pack_shape(seg, f1f, true);
      if (std::find(out.begin(), out.end(), sh) == out.end()) out.push_back(sh);
    }
  }
  return out;
}

int tune_shape(rsv_ctx* ctx, cudaStream_t stream, int n, bool c64, StepParams* sp, double* vmat, KState* ks, double* part, void* x,
               void* z) {
  if (const int o = shape_override(n, c64, ctx->num_sms)) return o;
  const auto key = std::make_pair(n, c64 ? 1 : 0);
  int known = 0;
  if (tuned_lookup(ctx, n, c64, &known)) return known;
  int best = pack_shape(kMinSegmentBits, 0, false);
  float best_ms = 1e30f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int shape : tune_candidates()) {
    if (!shape_valid(n, c64, ctx->num_sms, shape)) continue;
    const Plan p = plan_for(n, c64, ctx->num_sms, shape);
    if (!p.two_pass) continue;
    TileArgs b = p.b;
    b.sp = sp;
    b.vmat = vmat;
    b.ks = ks;
    b.partials = part;
    b.err = err_ptr(ks);
    b.xin = x;
    b.out = z;
    TileMaps maps;
    if (!encode_tile_map(&maps.x, x, p.b, c64) || !encode_tile_map(&maps.z, z, p.b, c64)) continue;
    bool ok = launch_tile(b, &maps, TileMode::kMatvecSecond, c64, false, p.grid_b, stream) == cudaSuccess;
    cudaEventRecord(e0, stream);
    for (int r = 0; r < 3 && ok; ++r)
      ok = launch_tile(b, &maps, TileMode::kMatvecSecond, c64, false, p.grid_b, stream) == cudaSuccess;
    cudaEventRecord(e1, stream);
    if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = shape;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaMemsetAsync(err_ptr(ks), 0, sizeof(int), stream);
  ctx->tuned_segment[key] = best;
  std::lock_guard<std::mutex> lk(g_tuned_mu);
  g_tuned[std::make_tuple(ctx->device, n, c64 ? 1 : 0)] = best;
  return best;
}

// Launch one streaming pass.
rsv_status run_pass(rsv_ctx* ctx, TileArgs args, const TileMaps* maps, TileMode mode, bool c64, bool phi, int grid) {
  cudaError_t e = launch_tile(args, maps, mode, c64, phi, grid, ctx->stream);
  if (e != cudaSuccess) return fail(RSV_ERR_CUDA, std::string("tile kernel launch: ") + cudaGetErrorString(e));
  return RSV_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Solver
// ---------------------------------------------------------------------------
struct rsv_solver {
  rsv_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;  // the context stream, or a served request's own stream
  bool own_stream = false;        // destroy `stream` with the solver
  int n = 0;
  int precision = RSV_C128;
  bool c64 = false;
  bool phi = false;
  int64_t dim = 0;
  rsv_config cfg{};
  Plan plan;
  int nsteps = 0, done = 0;
  std::vector<StepParams> h_sp;
  // device buffers
  StepParams* d_sp = nullptr;
  double* d_vmat = nullptr;
  void* d_qtab = nullptr;
  void* d_diag = nullptr;    // per-tile diagonal half tables of the current step
  void* d_phase = nullptr;   // laser-phase gauge tables of the current step (two-pass plans with phi)
  int phase_bits = 0;        // their split bit L
  bool phi_now = false;      // the passes of the running step use complex flip coefficients
  void* d_psi = nullptr;
  void* d_u[2] = {nullptr, nullptr};
  std::vector<void*> basis;
  void** d_basis = nullptr;
  std::vector<CUtensorMap> map_basis;  // strided-pass tensor maps over basis[j]
  CUtensorMap map_u[2];                // ... over the two work vectors
  KState* d_ks = nullptr;
  ChebWork* d_cheb = nullptr;  // the control step's kept Chebyshev expansion
  bool fused_control = true;  // the control step runs in the last pass (not RSV_FLAG_CONTROL_LAUNCH)
  double* d_part = nullptr;
  double* d_cpart = nullptr;
  double* d_occ = nullptr;   // [max_rows][n]
  int max_rows = 0, rows = 0;
  KState* h_ks = nullptr;    // pinned status mirror
  int last_m = 0;
  rsv_stats stats{};
  std::vector<void*> owned;  // arena allocations
  // live per-launch timing (rsv_solver_set_profiling)
  bool profiling = false;
  rsv_kernel_times ktimes{};
  struct Pending {
    int kind;
    double bytes;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  std::vector<char> init_host;  // caller's initial state (empty: |0...0>)

  // State <- initial state, step counter and recorded rows <- 0, row 0 recorded.
  // `direct`: the caller's initial state, copied straight to the device (a
  // one-shot solver, which never rewinds and so keeps no host copy).
  rsv_status reset_to_initial(const void* direct = nullptr) {
    const size_t vbytes = (size_t)dim * amp_bytes(precision);
    if (direct) {
      RSV_CUDA(cudaMemcpyAsync(d_psi, direct, vbytes, cudaMemcpyHostToDevice, stream));
    } else if (!init_host.empty()) {
      RSV_CUDA(cudaMemcpyAsync(d_psi, init_host.data(), vbytes, cudaMemcpyHostToDevice, stream));
    } else {
      RSV_CUDA(cudaMemsetAsync(d_psi, 0, vbytes, stream));
      const double one_d[2] = {1.0, 0.0};
      const float one_f[2] = {1.f, 0.f};
      RSV_CUDA(cudaMemcpyAsync(d_psi, c64 ? (const void*)one_f : (const void*)one_d, c64 ? sizeof(one_f) : sizeof(one_d),
                               cudaMemcpyHostToDevice, stream));
    }
    std::vector<char> zero_ks(sizeof(KState), 0);
    RSV_CUDA(cudaMemcpyAsync(d_ks, zero_ks.data(), sizeof(KState), cudaMemcpyHostToDevice, stream));
    RSV_CUDA(cudaMemsetAsync(d_cheb, 0, cheb_cache_bytes(), stream));
    for (auto& v : ctl_seen) v = 0;
    done = 0;
    rows = 0;
    last_m = 0;
    RSV_TRY(observe_into_partials());
    RSV_TRY(record_row());
    RSV_CUDA(cudaStreamSynchronize(stream));
    return RSV_OK;
  }

  rsv_status alloc(size_t bytes, void** out) {
    RSV_TRY(ctx->arena.alloc(bytes, out));
    owned.push_back(*out);
    return RSV_OK;
  }
  // Arena bytes of the state allocation (the arena rounds to 256 bytes).
  size_t state_alloc_bytes() const { return ((size_t)dim * amp_bytes(precision) + 255) & ~size_t(255); }
  // A finished solve kept only for its final state: returns every other
  // device allocation to the arena. The solver can no longer step.
  bool trimmed = false;
  void trim_to_state() {
    cudaStreamSynchronize(stream);
    for (void* p : owned)
      if (p != d_psi) ctx->arena.release(p);
    owned.assign(1, d_psi);
    d_sp = nullptr;
    d_vmat = nullptr;
    d_qtab = nullptr;
    d_diag = nullptr;
    d_phase = nullptr;
    d_u[0] = d_u[1] = nullptr;
    basis.clear();
    d_basis = nullptr;
    d_ks = nullptr;
    d_cheb = nullptr;
    d_part = nullptr;
    d_cpart = nullptr;
    d_occ = nullptr;
    trimmed = true;
  }
  ~rsv_solver() {
    if (ctx) cudaStreamSynchronize(stream);
    for (auto& p : pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : event_pool) cudaEventDestroy(e);
    for (void* p : owned) ctx->arena.release(p);
    if (h_ks) cudaFreeHost(h_ks);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }

  cudaEvent_t take_event() {
    if (!event_pool.empty()) {
      cudaEvent_t e = event_pool.back();
      event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }

  // Launches through `fn` (returning cudaError_t); with profiling on, brackets
  // the launch with events on the context stream.
  template <typename F>
  rsv_status launch(int kind, double bytes, F&& fn) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (profiling) {
      a = take_event();
      b = take_event();
      RSV_CUDA(cudaEventRecord(a, stream));
    }
    cudaError_t e = fn();
    if (e != cudaSuccess) return fail(RSV_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    stats.kernel_launches += 1;
    if (profiling) {
      RSV_CUDA(cudaEventRecord(b, stream));
      pending.push_back({kind, bytes, a, b});
    }
    return RSV_OK;
  }

  // Folds completed launch timings into ktimes (call after a stream sync).
  void drain_timings() {
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        ktimes.ms[p.kind] += ms;
        ktimes.launches[p.kind] += 1;
        ktimes.bytes[p.kind] += p.bytes;
      }
      event_pool.push_back(p.a);
      event_pool.push_back(p.b);
    }
    pending.clear();
  }

  rsv_status read_status() {
    RSV_CUDA(cudaMemcpyAsync(h_ks, d_ks, kStatusBytes, cudaMemcpyDeviceToHost, stream));
    RSV_CUDA(cudaStreamSynchronize(stream));
    if (profiling) {
      drain_timings();
      account_control();
    }
    return RSV_OK;
  }

  // The device's control-step counters (KState, zeroed with the state) as
  // last read, and what profiling has added up from them.
  uint64_t ctl_seen[4] = {0, 0, 0, 0};
  uint64_t ctl_acc[4] = {0, 0, 0, 0};
  void account_control() {
    const uint64_t cur[4] = {h_ks->ctl_ns, h_ks->ctl_steps, h_ks->chk_ns, h_ks->chk_steps};
    for (int i = 0; i < 4; ++i) {
      ctl_acc[i] += cur[i] >= ctl_seen[i] ? cur[i] - ctl_seen[i] : cur[i];  // zeroed by a rewind
      ctl_seen[i] = cur[i];
    }
  }

  double vec_bytes() const { return (double)dim * (double)amp_bytes(precision); }

  rsv_status combine(int combine_flag, int m) {
    CombineArgs ca{};
    ca.n = n;
    ca.dim = dim;
    ca.basis = (const void* const*)d_basis;
    ca.ks = d_ks;
    ca.psi = d_psi;
    ca.partials = d_cpart;
    ca.combine = combine_flag;
    ca.err = err_ptr(d_ks);
    const double bytes = combine_flag ? vec_bytes() * (m + 1) : vec_bytes();
    return launch(RSV_KERNEL_COMBINE, bytes, [&] { return launch_combine(ca, c64, plan.grid_c, stream); });
  }

  rsv_status observe_into_partials() { return combine(0, 0); }

  rsv_status begin(double new_tau, int reset_only, double* occ_row) {
    BeginArgs ba{};
    ba.ks = d_ks;
    ba.partials = d_cpart;
    ba.nparts = plan.grid_c;
    ba.n = n;
    ba.new_tau = new_tau;
    ba.occ_out = occ_row;
    ba.reset_only = reset_only;
    return launch(RSV_KERNEL_SETUP, 0.0, [&] { return launch_begin(ba, stream); });
  }

  rsv_status record_row() {
    if (rows >= max_rows) return RSV_OK;
    RSV_TRY(begin(0.0, 1, d_occ + (size_t)rows * n));
    ++rows;
    return RSV_OK;
  }

  TileArgs base_args(const TileArgs& g, int step) const {
    TileArgs a = g;
    a.sp = d_sp + step;
    a.vmat = d_vmat;
    a.qtab = d_qtab;
    a.ks = d_ks;
    a.partials = d_part;
    a.err = err_ptr(d_ks);
    a.diag = d_diag;
    return a;
  }

  // Algorithmic bytes: first pass reads u_{j-1} (and v_{j-1} for j > 0) and
  // writes v_j and its output; the second pass reads v_j and the first pass's
  // output and writes u_j.
  // ctl: the control step to fuse into the iteration's last pass (nullptr: a
  // separate scalar launch follows).
  rsv_status iteration(int j, int step, const ScalarArgs* ctl) {
    void* u_in = j == 0 ? d_psi : d_u[(j - 1) & 1];
    void* u_out = d_u[j & 1];
    TileArgs a = base_args(plan.a, step);
    a.xin = u_in;
    a.xprev = j > 0 ? basis[j - 1] : nullptr;
    a.xout = basis[j];
    a.out = u_out;
    const double first_bytes = vec_bytes() * (j > 0 ? 4 : 3);
    if (!plan.two_pass) {
      if (ctl) a.ctl = *ctl;
      RSV_TRY(launch(RSV_KERNEL_PASS_FIRST, first_bytes,
                     [&] { return launch_tile(a, nullptr, TileMode::kLanczosSingle, c64, phi_now, plan.grid_a, stream); }));
    } else {
      RSV_TRY(launch(RSV_KERNEL_PASS_FIRST, first_bytes,
                     [&] { return launch_tile(a, nullptr, TileMode::kLanczosFirst, c64, phi_now, plan.grid_a, stream); }));
      TileArgs b = base_args(plan.b, step);
      b.xin = basis[j];
      b.out = u_out;
      if (ctl) b.ctl = *ctl;
      RSV_TRY(launch(RSV_KERNEL_PASS_SECOND, vec_bytes() * 3,
                     [&] {
                       TileMaps maps{map_basis[j], map_u[j & 1]};
                       return launch_tile(b, &maps, TileMode::kLanczosSecond, c64, phi_now, plan.grid_b, stream);
                     }));
    }
    return RSV_OK;
  }

  // d_psi <- exp(-i tau H_k) d_psi under the parameters of step k (tau > 0,
  // in us; Krylov restarts as needed). d_cpart must hold the observation
  // partials of d_psi (left by the previous combine or observation).
  rsv_status evolve(int k, double tau) {
    RSV_TRY(begin(tau, 0, nullptr));
    RSV_TRY(launch(RSV_KERNEL_SETUP, 0.0, [&] {
      return launch_diag_table(d_sp + k, d_vmat, n, plan.a.L, plan.a.num_tiles, d_diag, c64, stream);
    }));
    // A step with a laser phase on the two-pass plan runs in the gauge frame:
    // exp(-i tau H(phi)) = U exp(-i tau H(0)) U^dagger with the diagonal
    // U = exp(-i sum_q phi_q n_q), so the passes keep real flip coefficients.
    // Norm and occupations are the same in both frames.
    const bool gauge = d_phase && step_has_phi(k);
    phi_now = phi && !gauge;
    const int phase_grid = ctx->num_sms * 8;
    if (gauge) {
      RSV_TRY(launch(RSV_KERNEL_SETUP, 0.0, [&] {
        return launch_phase_table(d_sp + k, n, phase_bits, d_phase, c64, stream);
      }));
      RSV_TRY(launch(RSV_KERNEL_SETUP, 2.0 * vec_bytes(), [&] {
        return launch_phase_apply(d_psi, n, phase_bits, d_phase, false, c64, phase_grid, stream);
      }));
    }
    const int m_max = cfg.m_max;
    int restarts = 0;
    while (true) {
      const int check_from = std::max(1, last_m - 2);
      ScalarArgs sa{};
      sa.ks = d_ks;
      sa.cache = d_cheb;
      sa.partials = d_part;
      sa.nparts = plan.two_pass ? plan.grid_b : plan.grid_a;
      sa.m_max = m_max;
      sa.check_from = check_from;
      sa.tol = cfg.krylov_tol;
      sa.breakdown = 1e-13;
      int j = 0;
      bool finished = false;
      for (; j < m_max; ++j) {
        if (fused_control) {
          RSV_TRY(iteration(j, k, &sa));
        } else {
          RSV_TRY(iteration(j, k, nullptr));
          RSV_TRY(launch(RSV_KERNEL_CONTROL, 0.0, [&] { return launch_scalar(sa, stream); }));
        }
        if (j + 1 >= check_from) {
          RSV_TRY(read_status());
          if (h_ks->error) return fail(RSV_ERR_TIMEOUT, "a device-side wait timed out (kernel aborted)");
          if (h_ks->status == kIdle) return fail(RSV_ERR_INVALID_ARG, "state has zero norm");
          if (h_ks->status != kContinue) {
            finished = true;
            break;
          }
        }
      }
      if (!finished) return fail(RSV_ERR_NOT_CONVERGED, "Krylov control did not finish (non-finite values?)");
      last_m = h_ks->m;
      stats.krylov_iterations += h_ks->m;
      stats.max_error_estimate = std::max(stats.max_error_estimate, h_ks->err_est);
      RSV_TRY(combine(1, h_ks->m));
      if (h_ks->tau_rem <= 0.0) break;
      if (++restarts > cfg.max_substeps)
        return fail(RSV_ERR_NOT_CONVERGED, "step " + std::to_string(k) + " needed more than max_substeps restarts");
      stats.substeps += 1;
      RSV_TRY(begin(0.0, 0, nullptr));
    }
    if (gauge) {
      RSV_TRY(launch(RSV_KERNEL_SETUP, 2.0 * vec_bytes(), [&] {
        return launch_phase_apply(d_psi, n, phase_bits, d_phase, true, c64, phase_grid, stream);
      }));
      stats.phase_gauge_steps += 1;
    }
    return RSV_OK;
  }

  bool step_has_phi(int k) const {
    for (int q = 0; q < n; ++q)
      if (h_sp[k].phi[q] != 0.0) return true;
    return false;
  }

  rsv_status step_once() {
    const int k = done;
    RSV_TRY(evolve(k, h_sp[k].tau));
    ++done;
    stats.steps += 1;
    const bool rec = (cfg.obs_stride > 0 && done % cfg.obs_stride == 0) || done == nsteps;
    if (rec) RSV_TRY(record_row());
    return RSV_OK;
  }
};

// ---------------------------------------------------------------------------
// Result
// ---------------------------------------------------------------------------
// Admission accounting of a server, shared with the results it hands out:
// bytes admitted and not yet released, guarded by `mu`, whose waiters (the
// server's workers) are woken on `cv_work` whenever bytes are released. It
// outlives the server while any of its results is unfreed.
struct ServeLedger {
  std::mutex mu;
  std::condition_variable cv_work;
  size_t in_use = 0;
  void release(size_t bytes) {
    {
      std::lock_guard<std::mutex> lk(mu);
      in_use -= bytes;
    }
    cv_work.notify_all();
  }
};

struct rsv_result {
  rsv_ctx* ctx = nullptr;
  int n = 0, precision = 0;
  rsv_solver* solver = nullptr;           // a streaming solve, owned by the result
  std::shared_ptr<rsv_batch> batch;       // or a register of a batched solve (shared by its results)
  int index = 0;
  std::vector<double> occ;
  int rows = 0;
  double wait_s = 0.0;     // served requests: submission to admission
  double service_s = 0.0;  // admission (or call) to completion
  // served requests: device bytes the result still holds, charged to the
  // server's admission budget until rsv_result_free (a batched group's charge
  // rides on the shared batch instead and is released with it)
  std::shared_ptr<ServeLedger> ledger;
  size_t charged = 0;
};

// A prepared H (Eq. (3)) for repeated y = H x: tables and per-tile diagonal
// rows are built once, each apply enqueues only the streaming passes.
struct rsv_hamiltonian {
  rsv_ctx* ctx = nullptr;
  int n = 0;
  bool c64 = true, phi = false;
  Plan plan;
  StepParams* d_sp = nullptr;
  double* d_vmat = nullptr;
  void* d_qtab = nullptr;
  void* d_diag = nullptr;
  KState* d_ks = nullptr;  // error word of the bounded waits
  double* d_part = nullptr;
  const void* map_x = nullptr;  // operands the cached tensor maps describe
  const void* map_y = nullptr;
  TileMaps maps;
  std::vector<void*> owned;
  rsv_status alloc(size_t bytes, void** p) {
    RSV_TRY(ctx->arena.alloc(bytes, p));
    owned.push_back(*p);
    return RSV_OK;
  }
  ~rsv_hamiltonian() {
    if (ctx && ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (void* p : owned) ctx->arena.release(p);
  }
};

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* rsv_last_error(void) { return g_last_error.c_str(); }
const char* rsv_version(void) { return "rsv 0.1 (sm_103a)"; }

rsv_status rsv_create(rsv_ctx** out, int32_t device, size_t arena_bytes, void* cuda_stream) {
  g_last_error.clear();
  if (!out) return fail(RSV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int count = 0;
  RSV_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return fail(RSV_ERR_INVALID_ARG, "no such CUDA device");
  RSV_CUDA(cudaSetDevice(device));
  rsv_ctx* c = new rsv_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return fail(RSV_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    c->own_stream = true;
  }
  rsv_status st = c->arena.init(arena_bytes);
  auto A = [&](size_t b, void** p) { return st == RSV_OK ? (st = c->arena.alloc(b, p)) : st; };
  A(sizeof(StepParams), (void**)&c->d_sp);
  A(sizeof(double) * kMaxAtoms * kMaxAtoms, (void**)&c->d_vmat);
  A(sizeof(double) << kTileBitsC64, &c->d_qtab);
  A(sizeof(KState), (void**)&c->d_ks);
  A(sizeof(double) * partials_doubles(c->num_sms), (void**)&c->d_part);
  A(sizeof(double) * kMaxAtoms, (void**)&c->d_occ);
  if (st == RSV_OK) {
    cudaError_t e = cudaMallocHost(&c->h_ks, sizeof(KState));
    if (e != cudaSuccess) st = fail(RSV_ERR_CUDA, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
  }
  if (st != RSV_OK) {
    rsv_destroy(c);
    return st;
  }
  *out = c;
  return RSV_OK;
}

void rsv_destroy(rsv_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  // free what the caller left open (their handles become invalid)
  while (!ctx->servers.empty()) rsv_server_destroy(*ctx->servers.begin());
  while (!ctx->hamiltonians.empty()) rsv_hamiltonian_destroy(*ctx->hamiltonians.begin());
  while (!ctx->results.empty()) rsv_result_free(*ctx->results.begin());
  while (!ctx->solvers.empty()) rsv_solver_destroy(*ctx->solvers.begin());
  while (!ctx->batches.empty()) rsv_batch_destroy(*ctx->batches.begin());
  ctx->arena.release(ctx->d_sp);
  ctx->arena.release(ctx->d_vmat);
  ctx->arena.release(ctx->d_qtab);
  ctx->arena.release(ctx->d_ks);
  ctx->arena.release(ctx->d_part);
  ctx->arena.release(ctx->d_occ);
  if (ctx->h_ks) cudaFreeHost(ctx->h_ks);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

size_t rsv_footprint_bytes(int32_t n_atoms, int32_t precision, int32_t m_max) {
  if (n_atoms < 1 || n_atoms > 31) return 0;
  if (m_max <= 0) m_max = 30;
  const size_t D = size_t(1) << n_atoms;
  const size_t vec = D * (size_t)amp_bytes(precision);
  const int L = precision == RSV_C64 ? kTileBitsC64 : kTileBitsC128;
  const size_t diag = (size_t)amp_bytes(precision) / 2 * kDiagStride * (n_atoms > L ? size_t(1) << (n_atoms - L) : 1);
  // state + m_max basis vectors + two work vectors + per-tile diagonal rows +
  // parameter tables, partial sums and allocation rounding
  return vec * (size_t)(m_max + 3) + diag + (size_t(2) << 20);
}

rsv_status rsv_pair_energies(int32_t n_atoms, int32_t dim, const double* positions_um, double c6, double* v_out) {
  g_last_error.clear();
  if (n_atoms < 1 || (dim != 2 && dim != 3) || !positions_um || !v_out)
    return fail(RSV_ERR_INVALID_ARG, "bad arguments");
  std::vector<double> v;
  RSV_TRY(pair_energies(n_atoms, dim, positions_um, c6, v));
  std::memcpy(v_out, v.data(), v.size() * sizeof(double));
  return RSV_OK;
}

int32_t rsv_num_steps(int32_t t_ns, int32_t dt_ns) {
  if (t_ns < 1 || dt_ns < 1) return 0;
  return num_steps(t_ns, dt_ns);
}

rsv_status rsv_midpoint_parameters(const rsv_problem* problem, int32_t dt_ns, double* omega_out, double* delta_out,
                                   double* phi_out, double* tau_us_out) {
  g_last_error.clear();
  RSV_TRY(validate_problem(problem));
  if (dt_ns < 1) return fail(RSV_ERR_INVALID_ARG, "dt_ns must be >= 1");
  std::vector<StepParams> sp;
  RSV_TRY(step_params(problem, dt_ns, sp));
  const int n = problem->n_atoms;
  for (size_t k = 0; k < sp.size(); ++k) {
    for (int i = 0; i < n; ++i) {
      const int q = n - 1 - i;
      if (omega_out) omega_out[k * n + i] = 2.0 * sp[k].half_omega[q];
      if (delta_out) delta_out[k * n + i] = sp[k].delta[q];
      if (phi_out) phi_out[k * n + i] = sp[k].phi[q];
    }
    if (tau_us_out) tau_us_out[k] = sp[k].tau;
  }
  return RSV_OK;
}

rsv_status rsv_apply_hamiltonian(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const double* v_pairs,
                                 const double* omega, const double* delta, const double* phi, const void* x_dev,
                                 void* y_dev) {
  g_last_error.clear();
  if (!ctx || !v_pairs || !omega || !delta || !x_dev || !y_dev) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (n_atoms < 1 || n_atoms > 31) return fail(RSV_ERR_INVALID_ARG, "n_atoms out of range");
  if (precision != RSV_C64 && precision != RSV_C128) return fail(RSV_ERR_INVALID_ARG, "bad precision");
  if ((reinterpret_cast<uintptr_t>(x_dev) | reinterpret_cast<uintptr_t>(y_dev)) & 15)
    return fail(RSV_ERR_INVALID_ARG, "device buffers must be 16-byte aligned");
  if (x_dev == y_dev) return fail(RSV_ERR_INVALID_ARG, "x and y must not alias");
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  const int n = n_atoms;
  const bool c64 = precision == RSV_C64;
  StepParams sp{};
  std::memset(&sp, 0, sizeof(sp));
  bool has_phi = false;
  for (int i = 0; i < n; ++i) {
    const int q = n - 1 - i;
    sp.half_omega[q] = 0.5 * omega[i];
    sp.delta[q] = delta[i];
    sp.phi[q] = phi ? phi[i] : 0.0;
    has_phi = has_phi || (phi && phi[i] != 0.0);
  }
  sp.has_phi = has_phi;
  const std::vector<double> vb = to_bit_matrix(n, v_pairs);
  const int shape = shape_for(ctx, n, c64);
  Plan plan = plan_for(n, c64, ctx->num_sms, shape);
  RSV_CUDA(cudaMemcpyAsync(ctx->d_sp, &sp, sizeof(sp), cudaMemcpyHostToDevice, ctx->stream));
  RSV_CUDA(cudaMemcpyAsync(ctx->d_vmat, vb.data(), vb.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  std::vector<float> qf;
  std::vector<double> qd;
  if (c64) {
    qf = q_table<float>(vb, plan.L_a);
    RSV_CUDA(cudaMemcpyAsync(ctx->d_qtab, qf.data(), qf.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  } else {
    qd = q_table<double>(vb, plan.L_a);
    RSV_CUDA(cudaMemcpyAsync(ctx->d_qtab, qd.data(), qd.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  }
  RSV_CUDA(cudaMemsetAsync(err_ptr(ctx->d_ks), 0, sizeof(int), ctx->stream));
  void* d_diag = nullptr;
  RSV_TRY(ctx->arena.alloc((c64 ? sizeof(float) : sizeof(double)) * kDiagStride * plan.a.num_tiles, &d_diag));
  struct DiagGuard {
    rsv_ctx* c;
    void* p;
    ~DiagGuard() {
      cudaStreamSynchronize(c->stream);
      c->arena.release(p);
    }
  } diag_guard{ctx, d_diag};
  {
    cudaError_t e = launch_diag_table(ctx->d_sp, ctx->d_vmat, n, plan.a.L, plan.a.num_tiles, d_diag, c64, ctx->stream);
    if (e != cudaSuccess) return fail(RSV_ERR_CUDA, std::string("diag table: ") + cudaGetErrorString(e));
  }
  TileArgs a = plan.a;
  a.sp = ctx->d_sp;
  a.vmat = ctx->d_vmat;
  a.qtab = ctx->d_qtab;
  a.ks = ctx->d_ks;
  a.partials = ctx->d_part;
  a.err = err_ptr(ctx->d_ks);
  a.diag = d_diag;
  a.xin = x_dev;
  a.out = y_dev;
  RSV_TRY(run_pass(ctx, a, nullptr, TileMode::kMatvecFirst, c64, has_phi, plan.grid_a));
  if (plan.two_pass) {
    TileArgs b = plan.b;
    b.sp = ctx->d_sp;
    b.vmat = ctx->d_vmat;
    b.ks = ctx->d_ks;
    b.partials = ctx->d_part;
    b.err = err_ptr(ctx->d_ks);
    b.xin = x_dev;
    b.out = y_dev;
    TileMaps maps;
    if (!encode_tile_map(&maps.x, x_dev, plan.b, c64) || !encode_tile_map(&maps.z, y_dev, plan.b, c64))
      return fail(RSV_ERR_CUDA, "tensor map encoding failed");
    RSV_TRY(run_pass(ctx, b, &maps, TileMode::kMatvecSecond, c64, has_phi, plan.grid_b));
  }
  // keep host staging alive until the copies are done
  RSV_CUDA(cudaMemcpyAsync(ctx->h_ks, ctx->d_ks, kStatusBytes, cudaMemcpyDeviceToHost, ctx->stream));
  RSV_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ctx->h_ks->error) return fail(RSV_ERR_TIMEOUT, "a device-side wait timed out (kernel aborted)");
  return RSV_OK;
}

rsv_status rsv_hamiltonian_create(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const double* v_pairs,
                                  const double* omega, const double* delta, const double* phi, rsv_hamiltonian** out) {
  g_last_error.clear();
  if (!ctx || !v_pairs || !omega || !delta || !out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (n_atoms < 1 || n_atoms > 31) return fail(RSV_ERR_INVALID_ARG, "n_atoms out of range");
  if (precision != RSV_C64 && precision != RSV_C128) return fail(RSV_ERR_INVALID_ARG, "bad precision");
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  std::unique_ptr<rsv_hamiltonian> h(new rsv_hamiltonian());
  h->ctx = ctx;
  h->n = n_atoms;
  h->c64 = precision == RSV_C64;
  StepParams sp{};
  std::memset(&sp, 0, sizeof(sp));
  for (int i = 0; i < n_atoms; ++i) {
    const int q = n_atoms - 1 - i;
    sp.half_omega[q] = 0.5 * omega[i];
    sp.delta[q] = delta[i];
    sp.phi[q] = phi ? phi[i] : 0.0;
    h->phi = h->phi || (phi && phi[i] != 0.0);
  }
  sp.has_phi = h->phi;
  const std::vector<double> vb = to_bit_matrix(n_atoms, v_pairs);
  const int shape = shape_for(ctx, n_atoms, h->c64);
  h->plan = plan_for(n_atoms, h->c64, ctx->num_sms, shape);
  if (h->plan.two_pass && h->plan.b.nG > kMaxGBits) return fail(RSV_ERR_INVALID_ARG, "n_atoms too large");
  RSV_TRY(h->alloc(sizeof(StepParams), (void**)&h->d_sp));
  RSV_TRY(h->alloc(sizeof(double) * kMaxAtoms * kMaxAtoms, (void**)&h->d_vmat));
  RSV_TRY(h->alloc((h->c64 ? sizeof(float) : sizeof(double)) << h->plan.L_a, &h->d_qtab));
  RSV_TRY(h->alloc((h->c64 ? sizeof(float) : sizeof(double)) * kDiagStride * h->plan.a.num_tiles, &h->d_diag));
  RSV_TRY(h->alloc(sizeof(KState), (void**)&h->d_ks));
  RSV_TRY(h->alloc(sizeof(double) * partials_doubles(ctx->num_sms), (void**)&h->d_part));
  RSV_CUDA(cudaMemcpyAsync(h->d_sp, &sp, sizeof(sp), cudaMemcpyHostToDevice, ctx->stream));
  RSV_CUDA(cudaMemcpyAsync(h->d_vmat, vb.data(), vb.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  if (h->c64) {
    const std::vector<float> q = q_table<float>(vb, h->plan.L_a);
    RSV_CUDA(cudaMemcpyAsync(h->d_qtab, q.data(), q.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    RSV_CUDA(cudaStreamSynchronize(ctx->stream));
  } else {
    const std::vector<double> q = q_table<double>(vb, h->plan.L_a);
    RSV_CUDA(cudaMemcpyAsync(h->d_qtab, q.data(), q.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    RSV_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  RSV_CUDA(cudaMemsetAsync(h->d_ks, 0, sizeof(KState), ctx->stream));
  RSV_CUDA(launch_diag_table(h->d_sp, h->d_vmat, n_atoms, h->plan.a.L, h->plan.a.num_tiles, h->d_diag, h->c64,
                             ctx->stream));
  RSV_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->hamiltonians.insert(h.get());
  *out = h.release();
  return RSV_OK;
}

rsv_status rsv_hamiltonian_apply(rsv_hamiltonian* h, const void* x_dev, void* y_dev) {
  g_last_error.clear();
  if (!h || !x_dev || !y_dev) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if ((reinterpret_cast<uintptr_t>(x_dev) | reinterpret_cast<uintptr_t>(y_dev)) & 15)
    return fail(RSV_ERR_INVALID_ARG, "device buffers must be 16-byte aligned");
  if (x_dev == y_dev) return fail(RSV_ERR_INVALID_ARG, "x and y must not alias");
  rsv_ctx* ctx = h->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  TileArgs a = h->plan.a;
  a.sp = h->d_sp;
  a.vmat = h->d_vmat;
  a.qtab = h->d_qtab;
  a.ks = h->d_ks;
  a.partials = h->d_part;
  a.err = err_ptr(h->d_ks);
  a.diag = h->d_diag;
  a.xin = x_dev;
  a.out = y_dev;
  RSV_TRY(run_pass(ctx, a, nullptr, TileMode::kMatvecFirst, h->c64, h->phi, h->plan.grid_a));
  if (h->plan.two_pass) {
    if (x_dev != h->map_x || y_dev != h->map_y) {
      if (!encode_tile_map(&h->maps.x, x_dev, h->plan.b, h->c64) ||
          !encode_tile_map(&h->maps.z, y_dev, h->plan.b, h->c64))
        return fail(RSV_ERR_CUDA, "tensor map encoding failed");
      h->map_x = x_dev;
      h->map_y = y_dev;
    }
    TileArgs b = h->plan.b;
    b.sp = h->d_sp;
    b.vmat = h->d_vmat;
    b.ks = h->d_ks;
    b.partials = h->d_part;
    b.err = err_ptr(h->d_ks);
    b.xin = x_dev;
    b.out = y_dev;
    RSV_TRY(run_pass(ctx, b, &h->maps, TileMode::kMatvecSecond, h->c64, h->phi, h->plan.grid_b));
  }
  return RSV_OK;
}

rsv_status rsv_hamiltonian_sync(rsv_hamiltonian* h) {
  g_last_error.clear();
  if (!h) return fail(RSV_ERR_INVALID_ARG, "NULL operator");
  rsv_ctx* ctx = h->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  int err = 0;
  RSV_CUDA(cudaMemcpyAsync(&err, err_ptr(h->d_ks), sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RSV_CUDA(cudaStreamSynchronize(ctx->stream));
  if (err) return fail(RSV_ERR_TIMEOUT, "a device-side wait timed out (kernel aborted)");
  return RSV_OK;
}

void rsv_hamiltonian_destroy(rsv_hamiltonian* h) {
  if (!h) return;
  {
    std::lock_guard<std::mutex> lk(h->ctx->mu);
    h->ctx->hamiltonians.erase(h);
  }
  delete h;
}

rsv_status rsv_observe(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const void* psi_dev, double* norm2_out,
                       double* occ_out) {
  g_last_error.clear();
  if (!ctx || !psi_dev) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (n_atoms < 1 || n_atoms > 31) return fail(RSV_ERR_INVALID_ARG, "n_atoms out of range");
  if (precision != RSV_C64 && precision != RSV_C128) return fail(RSV_ERR_INVALID_ARG, "bad precision");
  if (reinterpret_cast<uintptr_t>(psi_dev) & 15) return fail(RSV_ERR_INVALID_ARG, "psi must be 16-byte aligned");
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  const bool c64 = precision == RSV_C64;
  Plan plan = make_plan(n_atoms, c64, ctx->num_sms);
  CombineArgs ca{};
  ca.n = n_atoms;
  ca.dim = int64_t(1) << n_atoms;
  ca.ks = ctx->d_ks;
  ca.psi = const_cast<void*>(psi_dev);
  ca.partials = ctx->d_part;
  ca.combine = 0;
  RSV_CUDA(launch_combine(ca, c64, plan.grid_c, ctx->stream));
  BeginArgs ba{};
  ba.ks = ctx->d_ks;
  ba.partials = ctx->d_part;
  ba.nparts = plan.grid_c;
  ba.n = n_atoms;
  ba.occ_out = ctx->d_occ;
  ba.reset_only = 1;
  RSV_CUDA(launch_begin(ba, ctx->stream));
  RSV_CUDA(cudaMemcpyAsync(ctx->h_ks, ctx->d_ks, kStatusBytes, cudaMemcpyDeviceToHost, ctx->stream));
  std::vector<double> occ(n_atoms);
  RSV_CUDA(cudaMemcpyAsync(occ.data(), ctx->d_occ, sizeof(double) * n_atoms, cudaMemcpyDeviceToHost, ctx->stream));
  RSV_CUDA(cudaStreamSynchronize(ctx->stream));
  if (norm2_out) *norm2_out = ctx->h_ks->norm2;
  if (occ_out) std::memcpy(occ_out, occ.data(), sizeof(double) * n_atoms);
  return RSV_OK;
}

rsv_status rsv_correlations(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const void* psi_dev, double* out) {
  g_last_error.clear();
  if (!ctx || !psi_dev || !out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (n_atoms < 1 || n_atoms > 31) return fail(RSV_ERR_INVALID_ARG, "n_atoms out of range");
  if (precision != RSV_C64 && precision != RSV_C128) return fail(RSV_ERR_INVALID_ARG, "bad precision");
  if (reinterpret_cast<uintptr_t>(psi_dev) & 15) return fail(RSV_ERR_INVALID_ARG, "psi must be 16-byte aligned");
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  const bool c64 = precision == RSV_C64;
  const Plan plan = make_plan(n_atoms, c64, ctx->num_sms);
  std::vector<double> rows((size_t)n_atoms * n_atoms);
  for (int i = 0; i < n_atoms; ++i) {
    // row i: the occupations of psi restricted to amplitudes with atom i excited
    CombineArgs ca{};
    ca.n = n_atoms;
    ca.dim = int64_t(1) << n_atoms;
    ca.ks = ctx->d_ks;
    ca.psi = const_cast<void*>(psi_dev);
    ca.partials = ctx->d_part;
    ca.combine = 0;
    ca.mask_bit = n_atoms - 1 - i;
    RSV_CUDA(launch_combine(ca, c64, plan.grid_c, ctx->stream));
    BeginArgs ba{};
    ba.ks = ctx->d_ks;
    ba.partials = ctx->d_part;
    ba.nparts = plan.grid_c;
    ba.n = n_atoms;
    ba.occ_out = ctx->d_occ;
    ba.reset_only = 1;
    RSV_CUDA(launch_begin(ba, ctx->stream));
    RSV_CUDA(cudaMemcpyAsync(rows.data() + (size_t)i * n_atoms, ctx->d_occ, sizeof(double) * n_atoms,
                             cudaMemcpyDeviceToHost, ctx->stream));
  }
  RSV_CUDA(cudaStreamSynchronize(ctx->stream));
  std::memcpy(out, rows.data(), rows.size() * sizeof(double));
  return RSV_OK;
}

rsv_status rsv_hamiltonian_expectation(rsv_hamiltonian* h, const void* psi_dev, double* out) {
  g_last_error.clear();
  if (!h || !psi_dev || !out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (reinterpret_cast<uintptr_t>(psi_dev) & 15) return fail(RSV_ERR_INVALID_ARG, "psi must be 16-byte aligned");
  rsv_ctx* ctx = h->ctx;
  const int64_t dim = int64_t(1) << h->n;
  const size_t vbytes = (size_t)dim * amp_bytes(h->c64 ? RSV_C64 : RSV_C128);
  void* y = nullptr;
  RSV_TRY(ctx->arena.alloc(vbytes, &y));
  struct Release {
    rsv_ctx* c;
    void* p;
    ~Release() {
      cudaStreamSynchronize(c->stream);
      c->arena.release(p);
    }
  } release{ctx, y};
  RSV_TRY(rsv_hamiltonian_apply(h, psi_dev, y));
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  const int grid = 4 * ctx->num_sms;
  RSV_CUDA(launch_dot3(psi_dev, y, dim, h->c64, ctx->d_part, grid, ctx->stream));
  std::vector<double> part((size_t)grid * 3);
  int err = 0;
  RSV_CUDA(cudaMemcpyAsync(part.data(), ctx->d_part, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
  RSV_CUDA(cudaMemcpyAsync(&err, err_ptr(h->d_ks), sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RSV_CUDA(cudaStreamSynchronize(ctx->stream));
  if (err) return fail(RSV_ERR_TIMEOUT, "a device-side wait timed out (kernel aborted)");
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < grid; ++b)
    for (int k = 0; k < 3; ++k) s[k] += part[(size_t)b * 3 + k];
  out[0] = s[0];
  out[1] = s[1];
  out[2] = s[2];
  return RSV_OK;
}

rsv_status rsv_sample(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const void* psi_dev, int64_t shots,
                      uint64_t seed, uint64_t* out) {
  g_last_error.clear();
  if (!ctx || !psi_dev || (!out && shots > 0)) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (n_atoms < 1 || n_atoms > 31 || shots < 0) return fail(RSV_ERR_INVALID_ARG, "bad size");
  if (precision != RSV_C64 && precision != RSV_C128) return fail(RSV_ERR_INVALID_ARG, "bad precision");
  if (shots == 0) return RSV_OK;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  const bool c64 = precision == RSV_C64;
  const int64_t dim = int64_t(1) << n_atoms;
  const int64_t chunk = std::min<int64_t>(dim, kSampleChunk);
  const int64_t nchunks = (dim + chunk - 1) / chunk;
  double* d_sums = nullptr;
  uint64_t* d_out = nullptr;
  RSV_TRY(ctx->arena.alloc(sizeof(double) * nchunks, (void**)&d_sums));
  rsv_status st = ctx->arena.alloc(sizeof(uint64_t) * shots, (void**)&d_out);
  if (st != RSV_OK) {
    ctx->arena.release(d_sums);
    return st;
  }
  auto cleanup = [&]() {
    cudaStreamSynchronize(ctx->stream);
    ctx->arena.release(d_sums);
    ctx->arena.release(d_out);
  };
  std::vector<double> sums(nchunks), cdf(nchunks);
  cudaError_t e = launch_block_sums(psi_dev, dim, c64, chunk, d_sums, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sums.data(), d_sums, sizeof(double) * nchunks, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    cleanup();
    return fail(RSV_ERR_CUDA, std::string("sampling sums: ") + cudaGetErrorString(e));
  }
  double run = 0.0;
  for (int64_t c = 0; c < nchunks; ++c) {
    cdf[c] = run;
    run += sums[c];
  }
  const double total = run;
  if (!(total > 0.0)) {
    cleanup();
    return fail(RSV_ERR_INVALID_ARG, "state has zero norm");
  }
  e = cudaMemcpyAsync(d_sums, cdf.data(), sizeof(double) * nchunks, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = launch_sample(psi_dev, dim, c64, chunk, d_sums, nchunks, total, shots, seed, d_out, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, sizeof(uint64_t) * shots, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cleanup();
  if (e != cudaSuccess) return fail(RSV_ERR_CUDA, std::string("sampling: ") + cudaGetErrorString(e));
  return RSV_OK;
}

// one_shot: the solver will be stepped to the end and never rewound (rsv_run,
// served requests), so it keeps no host copy of the caller's initial state.
static rsv_status solver_create(rsv_ctx* ctx, const rsv_problem* problem, const rsv_config* config,
                                cudaStream_t stream, rsv_solver** out, bool one_shot = false) {
  g_last_error.clear();
  if (!ctx || !config || !out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  RSV_TRY(validate_problem(problem));
  rsv_config cfg = *config;
  if (cfg.dt_ns < 1) return fail(RSV_ERR_INVALID_ARG, "dt_ns must be >= 1");
  if (cfg.precision != RSV_C64 && cfg.precision != RSV_C128) return fail(RSV_ERR_INVALID_ARG, "bad precision");
  if (cfg.m_max == 0) cfg.m_max = 30;
  if (cfg.m_max < 2 || cfg.m_max > kMaxKrylov) return fail(RSV_ERR_INVALID_ARG, "m_max must be in [2, 64]");
  if (cfg.krylov_tol <= 0.0) cfg.krylov_tol = cfg.precision == RSV_C64 ? 1e-7 : 1e-12;
  if (cfg.max_substeps <= 0) cfg.max_substeps = 64;
  if (cfg.obs_stride < 0) return fail(RSV_ERR_INVALID_ARG, "obs_stride must be >= 0");
  if (cfg.flags & ~RSV_FLAG_CONTROL_LAUNCH) return fail(RSV_ERR_INVALID_ARG, "unknown flags");
  const int n = problem->n_atoms;
  if (cfg.precision == RSV_C128 && n > 30) return fail(RSV_ERR_INVALID_ARG, "n_atoms too large for complex128");
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  if (ctx->arena.cap() > 0 &&
      solver_bytes(problem, cfg) > ctx->arena.cap() - ctx->arena.used())
    return fail(RSV_ERR_OUT_OF_MEMORY, "footprint exceeds the free arena");
  std::vector<double> v_atoms;
  RSV_TRY(pair_energies(n, problem->dim, problem->positions_um, problem->c6, v_atoms));
  auto s = new rsv_solver();
  s->ctx = ctx;
  s->stream = stream ? stream : ctx->stream;
  s->n = n;
  s->precision = cfg.precision;
  s->c64 = cfg.precision == RSV_C64;
  s->dim = int64_t(1) << n;
  s->cfg = cfg;
  s->fused_control = !(cfg.flags & RSV_FLAG_CONTROL_LAUNCH);
  s->plan = make_plan(n, s->c64, ctx->num_sms);  // strided-pass shape tuned below
  RSV_TRY(step_params(problem, cfg.dt_ns, s->h_sp));
  s->nsteps = (int)s->h_sp.size();
  s->phi = any_phi(s->h_sp, n);
  const std::vector<double> vb = to_bit_matrix(n, v_atoms.data());
  const size_t vbytes = (size_t)s->dim * amp_bytes(cfg.precision);
  s->max_rows = (cfg.obs_stride > 0 ? s->nsteps / cfg.obs_stride : 0) + 2;
  rsv_status st = RSV_OK;
  auto A = [&](size_t b, void** p) {
    if (st == RSV_OK) st = s->alloc(b, p);
  };
  A(sizeof(StepParams) * s->nsteps, (void**)&s->d_sp);
  A(sizeof(double) * kMaxAtoms * kMaxAtoms, (void**)&s->d_vmat);
  A(amp_bytes(cfg.precision) / 2 * (size_t(1) << s->plan.L_a), &s->d_qtab);
  A((s->c64 ? sizeof(float) : sizeof(double)) * kDiagStride * s->plan.a.num_tiles, &s->d_diag);
  A(vbytes, &s->d_psi);
  A(vbytes, &s->d_u[0]);
  A(vbytes, &s->d_u[1]);
  s->basis.assign(cfg.m_max, nullptr);
  for (int k = 0; k < cfg.m_max; ++k) A(vbytes, &s->basis[k]);
  A(sizeof(void*) * cfg.m_max, (void**)&s->d_basis);
  A(sizeof(KState), (void**)&s->d_ks);
  A(cheb_cache_bytes(), (void**)&s->d_cheb);
  A(sizeof(double) * partials_doubles(ctx->num_sms), (void**)&s->d_part);
  A(sizeof(double) * partials_doubles(ctx->num_sms), (void**)&s->d_cpart);
  A(sizeof(double) * n * s->max_rows, (void**)&s->d_occ);
  if (s->phi && s->plan.two_pass) {
    // gauge tables (within the footprint's 2 MiB of tables: at most 1 MiB, at 30 atoms complex128)
    s->phase_bits = (n + 1) / 2;
    A(phase_table_bytes(n, s->phase_bits, s->c64), &s->d_phase);
  }
  if (st != RSV_OK) {
    delete s;
    return st;
  }
  cudaError_t e = cudaMallocHost(&s->h_ks, sizeof(KState));
  if (e != cudaSuccess) {
    delete s;
    return fail(RSV_ERR_CUDA, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
  }
  if (s->plan.two_pass) {
    const int shape = tune_shape(ctx, s->stream, n, s->c64, s->d_sp, s->d_vmat, s->d_ks, s->d_part, s->basis[0], s->d_u[0]);
    s->plan = plan_for(n, s->c64, ctx->num_sms, shape);
    s->map_basis.resize(cfg.m_max);
    bool ok = true;
    for (int k = 0; k < cfg.m_max; ++k) ok = ok && encode_tile_map(&s->map_basis[k], s->basis[k], s->plan.b, s->c64);
    ok = ok && encode_tile_map(&s->map_u[0], s->d_u[0], s->plan.b, s->c64) &&
         encode_tile_map(&s->map_u[1], s->d_u[1], s->plan.b, s->c64);
    if (!ok) {
      delete s;
      return fail(RSV_ERR_CUDA, "tensor map encoding failed");
    }
  }
  auto fin = [&](rsv_status r) {
    if (r != RSV_OK) delete s;
    return r;
  };
  std::vector<char> zero_ks(sizeof(KState), 0);
  if (cudaMemcpyAsync(s->d_sp, s->h_sp.data(), sizeof(StepParams) * s->nsteps, cudaMemcpyHostToDevice, s->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(s->d_vmat, vb.data(), vb.size() * sizeof(double), cudaMemcpyHostToDevice, s->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(s->d_basis, s->basis.data(), sizeof(void*) * cfg.m_max, cudaMemcpyHostToDevice, s->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(s->d_ks, zero_ks.data(), sizeof(KState), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
    return fin(fail(RSV_ERR_CUDA, "upload failed"));
  if (s->c64) {
    auto q = q_table<float>(vb, s->plan.L_a);
    if (cudaMemcpyAsync(s->d_qtab, q.data(), q.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream) !=
        cudaSuccess)
      return fin(fail(RSV_ERR_CUDA, "upload failed"));
    cudaStreamSynchronize(s->stream);
  } else {
    auto q = q_table<double>(vb, s->plan.L_a);
    if (cudaMemcpyAsync(s->d_qtab, q.data(), q.size() * sizeof(double), cudaMemcpyHostToDevice, s->stream) !=
        cudaSuccess)
      return fin(fail(RSV_ERR_CUDA, "upload failed"));
    cudaStreamSynchronize(s->stream);
  }
  if (problem->initial_state && !one_shot) {
    const char* p = static_cast<const char*>(problem->initial_state);
    s->init_host.assign(p, p + vbytes);
  }
  rsv_status r = s->reset_to_initial(one_shot ? problem->initial_state : nullptr);
  if (r != RSV_OK) return fin(r);
  ctx->solvers.insert(s);
  *out = s;
  return RSV_OK;
}

rsv_status rsv_solver_create(rsv_ctx* ctx, const rsv_problem* problem, const rsv_config* config, rsv_solver** out) {
  return solver_create(ctx, problem, config, nullptr, out);
}

rsv_status rsv_solver_rewind(rsv_solver* s) {
  g_last_error.clear();
  if (!s) return fail(RSV_ERR_INVALID_ARG, "NULL solver");
  std::lock_guard<std::mutex> lk(s->ctx->mu);
  cudaSetDevice(s->ctx->device);
  return s->reset_to_initial();
}

void rsv_solver_destroy(rsv_solver* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->ctx->mu);
    s->ctx->solvers.erase(s);
  }
  delete s;
}

// Advances a solver on its own stream. Callers serialise access to `s`; the
// context lock is not needed (the arena has its own).
static rsv_status solver_step(rsv_solver* s, int32_t n_steps) {
  if (s->trimmed) return fail(RSV_ERR_INVALID_ARG, "the solve has finished and kept only its state");
  cudaSetDevice(s->ctx->device);
  const auto t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < n_steps && s->done < s->nsteps; ++i) RSV_TRY(s->step_once());
  RSV_CUDA(cudaStreamSynchronize(s->stream));
  if (s->profiling) s->drain_timings();
  s->stats.seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return RSV_OK;
}

rsv_status rsv_solver_step(rsv_solver* s, int32_t n_steps) {
  g_last_error.clear();
  if (!s || n_steps < 0) return fail(RSV_ERR_INVALID_ARG, "bad arguments");
  std::lock_guard<std::mutex> lk(s->ctx->mu);
  return solver_step(s, n_steps);
}

rsv_status rsv_solver_progress(const rsv_solver* s, int32_t* done, int32_t* total) {
  if (!s) return fail(RSV_ERR_INVALID_ARG, "NULL solver");
  if (done) *done = s->done;
  if (total) *total = s->nsteps;
  return RSV_OK;
}

rsv_status rsv_solver_state_device(rsv_solver* s, void** dev_ptr, size_t* bytes) {
  if (!s || !dev_ptr) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  *dev_ptr = s->d_psi;
  if (bytes) *bytes = (size_t)s->dim * amp_bytes(s->precision);
  return RSV_OK;
}

rsv_status rsv_solver_get_state(rsv_solver* s, void* host_dst, size_t bytes) {
  g_last_error.clear();
  if (!s || !host_dst) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (bytes != (size_t)s->dim * amp_bytes(s->precision)) return fail(RSV_ERR_INVALID_ARG, "size mismatch");
  std::lock_guard<std::mutex> lk(s->ctx->mu);
  RSV_CUDA(cudaMemcpyAsync(host_dst, s->d_psi, bytes, cudaMemcpyDeviceToHost, s->stream));
  RSV_CUDA(cudaStreamSynchronize(s->stream));
  return RSV_OK;
}

rsv_status rsv_solver_set_state(rsv_solver* s, const void* host_src, size_t bytes) {
  g_last_error.clear();
  if (!s || !host_src) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (bytes != (size_t)s->dim * amp_bytes(s->precision)) return fail(RSV_ERR_INVALID_ARG, "size mismatch");
  std::lock_guard<std::mutex> lk(s->ctx->mu);
  RSV_CUDA(cudaMemcpyAsync(s->d_psi, host_src, bytes, cudaMemcpyHostToDevice, s->stream));
  RSV_TRY(s->observe_into_partials());
  RSV_CUDA(cudaStreamSynchronize(s->stream));
  return RSV_OK;
}

rsv_status rsv_solver_set_state_device(rsv_solver* s, const void* dev_src, size_t bytes) {
  g_last_error.clear();
  if (!s || !dev_src) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (bytes != (size_t)s->dim * amp_bytes(s->precision)) return fail(RSV_ERR_INVALID_ARG, "size mismatch");
  std::lock_guard<std::mutex> lk(s->ctx->mu);
  RSV_CUDA(cudaMemcpyAsync(s->d_psi, dev_src, bytes, cudaMemcpyDeviceToDevice, s->stream));
  RSV_TRY(s->observe_into_partials());
  RSV_CUDA(cudaStreamSynchronize(s->stream));
  return RSV_OK;
}

rsv_status rsv_solver_occupations(rsv_solver* s, double* dst, int32_t capacity_rows, int32_t* n_rows) {
  g_last_error.clear();
  if (!s || !n_rows) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  *n_rows = s->rows;
  if (!dst) return RSV_OK;
  const int rows = std::min(capacity_rows, s->rows);
  std::lock_guard<std::mutex> lk(s->ctx->mu);
  RSV_CUDA(cudaMemcpyAsync(dst, s->d_occ, sizeof(double) * s->n * rows, cudaMemcpyDeviceToHost, s->stream));
  RSV_CUDA(cudaStreamSynchronize(s->stream));
  return RSV_OK;
}

rsv_status rsv_solver_set_profiling(rsv_solver* s, int32_t on) {
  g_last_error.clear();
  if (!s) return fail(RSV_ERR_INVALID_ARG, "NULL solver");
  std::lock_guard<std::mutex> lk(s->ctx->mu);
  RSV_CUDA(cudaStreamSynchronize(s->stream));
  s->drain_timings();
  s->profiling = on != 0;
  if (s->profiling) {
    s->ktimes = rsv_kernel_times{};
    RSV_TRY(s->read_status());  // the control counters' starting point
    for (auto& v : s->ctl_acc) v = 0;
  }
  return RSV_OK;
}

rsv_status rsv_solver_kernel_times(const rsv_solver* s, rsv_kernel_times* out) {
  if (!s || !out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  *out = s->ktimes;
  out->control_step_ms = s->ctl_acc[0] * 1e-6;
  out->control_steps = (int64_t)s->ctl_acc[1];
  out->control_check_ms = s->ctl_acc[2] * 1e-6;
  out->control_checks = (int64_t)s->ctl_acc[3];
  return RSV_OK;
}

rsv_status rsv_solver_stats(const rsv_solver* s, rsv_stats* out) {
  if (!s || !out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  *out = s->stats;
  out->tile_passes = s->plan.two_pass ? 2 : 1;
  out->segment_bits = s->plan.two_pass ? s->plan.b.c : s->plan.a.c;
  out->l2_partner_bits = s->plan.two_pass ? s->plan.b.nG : s->plan.a.nG;
  out->tile_order_bits = s->plan.two_pass ? s->plan.b.f1_fast : 0;
  out->krylov_dim_max = s->cfg.m_max;
  out->strided_tile_bits = s->plan.two_pass ? s->plan.b.L : 0;
  return RSV_OK;
}

// A finished solver becomes a result (owned by the context until freed).
static rsv_status make_result(rsv_solver* s, rsv_result** out) {
  rsv_ctx* ctx = s->ctx;
  auto r = new rsv_result();
  r->ctx = ctx;
  r->n = s->n;
  r->precision = s->precision;
  r->solver = s;
  r->service_s = s->stats.seconds;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->solvers.erase(s);
    ctx->results.insert(r);
  }
  r->rows = s->rows;
  r->occ.resize((size_t)s->rows * s->n);
  int32_t rows = 0;
  const rsv_status st = rsv_solver_occupations(s, r->occ.data(), s->rows, &rows);
  if (st != RSV_OK) {
    rsv_result_free(r);
    return st;
  }
  *out = r;
  return RSV_OK;
}

rsv_status rsv_run(rsv_ctx* ctx, const rsv_problem* problem, const rsv_config* config, rsv_result** out) {
  g_last_error.clear();
  if (!out) return fail(RSV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  rsv_solver* s = nullptr;
  RSV_TRY(solver_create(ctx, problem, config, nullptr, &s, /*one_shot=*/true));
  rsv_status st = rsv_solver_step(s, s->nsteps);
  if (st != RSV_OK) {
    rsv_solver_destroy(s);
    return st;
  }
  return make_result(s, out);
}

rsv_status rsv_result_state(const rsv_result* r, void* host_dst, size_t bytes) {
  if (!r) return fail(RSV_ERR_INVALID_ARG, "NULL result");
  if (r->batch) return rsv_batch_state(r->batch.get(), r->index, host_dst, bytes);
  return rsv_solver_get_state(r->solver, host_dst, bytes);
}

rsv_status rsv_result_state_device(const rsv_result* r, void** dev_ptr, size_t* bytes) {
  if (!r) return fail(RSV_ERR_INVALID_ARG, "NULL result");
  if (r->batch) return rsv_batch_state_device(r->batch.get(), r->index, dev_ptr, bytes);
  return rsv_solver_state_device(r->solver, dev_ptr, bytes);
}

rsv_status rsv_result_occupations(const rsv_result* r, double* dst, int32_t capacity_rows, int32_t* n_rows) {
  if (!r || !n_rows) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  *n_rows = r->rows;
  if (dst) {
    const int rows = std::min(capacity_rows, r->rows);
    std::memcpy(dst, r->occ.data(), sizeof(double) * rows * r->n);
  }
  return RSV_OK;
}

rsv_status rsv_result_sample(const rsv_result* r, int64_t shots, uint64_t seed, uint64_t* out) {
  if (!r) return fail(RSV_ERR_INVALID_ARG, "NULL result");
  void* psi = nullptr;
  size_t bytes = 0;
  RSV_TRY(rsv_result_state_device(r, &psi, &bytes));
  return rsv_sample(r->ctx, r->n, r->precision, psi, shots, seed, out);
}

rsv_status rsv_result_stats(const rsv_result* r, rsv_stats* out) {
  if (!r) return fail(RSV_ERR_INVALID_ARG, "NULL result");
  if (r->batch) return rsv_batch_stats(r->batch.get(), r->index, out);
  return rsv_solver_stats(r->solver, out);
}

rsv_status rsv_result_times(const rsv_result* r, double* wait_s, double* service_s) {
  if (!r) return fail(RSV_ERR_INVALID_ARG, "NULL result");
  if (wait_s) *wait_s = r->wait_s;
  if (service_s) *service_s = r->service_s;
  return RSV_OK;
}

void rsv_result_free(rsv_result* r) {
  if (!r) return;
  {
    std::lock_guard<std::mutex> lk(r->ctx->mu);
    r->ctx->results.erase(r);
  }
  delete r->solver;  // owned by the result, not in the context's solver set
  if (r->ledger) r->ledger->release(r->charged);
  delete r;          // a batch goes with its last result (and releases its group's charge)
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batch: many independent registers evolved by one persistent launch
// (batch_kernels.cu), replayed from a captured CUDA graph.
// ---------------------------------------------------------------------------
struct rsv_batch {
  rsv_ctx* ctx = nullptr;
  int count = 0;
  rsv_config cfg{};
  bool c64 = true;
  int nmax = 0;
  int grid = 0;
  int blocks_per_sm = 0;
  int count_large = 0;  // registers solved by whole clusters (the front of `order`)
  int cluster = 1;      // CTAs per cluster of the launch
  int64_t work_stride = 0;
  size_t state_amps = 0;
  std::vector<BatchItem> items;
  std::vector<int> order;
  std::vector<BatchOut> out;
  bool have_out = false;
  int runs = 0;
  float last_ms = 0.f;
  float tuned_ms = 0.f;  // sample time of the chosen Krylov depth (autotuned batches)
  std::vector<void*> allocs;
  BatchItem* d_items = nullptr;
  int* d_order = nullptr;
  int* d_next = nullptr;
  void* d_states = nullptr;
  void* d_init = nullptr;
  double* d_params = nullptr;
  double* d_vmat = nullptr;
  double* d_occ = nullptr;
  BatchOut* d_out = nullptr;
  void* d_work = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev0 = nullptr, ev1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;

  rsv_status alloc(size_t bytes, void** p) {
    RSV_TRY(ctx->arena.alloc(bytes, p));
    allocs.push_back(*p);
    return RSV_OK;
  }
  ~rsv_batch() {
    if (stream) cudaStreamSynchronize(stream);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (void* p : allocs) ctx->arena.release(p);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (stream) cudaStreamDestroy(stream);
  }
  BatchArgs args() const {
    BatchArgs a{};
    a.items = d_items;
    a.order = d_order;
    a.count = count;
    a.count_large = count_large;
    a.cluster = cluster;
    a.next = d_next;
    a.states = d_states;
    a.params = d_params;
    a.vmat = d_vmat;
    a.occ = d_occ;
    a.out = d_out;
    a.work = d_work;
    a.work_stride = work_stride;
    a.m_max = cfg.m_max;
    a.max_substeps = cfg.max_substeps;
    a.step_limit = 0;
    a.tol = cfg.krylov_tol;
    a.breakdown = 1e-13;
    return a;
  }
};

namespace {

constexpr int kBatchTuneMax = 40;
constexpr int kBatchTuneSteps = 10;  // steps of each sampled register per candidate

// Krylov-depth autotuner of a batch: evolves a sample of the registers (spread
// over the largest-first order) over their first kBatchTuneSteps steps with
// each candidate m_max (see the choice rule below). A larger m_max means fewer substeps but more FP64 exponentials per
// step and a larger workspace; the best value depends on the registers'
// spectra and time steps. The workspace is then shrunk to the chosen depth.
rsv_status batch_tune_krylov(rsv_batch* b) {
  static const int cand[] = {12, 16, 20, 24, 32, kBatchTuneMax};
  const int ns = std::min(b->count, 48);
  std::vector<int> sample(ns);
  for (int i = 0; i < ns; ++i) sample[i] = b->order[(size_t)i * b->count / ns];
  int ns_large = 0;  // the sample keeps the order: cooperative registers first
  for (int i = 0; i < ns; ++i) ns_large += i * b->count / ns < b->count_large ? 1 : 0;
  const int sample_grid =
      std::min(b->grid, (ns + b->cluster - 1) / b->cluster * b->cluster);  // a multiple of the cluster size
  int* d_sample = nullptr;
  RSV_TRY(b->alloc(sizeof(int) * ns, (void**)&d_sample));
  RSV_CUDA(cudaMemcpyAsync(d_sample, sample.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, b->stream));
  const size_t sbytes = b->state_amps * amp_bytes(b->cfg.precision);
  const int ncand = (int)(sizeof(cand) / sizeof(cand[0]));
  std::vector<float> cand_ms(ncand, 1e30f);
  for (int c = -1; c < ncand; ++c) {
    BatchArgs a = b->args();
    a.order = d_sample;
    a.count = ns;
    a.count_large = ns_large;
    a.m_max = cand[c < 0 ? 0 : c];  // c = -1: warm-up launch
    a.step_limit = kBatchTuneSteps;
    RSV_CUDA(cudaMemcpyAsync(b->d_states, b->d_init, sbytes, cudaMemcpyDeviceToDevice, b->stream));
    RSV_CUDA(cudaMemsetAsync(b->d_next, 0, sizeof(int) * 2, b->stream));
    RSV_CUDA(cudaEventRecord(b->ev0, b->stream));
    RSV_CUDA(launch_batch(a, b->c64, sample_grid, b->stream));
    RSV_CUDA(cudaEventRecord(b->ev1, b->stream));
    RSV_CUDA(cudaStreamSynchronize(b->stream));
    float ms = 0.f;
    RSV_CUDA(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    std::vector<BatchOut> o(b->count);
    RSV_CUDA(cudaMemcpy(o.data(), b->d_out, sizeof(BatchOut) * b->count, cudaMemcpyDeviceToHost));
    bool ok = true;
    for (int i : sample) ok = ok && o[i].status == 0;
    if (c >= 0 && ok) cand_ms[c] = ms;
  }
  // The sample covers only the first steps, while later steps of a sequence
  // (a more entangled state) need larger Krylov spaces: take the largest depth
  // within 10% of the fastest sample time.
  float best_ms = 1e30f;
  for (int c = 0; c < ncand; ++c) best_ms = std::min(best_ms, cand_ms[c]);
  int best = b->cfg.m_max;
  for (int c = 0; c < ncand; ++c)
    if (cand_ms[c] <= 1.10f * best_ms) best = cand[c];
  b->cfg.m_max = best;
  b->tuned_ms = best_ms;
  // shrink the workspace to the chosen depth
  const int64_t stride = (int64_t)(best + 1) << b->nmax;
  if (stride < b->work_stride) {
    const size_t bytes = (size_t)stride * b->grid * amp_bytes(b->cfg.precision);
    void* w = nullptr;
    if (b->ctx->arena.alloc(bytes, &w) == RSV_OK) {
      b->ctx->arena.release(b->d_work);
      b->allocs.erase(std::find(b->allocs.begin(), b->allocs.end(), b->d_work));
      b->allocs.push_back(w);
      b->d_work = w;
      b->work_stride = stride;
    }
  }
  return RSV_OK;
}

rsv_status batch_capture(rsv_batch* b) {
  const size_t sbytes = b->state_amps * amp_bytes(b->cfg.precision);
  RSV_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemcpyAsync(b->d_states, b->d_init, sbytes, cudaMemcpyDeviceToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_next, 0, sizeof(int) * 2, b->stream);
  if (e == cudaSuccess) e = launch_batch(b->args(), b->c64, b->grid, b->stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(RSV_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  b->graph = g;
  RSV_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
  return RSV_OK;
}

}  // namespace

extern "C" {

rsv_status rsv_batch_create(rsv_ctx* ctx, const rsv_problem* problems, int32_t count, const rsv_config* config,
                            rsv_batch** out) {
  g_last_error.clear();
  if (!ctx || !problems || !config || !out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (count < 1) return fail(RSV_ERR_INVALID_ARG, "count must be >= 1");
  rsv_config cfg = *config;
  if (cfg.dt_ns < 1) return fail(RSV_ERR_INVALID_ARG, "dt_ns must be >= 1");
  if (cfg.precision != RSV_C64 && cfg.precision != RSV_C128) return fail(RSV_ERR_INVALID_ARG, "bad precision");
  const bool tune_m = cfg.m_max < 0;
  if (cfg.m_max == 0) cfg.m_max = 30;
  if (tune_m) cfg.m_max = kBatchTuneMax;
  if (cfg.m_max < 2 || cfg.m_max > kMaxKrylov) return fail(RSV_ERR_INVALID_ARG, "m_max must be in [2, 64]");
  if (cfg.krylov_tol <= 0.0) cfg.krylov_tol = cfg.precision == RSV_C64 ? 1e-7 : 1e-12;
  if (cfg.max_substeps <= 0) cfg.max_substeps = 64;
  if (cfg.obs_stride < 0) return fail(RSV_ERR_INVALID_ARG, "obs_stride must be >= 0");
  const int64_t ab = amp_bytes(cfg.precision);
  std::unique_ptr<rsv_batch> b(new rsv_batch());
  b->ctx = ctx;
  b->count = count;
  b->cfg = cfg;
  b->c64 = cfg.precision == RSV_C64;
  // host tables
  std::vector<double> params, vmat;
  std::vector<char> init;
  size_t occ_doubles = 0;
  b->items.resize(count);
  for (int r = 0; r < count; ++r) {
    const rsv_problem* p = problems + r;
    RSV_TRY(validate_problem(p));
    const int n = p->n_atoms;
    if (n > kBatchMaxAtoms)
      return fail(RSV_ERR_INVALID_ARG, "problem " + std::to_string(r) + ": n_atoms = " + std::to_string(n) +
                                           " exceeds the batched limit of " + std::to_string(kBatchMaxAtoms));
    std::vector<double> v_atoms;
    RSV_TRY(pair_energies(n, p->dim, p->positions_um, p->c6, v_atoms));
    std::vector<StepParams> sp;
    RSV_TRY(step_params(p, cfg.dt_ns, sp));
    BatchItem& it = b->items[r];
    std::memset(&it, 0, sizeof(it));
    it.n = n;
    it.steps = (int)sp.size();
    it.obs_stride = cfg.obs_stride;
    it.has_phi = any_phi(sp, n) ? 1 : 0;
    it.occ_rows = (cfg.obs_stride > 0 ? it.steps / cfg.obs_stride : 0) + 2;
    it.state_off = (int64_t)b->state_amps;
    it.param_off = (int64_t)params.size();
    it.vmat_off = (int64_t)vmat.size();
    it.occ_off = (int64_t)occ_doubles;
    for (const StepParams& s : sp) {
      params.push_back(s.tau);
      for (int q = 0; q < n; ++q) params.push_back(2.0 * s.half_omega[q]);
      for (int q = 0; q < n; ++q) params.push_back(s.delta[q]);
      for (int q = 0; q < n; ++q) params.push_back(s.phi[q]);
    }
    for (int q = 0; q < n; ++q)
      for (int r2 = 0; r2 < n; ++r2) vmat.push_back(v_atoms[(size_t)(n - 1 - q) * n + (n - 1 - r2)]);
    occ_doubles += (size_t)it.occ_rows * n;
    const size_t D = size_t(1) << n;
    const size_t old = init.size();
    init.resize(old + D * ab, 0);
    if (p->initial_state) {
      std::memcpy(init.data() + old, p->initial_state, D * ab);
    } else if (b->c64) {
      const float one = 1.0f;
      std::memcpy(init.data() + old, &one, sizeof(float));
    } else {
      const double one = 1.0;
      std::memcpy(init.data() + old, &one, sizeof(double));
    }
    b->state_amps += D;
    b->nmax = std::max(b->nmax, n);
  }
  // largest registers first
  b->order.resize(count);
  for (int r = 0; r < count; ++r) b->order[r] = r;
  // registers of kBatchCoopAtoms or more atoms first (each solved by a whole
  // cluster), then the rest; largest work first within each group
  auto large = [&](int x) { return b->items[x].n >= kBatchCoopAtoms; };
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
    if (large(x) != large(y)) return large(x);
    const int64_t wx = (int64_t)b->items[x].steps << b->items[x].n, wy = (int64_t)b->items[y].steps << b->items[y].n;
    return wx > wy;
  });
  for (int r = 0; r < count; ++r) b->count_large += large(r) ? 1 : 0;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  int max_clusters = 0;
  b->blocks_per_sm = batch_prepare(b->c64, b->count_large > 0 ? kBatchCluster : 1, &max_clusters);
  if (b->blocks_per_sm < 1) return fail(RSV_ERR_CUDA, "batched kernel does not fit on an SM");
  if (b->count_large > 0 && max_clusters > 0) {
    b->cluster = kBatchCluster;
    const int want = (count + kBatchCluster - 1) / kBatchCluster;
    b->grid = std::min(want, max_clusters) * kBatchCluster;
  } else {
    b->count_large = 0;  // no cluster launch possible: every register on one CTA
    b->grid = std::min(count, b->blocks_per_sm * ctx->num_sms);
  }
  b->work_stride = (int64_t)(cfg.m_max + 1) << b->nmax;
  rsv_status st = RSV_OK;
  auto A = [&](size_t bytes, void** p) {
    if (st == RSV_OK) st = b->alloc(std::max<size_t>(bytes, 16), p);
  };
  A(sizeof(BatchItem) * count, (void**)&b->d_items);
  A(sizeof(int) * count, (void**)&b->d_order);
  A(sizeof(int) * 2, (void**)&b->d_next);
  A(b->state_amps * ab, &b->d_states);
  A(b->state_amps * ab, &b->d_init);
  A(sizeof(double) * params.size(), (void**)&b->d_params);
  A(sizeof(double) * vmat.size(), (void**)&b->d_vmat);
  A(sizeof(double) * occ_doubles, (void**)&b->d_occ);
  A(sizeof(BatchOut) * count, (void**)&b->d_out);
  A((size_t)b->work_stride * b->grid * ab, &b->d_work);
  if (st != RSV_OK) return st;
  RSV_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
  RSV_CUDA(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
  RSV_CUDA(cudaEventCreate(&b->ev0));
  RSV_CUDA(cudaEventCreate(&b->ev1));
  RSV_CUDA(cudaMemcpyAsync(b->d_items, b->items.data(), sizeof(BatchItem) * count, cudaMemcpyHostToDevice, b->stream));
  RSV_CUDA(cudaMemcpyAsync(b->d_order, b->order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, b->stream));
  RSV_CUDA(cudaMemcpyAsync(b->d_init, init.data(), init.size(), cudaMemcpyHostToDevice, b->stream));
  RSV_CUDA(cudaMemcpyAsync(b->d_params, params.data(), sizeof(double) * params.size(), cudaMemcpyHostToDevice,
                           b->stream));
  RSV_CUDA(cudaMemcpyAsync(b->d_vmat, vmat.data(), sizeof(double) * vmat.size(), cudaMemcpyHostToDevice, b->stream));
  RSV_CUDA(cudaMemsetAsync(b->d_occ, 0, sizeof(double) * std::max<size_t>(occ_doubles, 1), b->stream));
  RSV_CUDA(cudaStreamSynchronize(b->stream));
  if (tune_m) RSV_TRY(batch_tune_krylov(b.get()));
  RSV_TRY(batch_capture(b.get()));
  ctx->batches.insert(b.get());
  *out = b.release();
  return RSV_OK;
}

}  // extern "C"

// Replays the batch's graph and waits for it. `after_ctx`: first order it
// after the context stream's earlier work (the caller's inputs).
static rsv_status batch_run(rsv_batch* b, bool after_ctx) {
  cudaSetDevice(b->ctx->device);
  b->have_out = false;
  if (after_ctx) {
    RSV_CUDA(cudaEventRecord(b->ev_in, b->ctx->stream));
    RSV_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
  }
  RSV_CUDA(cudaEventRecord(b->ev0, b->stream));
  RSV_CUDA(cudaGraphLaunch(b->exec, b->stream));
  RSV_CUDA(cudaEventRecord(b->ev1, b->stream));
  b->out.resize(b->count);
  RSV_CUDA(cudaMemcpyAsync(b->out.data(), b->d_out, sizeof(BatchOut) * b->count, cudaMemcpyDeviceToHost, b->stream));
  RSV_CUDA(cudaStreamSynchronize(b->stream));
  RSV_CUDA(cudaEventElapsedTime(&b->last_ms, b->ev0, b->ev1));
  b->have_out = true;
  ++b->runs;
  for (int r = 0; r < b->count; ++r)
    if (b->out[r].status != 0)
      return fail(RSV_ERR_NOT_CONVERGED, "register " + std::to_string(r) + ": Krylov step needed more than " +
                                             std::to_string(b->cfg.max_substeps) + " substeps");
  return RSV_OK;
}

extern "C" {

rsv_status rsv_batch_run(rsv_batch* b) {
  g_last_error.clear();
  if (!b) return fail(RSV_ERR_INVALID_ARG, "NULL batch");
  std::lock_guard<std::mutex> lk(b->ctx->mu);
  return batch_run(b, true);
}

rsv_status rsv_batch_state_device(const rsv_batch* b, int32_t index, void** dev_ptr, size_t* bytes) {
  g_last_error.clear();
  if (!b || !dev_ptr || !bytes) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (index < 0 || index >= b->count) return fail(RSV_ERR_INVALID_ARG, "index out of range");
  const BatchItem& it = b->items[index];
  const int64_t ab = amp_bytes(b->cfg.precision);
  *dev_ptr = static_cast<char*>(b->d_states) + it.state_off * ab;
  *bytes = (size_t(1) << it.n) * ab;
  return RSV_OK;
}

rsv_status rsv_batch_state(const rsv_batch* b, int32_t index, void* host_dst, size_t bytes) {
  void* p = nullptr;
  size_t need = 0;
  RSV_TRY(rsv_batch_state_device(b, index, &p, &need));
  if (!host_dst || bytes < need) return fail(RSV_ERR_INVALID_ARG, "destination too small");
  RSV_CUDA(cudaMemcpyAsync(host_dst, p, need, cudaMemcpyDeviceToHost, b->stream));
  RSV_CUDA(cudaStreamSynchronize(b->stream));
  return RSV_OK;
}

rsv_status rsv_batch_occupations(const rsv_batch* b, int32_t index, double* dst, int32_t capacity_rows,
                                 int32_t* n_rows) {
  g_last_error.clear();
  if (!b || !n_rows) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (index < 0 || index >= b->count) return fail(RSV_ERR_INVALID_ARG, "index out of range");
  if (!b->have_out) return fail(RSV_ERR_INVALID_ARG, "batch has not run");
  const BatchItem& it = b->items[index];
  *n_rows = b->out[index].rows;
  if (dst) {
    const int rows = std::min(capacity_rows, b->out[index].rows);
    if (rows > 0) {
      RSV_CUDA(cudaMemcpyAsync(dst, b->d_occ + it.occ_off, sizeof(double) * rows * it.n, cudaMemcpyDeviceToHost,
                               b->stream));
      RSV_CUDA(cudaStreamSynchronize(b->stream));
    }
  }
  return RSV_OK;
}

rsv_status rsv_batch_stats(const rsv_batch* b, int32_t index, rsv_stats* out) {
  g_last_error.clear();
  if (!b || !out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (index < -1 || index >= b->count) return fail(RSV_ERR_INVALID_ARG, "index out of range");
  std::memset(out, 0, sizeof(*out));
  if (!b->have_out) return RSV_OK;
  for (int r = 0; r < b->count; ++r) {
    if (index >= 0 && r != index) continue;
    out->steps += b->out[r].status == 0 ? b->items[r].steps : 0;
    out->krylov_iterations += b->out[r].iterations;
    out->substeps += b->out[r].substeps;
    out->max_error_estimate = std::max(out->max_error_estimate, b->out[r].max_err);
  }
  out->seconds = b->last_ms * 1e-3;
  out->kernel_launches = b->runs;
  out->tile_passes = b->grid;
  out->krylov_dim_max = b->cfg.m_max;
  return RSV_OK;
}

void rsv_batch_destroy(rsv_batch* b) {
  if (!b) return;
  {
    std::lock_guard<std::mutex> lk(b->ctx->mu);
    b->ctx->batches.erase(b);
  }
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Shot-to-shot noise: perturbed copies of one problem, occupations averaged.
// ---------------------------------------------------------------------------
// Many problems in one call: registers of at most kBatchMaxAtoms atoms share
// one batched persistent launch (their results share the batch), larger ones
// run on the streaming solver one by one.
extern "C" rsv_status rsv_run_batch(rsv_ctx* ctx, const rsv_problem* problems, int32_t count,
                                    const rsv_config* config, rsv_result** outs) {
  g_last_error.clear();
  if (!ctx || !problems || !config || !outs) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (count < 1) return fail(RSV_ERR_INVALID_ARG, "count must be >= 1");
  for (int i = 0; i < count; ++i) outs[i] = nullptr;
  std::vector<int> small, large;
  for (int i = 0; i < count; ++i) {
    RSV_TRY(validate_problem(&problems[i]));
    (problems[i].n_atoms <= kBatchMaxAtoms ? small : large).push_back(i);
  }
  auto release = [&](rsv_status st) {
    for (int i = 0; i < count; ++i) {
      if (outs[i]) rsv_result_free(outs[i]);
      outs[i] = nullptr;
    }
    return st;
  };
  if (!small.empty()) {
    std::vector<rsv_problem> probs;
    for (int i : small) probs.push_back(problems[i]);
    rsv_batch* b = nullptr;
    rsv_status st = rsv_batch_create(ctx, probs.data(), (int32_t)probs.size(), config, &b);
    if (st == RSV_OK) st = rsv_batch_run(b);
    if (st != RSV_OK) {
      if (b) rsv_batch_destroy(b);
      return release(st);
    }
    std::shared_ptr<rsv_batch> holder(b, [](rsv_batch* p) { rsv_batch_destroy(p); });
    for (size_t k = 0; k < small.size(); ++k) {
      auto res = new rsv_result();
      res->ctx = ctx;
      res->n = probs[k].n_atoms;
      res->precision = config->precision;
      res->batch = holder;
      res->index = (int)k;
      int32_t rows = 0;
      rsv_batch_occupations(b, (int32_t)k, nullptr, 0, &rows);
      res->occ.resize((size_t)rows * res->n);
      rsv_batch_occupations(b, (int32_t)k, res->occ.data(), rows, &rows);
      res->rows = rows;
      {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->results.insert(res);
      }
      outs[small[k]] = res;
    }
  }
  rsv_config streaming = *config;
  if (streaming.m_max < 0) streaming.m_max = 0;  // the depth autotuner is the batch's; the solver takes its default
  for (int i : large) {
    const rsv_status st = rsv_run(ctx, &problems[i], &streaming, &outs[i]);
    if (st != RSV_OK) return release(st);
  }
  return RSV_OK;
}

extern "C" rsv_status rsv_run_shots(rsv_ctx* ctx, const rsv_problem* problem, const rsv_config* config,
                                    int32_t shots, const double* omega_scale, const double* delta_shift,
                                    const double* pos_shift_um, double* occ_mean, int32_t capacity_rows,
                                    int32_t* n_rows) {
  g_last_error.clear();
  if (!ctx || !config || !n_rows || !omega_scale || !delta_shift) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  RSV_TRY(validate_problem(problem));
  if (shots < 1) return fail(RSV_ERR_INVALID_ARG, "shots must be >= 1");
  if (config->dt_ns < 1) return fail(RSV_ERR_INVALID_ARG, "dt_ns must be >= 1");
  if (config->obs_stride < 0) return fail(RSV_ERR_INVALID_ARG, "obs_stride must be >= 0");
  const int n = problem->n_atoms, T = problem->t_ns, dim = problem->dim;
  const int steps = num_steps(T, config->dt_ns);
  const int stride = config->obs_stride;
  // rows recorded: t = 0, every stride-th step, and the end if not on a stride
  const int rows = 1 + (stride > 0 ? steps / stride : 0) + ((stride == 0 || steps % stride != 0) ? 1 : 0);
  if (!occ_mean) {
    *n_rows = rows;
    return RSV_OK;
  }
  // the perturbed copies (owned here for the duration of the call)
  std::vector<std::vector<double>> pos(shots), om(shots), de(shots);
  std::vector<rsv_problem> probs(shots);
  for (int k = 0; k < shots; ++k) {
    pos[k].assign(problem->positions_um, problem->positions_um + (size_t)n * dim);
    if (pos_shift_um)
      for (int i = 0; i < n * dim; ++i) pos[k][i] += pos_shift_um[(size_t)k * n * dim + i];
    om[k].assign(problem->omega, problem->omega + (size_t)problem->omega_rows * T);
    for (double& v : om[k]) v *= omega_scale[k];
    de[k].assign(problem->delta, problem->delta + (size_t)problem->delta_rows * T);
    for (double& v : de[k]) v += delta_shift[k];
    probs[k] = *problem;
    probs[k].positions_um = pos[k].data();
    probs[k].omega = om[k].data();
    probs[k].delta = de[k].data();
  }
  std::vector<double> sum((size_t)rows * n, 0.0);
  std::vector<double> buf((size_t)rows * n);
  int got_rows = rows;
  if (n <= kBatchMaxAtoms) {
    rsv_batch* b = nullptr;
    RSV_TRY(rsv_batch_create(ctx, probs.data(), shots, config, &b));
    rsv_status st = rsv_batch_run(b);
    for (int k = 0; k < shots && st == RSV_OK; ++k) {
      int32_t r = 0;
      st = rsv_batch_occupations(b, k, buf.data(), rows, &r);
      got_rows = std::min(got_rows, r);
      for (size_t i = 0; i < (size_t)r * n; ++i) sum[i] += buf[i];
    }
    rsv_batch_destroy(b);
    RSV_TRY(st);
  } else {
    for (int k = 0; k < shots; ++k) {
      rsv_result* r = nullptr;
      RSV_TRY(rsv_run(ctx, &probs[k], config, &r));
      int32_t nr = 0;
      const rsv_status st = rsv_result_occupations(r, buf.data(), rows, &nr);
      rsv_result_free(r);
      RSV_TRY(st);
      got_rows = std::min(got_rows, nr);
      for (size_t i = 0; i < (size_t)nr * n; ++i) sum[i] += buf[i];
    }
  }
  *n_rows = got_rows;
  const int r = std::min(capacity_rows, got_rows);
  for (size_t i = 0; i < (size_t)r * n; ++i) occ_mean[i] = sum[i] / shots;
  return RSV_OK;
}

// ---------------------------------------------------------------------------
// Pulse gradients (Sec. V: expectation values are differentiable with respect
// to the tensors that define the pulses), by the adjoint method.
//
// With psi_{k+1} = U_k psi_k, U_k = exp(-i tau_k H_k) (Eq. (6)) and an
// occupation observable O = sum_i w_i n_i, a parameter theta of H_k moves
// <O>(T) by 2 Re <lambda_{k+1}| dU_k/dtheta |psi_k>, lambda_K = O psi_K,
// lambda_k = U_k^dagger lambda_{k+1}. Duhamel's formula
//     dU_k/dtheta = -i int_0^tau U_k(tau - s) G U_k(s) ds,  G = dH_k/dtheta,
// turns it into 2 Im int_0^tau <lambda(s)| G |psi(s)> ds with lambda(s) and
// psi(s) both evolved from step k + 1 back to time s of step k. Conjugation
// makes those backward evolutions forward ones under conj(H_k) (H_k with the
// phases negated), so they run on the ordinary Lanczos path:
//     mu(s) = conj(lambda(s)) = exp(-i conj(H_k) (tau - s)) mu_{k+1},
//     nu(s) = conj(psi(s))    = exp(-i conj(H_k) (tau - s)) conj(psi_{k+1}).
// The integral is a composite Gauss-Legendre rule, 8 nodes per panel, taken
// from s = tau down to 0 in one sweep of both vectors; the forward states
// psi_k are kept (checkpoints) so nu restarts exactly at every step.
//
// Panels: for f(s) = <lambda_k| e^{iHs} G e^{-iHs} |psi_k> the 2Q-th
// derivative is bounded by W^{2Q} |G| |lambda| |psi|, W the spectral width of
// H_k (|ad_H| = W). The Q-point Gauss-Legendre error on a panel of width h is
// h^{2Q+1} (Q!)^4 / ((2Q + 1) ((2Q)!)^3) times that bound, about
// 1.7e-23 (W h)^16 relative for Q = 8, below 1e-13 while W h <= 4. W is bounded
// by Gershgorin: W <= sum_{i<j} V_ij + sum_i |delta_i| + sum_i |Omega_i|.
// ---------------------------------------------------------------------------
namespace {

constexpr int kGradNodesPerPanel = 8;
constexpr int kGradMaxPanels = 4096;

// Gauss-Legendre nodes (ascending) and weights on [-1, 1]: Newton's method on
// P_q from the three-term Legendre recurrence, with Tricomi's first guess.
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
  constexpr double kPi = 3.14159265358979323846;
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= q; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = q == 1 ? 1.0 : q * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) <= 1e-16) break;
    }
    x[q - 1 - i] = z;
    w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

int gradient_panels(const StepParams& sp, const std::vector<double>& v_atoms, int n) {
  double width = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) width += std::fabs(v_atoms[(size_t)i * n + j]);
  for (int q = 0; q < n; ++q) width += std::fabs(sp.delta[q]) + 2.0 * std::fabs(sp.half_omega[q]);
  const double p = std::ceil(width * sp.tau / 4.0);
  return (int)std::min<double>(kGradMaxPanels, std::max(1.0, p));
}

}  // namespace

extern "C" rsv_status rsv_gradient(rsv_ctx* ctx, const rsv_problem* problem, const rsv_config* config,
                                   const double* weights, int32_t panels, double* value_out, double* d_omega,
                                   double* d_delta, double* d_phi, int64_t* nodes_out, rsv_stats* stats_out) {
  g_last_error.clear();
  if (!ctx || !config || !weights || !value_out || !d_omega || !d_delta) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  RSV_TRY(validate_problem(problem));
  if (panels < 0 || panels > kGradMaxPanels)
    return fail(RSV_ERR_INVALID_ARG, "panels must be in [0, " + std::to_string(kGradMaxPanels) + "]");
  if (config->dt_ns < 1) return fail(RSV_ERR_INVALID_ARG, "dt_ns must be >= 1");
  const int n = problem->n_atoms, T = problem->t_ns;
  rsv_config cfg = *config;
  cfg.obs_stride = 0;
  const int K = num_steps(T, cfg.dt_ns);
  for (size_t i = 0; i < (size_t)problem->omega_rows * T; ++i) d_omega[i] = 0.0;
  for (size_t i = 0; i < (size_t)problem->delta_rows * T; ++i) d_delta[i] = 0.0;
  if (d_phi)
    for (size_t i = 0; i < (size_t)problem->phi_rows * T; ++i) d_phi[i] = 0.0;
  std::vector<double> v_atoms;
  RSV_TRY(pair_energies(n, problem->dim, problem->positions_um, problem->c6, v_atoms));
  std::vector<StepParams> sp;
  RSV_TRY(step_params(problem, cfg.dt_ns, sp));

  // everything the call holds on the device, released on every exit path
  struct Held {
    rsv_ctx* ctx;
    std::vector<rsv_solver*> solvers;
    std::vector<void*> bufs;
    ~Held() {
      for (rsv_solver* s : solvers) rsv_solver_destroy(s);
      if (!bufs.empty()) cudaStreamSynchronize(ctx->stream);
      for (void* p : bufs) ctx->arena.release(p);
    }
  } held{ctx, {}, {}};
  auto alloc = [&](size_t bytes, void** p) -> rsv_status {
    RSV_TRY(ctx->arena.alloc(bytes, p));
    held.bufs.push_back(*p);
    return RSV_OK;
  };
  const bool c64 = cfg.precision == RSV_C64;
  const int64_t dim = int64_t(1) << n;
  const size_t vbytes = (size_t)dim * amp_bytes(cfg.precision);
  std::vector<void*> ckpt(K + 1, nullptr);
  for (int k = 0; k <= K; ++k) {
    const rsv_status st = alloc(vbytes, &ckpt[k]);
    if (st != RSV_OK)
      return fail(st, "gradient checkpoints (" + std::to_string(K + 1) + " states of " + std::to_string(vbytes) +
                          " bytes) do not fit the arena");
  }
  const int64_t nvec = c64 ? dim / 2 : dim;
  const int nchunks = (int)std::max<int64_t>(
      1, std::min<int64_t>((nvec + kThreads - 1) / kThreads, (4 * ctx->num_sms + n - 1) / n));
  double *d_acc = nullptr, *d_wbits = nullptr, *d_gpart = nullptr;
  RSV_TRY(alloc(sizeof(double) * 6 * n, (void**)&d_acc));
  RSV_TRY(alloc(sizeof(double) * n, (void**)&d_wbits));
  RSV_TRY(alloc(sizeof(double) * 6 * n * (size_t)nchunks, (void**)&d_gpart));
  std::vector<double> wbits(n);
  for (int i = 0; i < n; ++i) wbits[n - 1 - i] = weights[i];  // atom i sits at bit n - 1 - i
  rsv_stats total{};
  auto add_stats = [&](const rsv_solver* s) {
    total.krylov_iterations += s->stats.krylov_iterations;
    total.substeps += s->stats.substeps;
    total.kernel_launches += s->stats.kernel_launches;
    total.max_error_estimate = std::max(total.max_error_estimate, s->stats.max_error_estimate);
  };
  const auto t0 = std::chrono::steady_clock::now();

  // forward sweep, keeping psi_0 .. psi_K
  rsv_solver* F = nullptr;
  RSV_TRY(solver_create(ctx, problem, &cfg, nullptr, &F));
  held.solvers.push_back(F);
  double value = 0.0;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    RSV_CUDA(cudaMemcpyAsync(d_wbits, wbits.data(), sizeof(double) * n, cudaMemcpyHostToDevice, F->stream));
    RSV_CUDA(cudaMemcpyAsync(ckpt[0], F->d_psi, vbytes, cudaMemcpyDeviceToDevice, F->stream));
    for (int k = 0; k < K; ++k) {
      RSV_TRY(F->step_once());
      RSV_CUDA(cudaMemcpyAsync(ckpt[k + 1], F->d_psi, vbytes, cudaMemcpyDeviceToDevice, F->stream));
    }
    std::vector<double> occ(n);
    RSV_CUDA(cudaMemcpyAsync(occ.data(), F->d_occ + (size_t)(F->rows - 1) * n, sizeof(double) * n,
                             cudaMemcpyDeviceToHost, F->stream));
    RSV_CUDA(cudaStreamSynchronize(F->stream));
    for (int i = 0; i < n; ++i) value += weights[i] * occ[i];
  }
  add_stats(F);
  total.steps = K;
  *value_out = value;
  held.solvers.pop_back();
  rsv_solver_destroy(F);

  // backward sweep on the conjugated problem
  std::vector<double> neg_phi;
  rsv_problem back = *problem;
  back.initial_state = nullptr;
  if (problem->phi_rows > 0) {
    neg_phi.assign(problem->phi, problem->phi + (size_t)problem->phi_rows * T);
    for (double& v : neg_phi) v = -v;
    back.phi = neg_phi.data();
  }
  // mu and nu evolve independently between nodes: each on its own stream,
  // driven by its own host thread, joined before every generator pass
  rsv_solver *Bmu = nullptr, *Bnu = nullptr;
  auto make_back = [&](rsv_solver** out) -> rsv_status {
    cudaStream_t bs = nullptr;
    RSV_CUDA(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
    const rsv_status c = solver_create(ctx, &back, &cfg, bs, out);
    if (c != RSV_OK) {
      cudaStreamDestroy(bs);
      return c;
    }
    (*out)->own_stream = true;
    held.solvers.push_back(*out);
    return RSV_OK;
  };
  RSV_TRY(make_back(&Bmu));
  RSV_TRY(make_back(&Bnu));
  auto evolve_pair = [&](int k, double t) -> rsv_status {
    auto nu_side = std::async(std::launch::async, [&, k, t] {
      cudaSetDevice(ctx->device);
      rsv_status r = Bnu->evolve(k, t);
      if (r == RSV_OK && cudaStreamSynchronize(Bnu->stream) != cudaSuccess) r = RSV_ERR_CUDA;
      return r;
    });
    rsv_status a = Bmu->evolve(k, t);
    if (a == RSV_OK && cudaStreamSynchronize(Bmu->stream) != cudaSuccess) a = fail(RSV_ERR_CUDA, "stream sync failed");
    const rsv_status b = nu_side.get();
    RSV_TRY(a);
    if (b != RSV_OK) return fail(b, "backward evolution of the state failed");
    return RSV_OK;
  };
  std::vector<double> gx, gw;
  gauss_legendre(kGradNodesPerPanel, gx, gw);
  int64_t nodes = 0, launches = 0;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStream_t st = ctx->stream;
    const int grid = 4 * ctx->num_sms;
    // mu_K = O conj(psi_K); a vanishing costate leaves every derivative zero
    RSV_CUDA(launch_conj_weight(ckpt[K], Bmu->d_psi, dim, c64, n, d_wbits, grid, Bmu->stream));
    launches += 1;
    RSV_TRY(Bmu->observe_into_partials());
    RSV_TRY(Bmu->begin(0.0, 1, nullptr));
    RSV_TRY(Bmu->read_status());
    const bool live = Bmu->h_ks->norm2 > 0.0;
    std::vector<double> acc(6 * n);
    cudaEvent_t read_done = nullptr;
    RSV_CUDA(cudaEventCreateWithFlags(&read_done, cudaEventDisableTiming));
    struct EventGuard {
      cudaEvent_t e;
      ~EventGuard() { cudaEventDestroy(e); }
    } read_done_guard{read_done};
    for (int k = K - 1; k >= 0 && live; --k) {
      const double tau = sp[k].tau;
      const int P = panels > 0 ? panels : gradient_panels(sp[k], v_atoms, n);
      // nodes s_j and weights w_j of the composite rule on [0, tau], ascending
      std::vector<double> s, w;
      for (int p = 0; p < P; ++p) {
        const double a = tau * p / P, h = tau / P;
        for (int j = 0; j < kGradNodesPerPanel; ++j) {
          s.push_back(a + 0.5 * h * (1.0 + gx[j]));
          w.push_back(0.5 * h * gw[j]);
        }
      }
      nodes += (int64_t)s.size();
      RSV_CUDA(launch_conj_weight(ckpt[k + 1], Bnu->d_psi, dim, c64, n, nullptr, grid, Bnu->stream));
      launches += 1 + 2 * (int64_t)s.size();
      RSV_TRY(Bnu->observe_into_partials());
      RSV_CUDA(cudaMemsetAsync(d_acc, 0, sizeof(double) * 6 * n, st));
      double at = tau;
      for (int j = (int)s.size() - 1; j >= 0; --j) {
        const double step = at - s[j];
        if (step > 0.0) RSV_TRY(evolve_pair(k, step));
        at = s[j];
        RSV_CUDA(launch_generator(Bmu->d_psi, Bnu->d_psi, dim, c64, n, nchunks, d_gpart, w[j], d_acc, st));
        // the next evolutions overwrite what this pass reads
        RSV_CUDA(cudaEventRecord(read_done, st));
        RSV_CUDA(cudaStreamWaitEvent(Bmu->stream, read_done, 0));
        RSV_CUDA(cudaStreamWaitEvent(Bnu->stream, read_done, 0));
      }
      if (at > 0.0) RSV_TRY(Bmu->evolve(k, at));  // mu_k, the next step's costate
      RSV_CUDA(cudaStreamSynchronize(Bmu->stream));
      RSV_CUDA(cudaMemcpyAsync(acc.data(), d_acc, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, st));
      RSV_CUDA(cudaStreamSynchronize(st));
      // the step's samples under the midpoint rule, weight 1/2 each
      const int start = k * cfg.dt_ns, len = std::min(cfg.dt_ns, T - start);
      const int twice_m = 2 * start + len;
      const int lo = std::min(twice_m / 2, T - 1), hi = std::min((twice_m + 1) / 2, T - 1);
      for (int i = 0; i < n; ++i) {
        const int q = n - 1 - i;
        const std::complex<double> s0(acc[6 * q + 0], acc[6 * q + 1]), s1(acc[6 * q + 2], acc[6 * q + 3]),
            dd(acc[6 * q + 4], acc[6 * q + 5]);
        const double phase = sp[k].phi[q], om = 2.0 * sp[k].half_omega[q];
        const std::complex<double> e(std::cos(phase), std::sin(phase)), I(0.0, 1.0);
        // <0|dh/dOmega|1> = e/2, <1|dh/dOmega|0> = conj(e)/2; dh/ddelta = -n;
        // <0|dh/dphi|1> = i Omega/2 e, <1|dh/dphi|0> = -i Omega/2 conj(e)
        const double g_om = 2.0 * std::imag(0.5 * e * s0 + 0.5 * std::conj(e) * s1);
        const double g_de = 2.0 * std::imag(-dd);
        const double g_ph = 2.0 * std::imag(I * (0.5 * om) * (e * s0 - std::conj(e) * s1));
        double* ro = d_omega + (size_t)(problem->omega_rows == 1 ? 0 : i) * T;
        double* rd = d_delta + (size_t)(problem->delta_rows == 1 ? 0 : i) * T;
        ro[lo] += 0.5 * g_om;
        ro[hi] += 0.5 * g_om;
        rd[lo] += 0.5 * g_de;
        rd[hi] += 0.5 * g_de;
        if (d_phi && problem->phi_rows > 0) {
          double* rp = d_phi + (size_t)(problem->phi_rows == 1 ? 0 : i) * T;
          rp[lo] += 0.5 * g_ph;
          rp[hi] += 0.5 * g_ph;
        }
      }
    }
  }
  add_stats(Bmu);
  add_stats(Bnu);
  total.kernel_launches += launches;
  total.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  total.tile_passes = Bmu->plan.two_pass ? 2 : 1;
  total.krylov_dim_max = cfg.m_max;
  if (nodes_out) *nodes_out = nodes;
  if (stats_out) *stats_out = total;
  return RSV_OK;
}

// The error path of the bounded device waits, end to end: a kernel waits on a
// barrier nothing completes, gives up, sets an error word, and this call
// reports RSV_ERR_TIMEOUT the way every streaming pass's caller does.
extern "C" rsv_status rsv_check_bounded_wait(rsv_ctx* ctx) {
  g_last_error.clear();
  if (!ctx) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  int* d_err = reinterpret_cast<int*>(ctx->d_part);
  int err = 0;
  RSV_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), ctx->stream));
  RSV_CUDA(launch_wait_check(d_err, ctx->stream));
  RSV_CUDA(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RSV_CUDA(cudaStreamSynchronize(ctx->stream));
  if (err) return fail(RSV_ERR_TIMEOUT, "a device-side wait timed out (kernel aborted)");
  return RSV_OK;
}

// Overlap <a|b> with |a|^2 and |b|^2 (fidelity with a target state).
extern "C" rsv_status rsv_overlap(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const void* a_dev,
                                  const void* b_dev, double* out) {
  g_last_error.clear();
  if (!ctx || !a_dev || !b_dev || !out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  if (n_atoms < 1 || n_atoms > 31) return fail(RSV_ERR_INVALID_ARG, "n_atoms out of range");
  if (precision != RSV_C64 && precision != RSV_C128) return fail(RSV_ERR_INVALID_ARG, "bad precision");
  if ((reinterpret_cast<uintptr_t>(a_dev) | reinterpret_cast<uintptr_t>(b_dev)) & 15)
    return fail(RSV_ERR_INVALID_ARG, "states must be 16-byte aligned");
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  const int grid = 4 * ctx->num_sms;
  RSV_CUDA(launch_overlap(a_dev, b_dev, int64_t(1) << n_atoms, precision == RSV_C64, ctx->d_part, grid, ctx->stream));
  std::vector<double> part((size_t)grid * 4);
  RSV_CUDA(cudaMemcpyAsync(part.data(), ctx->d_part, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
  RSV_CUDA(cudaStreamSynchronize(ctx->stream));
  double sum[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < grid; ++b)
    for (int v = 0; v < 4; ++v) sum[v] += part[(size_t)b * 4 + v];
  for (int v = 0; v < 4; ++v) out[v] = sum[v];
  return RSV_OK;
}

// Fidelity |<a|b>|^2 / (|a|^2 |b|^2) from the overlap sums.
extern "C" rsv_status rsv_fidelity(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const void* a_dev,
                                   const void* b_dev, double* out) {
  if (!out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  double ov[4];
  RSV_TRY(rsv_overlap(ctx, n_atoms, precision, a_dev, b_dev, ov));
  if (!(ov[2] > 0.0) || !(ov[3] > 0.0)) return fail(RSV_ERR_INVALID_ARG, "a state has zero norm");
  *out = (ov[0] * ov[0] + ov[1] * ov[1]) / (ov[2] * ov[3]);
  return RSV_OK;
}

// ---------------------------------------------------------------------------
// Open-system dynamics (Sec. III.A): the Lindblad master equation, evolved
// step by step with the midpoint pulses of Sec. III by a Krylov exponential of
// the Liouvillian on vec(rho). The Liouvillian is not Hermitian, so the
// Krylov process is Arnoldi (classical Gram-Schmidt, twice) in place of
// Lanczos' three-term recurrence. The acceptance test is the same a-posteriori
// estimate: h_{m+1,m} |[exp(tau H_m) e_1]_{m-1}| <= p, with a step split by
// halving when m_max is reached.
// ---------------------------------------------------------------------------
namespace {

using cplx = std::complex<double>;

// exp(t A) e_1 for a small complex m x m matrix (row-major): scaling and
// squaring of a truncated Taylor series (Moler and Van Loan, "Nineteen
// dubious ways to compute the exponential of a matrix", method 3), with the
// scaled norm at most 1/2 so the series stops below 1e-18 relative.
std::vector<cplx> small_expm_e1(const std::vector<cplx>& A, int lda, int m, double t) {
  double nrm = 0.0;
  for (int j = 0; j < m; ++j) {
    double col = 0.0;
    for (int i = 0; i < m; ++i) col += std::abs(A[(size_t)i * lda + j]);
    nrm = std::max(nrm, col);
  }
  nrm *= std::fabs(t);
  int sq = 0;
  while (nrm > 0.5 && sq < 200) {
    nrm *= 0.5;
    ++sq;
  }
  const double scale = std::ldexp(t, -sq);
  std::vector<cplx> X((size_t)m * m), R((size_t)m * m, 0.0), term((size_t)m * m, 0.0), tmp((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) X[(size_t)i * m + j] = scale * A[(size_t)i * lda + j];
  for (int i = 0; i < m; ++i) R[(size_t)i * m + i] = term[(size_t)i * m + i] = 1.0;
  auto matmul = [&](const std::vector<cplx>& a, const std::vector<cplx>& b, std::vector<cplx>& c) {
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        cplx acc = 0.0;
        for (int k = 0; k < m; ++k) acc += a[(size_t)i * m + k] * b[(size_t)k * m + j];
        c[(size_t)i * m + j] = acc;
      }
  };
  for (int k = 1; k <= 40; ++k) {
    matmul(term, X, tmp);
    double tn = 0.0, rn = 0.0;
    for (size_t e = 0; e < tmp.size(); ++e) {
      term[e] = tmp[e] / (double)k;
      R[e] += term[e];
      tn = std::max(tn, std::abs(term[e]));
      rn = std::max(rn, std::abs(R[e]));
    }
    if (tn <= 1e-18 * rn) break;
  }
  for (int s = 0; s < sq; ++s) {
    matmul(R, R, tmp);
    R.swap(tmp);
  }
  std::vector<cplx> u(m);
  for (int i = 0; i < m; ++i) u[i] = R[(size_t)i * m];
  return u;
}

}  // namespace

extern "C" rsv_status rsv_lindblad_run(rsv_ctx* ctx, const rsv_problem* problem, const rsv_config* config,
                                       const double* g_dephasing, const double* g_relaxation, const void* rho0,
                                       void* rho_out, double* occ_out, int32_t capacity_rows, int32_t* n_rows,
                                       rsv_stats* stats_out) {
  g_last_error.clear();
  if (!ctx || !config || !n_rows) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  RSV_TRY(validate_problem(problem));
  const int n = problem->n_atoms, T = problem->t_ns;
  if (n > kLindbladMaxAtoms)
    return fail(RSV_ERR_INVALID_ARG, "Lindblad evolution holds 4^n_atoms amplitudes: n_atoms must be <= " +
                                         std::to_string(kLindbladMaxAtoms));
  if (problem->initial_state)
    return fail(RSV_ERR_INVALID_ARG, "pass the initial density matrix as rho0 (problem->initial_state must be NULL)");
  rsv_config cfg = *config;
  if (cfg.dt_ns < 1) return fail(RSV_ERR_INVALID_ARG, "dt_ns must be >= 1");
  if (cfg.precision != RSV_C128 && cfg.precision != RSV_C64) return fail(RSV_ERR_INVALID_ARG, "bad precision");
  const bool c64 = cfg.precision == RSV_C64;
  if (cfg.m_max == 0) cfg.m_max = 30;
  if (cfg.m_max < 2 || cfg.m_max > kLindbladMaxKrylov)
    return fail(RSV_ERR_INVALID_ARG, "m_max must be in [2, " + std::to_string(kLindbladMaxKrylov) + "]");
  if (cfg.krylov_tol <= 0.0) cfg.krylov_tol = c64 ? 1e-7 : 1e-12;
  if (cfg.max_substeps <= 0) cfg.max_substeps = 64;
  if (cfg.obs_stride < 0) return fail(RSV_ERR_INVALID_ARG, "obs_stride must be >= 0");
  for (int i = 0; i < n; ++i) {
    const double a = g_dephasing ? g_dephasing[i] : 0.0, b = g_relaxation ? g_relaxation[i] : 0.0;
    if (!(a >= 0.0 && b >= 0.0 && std::isfinite(a) && std::isfinite(b)))
      return fail(RSV_ERR_INVALID_ARG, "noise rates must be finite and >= 0");
  }
  const int K = num_steps(T, cfg.dt_ns);
  const int stride = cfg.obs_stride;
  const int rows = 1 + (stride > 0 ? K / stride : 0) + ((stride == 0 || K % stride != 0) ? 1 : 0);
  *n_rows = rows;
  if (!occ_out && !rho_out) return RSV_OK;
  std::vector<double> v_atoms;
  RSV_TRY(pair_energies(n, problem->dim, problem->positions_um, problem->c6, v_atoms));
  std::vector<StepParams> sp;
  RSV_TRY(step_params(problem, cfg.dt_ns, sp));

  struct Held {
    rsv_ctx* ctx;
    std::vector<void*> bufs;
    ~Held() {
      if (!bufs.empty()) cudaStreamSynchronize(ctx->stream);
      for (void* p : bufs) ctx->arena.release(p);
    }
  } held{ctx, {}};
  auto alloc = [&](size_t bytes, void** p) -> rsv_status {
    RSV_TRY(ctx->arena.alloc(bytes, p));
    held.bufs.push_back(*p);
    return RSV_OK;
  };
  const int64_t dim = int64_t(1) << n, total = dim * dim;
  const size_t abytes = c64 ? 8 : 16;  // bytes per amplitude
  const size_t vbytes = (size_t)total * abytes;
  const int m_max = cfg.m_max;
  void *rho = nullptr, *w = nullptr;
  std::vector<void*> basis(m_max, nullptr);
  RSV_TRY(alloc(vbytes, &rho));
  RSV_TRY(alloc(vbytes, &w));
  for (int k = 0; k < m_max; ++k) RSV_TRY(alloc(vbytes, &basis[k]));
  // device pointer slots: basis 0 .. m_max - 1, then rho, then w
  void** d_ptrs = nullptr;
  void* d_E = nullptr;
  double *d_coef = nullptr, *d_dots = nullptr, *d_norm = nullptr, *d_part = nullptr;
  const int grid = 4 * ctx->num_sms;
  RSV_TRY(alloc(sizeof(void*) * (m_max + 2), (void**)&d_ptrs));
  RSV_TRY(alloc(sizeof(double) * dim, &d_E));
  RSV_TRY(alloc(sizeof(double) * 2 * m_max, (void**)&d_coef));
  RSV_TRY(alloc(sizeof(double) * 2 * m_max, (void**)&d_dots));
  RSV_TRY(alloc(sizeof(double), (void**)&d_norm));
  RSV_TRY(alloc(sizeof(double) * std::max<size_t>((size_t)grid * 2 * m_max, (size_t)grid), (void**)&d_part));

  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  const auto t0 = std::chrono::steady_clock::now();
  rsv_stats stats{};
  stats.krylov_dim_max = m_max;
  std::vector<void*> ptrs(basis);
  ptrs.push_back(rho);
  ptrs.push_back(w);
  void** const rho_slot = d_ptrs + m_max;
  void** const w_slot = d_ptrs + m_max + 1;
  RSV_CUDA(cudaMemcpyAsync(d_ptrs, ptrs.data(), sizeof(void*) * ptrs.size(), cudaMemcpyHostToDevice, st));
  if (rho0) {
    RSV_CUDA(cudaMemcpyAsync(rho, rho0, vbytes, cudaMemcpyHostToDevice, st));
  } else {
    RSV_CUDA(cudaMemsetAsync(rho, 0, vbytes, st));
    const double one_d[2] = {1.0, 0.0};
    const float one_f[2] = {1.f, 0.f};
    RSV_CUDA(cudaMemcpyAsync(rho, c64 ? (const void*)one_f : (const void*)one_d, abytes, cudaMemcpyHostToDevice, st));
  }
  int64_t launches = 0;
  auto nchunks_for = [&](int nvec) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((total + kThreads - 1) / kThreads, (grid + nvec - 1) / nvec));
  };
  // <V_k, x> for k < nvec (slots from `first`), to the host
  std::vector<double> dots(2 * m_max);
  auto multi_dot = [&](void** first, int nvec, const void* x) -> rsv_status {
    RSV_CUDA(launch_multi_dot((const void* const*)first, nvec, x, total, c64, nchunks_for(nvec), d_part, d_dots, st));
    launches += 2;
    RSV_CUDA(cudaMemcpyAsync(dots.data(), d_dots, sizeof(double) * 2 * nvec, cudaMemcpyDeviceToHost, st));
    RSV_CUDA(cudaStreamSynchronize(st));
    return RSV_OK;
  };
  // y = (overwrite ? 0 : y) - sum_k c_k V_k; returns |y|^2
  auto multi_axpy = [&](void** first, const std::vector<double>& c, int nvec, void* y, bool overwrite,
                        double* norm2) -> rsv_status {
    RSV_CUDA(cudaMemcpyAsync(d_coef, c.data(), sizeof(double) * 2 * nvec, cudaMemcpyHostToDevice, st));
    RSV_CUDA(launch_multi_axpy((const void* const*)first, d_coef, nvec, y, total, c64, overwrite, grid, d_part,
                               d_norm, st));
    launches += 2;
    if (norm2) {
      RSV_CUDA(cudaMemcpyAsync(norm2, d_norm, sizeof(double), cudaMemcpyDeviceToHost, st));
      RSV_CUDA(cudaStreamSynchronize(st));
    }
    return RSV_OK;
  };
  // occupation rows: tr(rho n_i) from the diagonal
  std::vector<double> diag(2 * dim);  // the diagonal's amplitudes, as bytes of the working precision
  int row = 0;
  auto record = [&]() -> rsv_status {
    if (row < capacity_rows && occ_out) {
      RSV_CUDA(cudaMemcpy2DAsync(diag.data(), abytes, rho, (size_t)(dim + 1) * abytes, abytes, (size_t)dim,
                                 cudaMemcpyDeviceToHost, st));
      RSV_CUDA(cudaStreamSynchronize(st));
      const float* df = reinterpret_cast<const float*>(diag.data());
      for (int i = 0; i < n; ++i) {
        const int q = n - 1 - i;
        double s = 0.0;
        for (int64_t r = 0; r < dim; ++r)
          if ((r >> q) & 1) s += c64 ? (double)df[2 * r] : diag[2 * r];
        occ_out[(size_t)row * n + i] = s;
      }
    }
    ++row;
    return RSV_OK;
  };
  RSV_TRY(record());

  // bit-order pair energies and rates
  std::vector<double> vb((size_t)n * n), E(dim);
  std::vector<float> Ef(c64 ? dim : 0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) vb[(size_t)(n - 1 - i) * n + (n - 1 - j)] = v_atoms[(size_t)i * n + j];
  LindbladParams lp{};
  lp.n = n;
  for (int i = 0; i < n; ++i) {
    lp.gd[n - 1 - i] = g_dephasing ? g_dephasing[i] : 0.0;
    lp.gr[n - 1 - i] = g_relaxation ? g_relaxation[i] : 0.0;
  }
  std::vector<cplx> H((size_t)(m_max + 1) * m_max);
  for (int k = 0; k < K; ++k) {
    // E(b) = E(b without its lowest bit q) - delta_q + sum_{p in the rest} V_qp
    E[0] = 0.0;
    for (int64_t b = 1; b < dim; ++b) {
      const int q = __builtin_ctzll((unsigned long long)b);
      const int64_t rest = b & (b - 1);
      double e = E[rest] - sp[k].delta[q];
      for (int64_t r2 = rest; r2; r2 &= r2 - 1) e += vb[(size_t)q * n + __builtin_ctzll((unsigned long long)r2)];
      E[b] = e;
    }
    if (c64) {
      for (int64_t b = 0; b < dim; ++b) Ef[b] = (float)E[b];
      RSV_CUDA(cudaMemcpyAsync(d_E, Ef.data(), sizeof(float) * dim, cudaMemcpyHostToDevice, st));
    } else {
      RSV_CUDA(cudaMemcpyAsync(d_E, E.data(), sizeof(double) * dim, cudaMemcpyHostToDevice, st));
    }
    for (int q = 0; q < n; ++q) {
      lp.hre[q] = sp[k].half_omega[q] * std::cos(sp[k].phi[q]);
      lp.him[q] = sp[k].half_omega[q] * std::sin(sp[k].phi[q]);
    }
    double tau_rem = sp[k].tau;
    int restarts = 0;
    while (tau_rem > 0.0) {
      RSV_TRY(multi_dot(rho_slot, 1, rho));
      const double beta0 = std::sqrt(std::max(0.0, dots[0]));
      if (!(beta0 > 0.0)) break;  // rho = 0 stays 0
      RSV_TRY(multi_axpy(rho_slot, {-1.0 / beta0, 0.0}, 1, basis[0], true, nullptr));
      std::fill(H.begin(), H.end(), cplx(0.0));
      int m = 0;
      double tau_taken = 0.0, err = 0.0;
      std::vector<cplx> u;
      for (int j = 0; j < m_max; ++j) {
        RSV_CUDA(launch_lindblad_apply(basis[j], w, d_E, lp, c64, grid, st));
        launches += 1;
        std::vector<double> c(2 * (j + 1));
        double norm2 = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
          RSV_TRY(multi_dot(d_ptrs, j + 1, w));
          for (int i = 0; i <= j; ++i) {
            H[(size_t)i * m_max + j] += cplx(dots[2 * i], dots[2 * i + 1]);
            c[2 * i] = dots[2 * i];
            c[2 * i + 1] = dots[2 * i + 1];
          }
          RSV_TRY(multi_axpy(d_ptrs, c, j + 1, w, false, pass == 1 ? &norm2 : nullptr));
        }
        const double hn = std::sqrt(std::max(0.0, norm2));
        H[(size_t)(j + 1) * m_max + j] = hn;
        double hmax = 0.0;
        for (int i = 0; i <= j + 1; ++i)
          for (int l = 0; l <= j; ++l) hmax = std::max(hmax, std::abs(H[(size_t)i * m_max + l]));
        u = small_expm_e1(H, m_max, j + 1, tau_rem);
        err = hn * std::abs(u[j]);
        if (hn <= 1e-13 * std::max(1.0, hmax) || err <= cfg.krylov_tol) {
          m = j + 1;
          tau_taken = tau_rem;
          break;
        }
        if (j == m_max - 1) {
          double t = tau_rem;
          for (int h = 0; h < 200 && err > cfg.krylov_tol; ++h) {
            t *= 0.5;
            u = small_expm_e1(H, m_max, j + 1, t);
            err = hn * std::abs(u[j]);
          }
          if (err > cfg.krylov_tol)
            return fail(RSV_ERR_NOT_CONVERGED, "Arnoldi space did not reach the tolerance (non-finite values?)");
          m = j + 1;
          tau_taken = t;
          break;
        }
        RSV_TRY(multi_axpy(w_slot, {-1.0 / hn, 0.0}, 1, basis[j + 1], true, nullptr));
      }
      std::vector<double> c(2 * m);
      for (int i = 0; i < m; ++i) {
        c[2 * i] = -beta0 * u[i].real();
        c[2 * i + 1] = -beta0 * u[i].imag();
      }
      RSV_TRY(multi_axpy(d_ptrs, c, m, rho, true, nullptr));
      stats.krylov_iterations += m;
      stats.max_error_estimate = std::max(stats.max_error_estimate, err);
      tau_rem -= tau_taken;
      if (tau_rem <= 1e-15 * sp[k].tau) break;
      if (++restarts > cfg.max_substeps)
        return fail(RSV_ERR_NOT_CONVERGED, "step " + std::to_string(k) + " needed more than max_substeps restarts");
      stats.substeps += 1;
    }
    stats.steps += 1;
    if ((stride > 0 && (k + 1) % stride == 0) || k + 1 == K) RSV_TRY(record());
  }
  if (rho_out) RSV_CUDA(cudaMemcpyAsync(rho_out, rho, vbytes, cudaMemcpyDeviceToHost, st));
  RSV_CUDA(cudaStreamSynchronize(st));
  stats.kernel_launches = launches;
  stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  stats.tile_passes = 1;
  *n_rows = row;
  if (stats_out) *stats_out = stats;
  return RSV_OK;
}

// ---------------------------------------------------------------------------
// Serving: requests are admitted by device-memory footprint; each admitted
// solve runs on a worker thread with its own CUDA stream, so solves of
// different requests overlap on the device.
// ---------------------------------------------------------------------------
namespace {

struct ServeRequest {
  uint64_t ticket = 0;
  std::vector<double> pos, om, de, ph;
  std::vector<char> init;
  rsv_problem prob{};
  rsv_config cfg{};
  size_t bytes = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  rsv_status status = RSV_OK;
  std::string error;
  rsv_result* result = nullptr;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
};

}  // namespace

constexpr int kServeBatchMax = 64;  // requests per batched launch

struct rsv_server {
  rsv_ctx* ctx = nullptr;
  int slots = 0;
  int batch_atoms = 0;  // 0: every request on the streaming solver
  size_t budget = 0;
  // admitted bytes: running requests' footprints plus what finished results
  // still hold until they are freed (shared with those results)
  std::shared_ptr<ServeLedger> ledger = std::make_shared<ServeLedger>();
  size_t& in_use = ledger->in_use;
  std::mutex& mu = ledger->mu;
  std::condition_variable& cv_work = ledger->cv_work;
  double max_bypass_s = 0.5;
  std::condition_variable cv_done;
  std::deque<ServeRequest*> queue;
  std::map<uint64_t, std::unique_ptr<ServeRequest>> reqs;
  uint64_t next_ticket = 1;
  int running = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  const std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }

  // The first queued request that fits; requests behind a head that does not
  // fit may pass it only while it has waited less than max_bypass_s.
  std::deque<ServeRequest*>::iterator pick() {
    if (queue.empty()) return queue.end();
    const size_t room = budget - in_use;
    auto head = queue.begin();
    if ((*head)->bytes <= room) return head;
    if (max_bypass_s < 0.0 || now() - (*head)->t_submit >= max_bypass_s) return queue.end();
    for (auto it = std::next(head); it != queue.end(); ++it)
      if ((*it)->bytes <= room) return it;
    return queue.end();
  }

  // Requests of up to batch_atoms atoms with the same config are taken from the
  // queue together and solved by one batched-kernel launch (every step on the
  // device, no host round trip per iteration); sizes and durations may differ,
  // since each register of a batch runs its own sequence. A request with no
  // such companion queued runs on the streaming solver, which is faster for a
  // single register than a batch of one.
  // complex64 only: a complex128 batch runs FP64 arithmetic on one CTA (or one
  // 4-CTA cluster) per register, which on this part is far slower than the
  // streaming solver spread over every SM.
  bool batchable(const ServeRequest* r) const {
    return r->prob.n_atoms <= batch_atoms && r->cfg.precision == RSV_C64;
  }
  static bool same_class(const ServeRequest* a, const ServeRequest* b) {
    return std::memcmp(&a->cfg, &b->cfg, sizeof(rsv_config)) == 0;
  }

  // Solves a group of like requests in one batched launch. On success the
  // group's footprint stays charged until its last result is freed (the
  // shared batch's deleter releases it); `charged_out` is set to that sum.
  rsv_status serve_group(const std::vector<ServeRequest*>& g, std::vector<rsv_result*>& out, size_t* charged_out) {
    std::vector<rsv_problem> probs;
    size_t group_bytes = 0;
    for (const ServeRequest* q : g) {
      probs.push_back(q->prob);
      group_bytes += q->bytes;
    }
    rsv_batch* b = nullptr;
    rsv_status st = rsv_batch_create(ctx, probs.data(), (int32_t)g.size(), &g[0]->cfg, &b);
    if (st == RSV_OK) st = batch_run(b, false);
    if (st != RSV_OK) {
      if (b) rsv_batch_destroy(b);
      return st;
    }
    std::shared_ptr<ServeLedger> led = ledger;
    std::shared_ptr<rsv_batch> holder(b, [led, group_bytes](rsv_batch* p) {
      rsv_batch_destroy(p);
      led->release(group_bytes);
    });
    *charged_out = group_bytes;
    for (size_t i = 0; i < g.size(); ++i) {
      auto res = new rsv_result();
      res->ctx = ctx;
      res->n = g[i]->prob.n_atoms;
      res->precision = g[i]->cfg.precision;
      res->batch = holder;
      res->index = (int)i;
      int32_t rows = 0;
      rsv_batch_occupations(b, (int32_t)i, nullptr, 0, &rows);
      res->occ.resize((size_t)rows * res->n);
      rsv_batch_occupations(b, (int32_t)i, res->occ.data(), rows, &rows);
      res->rows = rows;
      {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->results.insert(res);
      }
      out[i] = res;
    }
    return RSV_OK;
  }

  rsv_status serve(ServeRequest* r, rsv_result** out) {
    cudaStream_t st = nullptr;
    RSV_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    rsv_solver* s = nullptr;
    const rsv_status c = solver_create(ctx, &r->prob, &r->cfg, st, &s, /*one_shot=*/true);
    if (c != RSV_OK) {
      cudaStreamDestroy(st);
      return c;
    }
    s->own_stream = true;
    const rsv_status k = solver_step(s, s->nsteps);
    if (k != RSV_OK) {
      rsv_solver_destroy(s);
      return k;
    }
    RSV_TRY(make_result(s, out));
    // the result only needs the final state: give the Krylov basis, work
    // vectors and tables back now, and keep the state charged until it is freed
    s->trim_to_state();
    (*out)->ledger = ledger;
    (*out)->charged = s->state_alloc_bytes();
    return RSV_OK;
  }

  void worker() {
    cudaSetDevice(ctx->device);
    for (;;) {
      std::vector<ServeRequest*> g;
      {
        std::unique_lock<std::mutex> lk(mu);
        // a bypass window closing changes pick(): re-check at least every 50 ms
        while (!stop && pick() == queue.end()) cv_work.wait_for(lk, std::chrono::milliseconds(50));
        if (stop) return;
        auto it = pick();
        g.push_back(*it);
        queue.erase(it);
        in_use += g[0]->bytes;
        if (batchable(g[0])) {
          for (auto jt = queue.begin(); jt != queue.end() && (int)g.size() < kServeBatchMax;) {
            ServeRequest* q = *jt;
            if (batchable(q) && same_class(q, g[0]) && q->bytes <= budget - in_use) {
              in_use += q->bytes;
              g.push_back(q);
              jt = queue.erase(jt);
            } else {
              ++jt;
            }
          }
        }
        const double t = now();
        for (ServeRequest* q : g) {
          q->state = 1;
          q->t_admit = t;
        }
        running += (int)g.size();
      }
      std::vector<rsv_result*> res(g.size(), nullptr);
      size_t group_charge = 0;  // equals the sum of the group's footprints
      const bool grouped = g.size() > 1;
      const rsv_status st = grouped ? serve_group(g, res, &group_charge) : serve(g[0], &res[0]);
      const std::string err = st == RSV_OK ? std::string() : g_last_error;
      {
        std::lock_guard<std::mutex> lk(mu);
        const double t = now();
        for (size_t i = 0; i < g.size(); ++i) {
          ServeRequest* q = g[i];
          q->t_done = t;
          q->status = st;
          q->error = err;
          q->result = res[i];
          if (res[i]) {
            res[i]->wait_s = q->t_admit - q->t_submit;
            res[i]->service_s = q->t_done - q->t_admit;
          }
          q->state = 2;
          // bytes a result keeps stay charged until it is freed: the state of
          // a streaming result; a batched group's whole footprint, which the
          // shared batch's deleter releases with the group's last result
          const bool group_held = grouped && st == RSV_OK;
          const size_t kept = group_held ? q->bytes : (res[i] ? res[i]->charged : 0);
          in_use -= q->bytes - kept;
          --running;
        }
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

extern "C" {

rsv_status rsv_server_create(rsv_ctx* ctx, const rsv_server_config* config, rsv_server** out) {
  g_last_error.clear();
  if (!ctx || !out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  rsv_server_config cfg{};
  if (config) cfg = *config;
  if (cfg.batch_atoms < 0 || cfg.batch_atoms > kBatchMaxAtoms)
    return fail(RSV_ERR_INVALID_ARG, "batch_atoms must be in [0, " + std::to_string(kBatchMaxAtoms) + "]");
  if (cfg.slots == 0) cfg.slots = 4;
  if (cfg.slots < 1 || cfg.slots > 64) return fail(RSV_ERR_INVALID_ARG, "slots must be in [1, 64]");
  std::unique_ptr<rsv_server> srv(new rsv_server());
  srv->ctx = ctx;
  srv->slots = cfg.slots;
  srv->batch_atoms = cfg.batch_atoms;
  srv->max_bypass_s = cfg.max_bypass_s == 0.0 ? 0.5 : cfg.max_bypass_s;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    size_t budget = cfg.memory_bytes;
    const size_t arena_free = ctx->arena.cap() > 0 ? ctx->arena.cap() - ctx->arena.used() : 0;
    if (budget == 0) {
      if (ctx->arena.cap() > 0) {
        budget = arena_free;
      } else {
        size_t fr = 0, tot = 0;
        RSV_CUDA(cudaMemGetInfo(&fr, &tot));
        budget = fr / 10 * 9;
      }
    } else if (ctx->arena.cap() > 0 && budget > arena_free) {
      return fail(RSV_ERR_OUT_OF_MEMORY, "memory_bytes exceeds the context arena's free bytes");
    }
    srv->budget = budget;
    ctx->servers.insert(srv.get());
  }
  rsv_server* p = srv.release();
  for (int i = 0; i < p->slots; ++i) p->workers.emplace_back([p] { p->worker(); });
  *out = p;
  return RSV_OK;
}

rsv_status rsv_submit(rsv_server* srv, const rsv_problem* problem, const rsv_config* config, uint64_t* ticket) {
  g_last_error.clear();
  if (!srv || !config || !ticket) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  RSV_TRY(validate_problem(problem));
  rsv_config cfg = *config;
  if (cfg.dt_ns < 1) return fail(RSV_ERR_INVALID_ARG, "dt_ns must be >= 1");
  if (cfg.precision != RSV_C64 && cfg.precision != RSV_C128) return fail(RSV_ERR_INVALID_ARG, "bad precision");
  if (cfg.m_max == 0) cfg.m_max = 30;
  if (cfg.m_max < 2 || cfg.m_max > kMaxKrylov) return fail(RSV_ERR_INVALID_ARG, "m_max must be in [2, 64]");
  if (cfg.obs_stride < 0) return fail(RSV_ERR_INVALID_ARG, "obs_stride must be >= 0");
  std::unique_ptr<ServeRequest> r(new ServeRequest());
  const int n = problem->n_atoms;
  const size_t T = (size_t)problem->t_ns;
  r->pos.assign(problem->positions_um, problem->positions_um + (size_t)n * problem->dim);
  r->om.assign(problem->omega, problem->omega + (size_t)problem->omega_rows * T);
  r->de.assign(problem->delta, problem->delta + (size_t)problem->delta_rows * T);
  if (problem->phi_rows > 0) r->ph.assign(problem->phi, problem->phi + (size_t)problem->phi_rows * T);
  if (problem->initial_state) {
    const char* c = static_cast<const char*>(problem->initial_state);
    r->init.assign(c, c + (size_t(1) << n) * amp_bytes(cfg.precision));
  }
  r->prob = *problem;
  r->prob.positions_um = r->pos.data();
  r->prob.omega = r->om.data();
  r->prob.delta = r->de.data();
  r->prob.phi = r->ph.empty() ? nullptr : r->ph.data();
  r->prob.initial_state = r->init.empty() ? nullptr : r->init.data();
  r->cfg = cfg;
  r->bytes = solver_bytes(&r->prob, cfg);
  std::lock_guard<std::mutex> lk(srv->mu);
  if (r->bytes > srv->budget)
    return fail(RSV_ERR_OUT_OF_MEMORY, "request footprint " + std::to_string(r->bytes) + " B exceeds the server's " +
                                           std::to_string(srv->budget) + " B");
  r->ticket = srv->next_ticket++;
  r->t_submit = srv->now();
  *ticket = r->ticket;
  srv->queue.push_back(r.get());
  srv->reqs[r->ticket] = std::move(r);
  srv->cv_work.notify_one();
  return RSV_OK;
}

rsv_status rsv_poll(rsv_server* srv, uint64_t ticket, int32_t timeout_ms, rsv_result** out) {
  g_last_error.clear();
  if (!srv || !out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return fail(RSV_ERR_NOT_FOUND, "unknown ticket " + std::to_string(ticket));
  ServeRequest* r = it->second.get();
  auto done = [&] { return r->state == 2; };
  if (timeout_ms < 0)
    srv->cv_done.wait(lk, done);
  else if (timeout_ms > 0)
    srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
  if (!done()) return fail(RSV_ERR_TIMEOUT, "ticket " + std::to_string(ticket) + " is still pending");
  const rsv_status st = r->status;
  const std::string err = r->error;
  *out = r->result;
  srv->reqs.erase(it);
  if (st != RSV_OK) return fail(st, err);
  return RSV_OK;
}

rsv_status rsv_request_bytes(const rsv_problem* problem, const rsv_config* config, size_t* out) {
  g_last_error.clear();
  if (!config || !out) return fail(RSV_ERR_INVALID_ARG, "NULL argument");
  RSV_TRY(validate_problem(problem));
  rsv_config cfg = *config;
  if (cfg.dt_ns < 1) return fail(RSV_ERR_INVALID_ARG, "dt_ns must be >= 1");
  if (cfg.precision != RSV_C64 && cfg.precision != RSV_C128) return fail(RSV_ERR_INVALID_ARG, "bad precision");
  if (cfg.m_max == 0) cfg.m_max = 30;
  if (cfg.m_max < 2 || cfg.m_max > kMaxKrylov) return fail(RSV_ERR_INVALID_ARG, "m_max must be in [2, 64]");
  if (cfg.obs_stride < 0) return fail(RSV_ERR_INVALID_ARG, "obs_stride must be >= 0");
  *out = solver_bytes(problem, cfg);
  return RSV_OK;
}

rsv_status rsv_server_load(rsv_server* srv, int32_t* queued, int32_t* running, size_t* bytes_in_use) {
  if (!srv) return fail(RSV_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(srv->mu);
  if (queued) *queued = (int32_t)srv->queue.size();
  if (running) *running = srv->running;
  if (bytes_in_use) *bytes_in_use = srv->in_use;
  return RSV_OK;
}

void rsv_server_destroy(rsv_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->queue.clear();
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  {
    std::lock_guard<std::mutex> lk(srv->ctx->mu);
    srv->ctx->servers.erase(srv);
  }
  for (auto& kv : srv->reqs)
    if (kv.second->result) rsv_result_free(kv.second->result);
  delete srv;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// rsv_observe_static: the observation reduction of rsv_observe (combine
// kernel in observe mode, then the begin kernel's FP64 reduction) with its
// scratch in a fixed device array of this library instead of context memory,
// so the call allocates nothing.
//
// Scratch layout (one copy per device, as every __device__ variable):
//   [0, kStaticKsBytes)         a KState; the begin kernel writes its norm2
//   [kStaticKsBytes, ...)       partial sums, grid rows of n + 1 doubles
// Every scratch word the call reads is written earlier in the same call, so
// nothing has to start at zero. Two calls in flight at once on one device
// share the array and race.
// ---------------------------------------------------------------------------
namespace {

constexpr int kStaticMaxAtoms = 31;                 // a partial row is n + 1 <= 32 doubles
constexpr int kStaticPartialDoubles = 1024 * 32;    // 256 KiB of partial rows
constexpr size_t kStaticKsBytes = (sizeof(KState) + 255) / 256 * 256;
constexpr size_t kStaticScratchBytes = kStaticKsBytes + sizeof(double) * kStaticPartialDoubles;
constexpr int kStaticMaxDevices = 64;

struct StaticSlot {
  std::atomic<unsigned char*> ptr{nullptr};
  int num_sms = 0;
};
StaticSlot g_static_slots[kStaticMaxDevices];
std::mutex g_static_mu;

}  // namespace

static __device__ __align__(256) unsigned char g_observe_scratch[kStaticScratchBytes];

namespace {

// Set-up, once per device, with that device current: the device address of
// the scratch array and the SM count. The first call on a device does it.
rsv_status static_scratch(int device, unsigned char** ptr, int* num_sms) {
  StaticSlot& s = g_static_slots[device];
  unsigned char* p = s.ptr.load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lk(g_static_mu);
    p = s.ptr.load(std::memory_order_relaxed);
    if (!p) {
      int sms = 0;
      RSV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
      void* q = nullptr;
      RSV_CUDA(cudaGetSymbolAddress(&q, g_observe_scratch));
      if (!q || (reinterpret_cast<uintptr_t>(q) & 255))
        return fail(RSV_ERR_CUDA, "rsv_observe_static: scratch array missing or not 256-byte aligned");
      s.num_sms = sms;
      p = static_cast<unsigned char*>(q);
      s.ptr.store(p, std::memory_order_release);
    }
  }
  *ptr = p;
  *num_sms = s.num_sms;
  return RSV_OK;
}

}  // namespace

extern "C" {

rsv_status rsv_observe_static(int32_t n_atoms, int32_t precision, const void* psi_dev, double* out_dev,
                              void* cuda_stream) {
  g_last_error.clear();
  if (!psi_dev || !out_dev) return fail(RSV_ERR_INVALID_ARG, "rsv_observe_static: NULL argument");
  if (precision != RSV_C64 && precision != RSV_C128) return fail(RSV_ERR_INVALID_ARG, "rsv_observe_static: bad precision");
  if (n_atoms < 1) return fail(RSV_ERR_INVALID_ARG, "rsv_observe_static: n_atoms must be >= 1");
  if (n_atoms > kStaticMaxAtoms)
    return fail(RSV_ERR_INVALID_ARG, "rsv_observe_static: n_atoms = " + std::to_string(n_atoms) +
                                         " exceeds the static scratch limit of " + std::to_string(kStaticMaxAtoms) +
                                         " atoms (partial rows of at most 32 doubles)");
  if (reinterpret_cast<uintptr_t>(psi_dev) & 15)
    return fail(RSV_ERR_INVALID_ARG, "rsv_observe_static: psi must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(out_dev) & 7)
    return fail(RSV_ERR_INVALID_ARG, "rsv_observe_static: out must be 8-byte aligned");
  int device = -1;
  RSV_CUDA(cudaGetDevice(&device));
  if (device < 0 || device >= kStaticMaxDevices)
    return fail(RSV_ERR_INVALID_ARG, "rsv_observe_static: device index beyond " + std::to_string(kStaticMaxDevices - 1));
  // both buffers must be device memory of the current device: a kernel given
  // another device's (or host) memory would fault or read the wrong bytes
  for (const void* p : {psi_dev, static_cast<const void*>(out_dev)}) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
      cudaGetLastError();
      return fail(RSV_ERR_INVALID_ARG, "rsv_observe_static: a buffer is not CUDA memory");
    }
    const bool dev_mem = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
    if (!dev_mem || pa.device != device)
      return fail(RSV_ERR_INVALID_ARG, "rsv_observe_static: psi_dev and out_dev must be device memory of the "
                                       "current device " + std::to_string(device));
  }
  unsigned char* scratch = nullptr;
  int sms = 0;
  RSV_TRY(static_scratch(device, &scratch, &sms));
  const bool c64 = precision == RSV_C64;
  const int nv = n_atoms + 1;
  // same grid as rsv_observe (chunks of 2^T amplitudes, up to 4 CTAs per SM),
  // capped by the rows the array holds
  const int T = std::min(n_atoms, (c64 ? 1 : 0) + 8 + 4);
  const int64_t chunks = int64_t(1) << (n_atoms - T);
  int grid = (int)std::min<int64_t>(chunks, 4 * (int64_t)std::max(sms, 1));
  grid = std::min(grid, kStaticPartialDoubles / nv);
  const size_t need = kStaticKsBytes + sizeof(double) * (size_t)grid * nv;
  if (need > kStaticScratchBytes)
    return fail(RSV_ERR_INVALID_ARG, "rsv_observe_static: needs " + std::to_string(need) +
                                         " bytes of scratch, the static array holds " +
                                         std::to_string(kStaticScratchBytes));
  KState* ks = reinterpret_cast<KState*>(scratch);
  double* part = reinterpret_cast<double*>(scratch + kStaticKsBytes);
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  CombineArgs ca{};
  ca.n = n_atoms;
  ca.dim = int64_t(1) << n_atoms;
  ca.ks = ks;
  ca.psi = const_cast<void*>(psi_dev);
  ca.partials = part;
  ca.combine = 0;
  RSV_CUDA(launch_combine(ca, c64, grid, stream));
  BeginArgs ba{};
  ba.ks = ks;
  ba.partials = part;
  ba.nparts = grid;
  ba.n = n_atoms;
  ba.occ_out = out_dev + 1;
  ba.reset_only = 1;
  RSV_CUDA(launch_begin(ba, stream));
  RSV_CUDA(cudaMemcpyAsync(out_dev, scratch + offsetof(KState, norm2), sizeof(double), cudaMemcpyDeviceToDevice,
                           stream));
  return RSV_OK;
}

}  // extern "C"
