// Fused structured matvec y = H x for the Rydberg Hamiltonian (arXiv 2510.09813,
// Eq. (3)) and the Lanczos iteration built on it (Sec. III.A).
//
// H x is "apply the diagonal, then add the Omega-scaled bit-flip permutations"
// (Sec. III.A). The diagonal is never stored: each tile rebuilds
//     E(b) = sum_{q<r} V_qr b_q b_r - sum_q delta_q b_q
// from FP64 pair energies as E_hi(tile) + sum_{q<L} w_q(tile) b_q + Q[b_lo].
//
// Tiles. A tile is a 2^L-amplitude sub-cube of the state: tile bits [0,c) are
// amplitude bits [0,c) (contiguous in memory) and tile bits [c,L) are amplitude
// bits [a, a+L-c). The remaining bits are fixed per tile; the lowest nG of the
// top fixed range are "G bits" whose partners are read from the neighbouring
// tile through L2 (neighbours differ in the low bits of the tile index, so they
// are processed at the same time by other CTAs). A full matvec is one pass when
// the tile plus G bits cover the state, else two: a contiguous pass over bits
// [0, L) that also adds the diagonal, and a strided pass over the rest.
//
// Execution. One persistent CTA of 16 warps per SM (4 per SM sub-partition, so
// each thread may hold 128 registers). The CTA's input tiles stream into a
// 3-stage shared-memory ring by TMA (1D bulk copies for contiguous tiles, tiled
// tensor copies for strided ones) with mbarrier completion; warp 0 issues the
// copies two tiles ahead before computing its own share. All warps compute from
// shared memory and store results straight to global memory. Every flip partner
// inside the tile is a 16-byte shared-memory load; complex64 arithmetic uses
// packed FP32x2 FMAs. Every mbarrier wait is bounded.
//
// Lanczos fusion. The first pass forms v_j = (u_{j-1} - alpha_{j-1} v_{j-1}) /
// beta_j in place from the staged tiles, writes v_j to the Krylov basis and
// subtracts beta_j v_{j-1}; the last pass accumulates Re<v_j,u_j>, |u_j|^2 and
// |v_j|^2, from which the scalar kernel derives alpha_j and beta_{j+1}.
#include <type_traits>

#include "kernels.h"
#include "krylov_control.cuh"
#include "rsv_common.cuh"
#include "tma.cuh"
#include "vec_ops.cuh"

namespace rsv {

static_assert(sizeof(ControlSmem) <= (size_t)kStages * 2 * 32768, "the control step fits the idle ring");

template <typename Real>
struct TileCfg {
  static constexpr bool kF = std::is_same<Real, float>::value;
  static constexpr int V = CplxT<Real>::kLogVec;  // log2 amplitudes per 16-byte vector
  static constexpr int NV = 1 << V;
  static constexpr int L = kF ? kTileBitsF : kTileBitsD;
  static constexpr int KT = 9;               // consumer-thread bits of a full tile
  static constexpr int KK = L - V - KT;      // register ("k") bits of a full tile
  static constexpr int K = 1 << KK;          // vectors per consumer thread
  static constexpr uint32_t kTileBytes = (1u << L) * 2u * sizeof(Real);
};
static_assert(TileCfg<float>::KK == 2 && TileCfg<double>::KK == 2, "tile layout");

constexpr int kMaxG = 12;

// ---------------------------------------------------------------------------
// The streaming pass.
// ---------------------------------------------------------------------------
template <typename Real, bool LANCZOS, bool FIRST, bool LAST, bool PHI, bool FULL>
__global__ void __launch_bounds__(kTileThreads, 1)
    tile_kernel(const TileArgs args, const __grid_constant__ TileMaps maps) {
  using C = TileCfg<Real>;
  using Acc = typename AccFor<Real>::type;
  constexpr int V = C::V;
  constexpr int KT = C::KT, KK = C::KK, K = C::K;
  constexpr bool FORM = LANCZOS && FIRST;  // v_j is formed from (u_{j-1}, v_{j-1})

  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], formed[kStages];
  __shared__ __align__(128) Real s_t[kStages][kDiagStride];  // the staged tile's diagonal half tables (first pass)
  __shared__ Coef s_cp[kMaxAtoms][2];         // [amplitude bit][bit of the target], apply form
  __shared__ double s_red[3][kConsumerWarps];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = args.n, L = args.L, c = args.c, a = args.a, f2 = args.f2;
  // FULL: the standard tile layout, known at compile time (no per-vector guards)
  const int nF2 = args.nF2, nG = args.nG, kt = FULL ? KT : args.kt, kk = FULL ? KK : L - V - kt;
  const StepParams* sp = args.sp;
  const int64_t num_tiles = args.num_tiles;
  const uint32_t tile_bytes = (1u << L) * 2u * sizeof(Real);
  const int64_t cmask = (int64_t(1) << c) - 1, f2mask = (int64_t(1) << nF2) - 1;

  if (LANCZOS && args.ks->status != kContinue) return;  // uniform: Krylov space already accepted
  const int jj = FORM ? args.ks->j : 0;
  const bool has_prev = FORM && jj > 0;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
      mbar_init(&formed[s], kConsumerWarps);
    }
    mbar_fence_init();
  }
  if (tid >= 32 && tid < 32 + n) {
    const int q = tid - 32;
    const double ho = sp->half_omega[q];
    double sn = 0.0, cs = 1.0;
    if (PHI) sincos(sp->phi[q], &sn, &cs);
    // target bit 0: <0|h|1> = Omega/2 e^{+i phi}; target bit 1: <1|h|0> = Omega/2 e^{-i phi}
    s_cp[q][0] = make_coef<Real, PHI>((Real)(ho * cs), (Real)(ho * sn));
    s_cp[q][1] = make_coef<Real, PHI>((Real)(ho * cs), (Real)(-ho * sn));
  }
  Real* s_q = reinterpret_cast<Real*>(smem + (size_t)kStages * 2 * C::kTileBytes);
  if (FIRST) {
    const Real* qg = reinterpret_cast<const Real*>(args.qtab);
    for (int i = tid; i < (1 << L); i += kConsumers) s_q[i] = qg[i];
  }
  __syncthreads();

  auto stage_tile = [&](int s, int op) -> unsigned char* {
    return smem + ((size_t)s * 2 + op) * C::kTileBytes;
  };
  // Tile index -> fixed bits: the lowest f1f index bits are segment-index (F1)
  // bits, then the nF2 top-range (F2) bits, then the remaining F1 bits. f1f > 0
  // makes neighbouring CTAs read adjacent segments (DRAM row locality); F2
  // neighbours, whose partners come through L2, stay 2^(f1f + g) tiles apart.
  const int f1f = args.f1_fast;
  const int64_t f1fmask = (int64_t(1) << f1f) - 1;
  auto f2_of = [&](int64_t t) -> int64_t { return (t >> f1f) & f2mask; };
  auto f1_of = [&](int64_t t) -> int64_t { return (t & f1fmask) | ((t >> (f1f + nF2)) << f1f); };
  auto tile_base = [&](int64_t tile) -> int64_t { return (f1_of(tile) << c) | (f2_of(tile) << f2); };

  // ---- producer duties (warp 0): stream this CTA's tile number ip into stage
  // ip % kStages with TMA; the next kStages - 1 tiles are always in flight ----
  int produced = 0;
  bool prod_ok = true;
  auto produce = [&](int ip) {
    const int64_t tile = blockIdx.x + (int64_t)ip * gridDim.x;
    if (tile >= num_tiles || !prod_ok) return;
    const int s = ip % kStages, r = ip / kStages;
    if (ip >= kStages) {
      // all warps released round r-1 of this stage
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&empty[s], (r - 1) & 1) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        prod_ok = false;
        if (lane == 0) atomicOr(args.err, 1);
        return;
      }
    }
    if (lane == 0) {
      if (FIRST) {
        // contiguous tile: amplitude offset tile << L; its diagonal half tables
        // (c == L: tile bits are amplitude bits [0, L)) ride on the same
        // barrier, so no thread waits on a global load for them
        const size_t off = (size_t)tile * tile_bytes;
        constexpr uint32_t row_bytes = kDiagStride * sizeof(Real);
        mbar_arrive_expect_tx(&full[s], tile_bytes * (has_prev ? 2 : 1) + row_bytes);
        tma_load_1d(s_t[s], static_cast<const Real*>(args.diag) + tile * kDiagStride, row_bytes, &full[s]);
        tma_load_1d(stage_tile(s, 0), static_cast<const unsigned char*>(args.xin) + off, tile_bytes, &full[s]);
        if (has_prev)
          tma_load_1d(stage_tile(s, 1), static_cast<const unsigned char*>(args.xprev) + off, tile_bytes, &full[s]);
        else if (tile + 2 * (int64_t)gridDim.x < num_tiles)
          // one operand per stage leaves half the ring's bytes in flight: keep
          // the DRAM reads of the tile two beyond this one going through L2
          prefetch_l2_1d(static_cast<const unsigned char*>(args.xin) + off + 2 * (size_t)gridDim.x * tile_bytes,
                         tile_bytes);
      } else {
        const int cf1 = (int)f1_of(tile), cf2 = (int)f2_of(tile);
        mbar_arrive_expect_tx(&full[s], tile_bytes * 2);
        if (args.split_h) {
          tma_load_5d(stage_tile(s, 0), &maps.x, 0, cf1, 0, 0, cf2, &full[s]);
          tma_load_5d(stage_tile(s, 1), &maps.z, 0, cf1, 0, 0, cf2, &full[s]);
        } else {
          tma_load_5d(stage_tile(s, 0), &maps.x, 0, 0, cf1, 0, cf2, &full[s]);
          tma_load_5d(stage_tile(s, 1), &maps.z, 0, 0, cf1, 0, cf2, &full[s]);
        }
      }
    }
    __syncwarp();
    produced = ip + 1;
  };
  if (warp == 0)
    for (int ip = 0; ip < kStages - 1; ++ip) produce(ip);

  {
    // ---------------- consumers ----------------
    const int ct = tid;
    const bool active = ct < (1 << kt);
    const int keff = 1 << kk;
    // Without a phase a flip coefficient is the real Omega_q / 2 for both target
    // bit states and lives in a register; with a phase it is read from s_cp.
    unsigned long long cre_t[KT], cre_r[KK], cre_l = 0ull;
    bool flip_t[KT], flip_r[KK];
#pragma unroll
    for (int j = 0; j < KT; ++j) {
      const int tb = V + j;
      flip_t[j] = j < kt && (FIRST || tb >= c);
      cre_t[j] = flip_t[j] ? s_cp[tb < c ? tb : a + (tb - c)][0].rr : 0ull;
    }
#pragma unroll
    for (int j = 0; j < KK; ++j) {
      const int tb = V + kt + j;
      flip_r[j] = j < kk && (FIRST || tb >= c);
      cre_r[j] = flip_r[j] ? s_cp[tb < c ? tb : a + (tb - c)][0].rr : 0ull;
    }
    if (V == 1 && FIRST) cre_l = s_cp[0][0].rr;
    auto coef_thread = [&](int j) -> Coef {
      if (!PHI) return Coef{cre_t[j], 0ull};
      const int tb = V + j;
      return s_cp[tb < c ? tb : a + (tb - c)][(ct >> j) & 1];
    };
    auto coef_reg = [&](int j, int k) -> Coef {
      if (!PHI) return Coef{cre_r[j], 0ull};
      const int tb = V + kt + j;
      return s_cp[tb < c ? tb : a + (tb - c)][(k >> j) & 1];
    };
    const Real fa = FORM ? (Real)args.ks->form_a : (Real)0;
    const Real fs = FORM ? (Real)args.ks->form_s : (Real)1;
    const Real bp = FORM ? (Real)args.ks->beta_prev : (Real)0;

    Acc r0, r1, r2;
    int i = 0;
    for (int64_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++i) {
      if (warp == 0) produce(i + kStages - 1);
      const int s = i % kStages, r = i / kStages;
      if (!mbar_wait(&full[s], r & 1)) {
        if (lane == 0) atomicOr(args.err, 1);
        break;
      }
      unsigned char* T0 = stage_tile(s, 0);
      unsigned char* T1 = stage_tile(s, 1);
      const int64_t base = tile_base(tile);
      const int64_t tf2 = f2_of(tile);
      if (FORM) {
        // v_j = (u_{j-1} - alpha_{j-1} v_{j-1}) / beta_j, in place, and into the basis
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (!active || k >= keff) continue;
          const int tv = ct | (k << kt);
          const Vec u = lds_vec(T0, tv);
          const Vec v = has_prev ? lds_vec(T1, tv) : Vec{0ull, 0ull};
          const Vec x = form<Real>(u, v, fa, fs, has_prev);
          sts_vec(T0, tv, x);
          const int t = tv << V;
          const int64_t amp = base | (t & cmask) | ((int64_t)(t >> c) << a);
          stg_vec(args.xout, amp >> V, x);
        }
        // every consumer's v_j is in shared memory before anyone reads partners
        __syncwarp();
        if (lane == 0) mbar_arrive(&formed[s]);
        if (!mbar_wait(&formed[s], r & 1)) {
          if (lane == 0) atomicOr(args.err, 1);
          break;
        }
      }
      if (active) {
        // this thread's vectors: tile-local index, global vector index, value
        int tvk[K];
        int64_t vidx[K];
        Vec x[K], o[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          tvk[k] = ct | (k << kt);
          const int t = tvk[k] << V;
          vidx[k] = (base | (t & cmask) | ((int64_t)(t >> c) << a)) >> V;
          x[k] = k < keff ? lds_vec(T0, tvk[k]) : Vec{0ull, 0ull};
        }
        if (FIRST) {
          // E(t) = T1[t mod 64] + T2[t / 64] + Q[t]: three terms, each rounded
          // once from FP64, so the working-precision error is a few units of
          // roundoff of |E| (a running sum over the tile bits would round at
          // every bit)
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int t = tvk[k] << V;
            const Real hi = s_t[s][kDiagHalf + (t >> 6)];
            const Real e0 = (s_t[s][t & (kDiagHalf - 1)] + hi) + s_q[t];
            const Real e1 = V == 1 ? (s_t[s][(t + 1) & (kDiagHalf - 1)] + hi) + s_q[t + 1] : e0;
            o[k] = scale2<Real>(x[k], e0, e1);
            if constexpr (C::kF) {
              // vector-lane bit: amplitude bit 0, the partner is the other half of the vector
              cmac_word<PHI>(o[k].w0, PHI ? s_cp[0][0] : Coef{cre_l, 0ull}, x[k].w1);
              cmac_word<PHI>(o[k].w1, PHI ? s_cp[0][1] : Coef{cre_l, 0ull}, x[k].w0);
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < K; ++k) o[k] = k < keff ? lds_vec(T1, tvk[k]) : Vec{0ull, 0ull};
        }
        // thread bits, bit-major: the K partner loads of one bit are independent
#pragma unroll
        for (int j = 0; j < KT; ++j) {
          if (!flip_t[j]) continue;
          const Coef cf = coef_thread(j);
          Vec pp[K];
#pragma unroll
          for (int k = 0; k < K; ++k) pp[k] = k < keff ? lds_vec(T0, tvk[k] ^ (1 << j)) : Vec{0ull, 0ull};
#pragma unroll
          for (int k = 0; k < K; ++k) cmac<Real, PHI>(o[k], cf, pp[k]);
        }
        // register bits: the partner is another of this thread's own vectors
#pragma unroll
        for (int j = 0; j < KK; ++j) {
          if (!flip_r[j]) continue;
#pragma unroll
          for (int k = 0; k < K; ++k)
            if (k < keff) cmac<Real, PHI>(o[k], coef_reg(j, k), x[k ^ (1 << j)]);
        }
        if (has_prev) {
#pragma unroll
          for (int k = 0; k < K; ++k)
            if (k < keff) axpy<Real>(o[k], -bp, lds_vec(T1, tvk[k]));
        }
        // G bits: partners in neighbouring tiles, read through L2, two bits at a
        // time for all of this thread's vectors (8 loads in flight per thread)
        // (the strided pass re-reads x from shared memory for its reductions, so
        // x's registers hold a third bit of partner loads instead)
        constexpr int GB = FIRST ? 2 : 3;
        for (int g0 = 0; g0 < nG; g0 += GB) {
          Vec p[GB][K];
#pragma unroll
          for (int g = 0; g < GB; ++g) {
            // a G bit is fixed per tile, so the partner sits at a uniform offset
            const int64_t gstep = int64_t(1) << (f2 + g0 + g - V);
            const int64_t goff = ((tf2 >> (g0 + g)) & 1) ? -gstep : gstep;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              p[g][k] = Vec{0ull, 0ull};
              if (g0 + g >= nG || k >= keff) continue;
              const int64_t pidx = vidx[k] + goff;
              if (FORM) {
                const Vec u = ldg_vec(args.xin, pidx);
                const Vec v = has_prev ? ldg_vec(args.xprev, pidx) : Vec{0ull, 0ull};
                p[g][k] = form<Real>(u, v, fa, fs, has_prev);
              } else {
                p[g][k] = ldg_vec(args.xin, pidx);
              }
            }
          }
#pragma unroll
          for (int g = 0; g < GB; ++g) {
            if (g0 + g >= nG) continue;
            const Coef cg = s_cp[f2 + g0 + g][(tf2 >> (g0 + g)) & 1];
#pragma unroll
            for (int k = 0; k < K; ++k)
              if (k < keff) cmac<Real, PHI>(o[k], cg, p[g][k]);
          }
        }
        // store (and reduce)
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (k >= keff) continue;
          if (LANCZOS && LAST) reduce_vec<Real>(FIRST ? x[k] : lds_vec(T0, tvk[k]), o[k], r0, r1, r2);
          stg_vec(args.out, vidx[k], o[k]);
        }
      }
      // release the stage (generic writes to it must precede the next TMA write)
      if (FORM) fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (LANCZOS && LAST) {
      Acc acc[3] = {r0, r1, r2};
#pragma unroll
      for (int v = 0; v < 3; ++v) warp_merge(acc[v]);
      if (lane == 0) {
#pragma unroll
        for (int v = 0; v < 3; ++v) s_red[v][warp] = acc[v].value();
      }
    }
  }
  // On an aborted run, let copies still in flight into the ring land before the
  // CTA exits (bounded); on a normal run these phases have already completed.
  if (warp == 0 && lane == 0 && *args.err) {
    for (int ip = produced - 1; ip >= 0 && ip >= produced - kStages; --ip)
      mbar_wait(&full[ip % kStages], (ip / kStages) & 1);
  }
  // every thread of the CTA reaches this point: all waits above are bounded
  __syncthreads();
  if (LANCZOS && LAST) pass_tail(args.ctl, args.partials, s_red, args.err, smem);
}

// ---------------------------------------------------------------------------
// Host-side launch
// ---------------------------------------------------------------------------
template <typename Real>
size_t tile_smem_bytes() {
  return (size_t)kStages * 2 * TileCfg<Real>::kTileBytes + (sizeof(Real) << TileCfg<Real>::L);
}

template <typename Real, bool LANCZOS, bool FIRST, bool LAST, bool PHI, bool FULL>
static cudaError_t launch_full(const TileArgs& args, const TileMaps* maps, int grid, cudaStream_t stream) {
  auto fn = tile_kernel<Real, LANCZOS, FIRST, LAST, PHI, FULL>;
  const size_t smem = tile_smem_bytes<Real>();
  static bool configured = false;  // per instantiation
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  static const TileMaps empty_maps{};
  fn<<<grid, kTileThreads, smem, stream>>>(args, maps ? *maps : empty_maps);
  return cudaGetLastError();
}



template <typename Real, bool LANCZOS, bool FIRST, bool LAST, bool PHI>
static cudaError_t launch_one(const TileArgs& args, const TileMaps* maps, int grid, cudaStream_t stream) {
  const bool full = args.kt == TileCfg<Real>::KT && args.L == TileCfg<Real>::L;
  return full ? launch_full<Real, LANCZOS, FIRST, LAST, PHI, true>(args, maps, grid, stream)
              : launch_full<Real, LANCZOS, FIRST, LAST, PHI, false>(args, maps, grid, stream);
}

template <typename Real>
static cudaError_t dispatch(const TileArgs& args, const TileMaps* maps, TileMode mode, bool phi, int grid,
                            cudaStream_t stream) {
  switch (mode) {
    case TileMode::kMatvecFirst:
      return phi ? launch_one<Real, false, true, false, true>(args, maps, grid, stream)
                 : launch_one<Real, false, true, false, false>(args, maps, grid, stream);
    case TileMode::kMatvecSecond:
      return phi ? launch_one<Real, false, false, false, true>(args, maps, grid, stream)
                 : launch_one<Real, false, false, false, false>(args, maps, grid, stream);
    case TileMode::kLanczosSingle:
      return phi ? launch_one<Real, true, true, true, true>(args, maps, grid, stream)
                 : launch_one<Real, true, true, true, false>(args, maps, grid, stream);
    case TileMode::kLanczosFirst:
      return phi ? launch_one<Real, true, true, false, true>(args, maps, grid, stream)
                 : launch_one<Real, true, true, false, false>(args, maps, grid, stream);
    case TileMode::kLanczosSecond:
      return phi ? launch_one<Real, true, false, true, true>(args, maps, grid, stream)
                 : launch_one<Real, true, false, true, false>(args, maps, grid, stream);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_tile(const TileArgs& args, const TileMaps* maps, TileMode mode, bool c64, bool phi, int grid,
                        cudaStream_t stream) {
  if (grid <= 0) return cudaErrorInvalidValue;
  // a strided geometry of 64 KiB x-only tiles goes to the strided kernel
  const bool second = mode == TileMode::kMatvecSecond || mode == TileMode::kLanczosSecond;
  if (second && args.L == (c64 ? kStridedTileBitsF : kStridedTileBitsD))
    return launch_strided(args, maps, mode == TileMode::kLanczosSecond, c64, phi, grid, stream);
  return c64 ? dispatch<float>(args, maps, mode, phi, grid, stream)
             : dispatch<double>(args, maps, mode, phi, grid, stream);
}

// ---------------------------------------------------------------------------
// Tensor maps of the strided pass (driver entry point, no link-time libcuda).
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

bool encode_tile_map(CUtensorMap* out, const void* base, const TileArgs& g, bool c64) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  // 8-byte elements: one per complex64 amplitude, two per complex128 amplitude.
  // Dimensions (innermost first): amplitude bits [0, c0), [c0, c), [c, a),
  // [a, a+h), [a+h, n); the box takes the first, second and fourth whole, so the
  // tile lands in shared memory in tile-local order. c0 keeps a box edge <= 256.
  // When the strided range is wider than a box edge (h > 8), the contiguous
  // segment is kept whole and the strided range is split instead (kernel side:
  // TileArgs::split_h selects the matching coordinate order).
  const int lepa = c64 ? 0 : 1;
  const uint64_t ab = c64 ? 8 : 16;
  const int h = g.L - g.c;
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5];
  if (!g.split_h) {
    const int c0 = g.c < 8 - lepa ? g.c : 8 - lepa;
    const cuuint64_t d[5] = {(cuuint64_t)1 << (c0 + lepa), (cuuint64_t)1 << (g.c - c0),
                             (cuuint64_t)1 << (g.a - g.c), (cuuint64_t)1 << h, (cuuint64_t)1 << (g.n - g.a - h)};
    const cuuint64_t st[4] = {(cuuint64_t)(ab << c0), (cuuint64_t)(ab << g.c), (cuuint64_t)(ab << g.a),
                              (cuuint64_t)(ab << (g.a + h))};
    const cuuint32_t b[5] = {(cuuint32_t)1 << (c0 + lepa), (cuuint32_t)1 << (g.c - c0), 1, (cuuint32_t)1 << h, 1};
    for (int i = 0; i < 5; ++i) dims[i] = d[i], box[i] = b[i];
    for (int i = 0; i < 4; ++i) strides[i] = st[i];
  } else {
    const int h0 = 8;
    const cuuint64_t d[5] = {(cuuint64_t)1 << (g.c + lepa), (cuuint64_t)1 << (g.a - g.c), (cuuint64_t)1 << h0,
                             (cuuint64_t)1 << (h - h0), (cuuint64_t)1 << (g.n - g.a - h)};
    const cuuint64_t st[4] = {(cuuint64_t)(ab << g.c), (cuuint64_t)(ab << g.a), (cuuint64_t)(ab << (g.a + h0)),
                              (cuuint64_t)(ab << (g.a + h))};
    const cuuint32_t b[5] = {(cuuint32_t)1 << (g.c + lepa), 1, (cuuint32_t)1 << h0, (cuuint32_t)1 << (h - h0), 1};
    for (int i = 0; i < 5; ++i) dims[i] = d[i], box[i] = b[i];
    for (int i = 0; i < 4; ++i) strides[i] = st[i];
  }
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  for (int i = 0; i < 5; ++i)
    if (box[i] > 256) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  const CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace rsv
