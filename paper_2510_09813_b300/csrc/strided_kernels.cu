// Second (strided) streaming pass of the two-pass matvec y = H x for the
// Rydberg Hamiltonian (arXiv 2510.09813, Eq. (3)) and of the Lanczos iteration
// built on it (Sec. III.A), with shared memory given to x alone.
//
// The first pass has added the diagonal and the flips of amplitude bits
// [0, a) into z. This pass adds the flips of bits [a, n): the h strided bits
// of its tile from shared memory and the nG bits above them ("G bits") from
// the neighbouring tiles through L2, and, in a Lanczos iteration, reduces
// Re<v_j, z>, |z|^2 and |v_j|^2.
//
// Tiles. A tile is 2^T amplitudes (64 KiB: T = 13 for complex64, 12 for
// complex128): tile bits [0, c) are amplitude bits [0, c), a contiguous
// segment of 2^c amplitudes, and tile bits [c, T) are amplitude bits
// [a, a + h), h = T - c. Only x (the vector the flips read) is staged, by TMA
// into a 3-stage ring of 64 KiB stages. z is read and written once per
// amplitude by the thread that owns it, so it needs no staging: the producer
// prefetches each tile's z region into L2 with a TMA prefetch two tiles ahead,
// and the owning threads load it from L2 and store the result. Staging x alone
// doubles the tile of a ring that stages x and z, which takes one partner bit
// off L2: each partner bit read through L2 costs 8 (complex64) or 16
// (complex128) bytes per amplitude of L2-to-SM traffic, the pass's bound.
//
// Segment width. With c small (2 or 3 bits: 32- or 64-byte segments) the tile
// holds more strided bits and fewer partner bits remain for L2. Consecutive
// tile numbers then take adjacent segments of the same rows (f1_fast), so the
// 256-byte L2 lines and DRAM bursts a segment belongs to are requested by
// neighbouring CTAs at the same time.
//
// Threads. 16 warps; thread ct owns tile vectors ct | k << 9 | b << 11 (K = 4
// register vectors per sub-batch b, two sub-batches). Flip partners are read
// from shared memory (thread and sub-batch bits), from the thread's own
// registers (register bits) or from global memory through L2 (G bits, two at
// a time: 8 loads in flight per thread). Issuing more partner loads at once
// (all G bits of a sub-batch before the shared-memory flips) measured slower.
//
// Every mbarrier wait is bounded; a timeout sets the error word and the CTA
// drains its copies in flight before it exits.
#include <type_traits>

#include "kernels.h"
#include "krylov_control.cuh"
#include "rsv_common.cuh"
#include "tma.cuh"
#include "vec_ops.cuh"

namespace rsv {

static_assert(sizeof(ControlSmem) <= (size_t)kStridedStages * 65536, "the control step fits the idle ring");

template <typename Real>
struct StridedCfg {
  static constexpr bool kF = std::is_same<Real, float>::value;
  static constexpr int V = CplxT<Real>::kLogVec;  // log2 amplitudes per 16-byte vector
  static constexpr int T = kF ? kStridedTileBitsF : kStridedTileBitsD;
  static constexpr int KT = 9;                    // thread bits
  static constexpr int KK = 2;                    // register bits
  static constexpr int K = 1 << KK;
  static constexpr int KB = T - V - KT - KK;      // sub-batch bits
  static constexpr int NB = 1 << KB;
  static constexpr int GB = 2;                    // G bits whose partner loads are in flight together
  static constexpr uint32_t kTileBytes = (1u << T) * 2u * sizeof(Real);
};
static_assert(StridedCfg<float>::KB == 1 && StridedCfg<double>::KB == 1, "strided tile layout");
static_assert(StridedCfg<float>::kTileBytes == 65536 && StridedCfg<double>::kTileBytes == 65536, "64 KiB tiles");

template <typename Real, bool LANCZOS, bool PHI>
__global__ void __launch_bounds__(kTileThreads, 1)
    strided_kernel(const TileArgs args, const __grid_constant__ TileMaps maps) {
  using C = StridedCfg<Real>;
  using Acc = typename AccFor<Real>::type;
  constexpr int V = C::V, KT = C::KT, KK = C::KK, K = C::K, KB = C::KB, NB = C::NB, GB = C::GB;

  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStridedStages], empty[kStridedStages];
  __shared__ Coef s_cp[kMaxAtoms][2];  // [amplitude bit][bit of the target], apply form
  __shared__ double s_red[3][kConsumerWarps];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = args.n, c = args.c, a = args.a, f2 = args.f2, nF2 = args.nF2, nG = args.nG;
  const int64_t num_tiles = args.num_tiles;
  const int64_t cmask = (int64_t(1) << c) - 1, f2mask = (int64_t(1) << nF2) - 1;

  if (LANCZOS && args.ks->status != kContinue) return;  // uniform: Krylov space already accepted

  if (tid == 0) {
    for (int s = 0; s < kStridedStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    mbar_fence_init();
  }
  if (tid >= 32 && tid < 32 + n) {
    const int q = tid - 32;
    const double ho = args.sp->half_omega[q];
    double sn = 0.0, cs = 1.0;
    if (PHI) sincos(args.sp->phi[q], &sn, &cs);
    // target bit 0: <0|h|1> = Omega/2 e^{+i phi}; target bit 1: <1|h|0> = Omega/2 e^{-i phi}
    s_cp[q][0] = make_coef<Real, PHI>((Real)(ho * cs), (Real)(ho * sn));
    s_cp[q][1] = make_coef<Real, PHI>((Real)(ho * cs), (Real)(-ho * sn));
  }
  __syncthreads();

  auto stage = [&](int s) -> unsigned char* { return smem + (size_t)s * C::kTileBytes; };
  // Tile number -> fixed bits: the lowest f1_fast bits are segment-index (F1)
  // bits, then the nF2 top-range (F2) bits, then the remaining F1 bits.
  const int f1f = args.f1_fast;
  const int64_t f1fmask = (int64_t(1) << f1f) - 1;
  auto f2_of = [&](int64_t t) -> int64_t { return (t >> f1f) & f2mask; };
  auto f1_of = [&](int64_t t) -> int64_t { return (t & f1fmask) | ((t >> (f1f + nF2)) << f1f); };
  auto tile_base = [&](int64_t t) -> int64_t { return (f1_of(t) << c) | (f2_of(t) << f2); };

  // ---- producer (warp 0): x tile ip into stage ip % kStridedStages, and the
  // tile's z region into L2 ----
  int produced = 0;
  bool prod_ok = true;
  auto produce = [&](int ip) {
    const int64_t tile = blockIdx.x + (int64_t)ip * gridDim.x;
    if (tile >= num_tiles || !prod_ok) return;
    const int s = ip % kStridedStages, r = ip / kStridedStages;
    if (ip >= kStridedStages) {
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
      const int cf1 = (int)f1_of(tile), cf2 = (int)f2_of(tile);
      mbar_arrive_expect_tx(&full[s], C::kTileBytes);
      if (args.split_h) {
        tma_load_5d(stage(s), &maps.x, 0, cf1, 0, 0, cf2, &full[s]);
        tma_prefetch_l2_5d(&maps.z, 0, cf1, 0, 0, cf2);
      } else {
        tma_load_5d(stage(s), &maps.x, 0, 0, cf1, 0, cf2, &full[s]);
        tma_prefetch_l2_5d(&maps.z, 0, 0, cf1, 0, cf2);
      }
    }
    __syncwarp();
    produced = ip + 1;
  };
  if (warp == 0)
    for (int ip = 0; ip < kStridedStages - 1; ++ip) produce(ip);

  const int ct = tid;
  // Flip coefficients, read from shared memory where they are used (every
  // thread of a warp reads the same word: a broadcast). Tile bit tb >= c is
  // amplitude bit a + tb - c; tile bits below c are the first pass's. Without
  // a phase a coefficient is the real Omega_q / 2 for both target bit states.
  auto qbit = [&](int tb) { return a + (tb - c); };
  auto coef = [&](int tb, int target_bit) -> Coef {
    if (!PHI) return Coef{s_cp[qbit(tb)][0].rr, 0ull};
    return s_cp[qbit(tb)][target_bit];
  };
  // global vector index of register vector k and sub-batch b, relative to
  // that of k = b = 0 (their tile bits lie above c, in the strided range)
  auto koff = [&](int k, int b) -> int64_t {
    const int t = ((k << KT) | (b << (KT + KK))) << V;
    return ((int64_t)(t >> c) << a) >> V;
  };

  Acc r0, r1, r2;
  int i = 0;
  for (int64_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++i) {
    if (warp == 0) produce(i + kStridedStages - 1);
    const int s = i % kStridedStages, r = i / kStridedStages;
    const int64_t base = tile_base(tile);
    const int64_t tf2 = f2_of(tile);
    if (!mbar_wait(&full[s], r & 1)) {
      if (lane == 0) atomicOr(args.err, 1);
      break;
    }
    const unsigned char* X = stage(s);
    // this thread's k = b = 0 vector: tile-local and global index
    const int64_t vidx0 = (base | ((int64_t)(ct << V) & cmask) | ((int64_t)((ct << V) >> c) << a)) >> V;
#pragma unroll 1
    for (int b = 0; b < NB; ++b) {
      Vec zv[K], x[K], o[K];
#pragma unroll
      for (int k = 0; k < K; ++k) zv[k] = ldcs_vec(args.out, vidx0 + koff(k, b));  // z from L2, used once
#pragma unroll
      for (int k = 0; k < K; ++k) {
        x[k] = lds_vec(X, ct | (k << KT) | (b << (KT + KK)));
        o[k] = Vec{0ull, 0ull};
      }
      // thread bits, bit-major: the K partner loads of one bit are independent
#pragma unroll
      for (int j = 0; j < KT; ++j) {
        if (V + j < c) continue;  // a contiguous bit: the first pass's
        const Coef cf = coef(V + j, (ct >> j) & 1);
        Vec pp[K];
#pragma unroll
        for (int k = 0; k < K; ++k) pp[k] = lds_vec(X, (ct ^ (1 << j)) | (k << KT) | (b << (KT + KK)));
#pragma unroll
        for (int k = 0; k < K; ++k) cmac<Real, PHI>(o[k], cf, pp[k]);
      }
      // sub-batch bits: the partner is in another sub-batch, in shared memory
#pragma unroll
      for (int j = 0; j < KB; ++j) {
        const Coef cf = coef(V + KT + KK + j, (b >> j) & 1);
        Vec pp[K];
#pragma unroll
        for (int k = 0; k < K; ++k) pp[k] = lds_vec(X, ct | (k << KT) | ((b ^ (1 << j)) << (KT + KK)));
#pragma unroll
        for (int k = 0; k < K; ++k) cmac<Real, PHI>(o[k], cf, pp[k]);
      }
      // register bits: the partner is another of this thread's own vectors
#pragma unroll
      for (int j = 0; j < KK; ++j) {
        const Coef c0 = coef(V + KT + j, 0), c1 = coef(V + KT + j, 1);
#pragma unroll
        for (int k = 0; k < K; ++k) cmac<Real, PHI>(o[k], ((k >> j) & 1) ? c1 : c0, x[k ^ (1 << j)]);
      }
      // G bits: partners in neighbouring tiles through L2, GB bits at a time
      for (int g0 = 0; g0 < nG; g0 += GB) {
        Vec p[GB][K];
#pragma unroll
        for (int g = 0; g < GB; ++g) {
          // a G bit is fixed per tile, so the partner sits at a uniform offset
          const int64_t gstep = int64_t(1) << (f2 + g0 + g - V);
          const int64_t goff = ((tf2 >> (g0 + g)) & 1) ? -gstep : gstep;
#pragma unroll
          for (int k = 0; k < K; ++k)
            p[g][k] = g0 + g < nG ? ldg_vec(args.xin, vidx0 + koff(k, b) + goff) : Vec{0ull, 0ull};
        }
#pragma unroll
        for (int g = 0; g < GB; ++g) {
          if (g0 + g >= nG) continue;
          const Coef cg = s_cp[f2 + g0 + g][(tf2 >> (g0 + g)) & 1];
#pragma unroll
          for (int k = 0; k < K; ++k) cmac<Real, PHI>(o[k], cg, p[g][k]);
        }
      }
      // z += flips; reduce; store
#pragma unroll
      for (int k = 0; k < K; ++k) {
        axpy<Real>(o[k], (Real)1, zv[k]);
        if (LANCZOS) reduce_vec<Real>(x[k], o[k], r0, r1, r2);
        stg_vec(args.out, vidx0 + koff(k, b), o[k]);
      }
    }
    // release the stage (only shared-memory reads of it were made)
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  if (LANCZOS) {
    Acc acc[3] = {r0, r1, r2};
#pragma unroll
    for (int v = 0; v < 3; ++v) warp_merge(acc[v]);
    if (lane == 0) {
#pragma unroll
      for (int v = 0; v < 3; ++v) s_red[v][warp] = acc[v].value();
    }
  }
  // On an aborted run, let copies still in flight into the ring land before the
  // CTA exits (bounded); on a normal run these phases have already completed.
  if (warp == 0 && lane == 0 && *args.err) {
    for (int ip = produced - 1; ip >= 0 && ip >= produced - kStridedStages; --ip)
      mbar_wait(&full[ip % kStridedStages], (ip / kStridedStages) & 1);
  }
  __syncthreads();
  if (LANCZOS) pass_tail(args.ctl, args.partials, s_red, args.err, smem);
}

template <typename Real, bool LANCZOS, bool PHI>
static cudaError_t launch_one(const TileArgs& args, const TileMaps* maps, int grid, cudaStream_t stream) {
  auto fn = strided_kernel<Real, LANCZOS, PHI>;
  const size_t smem = (size_t)kStridedStages * StridedCfg<Real>::kTileBytes;
  static bool configured = false;  // per instantiation
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  fn<<<grid, kTileThreads, smem, stream>>>(args, *maps);
  return cudaGetLastError();
}

template <typename Real>
static cudaError_t dispatch(const TileArgs& args, const TileMaps* maps, bool lanczos, bool phi, int grid,
                            cudaStream_t stream) {
  if (lanczos)
    return phi ? launch_one<Real, true, true>(args, maps, grid, stream)
               : launch_one<Real, true, false>(args, maps, grid, stream);
  return phi ? launch_one<Real, false, true>(args, maps, grid, stream)
             : launch_one<Real, false, false>(args, maps, grid, stream);
}

cudaError_t launch_strided(const TileArgs& args, const TileMaps* maps, bool lanczos, bool c64, bool phi, int grid,
                           cudaStream_t stream) {
  if (grid <= 0 || !maps) return cudaErrorInvalidValue;
  const int T = c64 ? kStridedTileBitsF : kStridedTileBitsD;
  // the kernel assumes a full tile: all T - c strided bits exist above a, and
  // the first pass owns the contiguous bits
  if (args.L != T || args.c < (c64 ? 1 : 0) || args.c > 8 || args.a + (T - args.c) > args.n || args.nG > 12)
    return cudaErrorInvalidValue;
  return c64 ? dispatch<float>(args, maps, lanczos, phi, grid, stream)
             : dispatch<double>(args, maps, lanczos, phi, grid, stream);
}

}  // namespace rsv
