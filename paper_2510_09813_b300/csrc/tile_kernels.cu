// Fused structured matvec y = H x for the Rydberg Hamiltonian (arXiv 2510.09813,
// Eq. (3)) and the Lanczos iteration built on it (Sec. III.A).
//
// H x is "apply the diagonal, then add the Omega-scaled bit-flip permutations"
// (Sec. III.A). Here the diagonal is never stored: each tile rebuilds
//     E(b) = sum_{q<r} V_qr b_q b_r - sum_q delta_q b_q
// from FP64 pair energies as E_hi(tile) + sum_{q<L} w_q(tile) b_q + Q[b_lo].
//
// A tile is a 2^L-amplitude sub-cube of the state: tile bits [0,c) are the
// amplitude bits [0,c) (contiguous in memory, for coalescing) and tile bits
// [c,L) are amplitude bits [a, a+L-c). Every other bit is fixed per tile. The
// tile is staged in shared memory, so flips of all L tile bits are resolved on
// chip: the vector lane bit in registers, the 8 "thread" bits through shared
// memory and the "register" bits inside each thread's register array. Flips of
// the lowest nG fixed bits (G bits) read the partner tile through L2; tiles
// that differ only in G bits are scheduled back to back so those partners are
// L2 hits. A full matvec over N > L bits is one pass (N <= L + nG) or two
// passes: a contiguous pass over bits [0, L) plus a strided pass over the rest.
//
// The Lanczos variant fuses, per amplitude: forming v_j = (u_{j-1} -
// alpha_{j-1} v_{j-1}) / beta_j from the previous pass's output, writing v_j
// into the Krylov basis, the matvec, the three-term subtraction -beta_j v_{j-1}
// and the three reductions Re<v_j,u_j>, |u_j|^2, |v_j|^2 from which the scalar
// kernel derives alpha_j and beta_{j+1} without another pass.
#include "kernels.h"
#include "rsv_common.cuh"

namespace rsv {

template <typename Real>
struct Lanes {
  static constexpr int kLogVec = CplxT<Real>::kLogVec;
  static constexpr int kNV = 1 << kLogVec;  // amplitudes per 16-byte vector
  static constexpr int kR = 2 * kNV;         // reals per vector
};

template <typename Real>
__device__ __forceinline__ void load_vec(Real (&d)[Lanes<Real>::kR], const void* base, int64_t vidx) {
  using vec = typename CplxT<Real>::vec;
  vec v = reinterpret_cast<const vec*>(base)[vidx];
  *reinterpret_cast<vec*>(d) = v;
}
template <typename Real>
__device__ __forceinline__ void load_vec_cs(Real (&d)[Lanes<Real>::kR], const void* base, int64_t vidx) {
  using vec = typename CplxT<Real>::vec;
  vec v = __ldcs(reinterpret_cast<const vec*>(base) + vidx);
  *reinterpret_cast<vec*>(d) = v;
}
template <typename Real>
__device__ __forceinline__ void store_vec(void* base, int64_t vidx, const Real (&s)[Lanes<Real>::kR]) {
  using vec = typename CplxT<Real>::vec;
  reinterpret_cast<vec*>(base)[vidx] = *reinterpret_cast<const vec*>(s);
}
template <typename Real>
__device__ __forceinline__ void store_vec_cs(void* base, int64_t vidx, const Real (&s)[Lanes<Real>::kR]) {
  using vec = typename CplxT<Real>::vec;
  __stcs(reinterpret_cast<vec*>(base) + vidx, *reinterpret_cast<const vec*>(s));
}

// o += coef * p for one complex amplitude; coef real unless PHI.
template <typename Real, bool PHI>
__device__ __forceinline__ void cmac(Real& ore, Real& oim, Real cr, Real ci, Real pre, Real pim) {
  if (PHI) {
    ore = fma(cr, pre, ore);
    ore = fma(-ci, pim, ore);
    oim = fma(cr, pim, oim);
    oim = fma(ci, pre, oim);
  } else {
    ore = fma(cr, pre, ore);
    oim = fma(cr, pim, oim);
  }
}

template <typename Real, int KK, bool LANCZOS, bool FIRST, bool LAST, bool PHI>
__global__ void __launch_bounds__(kThreads, 2) tile_kernel(const TileArgs args) {
  using L_ = Lanes<Real>;
  using Acc = typename AccFor<Real>::type;
  constexpr int V = L_::kLogVec;
  constexpr int NV = L_::kNV;
  constexpr int R = L_::kR;
  constexpr int K = 1 << KK;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sx = reinterpret_cast<Real*>(smem_raw);  // tile: [2^(L-V)] vectors of R reals
  __shared__ double s_w[kMaxAtoms];
  __shared__ double s_ehi;
  __shared__ Real s_linreg[K];
  __shared__ Real s_coef[kMaxAtoms][2][2];  // [amp bit][bit state of the target][re, im]
  __shared__ double s_red[3 * (kThreads / 32)];

  if (LANCZOS && args.ks->status != kContinue) return;

  const int tid = threadIdx.x;
  const int n = args.n, L = args.L, c = args.c, a = args.a, f2 = args.f2;
  const int nF2 = args.nF2, nG = args.nG, kt = args.kt;
  const bool active = tid < (1 << kt);
  const StepParams* sp = args.sp;

  if (tid < n) {
    const double ho = sp->half_omega[tid];
    if (PHI) {
      double sn, cs;
      sincos(sp->phi[tid], &sn, &cs);
      // target bit 0: <0|h|1> = Omega/2 e^{+i phi}; target bit 1: <1|h|0> = Omega/2 e^{-i phi}
      s_coef[tid][0][0] = (Real)(ho * cs);
      s_coef[tid][0][1] = (Real)(ho * sn);
      s_coef[tid][1][0] = (Real)(ho * cs);
      s_coef[tid][1][1] = (Real)(-ho * sn);
    } else {
      s_coef[tid][0][0] = s_coef[tid][1][0] = (Real)ho;
      s_coef[tid][0][1] = s_coef[tid][1][1] = (Real)0;
    }
  }

  double form_a = 0.0, form_s = 1.0, beta_prev = 0.0;
  int jj = 0;
  if (LANCZOS && FIRST) {
    form_a = args.ks->form_a;
    form_s = args.ks->form_s;
    beta_prev = args.ks->beta_prev;
    jj = args.ks->j;
  }
  const Real fa = (Real)form_a, fs = (Real)form_s, bp = (Real)beta_prev;
  const Real* qtab = reinterpret_cast<const Real*>(args.qtab);

  Acc r0, r1, r2;
  const int64_t cmask = (int64_t(1) << c) - 1;
  const int64_t f2mask = (int64_t(1) << nF2) - 1;

  for (int64_t tile = blockIdx.x; tile < args.num_tiles; tile += gridDim.x) {
    const int64_t base = ((tile >> nF2) << c) | ((tile & f2mask) << f2);
    __syncthreads();  // previous tile's shared-memory readers are done
    if (FIRST) {
      // Diagonal decomposition for this tile (c == L: tile bits == amplitude bits [0, L)).
      if (tid < L) {
        double w = -sp->delta[tid];
        for (int r = L; r < n; ++r)
          if ((tile >> (r - L)) & 1) w += args.vmat[tid * kMaxAtoms + r];
        s_w[tid] = w;
      }
      if (tid == 32) {
        double e = 0.0;
        for (int q = L; q < n; ++q) {
          if (!((tile >> (q - L)) & 1)) continue;
          e -= sp->delta[q];
          for (int r = q + 1; r < n; ++r)
            if ((tile >> (r - L)) & 1) e += args.vmat[q * kMaxAtoms + r];
        }
        s_ehi = e;
      }
    }
    // Load (or form) this thread's vectors and stage them in shared memory.
    Real xr[K][R];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!active) continue;
      const int tv = tid | (k << kt);
      const int t = tv << V;
      const int64_t amp = base | (t & cmask) | ((int64_t)(t >> c) << a);
      const int64_t vidx = amp >> V;
      if (LANCZOS && FIRST) {
        Real u[R];
        load_vec_cs<Real>(u, args.xin, vidx);
        if (jj > 0) {
          Real p[R];
          load_vec<Real>(p, args.xprev, vidx);
#pragma unroll
          for (int i = 0; i < R; ++i) xr[k][i] = (u[i] - fa * p[i]) * fs;
        } else {
#pragma unroll
          for (int i = 0; i < R; ++i) xr[k][i] = u[i] * fs;
        }
        store_vec<Real>(args.xout, vidx, xr[k]);
      } else {
        load_vec<Real>(xr[k], args.xin, vidx);
      }
#pragma unroll
      for (int i = 0; i < R; ++i) sx[tv * R + i] = xr[k][i];
    }
    __syncthreads();
    if (FIRST && tid < K) {
      double s = 0.0;
#pragma unroll
      for (int jr = 0; jr < KK; ++jr)
        if ((tid >> jr) & 1) s += s_w[V + kt + jr];
      s_linreg[tid] = (Real)s;
    }
    Real lin_thread = 0;
    if (FIRST) {
      double s = s_ehi;
      for (int j = 0; j < kt; ++j)
        if ((tid >> j) & 1) s += s_w[V + j];
      lin_thread = (Real)s;
    }
    if (FIRST) __syncthreads();  // s_linreg ready
    if (!active) continue;

#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int tv = tid | (k << kt);
      const int t = tv << V;
      const int64_t amp = base | (t & cmask) | ((int64_t)(t >> c) << a);
      const int64_t vidx = amp >> V;
      Real o[R];
      if (FIRST) {
        const Real lk = lin_thread + s_linreg[k];
#pragma unroll
        for (int e = 0; e < NV; ++e) {
          Real E = lk + qtab[t + e];
          if (V == 1 && e == 1) E += (Real)s_w[0];
          o[2 * e] = E * xr[k][2 * e];
          o[2 * e + 1] = E * xr[k][2 * e + 1];
        }
      } else {
        load_vec_cs<Real>(o, args.out, vidx);
      }
      // Tile bits [0, c) of the strided (second) pass are there only for
      // coalescing: their flips belong to the first pass, so they are skipped.
      // (a) vector-lane bit: tile bit 0 == amplitude bit 0 (requires c >= 1)
      if (V == 1 && FIRST) {
        cmac<Real, PHI>(o[0], o[1], s_coef[0][0][0], s_coef[0][0][1], xr[k][2], xr[k][3]);
        cmac<Real, PHI>(o[2], o[3], s_coef[0][1][0], s_coef[0][1][1], xr[k][0], xr[k][1]);
      }
      // (b) thread bits through shared memory
      for (int j = FIRST ? 0 : (c > V ? c - V : 0); j < kt; ++j) {
        const int tb = V + j;
        const int q = tb < c ? tb : a + (tb - c);
        const int bs = (tid >> j) & 1;
        const Real cr = s_coef[q][bs][0], ci = s_coef[q][bs][1];
        Real p[R];
        *reinterpret_cast<typename CplxT<Real>::vec*>(p) =
            *reinterpret_cast<const typename CplxT<Real>::vec*>(sx + (tv ^ (1 << j)) * R);
#pragma unroll
        for (int e = 0; e < NV; ++e) cmac<Real, PHI>(o[2 * e], o[2 * e + 1], cr, ci, p[2 * e], p[2 * e + 1]);
      }
      // (c) register bits
#pragma unroll
      for (int jr = 0; jr < KK; ++jr) {
        const int tb = V + kt + jr;
        if (!FIRST && tb < c) continue;
        const int q = tb < c ? tb : a + (tb - c);
        const int bs = (k >> jr) & 1;
        const Real cr = s_coef[q][bs][0], ci = s_coef[q][bs][1];
#pragma unroll
        for (int e = 0; e < NV; ++e)
          cmac<Real, PHI>(o[2 * e], o[2 * e + 1], cr, ci, xr[k ^ (1 << jr)][2 * e], xr[k ^ (1 << jr)][2 * e + 1]);
      }
      // (d) G bits: partner tiles through L2
      for (int g = 0; g < nG; ++g) {
        const int q = f2 + g;
        const int bs = (int)((tile >> g) & 1);
        const Real cr = s_coef[q][bs][0], ci = s_coef[q][bs][1];
        const int64_t pidx = vidx ^ (int64_t(1) << (q - V));
        Real p[R];
        if (LANCZOS && FIRST) {
          Real u[R];
          load_vec<Real>(u, args.xin, pidx);
          if (jj > 0) {
            Real pp[R];
            load_vec<Real>(pp, args.xprev, pidx);
#pragma unroll
            for (int i = 0; i < R; ++i) p[i] = (u[i] - fa * pp[i]) * fs;
          } else {
#pragma unroll
            for (int i = 0; i < R; ++i) p[i] = u[i] * fs;
          }
        } else {
          load_vec<Real>(p, args.xin, pidx);
        }
#pragma unroll
        for (int e = 0; e < NV; ++e) cmac<Real, PHI>(o[2 * e], o[2 * e + 1], cr, ci, p[2 * e], p[2 * e + 1]);
      }
      // (e) three-term recurrence
      if (LANCZOS && FIRST) {
        if (jj > 0) {
          Real p[R];
          load_vec<Real>(p, args.xprev, vidx);
#pragma unroll
          for (int i = 0; i < R; ++i) o[i] = fma(-bp, p[i], o[i]);
        }
      }
      if (LANCZOS && LAST) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          r0.dot(xr[k][i], o[i]);
          r1.dot(o[i], o[i]);
          r2.dot(xr[k][i], xr[k][i]);
        }
      }
      store_vec<Real>(args.out, vidx, o);
    }
  }
  if (LANCZOS && LAST) {
    Acc acc[3] = {r0, r1, r2};
    __syncthreads();
    block_reduce_write<3>(acc, s_red, args.partials + (int64_t)blockIdx.x * 3);
  }
}

// ---------------------------------------------------------------------------
// Host-side launch
// ---------------------------------------------------------------------------

template <typename Real, int KK, bool LANCZOS, bool FIRST, bool LAST, bool PHI>
static cudaError_t launch_one(const TileArgs& args, int grid, cudaStream_t stream) {
  auto fn = tile_kernel<Real, KK, LANCZOS, FIRST, LAST, PHI>;
  const int smem = (1 << args.L) * 2 * (int)sizeof(Real);
  static bool configured = false;  // per instantiation
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 1 << 16);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  fn<<<grid, kThreads, smem, stream>>>(args);
  return cudaGetLastError();
}

template <typename Real, bool LANCZOS, bool FIRST, bool LAST, bool PHI>
static cudaError_t dispatch_kk(const TileArgs& args, int kk, int grid, cudaStream_t stream) {
  switch (kk) {
    case 0: return launch_one<Real, 0, LANCZOS, FIRST, LAST, PHI>(args, grid, stream);
    case 1: return launch_one<Real, 1, LANCZOS, FIRST, LAST, PHI>(args, grid, stream);
    case 2: return launch_one<Real, 2, LANCZOS, FIRST, LAST, PHI>(args, grid, stream);
    case 3: return launch_one<Real, 3, LANCZOS, FIRST, LAST, PHI>(args, grid, stream);
    case 4: return launch_one<Real, 4, LANCZOS, FIRST, LAST, PHI>(args, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <typename Real>
static cudaError_t dispatch(const TileArgs& args, TileMode mode, bool phi, int grid, cudaStream_t stream) {
  const int kk = args.L - Lanes<Real>::kLogVec - args.kt;
  switch (mode) {
    case TileMode::kMatvecFirst:
      return phi ? dispatch_kk<Real, false, true, false, true>(args, kk, grid, stream)
                 : dispatch_kk<Real, false, true, false, false>(args, kk, grid, stream);
    case TileMode::kMatvecSecond:
      return phi ? launch_one<Real, 4, false, false, false, true>(args, grid, stream)
                 : launch_one<Real, 4, false, false, false, false>(args, grid, stream);
    case TileMode::kLanczosSingle:
      return phi ? dispatch_kk<Real, true, true, true, true>(args, kk, grid, stream)
                 : dispatch_kk<Real, true, true, true, false>(args, kk, grid, stream);
    case TileMode::kLanczosFirst:
      return phi ? launch_one<Real, 4, true, true, false, true>(args, grid, stream)
                 : launch_one<Real, 4, true, true, false, false>(args, grid, stream);
    case TileMode::kLanczosSecond:
      return phi ? launch_one<Real, 4, true, false, true, true>(args, grid, stream)
                 : launch_one<Real, 4, true, false, true, false>(args, grid, stream);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_tile(const TileArgs& args, TileMode mode, bool c64, bool phi, int grid, cudaStream_t stream) {
  if (grid <= 0) return cudaErrorInvalidValue;
  return c64 ? dispatch<float>(args, mode, phi, grid, stream) : dispatch<double>(args, mode, phi, grid, stream);
}

}  // namespace rsv
