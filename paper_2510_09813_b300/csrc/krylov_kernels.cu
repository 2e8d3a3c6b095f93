// Device-side Krylov control for exp(-i H_k dt) psi (arXiv 2510.09813, Sec. III.A
// and Eq. (6)): reduction of the streaming passes' partial sums into the
// Lanczos scalars alpha_j, beta_{j+1}; the small exponential exp(-i tau T_m) e_1
// in FP64; the convergence test; the Krylov combine psi' = |psi| sum_k u_k v_k;
// and the observables <n_i> fused into the combine.
#include "kernels.h"
#include "krylov_control.cuh"
#include "krylov_math.cuh"
#include "rsv_common.cuh"

namespace rsv {

// ---------------------------------------------------------------------------
// Scalar kernel: the Krylov control step of iteration j as a launch of its own
// (krylov_control.cuh). The streaming solver normally runs the same step in the
// last CTA of the iteration's last pass instead.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kControlThreads, 1) scalar_kernel(const ScalarArgs A) {
  __shared__ ControlSmem w;
  krylov_control(A, w);
}

size_t cheb_cache_bytes() { return sizeof(ChebWork); }

cudaError_t launch_scalar(const ScalarArgs& a, cudaStream_t stream) {
  if (!a.cache) return cudaErrorInvalidValue;
  scalar_kernel<<<1, kControlThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Begin kernel: reduce the combine/observe partials into |psi|^2 and <n_i>,
// record the occupations, and reset the Krylov run for the next (sub)step.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) begin_kernel(const BeginArgs A) {
  __shared__ double s_part[kMaxAtoms + 1][kThreads / 32];
  __shared__ double s_tot[kMaxAtoms + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nv = A.n + 1;
  for (int col = 0; col < nv; ++col) {
    double v = 0.0;
    for (int p = tid; p < A.nparts; p += kThreads) v += A.partials[(int64_t)p * nv + col];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) s_part[col][warp] = v;
  }
  __syncthreads();
  if (tid < nv) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += s_part[tid][w];
    s_tot[tid] = s;
  }
  __syncthreads();
  if (A.occ_out && tid < A.n) {
    // atom i sits at bit q = n - 1 - i
    A.occ_out[tid] = s_tot[1 + (A.n - 1 - tid)];
  }
  if (tid == 0) {
    KState* ks = A.ks;
    const double norm2 = s_tot[0];
    ks->norm2 = norm2;
    if (!A.reset_only) {
      const double b0 = sqrt(norm2);
      ks->beta[0] = b0;
      ks->form_a = 0.0;
      ks->form_s = b0 > 0.0 ? 1.0 / b0 : 0.0;
      ks->beta_prev = 0.0;
      ks->tnorm = 0.0;
      ks->arrivals = 0;
      ks->j = 0;
      ks->m = 0;
      ks->status = b0 > 0.0 ? kContinue : kIdle;
      if (A.new_tau > 0.0) {
        ks->tau_rem = A.new_tau;
        ks->substeps = 0;
      } else {
        ks->substeps += 1;
        ks->total_substeps += 1;
      }
    }
  }
}

cudaError_t launch_begin(const BeginArgs& a, cudaStream_t stream) {
  begin_kernel<<<1, kThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Combine + observe: psi = sum_k coef_k v_k (optional), then per-CTA partial
// sums of |psi|^2 and of |psi_b|^2 b_q for every bit q.
//
// Each CTA walks chunks of 2^T amplitudes (T = V + kt + KK bits). Inside a
// chunk a thread owns K consecutive-by-register vectors: the vector-lane bit,
// the 8 thread bits and the KK register bits are resolved from the thread's
// own sums; the chunk-index bits (>= T) get the thread's chunk total.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(kThreads) combine_kernel(const CombineArgs A) {
  using vec = typename CplxT<Real>::vec;
  using Acc = typename AccFor<Real>::type;
  constexpr int V = CplxT<Real>::kLogVec;
  constexpr int NV = 1 << V;
  constexpr int R = 2 * NV;
  constexpr int KKMAX = 4;
  __shared__ Real s_cr[kMaxKrylov], s_ci[kMaxKrylov];
  __shared__ const Real* s_basis[kMaxKrylov];
  __shared__ double s_red[(kMaxAtoms + 1) * (kThreads / 32)];
  constexpr int kMaxHi = kMaxAtoms - (V + 8 + KKMAX);  // chunk-index bits
  __shared__ double s_hi[kThreads / 32][kMaxHi];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (lane < kMaxHi) s_hi[warp][lane] = 0.0;
  const int n = A.n;
  int m = 0;
  if (A.combine) {
    m = A.ks->m;
    if (tid < m) {
      s_cr[tid] = (Real)A.ks->coef_re[tid];
      s_ci[tid] = (Real)A.ks->coef_im[tid];
      s_basis[tid] = reinterpret_cast<const Real*>(A.basis[tid]);
    }
  }
  __syncthreads();
  const int T = n < (V + 8 + KKMAX) ? n : (V + 8 + KKMAX);
  const int kt = (T - V) < 8 ? (T - V) : 8;
  const int kk = T - V - kt;
  const int K = 1 << kk;
  const bool active = tid < (1 << kt);
  const int64_t nchunks = A.dim >> T;

  // Every |psi_b|^2 product is made exact (TwoProduct) and every sum is
  // compensated; the per-thread accumulators stay in registers (compile-time
  // indices), the chunk-index bits use per-warp shared accumulators.
  Acc tot, lane_acc, reg_acc[KKMAX];
  constexpr int kObserveBatch = 8;  // observe mode: vectors loaded ahead of their use
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    Acc ct;
    vec pre[kObserveBatch];  // observe mode: the next kObserveBatch vectors of the chunk
#pragma unroll
    for (int k = 0; k < (1 << KKMAX); ++k) {
      if (k >= K || !active) continue;
      const int64_t vidx = ((ch << T) >> V) + (tid | (k << kt));
      if (!A.combine && (k % kObserveBatch) == 0) {
        // one batch of independent loads instead of one round trip per vector
#pragma unroll
        for (int u = 0; u < kObserveBatch; ++u)
          if (k + u < K) pre[u] = __ldcs(reinterpret_cast<const vec*>(A.psi) + ((ch << T) >> V) + (tid | ((k + u) << kt)));
      }
      Real x[R];
      if (A.combine) {
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = 0;
        // basis vectors kCombineBatch at a time: their loads are issued before
        // their FMAs (a combine of m vectors makes m / kCombineBatch dependent
        // DRAM round trips per amplitude; with 4 in flight it was latency-bound)
        constexpr int kCombineBatch = 8;
        for (int jb0 = 0; jb0 < m; jb0 += kCombineBatch) {
          Real b[kCombineBatch][R];
#pragma unroll
          for (int u = 0; u < kCombineBatch; ++u) {
            if (jb0 + u < m)
              *reinterpret_cast<vec*>(b[u]) = __ldcs(reinterpret_cast<const vec*>(s_basis[jb0 + u]) + vidx);
          }
#pragma unroll
          for (int u = 0; u < kCombineBatch; ++u) {
            if (jb0 + u >= m) continue;
            const Real cr = s_cr[jb0 + u], ci = s_ci[jb0 + u];
#pragma unroll
            for (int e = 0; e < NV; ++e) {
              x[2 * e] = fma(cr, b[u][2 * e], x[2 * e]);
              x[2 * e] = fma(-ci, b[u][2 * e + 1], x[2 * e]);
              x[2 * e + 1] = fma(cr, b[u][2 * e + 1], x[2 * e + 1]);
              x[2 * e + 1] = fma(ci, b[u][2 * e], x[2 * e + 1]);
            }
          }
        }
        reinterpret_cast<vec*>(A.psi)[vidx] = *reinterpret_cast<const vec*>(x);
      } else {
        *reinterpret_cast<vec*>(x) = pre[k % kObserveBatch];
        if (A.mask_bit >= 0) {
          // restrict to amplitudes whose bit mask_bit is 1
#pragma unroll
          for (int e = 0; e < NV; ++e) {
            const int64_t b = (vidx << V) | e;
            if (!((b >> A.mask_bit) & 1)) {
              x[2 * e] = 0;
              x[2 * e + 1] = 0;
            }
          }
        }
      }
      Acc pv;  // this vector's total
#pragma unroll
      for (int e = 0; e < NV; ++e) {
        Acc pe;
        pe.dot(x[2 * e], x[2 * e]);
        pe.dot(x[2 * e + 1], x[2 * e + 1]);
        if (V == 1 && e == 1) lane_acc.merge_acc(pe);
        pv.merge_acc(pe);
      }
      ct.merge_acc(pv);
#pragma unroll
      for (int jr = 0; jr < KKMAX; ++jr)
        if (jr < kk && ((k >> jr) & 1)) reg_acc[jr].merge_acc(pv);
    }
    tot.merge_acc(ct);
    // chunk-index bits: the warp's chunk total goes, by lane hq, into that warp's
    // shared accumulator for chunk bit hq (FP64)
    Acc cw = ct;
    warp_merge(cw);
    if (lane < kMaxHi && T + lane < n && ((ch >> lane) & 1)) s_hi[warp][lane] += cw.value();
  }
  __syncwarp();
  // per-bit contributions of this thread
  Acc out[kMaxAtoms + 1];
  out[0] = tot;
  for (int q = 0; q < n; ++q) {
    Acc v;
    if (q < V) v = lane_acc;
    else if (q < V + kt) { if ((tid >> (q - V)) & 1) v = tot; }
    else if (q < T) {
#pragma unroll
      for (int jr = 0; jr < KKMAX; ++jr)
        if (jr == q - V - kt) v = reg_acc[jr];
    }
    else if (lane == 0) {
      v.add_double(s_hi[warp][q - T]);
    }
    out[1 + q] = v;
  }
  block_reduce_write<kMaxAtoms + 1>(out, s_red, A.partials + (int64_t)blockIdx.x * (n + 1), n + 1);
}

// ---------------------------------------------------------------------------
// Combine through a TMA ring: combine_kernel's combine mode on registers of at
// least one full chunk, with the same arithmetic in the same order (psi summed
// over the basis in index order, then the observation sums over the thread's
// vectors). Each basis vector's 64 KiB chunk tile comes into shared memory by
// one bulk copy, two tiles ahead of the one being summed (128 KiB in flight per
// SM, where eight 16-byte loads per thread kept 64 KiB).
// ---------------------------------------------------------------------------
constexpr int kCombStages = 3;

template <typename Real>
struct CombTma {
  static constexpr int V = CplxT<Real>::kLogVec;
  static constexpr int KK = 4;                   // register bits
  static constexpr int T = V + 8 + KK;           // chunk bits: vector lane, 8 thread bits, register bits
  static constexpr int K = 1 << KK;              // vectors per thread
  static constexpr uint32_t kTileBytes = (1u << T) * 2u * (uint32_t)sizeof(Real);
};
static_assert(CombTma<float>::kTileBytes == 65536 && CombTma<double>::kTileBytes == 65536, "64 KiB tiles");

template <typename Real>
__global__ void __launch_bounds__(kThreads, 1) combine_tma_kernel(const CombineArgs A) {
  using C = CombTma<Real>;
  using vec = typename CplxT<Real>::vec;
  using Acc = typename AccFor<Real>::type;
  constexpr int V = C::V, NV = 1 << V, R = 2 * NV, T = C::T, K = C::K, KK = C::KK;
  constexpr uint32_t kTile = C::kTileBytes;
  extern __shared__ __align__(1024) unsigned char ring[];
  __shared__ __align__(8) uint64_t full[kCombStages], empty[kCombStages];
  __shared__ Real s_cr[kMaxKrylov], s_ci[kMaxKrylov];
  __shared__ const unsigned char* s_basis[kMaxKrylov];
  __shared__ double s_red[(kMaxAtoms + 1) * (kThreads / 32)];
  __shared__ double s_hi[kThreads / 32][kMaxAtoms];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = A.n;
  s_hi[warp][lane] = 0.0;
  const int m = A.ks->m;
  if (tid < m) {
    s_cr[tid] = (Real)A.ks->coef_re[tid];
    s_ci[tid] = (Real)A.ks->coef_im[tid];
    s_basis[tid] = static_cast<const unsigned char*>(A.basis[tid]);
  }
  if (tid == 0) {
    for (int s = 0; s < kCombStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kThreads / 32);
    }
    mbar_fence_init();
  }
  __syncthreads();
  const int64_t nchunks = A.dim >> T;
  const int64_t my_chunks =
      (int64_t)blockIdx.x < nchunks ? (nchunks - 1 - (int64_t)blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t items = my_chunks * m;  // item q: chunk q / m of this CTA, basis vector q % m

  // ---- producer (warp 0): item q into stage q % kCombStages ----
  int64_t produced = 0;
  bool prod_ok = true;
  auto produce = [&](int64_t q) {
    if (q >= items || !prod_ok) return;
    const int s = (int)(q % kCombStages);
    const int64_t r = q / kCombStages;
    if (q >= kCombStages) {
      int okw = 1;
      if (lane == 0) okw = mbar_wait(&empty[s], (uint32_t)((r - 1) & 1)) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) {
        prod_ok = false;
        if (lane == 0) atomicOr(A.err, 1);
        return;
      }
    }
    if (lane == 0) {
      const int64_t ch = (int64_t)blockIdx.x + (q / m) * gridDim.x;
      mbar_arrive_expect_tx(&full[s], kTile);
      tma_load_1d(ring + (size_t)s * kTile, s_basis[q % m] + ch * kTile, kTile, &full[s]);
    }
    __syncwarp();
    produced = q + 1;
  };
  if (warp == 0)
    for (int64_t q = 0; q < kCombStages - 1; ++q) produce(q);

  Acc tot, lane_acc, reg_acc[KK];
  bool ok = true;
  int64_t q = 0;
  for (int64_t i = 0; i < my_chunks && ok; ++i) {
    const int64_t ch = (int64_t)blockIdx.x + i * gridDim.x;
    Real x[K][R];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int e = 0; e < R; ++e) x[k][e] = 0;
    for (int j = 0; j < m; ++j, ++q) {
      if (warp == 0) produce(q + kCombStages - 1);
      const int s = (int)(q % kCombStages);
      if (!mbar_wait(&full[s], (uint32_t)((q / kCombStages) & 1))) {
        if (lane == 0) atomicOr(A.err, 1);
        ok = false;
        break;
      }
      const vec* tile = reinterpret_cast<const vec*>(ring + (size_t)s * kTile);
      const Real cr = s_cr[j], ci = s_ci[j];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        Real b[R];
        *reinterpret_cast<vec*>(b) = tile[tid | (k << 8)];
#pragma unroll
        for (int e = 0; e < NV; ++e) {
          x[k][2 * e] = fma(cr, b[2 * e], x[k][2 * e]);
          x[k][2 * e] = fma(-ci, b[2 * e + 1], x[k][2 * e]);
          x[k][2 * e + 1] = fma(cr, b[2 * e + 1], x[k][2 * e + 1]);
          x[k][2 * e + 1] = fma(ci, b[2 * e], x[k][2 * e + 1]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (!ok) break;
    // psi and this chunk's observation sums, vector by vector as combine_kernel
    Acc ct;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t vidx = ((ch << T) >> V) + (tid | (k << 8));
      reinterpret_cast<vec*>(A.psi)[vidx] = *reinterpret_cast<const vec*>(x[k]);
      Acc pv;
#pragma unroll
      for (int e = 0; e < NV; ++e) {
        Acc pe;
        pe.dot(x[k][2 * e], x[k][2 * e]);
        pe.dot(x[k][2 * e + 1], x[k][2 * e + 1]);
        if (V == 1 && e == 1) lane_acc.merge_acc(pe);
        pv.merge_acc(pe);
      }
      ct.merge_acc(pv);
#pragma unroll
      for (int jr = 0; jr < KK; ++jr)
        if ((k >> jr) & 1) reg_acc[jr].merge_acc(pv);
    }
    tot.merge_acc(ct);
    Acc cw = ct;
    warp_merge(cw);
    if (T + lane < n && ((ch >> lane) & 1)) s_hi[warp][lane] += cw.value();
  }
  // On an aborted run, let copies still in flight into the ring land (bounded)
  if (warp == 0 && lane == 0 && !ok)
    for (int64_t ip = produced - 1; ip >= 0 && ip >= produced - kCombStages; --ip)
      mbar_wait(&full[ip % kCombStages], (uint32_t)((ip / kCombStages) & 1));
  __syncthreads();
  Acc out[kMaxAtoms + 1];
  out[0] = tot;
  for (int qb = 0; qb < n; ++qb) {
    Acc v;
    if (qb < V) v = lane_acc;
    else if (qb < V + 8) { if ((tid >> (qb - V)) & 1) v = tot; }
    else if (qb < T) {
#pragma unroll
      for (int jr = 0; jr < KK; ++jr)
        if (jr == qb - V - 8) v = reg_acc[jr];
    }
    else if (lane == 0) {
      v.add_double(s_hi[warp][qb - T]);
    }
    out[1 + qb] = v;
  }
  block_reduce_write<kMaxAtoms + 1>(out, s_red, A.partials + (int64_t)blockIdx.x * (n + 1), n + 1);
}

template <typename Real>
static cudaError_t launch_combine_tma(const CombineArgs& a, int grid, cudaStream_t stream) {
  const size_t smem = (size_t)kCombStages * CombTma<Real>::kTileBytes;
  static bool configured = false;  // per instantiation
  if (!configured) {
    const cudaError_t e =
        cudaFuncSetAttribute(combine_tma_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  combine_tma_kernel<Real><<<grid, kThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_combine(const CombineArgs& a, bool c64, int grid, cudaStream_t stream) {
  // combine mode on registers of at least one full chunk, with an error word
  // for the ring's bounded waits: the TMA ring; otherwise per-thread loads
  const int T = c64 ? CombTma<float>::T : CombTma<double>::T;
  if (a.combine && a.err && a.n >= T)
    return c64 ? launch_combine_tma<float>(a, grid, stream) : launch_combine_tma<double>(a, grid, stream);
  if (c64)
    combine_kernel<float><<<grid, kThreads, 0, stream>>>(a);
  else
    combine_kernel<double><<<grid, kThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace rsv
