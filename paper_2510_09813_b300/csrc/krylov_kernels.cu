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

cudaError_t launch_combine(const CombineArgs& a, bool c64, int grid, cudaStream_t stream) {
  if (c64)
    combine_kernel<float><<<grid, kThreads, 0, stream>>>(a);
  else
    combine_kernel<double><<<grid, kThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace rsv
