// Device-side Krylov control for exp(-i H_k dt) psi (arXiv 2510.09813, Sec. III.A
// and Eq. (6)): reduction of the streaming passes' partial sums into the
// Lanczos scalars alpha_j, beta_{j+1}; the small exponential exp(-i tau T_m) e_1
// in FP64; the convergence test; the Krylov combine psi' = |psi| sum_k u_k v_k;
// and the observables <n_i> fused into the combine.
#include "kernels.h"
#include "krylov_math.cuh"
#include "rsv_common.cuh"

namespace rsv {

// ---------------------------------------------------------------------------
// Scalar kernel: after the last streaming pass of Krylov iteration j.
//
// One CTA of four warps, one per SM sub-partition: FP64 instructions occupy a
// sub-partition's FP64 unit for about 70 cycles each and do not pipeline
// within a warp, so the launch keeps their count on the critical path small.
// Every load the launch needs is issued first; the norm bound of T_m is kept
// in the state (one row added per iteration); the tridiagonal and the kept
// Chebyshev expansion are read only when the convergence test runs.
// ---------------------------------------------------------------------------
constexpr int kScalarThreads = 128;

__global__ void __launch_bounds__(kScalarThreads, 1) scalar_kernel(const ScalarArgs A) {
  __shared__ double s_part[3][kScalarThreads / 32];
  __shared__ double s_al[kMaxKrylov], s_be[kMaxKrylov + 1];
  __shared__ double s_ur[kMaxKrylov], s_ui[kMaxKrylov];
  __shared__ ChebWork s_w;
  KState* ks = A.ks;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // ---- loads, all issued before any of them is used ----
  const int status0 = ks->status;
  const int j = ks->j;
  double v[3] = {0.0, 0.0, 0.0};
  for (int p = tid; p < A.nparts; p += kScalarThreads) {
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] += A.partials[(int64_t)p * 3 + i];
  }
  const int m = j + 1;
  const bool maybe_check = m >= A.check_from || m >= A.m_max;
  double tn_prev = 0.0, beta_j = 0.0, tau_rem = 0.0, b0 = 0.0;
  double al_i = 0.0, al_i2 = 0.0, be_i = 0.0;  // rows of T_m by lane (and lane + 32)
  if (warp == 0) {
    tn_prev = ks->tnorm;
    beta_j = j > 0 ? ks->beta[j] : 0.0;  // beta[0] is |psi|, not an entry of T
    tau_rem = ks->tau_rem;
    b0 = ks->beta[0];
    if (maybe_check) {
      if (lane < j) al_i = ks->alpha[lane];
      if (lane <= j) be_i = ks->beta[lane];
      if (lane + 32 < j) al_i2 = ks->alpha[lane + 32];
    }
  }
  if (status0 != kContinue) return;  // uniform: the Krylov space is already accepted
  // ---- partial sums: per warp, then four rows ----
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) s_part[i][warp] = v[i];
  }
  __syncthreads();
  if (warp != 0) return;
  double rs = 0.0;  // lane i < 3: sum i
  if (lane < 3)
    for (int w = 0; w < kScalarThreads / 32; ++w) rs += s_part[lane][w];
  const double r0 = __shfl_sync(0xffffffffu, rs, 0), r1 = __shfl_sync(0xffffffffu, rs, 1),
               r2 = __shfl_sync(0xffffffffu, rs, 2);
  // alpha_j = Re<v_j, u_j> / |v_j|^2 and beta_{j+1} = |u_j - alpha_j v_j| expanded
  // as |u|^2 - 2 alpha Re<v,u> + alpha^2 |v|^2 = |u|^2 - alpha Re<v,u>.
  const LanczosScalars ls = lanczos_scalars(r0, r1, r2);
  const double alpha = ls.alpha, beta = ls.beta;
  const int mk = ls.vanished ? m - 1 : m;  // accepted dimension if this space ends here
  // Gershgorin bound of T_mk: the previous rows' maximum and row j
  const double tn = ls.vanished ? tn_prev : fmax(tn_prev, fabs(alpha) + fabs(beta_j) + fabs(beta));
  const bool breakdown = ls.vanished || beta <= A.breakdown * fmax(tn, 1e-300);
  const bool check = breakdown || maybe_check;
  KrylovDecision d{kContinue, 0.0, 0.0};
  if (check) {
    if (!maybe_check) {  // a breakdown before the expected dimension: load now
      if (lane < j) al_i = ks->alpha[lane];
      if (lane <= j) be_i = ks->beta[lane];
      if (lane + 32 < j) al_i2 = ks->alpha[lane + 32];
    }
    if (lane < m) s_al[lane] = (lane == j) ? alpha : al_i;
    if (lane + 32 < m) s_al[lane + 32] = (lane + 32 == j) ? alpha : al_i2;
    for (int i = lane; i <= m; i += 32) s_be[i] = (i == m) ? beta : (i <= j && i < 32 ? be_i : ks->beta[i]);
    // the kept expansion comes from the previous launch (global) and goes back
    // after use; only its header and the Bessel factors matter
    if (lane == 0) {
      s_w.c_valid = A.cache->c_valid;
      s_w.c_pieces = A.cache->c_pieces;
      s_w.kmax = A.cache->kmax;
      s_w.c_lo = A.cache->c_lo;
      s_w.c_hi = A.cache->c_hi;
      s_w.c_tau = A.cache->c_tau;
      s_w.c_pc = A.cache->c_pc;
      s_w.c_ps = A.cache->c_ps;
    }
    __syncwarp();
    if (s_w.c_valid) {
      for (int k = lane; k <= s_w.kmax; k += 32) {
        s_w.J[k] = A.cache->J[k];
        s_w.jh[k] = A.cache->jh[k];
        s_w.jl[k] = A.cache->jl[k];
      }
    }
    __syncwarp();
    d = krylov_decide(s_al, s_be, mk, ls.vanished ? 0.0 : beta, tau_rem, breakdown, true, A.m_max, A.tol, s_ur,
                      s_ui, s_w);
    if (s_w.c_valid) {
      for (int k = lane; k <= s_w.kmax; k += 32) {
        A.cache->J[k] = s_w.J[k];
        A.cache->jh[k] = s_w.jh[k];
        A.cache->jl[k] = s_w.jl[k];
      }
      if (lane == 0) {
        A.cache->c_pieces = s_w.c_pieces;
        A.cache->kmax = s_w.kmax;
        A.cache->c_lo = s_w.c_lo;
        A.cache->c_hi = s_w.c_hi;
        A.cache->c_tau = s_w.c_tau;
        A.cache->c_pc = s_w.c_pc;
        A.cache->c_ps = s_w.c_ps;
        A.cache->c_valid = 1;
      }
    }
  }
  const int status = d.status;
  const double tau_take = d.tau_take, err = d.err;
  if (lane == 0) {
    ks->alpha[j] = alpha;
    ks->beta[m] = beta;
    ks->tnorm = tn;
    ks->total_iterations += 1;
  }
  if (status != kContinue) {
    for (int i = lane; i < mk; i += 32) {
      ks->coef_re[i] = b0 * s_ur[i];
      ks->coef_im[i] = b0 * s_ui[i];
    }
    if (lane == 0) {
      double rem = tau_rem - tau_take;
      if (status == kDone || rem <= 1e-14 * tau_rem) rem = 0.0;
      ks->m = mk;
      ks->tau_taken = tau_take;
      ks->tau_rem = rem;
      ks->err_est = err;
      ks->max_err_est = fmax(ks->max_err_est, err);
      ks->status = status;
    }
  } else if (lane == 0) {
    ks->form_a = alpha;
    ks->form_s = 1.0 / beta;
    ks->beta_prev = beta;
    ks->j = j + 1;
  }
}

size_t cheb_cache_bytes() { return sizeof(ChebWork); }

cudaError_t launch_scalar(const ScalarArgs& a, cudaStream_t stream) {
  if (!a.cache) return cudaErrorInvalidValue;
  scalar_kernel<<<1, kScalarThreads, 0, stream>>>(a);
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
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    Acc ct;
#pragma unroll
    for (int k = 0; k < (1 << KKMAX); ++k) {
      if (k >= K || !active) continue;
      const int64_t vidx = ((ch << T) >> V) + (tid | (k << kt));
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
        *reinterpret_cast<vec*>(x) = reinterpret_cast<const vec*>(A.psi)[vidx];
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
