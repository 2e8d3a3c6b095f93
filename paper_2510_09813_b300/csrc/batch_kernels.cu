// Batched time evolution of many small registers in one persistent launch
// (arXiv 2510.09813, Eq. (3), Eq. (6), Sec. III.A for each register).
//
// Each CTA takes registers from a shared work counter (largest first) and
// runs a register's whole pulse sequence before taking the next: per time
// step the midpoint Hamiltonian, the Lanczos recurrence, the FP64
// tridiagonal exponential with its acceptance test and substeps, the combine
// psi = |psi| sum_k u_k v_k and the occupations <n_i>. Nothing returns to the
// host between steps.
//
// Matvec of one Krylov vector (2^n amplitudes in global memory, L2-resident for
// most of the sizes this kernel serves), in 16-byte vectors (two complex64 or
// one complex128 amplitude) with packed FP32x2 arithmetic for complex64:
//   - pass A walks contiguous chunks of 2^T amplitudes (T = min(n, TB)): it
//     forms v_j while staging the chunk in shared memory, adds the diagonal
//     E(b) = E_hi(chunk) + sum_{q<T} w_q b_q + Q[b mod 2^T] (never stored) and
//     the flips of bits < T: the in-vector bit from the vector itself, the 8
//     thread bits from shared memory, the 3 register bits from the thread's
//     own vectors;
//   - for n > TB, pass B walks strided chunks (2^(TB-h) contiguous amplitudes
//     times every value of the h = n - TB high bits) and adds their flips.
// Registers with n <= TB are one chunk, so an iteration is a single sweep.
#include "kernels.h"
#include "krylov_math.cuh"
#include "rsv_common.cuh"
#include "vec_ops.cuh"

namespace rsv {

template <typename Real>
struct BatchCfg;
template <>
struct BatchCfg<float> {
  static constexpr int TB = 12;  // 2^12 complex64 = 32 KiB chunk
};
template <>
struct BatchCfg<double> {
  static constexpr int TB = 11;  // 2^11 complex128 = 32 KiB chunk
};

// dynamic shared memory: the staged chunk (2^TB amplitudes, 32 KiB) and Q
template <typename Real>
size_t batch_dynamic_smem() {
  return (2 * sizeof(Real) + sizeof(Real)) << BatchCfg<Real>::TB;
}

namespace {

constexpr int kBK = 8;   // vectors per thread of a full chunk (2^11 vectors / 256 threads)
constexpr int kBKK = 3;  // register bits of a full chunk
constexpr int kLoadBatch = 4;  // global loads issued together ahead of their stores

// ---- thread-block cluster helpers (distributed shared memory) ----
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Every thread of every CTA of the cluster; release/acquire at cluster scope
// (shared and global memory written before it are visible after it).
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// Address of `p` (this CTA's shared memory) in the shared memory of cluster rank r.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, unsigned r) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(r));
  return out;
}
__device__ __forceinline__ void st_cluster(uint32_t a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t a, unsigned long long v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
template <typename T>
__device__ __forceinline__ void bcast(T* local_field, T v, unsigned ncl) {
  for (unsigned r = 0; r < ncl; ++r) st_cluster(cluster_addr(local_field, r), v);
}

// Loads of vectors another CTA of the cluster may have written: through L2
// (the cluster barrier orders the writes; L1 holds no stale copy).
template <bool COOP>
__device__ __forceinline__ Vec ld_vec(const void* base, int64_t idx) {
  if (COOP) {
    const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(base) + idx);
    return Vec{v.x, v.y};
  }
  return ldv_vec(base, idx);
}

template <typename Real>
struct Shared {
  double V[kBatchMaxAtoms][kBatchMaxAtoms];  // pair energies by bit position
  double delta[kBatchMaxAtoms];
  Coef cp[kBatchMaxAtoms][2];                // flip coefficient by [bit][target bit value], phase form
  Coef cf[kMaxKrylov];                       // combine coefficients |psi| u_k, phase form
  Real w[BatchCfg<Real>::TB];
  Real ehi;
  double al[kMaxKrylov], be[kMaxKrylov + 1], ur[kMaxKrylov], ui[kMaxKrylov];
  ChebWork cw;
  double red[(kBatchMaxAtoms + 1) * (kThreads / 32)];
  double tot[kBatchMaxAtoms + 1];
  double cpart[kBatchCluster][kBatchMaxAtoms + 1];  // cluster rank 0: the CTAs' partial sums
  double tau;
  double tau_take, err, alpha, beta;
  int status;
  int m;
  int item;
};

// Per-chunk diagonal row: s.w[q] = sum_{r >= T} V_qr b_r - delta_q (q < T) and
// s.ehi = sum_{T <= q < r} V_qr b_q b_r - sum_{q >= T} delta_q b_q for the high
// bits b_r of chunk c. One warp.
template <typename Real>
__device__ void chunk_row(Shared<Real>& s, int n, int T, int64_t c, int lane) {
  if (lane < T) {
    double w = -s.delta[lane];
    for (int r = T; r < n; ++r)
      if ((c >> (r - T)) & 1) w += s.V[lane][r];
    s.w[lane] = (Real)w;
  }
  if (lane == 0) {
    double e = 0.0;
    for (int q = T; q < n; ++q) {
      if (!((c >> (q - T)) & 1)) continue;
      e -= s.delta[q];
      for (int r = q + 1; r < n; ++r)
        if ((c >> (r - T)) & 1) e += s.V[q][r];
    }
    s.ehi = (Real)e;
  }
}

// Pass A over contiguous chunk c (see the file comment). `reduce`: this is the
// whole vector (n <= TB), so the Lanczos sums are taken here.
template <typename Real, bool PHI, bool COOP, typename Acc>
__device__ void pass_a(Shared<Real>& s, Vec* s_x, const Real* s_q, int n, int T, int64_t c, const Vec* src,
                       Vec* __restrict__ basis_j, const Vec* __restrict__ basis_prev, Vec* u, bool has_prev, Real a, Real sc, Real bprev,
                       bool reduce, Acc& r0, Acc& r1, Acc& r2) {
  constexpr int V = CplxT<Real>::kLogVec;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int vb = T - V;
  const int kt = vb < 8 ? vb : 8;
  const int kk = vb - kt;
  const int keff = 1 << kk;
  const bool active = tid < (1 << kt);
  const int64_t vbase = c << vb;
  if (warp == 0) chunk_row(s, n, T, c, lane);
#pragma unroll
  for (int k = 0; k < kBK; ++k) {
    if (!active || k >= keff) continue;
    const int t = tid | (k << kt);
    const Vec uu = ld_vec<COOP>(src, vbase + t);
    const Vec pv = has_prev ? ld_vec<COOP>(basis_prev, vbase + t) : Vec{0ull, 0ull};
    const Vec x = form<Real>(uu, pv, a, sc, has_prev);
    sts_vec(s_x, t, x);
    stg_vec(basis_j, vbase + t, x);
  }
  __syncthreads();
  if (active) {
    Real lin_t = s.ehi;
    for (int j = 0; j < kt; ++j)
      if ((tid >> j) & 1) lin_t += s.w[V + j];
    Vec o[kBK];
#pragma unroll
    for (int k = 0; k < kBK; ++k) {
      o[k] = Vec{0ull, 0ull};
      if (k >= keff) continue;
      Real lk = lin_t;
#pragma unroll
      for (int j = 0; j < kBKK; ++j)
        if (j < kk && ((k >> j) & 1)) lk += s.w[V + kt + j];
      const int t = tid | (k << kt);
      const int b0 = t << V;
      const Real e0 = lk + s_q[b0];
      const Real e1 = V == 1 ? lk + s.w[0] + s_q[b0 + 1] : e0;
      const Vec x = lds_vec(s_x, t);
      o[k] = scale2<Real>(x, e0, e1);
      if constexpr (V == 1) {
        // amplitude bit 0: the partner is the other half of the vector
        cmac_word<PHI>(o[k].w0, s.cp[0][0], x.w1);
        cmac_word<PHI>(o[k].w1, s.cp[0][1], x.w0);
      }
    }
    // thread bits: partners from shared memory, all K loads of one bit together
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (j >= kt) continue;
      const Coef cj = s.cp[V + j][(tid >> j) & 1];
      Vec pp[kBK];
#pragma unroll
      for (int k = 0; k < kBK; ++k) pp[k] = k < keff ? lds_vec(s_x, (tid | (k << kt)) ^ (1 << j)) : Vec{0ull, 0ull};
#pragma unroll
      for (int k = 0; k < kBK; ++k)
        if (k < keff) cmac<Real, PHI>(o[k], cj, pp[k]);
    }
    // register bits: the partner is another of this thread's vectors
#pragma unroll
    for (int j = 0; j < kBKK; ++j) {
      if (j >= kk) continue;
      const int q = V + kt + j;
#pragma unroll
      for (int k = 0; k < kBK; ++k)
        if (k < keff) cmac<Real, PHI>(o[k], s.cp[q][(k >> j) & 1], lds_vec(s_x, tid | ((k ^ (1 << j)) << kt)));
    }
#pragma unroll
    for (int k = 0; k < kBK; ++k) {
      if (k >= keff) continue;
      const int t = tid | (k << kt);
      const int64_t vg = vbase + t;
      if (has_prev) axpy<Real>(o[k], -bprev, ld_vec<COOP>(basis_prev, vg));  // this thread read it while staging
      stg_vec(u, vg, o[k]);
      if (reduce) reduce_vec<Real>(lds_vec(s_x, t), o[k], r0, r1, r2);
    }
  }
  __syncthreads();
}

// Pass B (n > TB): flips of the h = n - TB high bits over strided chunks; adds
// them to u and takes the Lanczos sums.
template <typename Real, bool PHI, bool COOP, typename Acc>
__device__ void pass_b(Shared<Real>& s, Vec* s_x, int n, const Vec* basis_j, Vec* u, unsigned g0, unsigned gstep,
                       Acc& r0, Acc& r1, Acc& r2) {
  constexpr int TB = BatchCfg<Real>::TB;
  constexpr int V = CplxT<Real>::kLogVec;
  constexpr int VB = TB - V;               // vector bits of a chunk (11)
  const int tid = threadIdx.x;
  const int h = n - TB;                    // 1 .. kBatchMaxAtoms - TB
  const int cbv = VB - h;                  // contiguous vector bits of a segment
  const int lowmask = (1 << cbv) - 1;
  const int64_t nsc = int64_t(1) << h;
  auto vidx_of = [&](int t, int64_t g) -> int64_t {
    return ((int64_t)(t >> cbv) << VB) | (g << cbv) | (t & lowmask);
  };
  for (int64_t g = g0; g < nsc; g += gstep) {
    {
      Vec x[kBK];
#pragma unroll
      for (int k = 0; k < kBK; ++k) x[k] = ld_vec<COOP>(basis_j, vidx_of(tid | (k << 8), g));
#pragma unroll
      for (int k = 0; k < kBK; ++k) sts_vec(s_x, tid | (k << 8), x[k]);
    }
    __syncthreads();
    // the partial u of the segment, kLoadBatch loads ahead of their stores
#pragma unroll
    for (int k0 = 0; k0 < kBK; k0 += kLoadBatch) {
      Vec y[kLoadBatch];
#pragma unroll
      for (int i = 0; i < kLoadBatch; ++i) y[i] = ld_vec<COOP>(u, vidx_of(tid | ((k0 + i) << 8), g));
#pragma unroll
      for (int i = 0; i < kLoadBatch; ++i) {
      const int k = k0 + i;
      const int t = tid | (k << 8);
#pragma unroll
      for (int r = 0; r < kBatchMaxAtoms - 11 + 1; ++r) {
        if (r >= h) break;
        const int tb = cbv + r;  // vector-index bit of amplitude bit TB + r
        cmac<Real, PHI>(y[i], s.cp[TB + r][(t >> tb) & 1], lds_vec(s_x, t ^ (1 << tb)));
      }
      stg_vec(u, vidx_of(t, g), y[i]);
      reduce_vec<Real>(lds_vec(s_x, t), y[i], r0, r1, r2);
      }
    }
    __syncthreads();
  }
}

// One Lanczos iteration j of a register (all threads of the CTA):
//   v_j = (u - a v_{j-1}) * sc (j > 0) or psi * sc (j = 0), written to basis[j];
//   u   = H v_j - bprev v_{j-1};
//   Re<v_j, u>, |u|^2, |v_j|^2 -> s.tot[0..2].
template <typename Real, bool PHI, bool COOP>
__device__ void lanczos_iteration(Shared<Real>& s, Vec* s_x, const Real* s_q, int n, int T, const Vec* src,
                                  Vec* basis_j, const Vec* basis_prev, Vec* u, int j, Real a, Real sc, Real bprev,
                                  unsigned rank, unsigned ncl) {
  using Acc = typename AccFor<Real>::type;
  const int64_t nch = int64_t(1) << (n - T);
  Acc r0, r1, r2;
  for (int64_t c = rank; c < nch; c += ncl)
    pass_a<Real, PHI, COOP>(s, s_x, s_q, n, T, c, src, basis_j, basis_prev, u, j > 0, a, sc, bprev, nch == 1, r0,
                            r1, r2);
  if (nch > 1) {
    if (COOP) cluster_sync();  // every chunk of v_j and of the partial u is written
    pass_b<Real, PHI, COOP>(s, s_x, n, basis_j, u, rank, ncl, r0, r1, r2);
  }
  Acc acc[3] = {r0, r1, r2};
  block_reduce_write<3>(acc, s.red, s.tot, 3);
}

// psi = sum_{k<m} cf_k basis_k (combine) or psi as is (observe), with
// |psi|^2 -> s.tot[0] and sum_b |psi_b|^2 b_q -> s.tot[1 + q]. Products are
// exact (TwoProduct) and sums compensated.
template <typename Real, bool COOP>
__device__ void combine_observe(Shared<Real>& s, int n, int T, Vec* psi, const Vec* __restrict__ basis, int64_t vstride, int m,
                                bool combine, unsigned rank, unsigned ncl) {
  using Acc = typename AccFor<Real>::type;
  constexpr int V = CplxT<Real>::kLogVec;
  constexpr int HB = kBatchMaxAtoms - 8 - V;  // chunk-index bits at most
  const int tid = threadIdx.x;
  const int vb = T - V;
  const int kt = vb < 8 ? vb : 8;
  const int kk = vb - kt;
  const int keff = 1 << kk;
  const bool active = tid < (1 << kt);
  const int64_t nch = int64_t(1) << (n - T);
  Acc tot, lane_acc, reg[kBKK], hi[HB];
  if (active) {
    for (int64_t c = rank; c < nch; c += ncl) {
      Acc ct;
#pragma unroll
      for (int k = 0; k < kBK; ++k) {
        if (k >= keff) continue;
        const int64_t vg = (c << vb) + (tid | (k << kt));
        Vec x;
        if (combine) {
          x = Vec{0ull, 0ull};
          for (int i0 = 0; i0 < m; i0 += 4) {
            Vec bv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (i0 + q < m) bv[q] = ld_vec<COOP>(basis, (int64_t)(i0 + q) * vstride + vg);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (i0 + q < m) cmac<Real, true>(x, s.cf[i0 + q], bv[q]);
          }
          stg_vec(psi, vg, x);
        } else {
          x = ld_vec<COOP>(psi, vg);
        }
        Acc pv;
        if constexpr (V == 1) {
          float re0, im0, re1, im1;
          f2_unpack(x.w0, re0, im0);
          f2_unpack(x.w1, re1, im1);
          Acc p1;
          pv.dot(re0, re0);
          pv.dot(im0, im0);
          p1.dot(re1, re1);
          p1.dot(im1, im1);
          lane_acc.merge_acc(p1);
          pv.merge_acc(p1);
        } else {
          pv.dot(dbl(x.w0), dbl(x.w0));
          pv.dot(dbl(x.w1), dbl(x.w1));
        }
        ct.merge_acc(pv);
#pragma unroll
        for (int r = 0; r < kBKK; ++r)
          if ((k >> r) & 1) reg[r].merge_acc(pv);
      }
      tot.merge_acc(ct);
#pragma unroll
      for (int hb = 0; hb < HB; ++hb)
        if (T + hb < n && ((c >> hb) & 1)) hi[hb].merge_acc(ct);
    }
  }
  Acc out[kBatchMaxAtoms + 1];
  out[0] = tot;
#pragma unroll
  for (int q = 0; q < kBatchMaxAtoms; ++q) {
    if (q >= n) continue;
    if (q < V) {
      out[1 + q] = lane_acc;
    } else if (q < V + kt) {
      if ((tid >> (q - V)) & 1) out[1 + q] = tot;
    } else if (q < T) {
#pragma unroll
      for (int r = 0; r < kBKK; ++r)
        if (r == q - V - kt) out[1 + q] = reg[r];
    } else {
#pragma unroll
      for (int hb = 0; hb < HB; ++hb)
        if (hb == q - T) out[1 + q] = hi[hb];
    }
  }
  block_reduce_write<kBatchMaxAtoms + 1>(out, s.red, s.tot, n + 1);
  if (COOP) {
    // the cluster's total, in rank order, broadcast by rank 0
    if (threadIdx.x <= n) st_cluster(cluster_addr(&s.cpart[rank][threadIdx.x], 0), s.tot[threadIdx.x]);
    cluster_sync();
    if (rank == 0 && threadIdx.x <= n) {
      double t = 0.0;
      for (unsigned r = 0; r < ncl; ++r) t += s.cpart[r][threadIdx.x];
      bcast(&s.tot[threadIdx.x], t, ncl);
    }
    cluster_sync();
  }
}

}  // namespace

// Evolves register `ri` over its whole pulse sequence. COOP: every CTA of the
// cluster runs this with the same register; chunks are split by cluster rank,
// partial sums meet in rank 0's shared memory, and rank 0 takes every Krylov
// decision and broadcasts it, so all CTAs follow the same control flow and
// meet at the same cluster barriers.
template <typename Real, bool COOP>
__device__ void process_register(const BatchArgs& A, Shared<Real>& s, Vec* s_x, Real* s_q, Vec* states, Vec* work,
                                 int ri, unsigned rank, unsigned ncl) {
  constexpr int TB = BatchCfg<Real>::TB;
  constexpr int V = CplxT<Real>::kLogVec;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const BatchItem it = A.items[ri];
  const int n = it.n;
  const int T = n < TB ? n : TB;
  const int64_t DV = (int64_t(1) << n) >> V;  // vectors per Krylov vector
  Vec* psi = states + (it.state_off >> V);
  Vec* u = work + (int64_t)A.m_max * DV;
  const double* Vm = A.vmat + it.vmat_off;
  for (int i = tid; i < n * n; i += kThreads) s.V[i / n][i % n] = Vm[i];
  __syncthreads();
  // Q[t] = sum_{q<r<T} V_qr t_q t_r over the low bits of b (FP64, rounded once)
  for (int t = tid; t < (1 << T); t += kThreads) {
    double e = 0.0;
    for (int r = 1; r < T; ++r) {
      if (!((t >> r) & 1)) continue;
      for (int q = 0; q < r; ++q)
        if ((t >> q) & 1) e += s.V[q][r];
    }
    s_q[t] = (Real)e;
  }
  // initial |psi|^2 and occupation row 0
  combine_observe<Real, COOP>(s, n, T, psi, nullptr, 0, 0, false, rank, ncl);
  double norm2 = s.tot[0];
  int row = 0;
  auto record = [&](int r) {
    if (rank == 0 && r < it.occ_rows && tid < n) A.occ[it.occ_off + (int64_t)r * n + tid] = s.tot[1 + (n - 1 - tid)];
  };
  record(row++);
  int last_m = 0;
  int64_t iters = 0, subs = 0;
  double max_err = 0.0;
  int status = 0;
  const int steps = A.step_limit > 0 && A.step_limit < it.steps ? A.step_limit : it.steps;
  for (int step = 0; step < steps && status == 0; ++step) {
    const double* P = A.params + it.param_off + (int64_t)step * (1 + 3 * n);
    __syncthreads();
    if (tid < n) {
      // target bit 0: <0|h|1> = Omega/2 e^{+i phi}; target bit 1: <1|h|0> = Omega/2 e^{-i phi}
      const double h = 0.5 * P[1 + tid];
      const double ph = it.has_phi ? P[1 + 2 * n + tid] : 0.0;
      const double cs = h * cos(ph), sn = h * sin(ph);
      s.cp[tid][0] = make_coef<Real, true>((Real)cs, (Real)sn);
      s.cp[tid][1] = make_coef<Real, true>((Real)cs, (Real)(-sn));
      s.delta[tid] = P[1 + n + tid];
    }
    if (tid == 0) s.tau = P[0];
    __syncthreads();
    double tau_rem = s.tau;
    int sub = 0;
    while (tau_rem > 0.0 && norm2 > 0.0) {
      const double b0 = sqrt(norm2);
      const int check_from = last_m > 2 ? last_m - 2 : 1;
      double a = 0.0, sc = 1.0 / b0, bprev = 0.0;
      int m = 0;
      for (int j = 0; j < A.m_max; ++j) {
        Vec* bj = work + (int64_t)j * DV;
        const Vec* bp = j > 0 ? work + (int64_t)(j - 1) * DV : nullptr;
        const Vec* src = j == 0 ? psi : u;
        if (it.has_phi)
          lanczos_iteration<Real, true, COOP>(s, s_x, s_q, n, T, src, bj, bp, u, j, (Real)a, (Real)sc, (Real)bprev,
                                              rank, ncl);
        else
          lanczos_iteration<Real, false, COOP>(s, s_x, s_q, n, T, src, bj, bp, u, j, (Real)a, (Real)sc,
                                               (Real)bprev, rank, ncl);
        ++iters;
        m = j + 1;
        if (COOP) {
          // the CTAs' sums meet in rank 0
          if (tid < 3) st_cluster(cluster_addr(&s.cpart[rank][tid], 0), s.tot[tid]);
          cluster_sync();
        }
        if (warp == 0 && (!COOP || rank == 0)) {
          double r3[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            r3[i] = s.tot[i];
            if (COOP) {
              r3[i] = 0.0;
              for (unsigned r = 0; r < ncl; ++r) r3[i] += s.cpart[r][i];
            }
          }
          const LanczosScalars ls = lanczos_scalars(r3[0], r3[1], r3[2]);
          const double alpha = ls.alpha, beta = ls.beta;
          const int mk = ls.vanished ? m - 1 : m;  // accepted dimension if the space ends here
          if (lane == 0) {
            s.al[j] = alpha;
            s.be[m] = beta;
          }
          __syncwarp();
          double tn = 0.0;
          for (int i = lane; i < mk; i += 32)
            tn = fmax(tn, fabs(s.al[i]) + fabs(s.be[i + 1]) + (i > 0 ? fabs(s.be[i]) : 0.0));
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, off));
          const bool breakdown = ls.vanished || beta <= A.breakdown * fmax(tn, 1e-300);
          const bool check = breakdown || m >= check_from || m >= A.m_max;
          const KrylovDecision d = krylov_decide(s.al, s.be, mk, ls.vanished ? 0.0 : beta, tau_rem, breakdown,
                                                 check, A.m_max, A.tol, s.ur, s.ui, s.cw);
          if (d.status != kContinue) {
            for (int i = lane; i < mk; i += 32) {
              const Coef cf = make_coef<Real, true>((Real)(b0 * s.ur[i]), (Real)(b0 * s.ui[i]));
              if (COOP) {
                bcast(&s.cf[i].rr, cf.rr, ncl);
                bcast(&s.cf[i].ii, cf.ii, ncl);
              } else {
                s.cf[i] = cf;
              }
            }
          }
          if (lane == 0) {
            if (COOP) {
              bcast(&s.m, mk, ncl);
              bcast(&s.status, (int)d.status, ncl);
              bcast(&s.tau_take, d.tau_take, ncl);
              bcast(&s.err, d.err, ncl);
              bcast(&s.alpha, alpha, ncl);
              bcast(&s.beta, beta, ncl);
            } else {
              s.m = mk;
              s.status = d.status;
              s.tau_take = d.tau_take;
              s.err = d.err;
              s.alpha = alpha;
              s.beta = beta;
            }
          }
        }
        if (COOP)
          cluster_sync();  // the decision is in every CTA's shared memory
        else
          __syncthreads();
        if (s.status != kContinue) {
          m = s.m;
          break;
        }
        a = s.alpha;
        sc = 1.0 / s.beta;
        bprev = s.beta;
      }
      const int st = s.status;
      const double take = s.tau_take;
      max_err = fmax(max_err, s.err);
      last_m = m;
      double rem = tau_rem - take;
      if (st == kDone || rem <= 1e-14 * tau_rem) rem = 0.0;
      combine_observe<Real, COOP>(s, n, T, psi, work, DV, m, true, rank, ncl);
      norm2 = s.tot[0];
      tau_rem = rem;
      if (tau_rem > 0.0) {
        ++sub;
        ++subs;
        if (sub > A.max_substeps) {
          status = -3;
          break;
        }
      }
    }
    const int done = step + 1;
    if ((it.obs_stride > 0 && done % it.obs_stride == 0) || done == steps) record(row++);
  }
  if (tid == 0 && rank == 0) {
    BatchOut o;
    o.iterations = iters;
    o.substeps = subs;
    o.max_err = max_err;
    o.norm2 = norm2;
    o.status = status;
    o.rows = row < it.occ_rows ? row : it.occ_rows;
    A.out[ri] = o;
  }
  __syncthreads();
}

template <typename Real>
__global__ void __launch_bounds__(kThreads, 2) batch_kernel(const BatchArgs A) {
  constexpr int TB = BatchCfg<Real>::TB;
  constexpr int V = CplxT<Real>::kLogVec;
  extern __shared__ __align__(16) unsigned char dyn[];
  Vec* s_x = reinterpret_cast<Vec*>(dyn);
  Real* s_q = reinterpret_cast<Real*>(dyn + (2 * sizeof(Real) << TB));
  __shared__ Shared<Real> s;
  const int tid = threadIdx.x;
  if (tid == 0) cheb_reset(s.cw);  // the kept expansion starts empty (first use is after barriers)
  Vec* states = reinterpret_cast<Vec*>(A.states);
  const int64_t wstride = A.work_stride >> V;
  Vec* work = reinterpret_cast<Vec*>(A.work) + (int64_t)blockIdx.x * wstride;

  // Phase 1: the large registers, one whole cluster each (the workspace of the
  // cluster's rank-0 CTA holds the shared Krylov vectors).
  const unsigned ncl = (unsigned)A.cluster;
  if (ncl > 1 && A.count_large > 0) {
    const unsigned rank = cluster_rank();
    Vec* cwork = reinterpret_cast<Vec*>(A.work) + (int64_t)(blockIdx.x - rank) * wstride;
    for (;;) {
      if (rank == 0 && tid == 0) bcast(&s.item, atomicAdd(&A.next[0], 1), ncl);
      cluster_sync();
      const int qi = s.item;
      cluster_sync();  // every CTA read s.item before the next broadcast
      if (qi >= A.count_large) break;
      process_register<Real, true>(A, s, s_x, s_q, states, cwork, A.order[qi], rank, ncl);
    }
  }
  // Phase 2: the other registers, one CTA each.
  for (;;) {
    if (tid == 0) s.item = A.count_large + atomicAdd(&A.next[1], 1);
    __syncthreads();
    const int qi = s.item;
    __syncthreads();
    if (qi >= A.count) break;
    process_register<Real, false>(A, s, s_x, s_q, states, work, A.order[qi], 0, 1);
  }
}

namespace {

template <typename Real>
cudaError_t launch_typed(const BatchArgs& a, int grid, cudaStream_t stream) {
  if (a.cluster <= 1) {
    batch_kernel<Real><<<grid, kThreads, batch_dynamic_smem<Real>(), stream>>>(a);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = batch_dynamic_smem<Real>();
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_kernel<Real>, a);
}

template <typename Real>
int prepare_typed(int cluster, int* max_clusters) {
  // several CTAs per SM need the shared-memory side of the L1/shared split
  cudaFuncSetAttribute(batch_kernel<Real>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  cudaFuncSetAttribute(batch_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)batch_dynamic_smem<Real>());
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<Real>, kThreads, batch_dynamic_smem<Real>());
  *max_clusters = 0;
  if (cluster > 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = batch_dynamic_smem<Real>();
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(max_clusters, batch_kernel<Real>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      *max_clusters = 0;
    }
  }
  return nb;
}

}  // namespace

cudaError_t launch_batch(const BatchArgs& a, bool c64, int grid, cudaStream_t stream) {
  return c64 ? launch_typed<float>(a, grid, stream) : launch_typed<double>(a, grid, stream);
}

int batch_prepare(bool c64, int cluster, int* max_clusters) {
  return c64 ? prepare_typed<float>(cluster, max_clusters) : prepare_typed<double>(cluster, max_clusters);
}

}  // namespace rsv
