// Shared device-side definitions of the B300 state-vector Rydberg library.
//
// Conventions (arXiv 2510.09813, Sec. II.B, Eq. (4)): a state of N atoms is a
// contiguous array of 2^N complex amplitudes; atom i lives at bit position
// q = N-1-i of the basis index (atom 0 is the most significant bit). Inside
// the library everything is indexed by bit position q.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rsv {

constexpr int kMaxAtoms = 32;   // bit positions 0..31
constexpr int kMaxKrylov = 64;  // Krylov dimension cap (tridiagonal size)
constexpr int kThreads = 256;   // block size of the streaming kernels

// Per-time-step Hamiltonian parameters of Eq. (3) after the midpoint rule of
// Sec. III, indexed by bit position q.
struct StepParams {
  double half_omega[kMaxAtoms];  // Omega_bar_q / 2, rad/us
  double phi[kMaxAtoms];         // phi_bar_q, rad
  double delta[kMaxAtoms];       // delta_bar_q, rad/us
  double tau;                    // step length, us
  int32_t has_phi;
  int32_t pad;
};

// Krylov status values written by the scalar kernel.
enum : int32_t { kContinue = 0, kDone = 1, kDonePartial = 2, kIdle = 3 };

// Device-resident scalars of one Lanczos run (Sec. III.A): the tridiagonal
// T_m, the exponential coefficients and the values the next streaming pass
// needs to form v_{j+1} = (u_j - alpha_j v_j) / beta_{j+1}.
struct KState {
  // --- status block (first 128 bytes; the host mirrors only this part) ---
  int32_t status;
  int32_t j;                     // index of the Krylov vector the next pass forms
  int32_t m;                     // accepted Krylov dimension
  int32_t substeps;              // Krylov restarts inside the current step
  double tau_rem;                // remaining time of the current step (us)
  double tau_taken;              // time covered by the accepted Krylov space
  double err_est;                // a-posteriori error estimate of the accepted space
  double max_err_est;            // running maximum over the solve
  double norm2;                  // |psi|^2 of the current state
  int64_t total_iterations;
  int64_t total_substeps;
  int32_t error;                 // set by kernels whose bounded waits timed out
  uint32_t arrivals;             // CTAs of the running last pass that have finished (fused control)
  double tnorm;                  // Gershgorin bound of T_m so far (max row sum), reset per Krylov space
  // device time of the control step (%globaltimer ns), over the solver's life
  uint64_t ctl_ns, ctl_steps;    // every step that did work
  uint64_t chk_ns, chk_steps;    // steps that evaluated the small exponential
  double pad_[1];
  // --- values consumed by the next "first" pass ---
  double form_a;                 // alpha_{j-1} (0 for j = 0)
  double form_s;                 // 1 / beta_j (1 / |psi| for j = 0)
  double beta_prev;              // beta_j (0 for j = 0)
  // --- tridiagonal T_m and the exponential coefficients ---
  double alpha[kMaxKrylov];      // diagonal of T
  double beta[kMaxKrylov + 1];   // beta[k] couples v_{k-1} and v_k; beta[0] = |psi|
  double coef_re[kMaxKrylov];    // |psi| * exp(-i tau T_m) e_1
  double coef_im[kMaxKrylov];
};
constexpr int kStatusBytes = 128;
static_assert(sizeof(int32_t) * 6 + sizeof(double) * 5 + sizeof(int64_t) * 2 + sizeof(double) * 1 +
                  sizeof(uint64_t) * 4 + sizeof(double) * 1 == kStatusBytes,
              "status block layout");

template <typename Real>
struct CplxT;
template <>
struct CplxT<float> {
  using type = float2;
  using vec = float4;  // 16-byte vector = 2 amplitudes
  static constexpr int kLogVec = 1;
};
template <>
struct CplxT<double> {
  using type = double2;
  using vec = double2;  // 16-byte vector = 1 amplitude
  static constexpr int kLogVec = 0;
};

// ---------------------------------------------------------------------------
// FP64-class accumulation for the complex64 path.
//
// B300's FP64 rate is a small fraction of its FP32 rate, so per-amplitude FP64
// arithmetic would dominate an HBM-bound kernel. Inner products and norms are
// therefore accumulated as unevaluated float pairs (hi + lo): products are
// made exact with an FMA (TwoProduct) and sums with Knuth's TwoSum, the
// cascaded scheme of Ogita, Rump and Oishi, "Accurate sum and dot product"
// (SIAM J. Sci. Comput. 26, 2005). Only block totals are promoted to FP64.
// The _rn intrinsics keep the compiler from contracting or reassociating.
// ---------------------------------------------------------------------------
struct AccF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float b) {
    float s = __fadd_rn(hi, b);
    float bp = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void dot(float x, float y) {
    float p = __fmul_rn(x, y);
    float e = __fmaf_rn(x, y, -p);
    add(p);
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void merge(float ohi, float olo) {
    add(ohi);
    lo = __fadd_rn(lo, olo);
  }
  __device__ __forceinline__ void merge_acc(const AccF& o) { merge(o.hi, o.lo); }
  // adds a double as an unevaluated float pair (exact to ~2^-48 relative)
  __device__ __forceinline__ void add_double(double d) {
    const float h = (float)d;
    merge(h, (float)(d - (double)h));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

struct AccD {
  double v = 0.0;
  __device__ __forceinline__ void add(double b) { v += b; }
  __device__ __forceinline__ void dot(double x, double y) { v = fma(x, y, v); }
  __device__ __forceinline__ void merge_acc(const AccD& o) { v += o.v; }
  __device__ __forceinline__ void add_double(double d) { v += d; }
  __device__ __forceinline__ double value() const { return v; }
};

template <typename Real>
struct AccFor;
template <>
struct AccFor<float> {
  using type = AccF;
};
template <>
struct AccFor<double> {
  using type = AccD;
};

__device__ __forceinline__ void warp_merge(AccF& a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    float oh = __shfl_xor_sync(0xffffffffu, a.hi, off);
    float ol = __shfl_xor_sync(0xffffffffu, a.lo, off);
    a.merge(oh, ol);
  }
}
__device__ __forceinline__ void warp_merge(AccD& a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a.v += __shfl_xor_sync(0xffffffffu, a.v, off);
}

// Block-wide sum of NV accumulators; the first `nout` totals are written to
// out[0 .. nout-1] as doubles. Requires blockDim.x == kThreads and `scratch` of
// NV * (kThreads / 32) doubles. Deterministic: fixed reduction tree.
template <int NV, typename A>
__device__ void block_reduce_write(A (&acc)[NV], double* scratch, double* out, int nout = NV) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) warp_merge(acc[i]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) scratch[i * (kThreads / 32) + warp] = acc[i].value();
  }
  __syncthreads();
  if (threadIdx.x < nout) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += scratch[threadIdx.x * (kThreads / 32) + w];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

}  // namespace rsv
