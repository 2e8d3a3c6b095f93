// Host-side declarations of the kernel launchers (internal to the library).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rsv_common.cuh"

namespace rsv {

// Streaming tile pass geometry (tile_kernels.cu).
constexpr int kTileBitsF = 12;  // complex64 tile: 2^12 amplitudes = 32 KiB
constexpr int kTileBitsD = 11;  // complex128 tile: 2^11 amplitudes = 32 KiB
constexpr int kConsumerWarps = 16;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kTileThreads = kConsumers;       // warp 0 also issues the TMA loads
constexpr int kStages = 3;                     // shared-memory ring depth (2 tiles per stage)
// Strided pass with x alone staged (strided_kernels.cu): 64 KiB tiles.
constexpr int kStridedTileBitsF = 13;          // complex64: 2^13 amplitudes
constexpr int kStridedTileBitsD = 12;          // complex128: 2^12 amplitudes
constexpr int kStridedStages = 3;

// Krylov control step of one Lanczos iteration (krylov_control.cuh).
struct ChebWork;
struct ScalarArgs {
  KState* ks;
  ChebWork* cache;    // device: the kept expansion, carried between launches
  const double* partials;
  int nparts;
  int m_max;
  int check_from;     // first Krylov dimension at which convergence is tested
  double tol;         // relative tolerance p of the step
  double breakdown;   // relative breakdown threshold for beta
};

struct TileArgs {
  int n;         // atoms = state bits
  int L;         // tile bits
  int c;         // tile bits [0, c) are amplitude bits [0, c)
  int a;         // tile bits [c, L) are amplitude bits [a, a + L - c)
  int f2;        // first amplitude bit of the top fixed range (a + L - c)
  int nF2;       // bits in the top fixed range (n - f2)
  int nG;        // lowest nG bits of the top range resolved by partner loads through L2 (<= 8)
  int kt;        // consumer-thread bits of the tile layout (<= 9)
  int split_h;   // strided pass with L - c > 8: tensor-map layout that splits the strided range
  int f1_fast;   // strided pass: segment-index bits varied fastest across tile numbers (0 = none)
  int64_t num_tiles;
  const StepParams* sp;  // device
  const double* vmat;    // device [kMaxAtoms][kMaxAtoms], FP64, by bit position
  const void* qtab;      // device [2^L] Real, first pass only
  const void* xin;
  const void* xprev;
  void* xout;
  void* out;
  const KState* ks;
  double* partials;      // [grid][3]
  int* err;              // device error word: bit 0 = a bounded wait timed out
  const void* diag;      // first pass: [num_tiles][kDiagStride] diagonal half tables (working precision)
  // Last pass of a Lanczos iteration with ctl.ks set: the CTA that finishes
  // last runs the Krylov control step with these arguments (partials are this
  // pass's), instead of a separate scalar launch.
  ScalarArgs ctl;
};

// Per-tile diagonal half tables (diag_kernels.cu). For the contiguous tile
// tau (amplitude bits >= L fixed to the bits of tau), with
//   w_q  = sum_{r >= L} V_qr tau_r - delta_q   (q < L)
//   E_hi = sum_{L <= q < r} V_qr tau_q tau_r - sum_{q >= L} delta_q tau_q,
// the row holds, computed in FP64 and rounded once to the working precision,
//   row[i]      = sum_{q < 6} w_q i_q                       (i < 64)
//   row[64 + i] = E_hi + sum_{6 <= q < L} w_q i_{q-6}      (i < 64)
// so that E(b) = row[b mod 64] + row[64 + (b mod 2^L) / 64] + Q[b mod 2^L].
constexpr int kDiagHalf = 64;
constexpr int kDiagStride = 2 * kDiagHalf;
cudaError_t launch_diag_table(const StepParams* sp, const double* vmat, int n, int L, int64_t num_tiles, void* out,
                              bool c64, cudaStream_t stream);

// Laser phase by the gauge transform U = exp(-i sum_q phi_q n_q) (phase_kernels.cu):
// a table of exp(i theta) split at bit L, theta(b) = sum_q phi_q b_q, and
// psi_b *= exp(+i theta(b)) (conj = false: U^dagger) or exp(-i theta(b)) (U).
size_t phase_table_bytes(int n, int L, bool c64);
cudaError_t launch_phase_table(const StepParams* sp, int n, int L, void* table, bool c64, cudaStream_t stream);
cudaError_t launch_phase_apply(void* psi, int n, int L, const void* table, bool conj, bool c64, int grid,
                               cudaStream_t stream);

// Tensor maps of the strided pass's two input tiles.
struct TileMaps {
  CUtensorMap x;
  CUtensorMap z;
};

enum class TileMode {
  kMatvecFirst,    // out = E x + flips(tile, G)
  kMatvecSecond,   // out += flips(tile, G)
  kLanczosSingle,  // form v_j, matvec, three-term, reductions in one pass
  kLanczosFirst,   // form v_j, diagonal + low flips - beta v_{j-1}
  kLanczosSecond,  // + high flips, reductions
};

cudaError_t launch_tile(const TileArgs& args, const TileMaps* maps, TileMode mode, bool c64, bool phi, int grid,
                        cudaStream_t stream);
// The strided pass with x alone staged in shared memory (64 KiB tiles, z
// prefetched into L2 and read/written by its owning threads): args.L must be
// kStridedTileBitsF (complex64) or kStridedTileBitsD (complex128) with every
// strided bit present (a + L - c <= n). lanczos: also reduce Re<x, z>, |z|^2,
// |x|^2 into partials (kLanczosSecond); else a plain matvec second pass.
cudaError_t launch_strided(const TileArgs& args, const TileMaps* maps, bool lanczos, bool c64, bool phi, int grid,
                           cudaStream_t stream);
// Tensor map over a state vector for the strided-pass tile geometry `g`.
bool encode_tile_map(CUtensorMap* out, const void* base, const TileArgs& g, bool c64);

// Krylov control kernels (krylov_kernels.cu).
// Bytes of the device buffer a solver keeps for the control kernel's reused
// Chebyshev expansion (zero-filled before first use).
size_t cheb_cache_bytes();
cudaError_t launch_scalar(const ScalarArgs& a, cudaStream_t stream);

struct BeginArgs {
  KState* ks;
  const double* partials;  // [nparts][n+1]: |psi|^2 then per-bit sums
  int nparts;
  int n;
  double new_tau;          // > 0: start a new time step of this length
  double* occ_out;         // nullable: [n] occupations by ATOM index
  int reset_only;          // 1: only reduce (no Krylov restart)
};
cudaError_t launch_begin(const BeginArgs& a, cudaStream_t stream);

struct CombineArgs {
  int n;
  int64_t dim;             // 2^n
  const void* const* basis;  // device array of m_max basis pointers
  const KState* ks;        // coefficients and m
  void* psi;               // output (COMBINE) or input (observe only)
  double* partials;        // [grid][n+1]
  int combine;
  int mask_bit = -1;       // observe only: >= 0 counts only amplitudes whose bit mask_bit is 1
  int* err = nullptr;      // device error word (bounded waits of the TMA combine); null: per-thread loads
};
cudaError_t launch_combine(const CombineArgs& a, bool c64, int grid, cudaStream_t stream);

// Batched evolution of many small registers (batch_kernels.cu).
constexpr int kBatchMaxAtoms = 20;
constexpr int kBatchCluster = 4;    // CTAs of a thread-block cluster sharing one large register
constexpr int kBatchCoopAtoms = 15; // registers of at least this many atoms go to a whole cluster

struct BatchItem {       // one register, device descriptor
  int32_t n;             // atoms
  int32_t steps;         // time steps
  int32_t obs_stride;    // occupation rows: t = 0, every obs_stride steps, and the end
  int32_t has_phi;
  int32_t occ_rows;      // capacity of the register's occupation rows
  int32_t pad;
  int64_t state_off;     // amplitudes into the state buffer
  int64_t param_off;     // doubles into the step parameters: per step [tau, omega[n], delta[n], phi[n]] by bit position
  int64_t vmat_off;      // doubles into the pair energies: [n][n] by bit position
  int64_t occ_off;       // doubles into the occupation rows: [rows][n] by atom index
};

struct BatchOut {        // per-register result, written once by the CTA that ran it
  int64_t iterations;
  int64_t substeps;
  double max_err;
  double norm2;
  int32_t status;        // 0, or RSV_ERR_NOT_CONVERGED
  int32_t rows;          // occupation rows written
};

struct BatchArgs {
  const BatchItem* items;
  const int* order;      // processing order (largest registers first)
  int count;
  int count_large;       // order[0 .. count_large) are solved by whole clusters
  int cluster;           // CTAs per cluster of the launch (1: no cooperative phase)
  int* next;             // work counters [large, small], 0 at launch
  void* states;
  const double* params;
  const double* vmat;
  double* occ;
  BatchOut* out;
  void* work;            // per-CTA Krylov basis + work vector, work_stride amplitudes each
  int64_t work_stride;
  int m_max;
  int max_substeps;
  int step_limit;        // > 0: stop every register after this many steps (autotuner samples)
  double tol;
  double breakdown;
};
cudaError_t launch_batch(const BatchArgs& a, bool c64, int grid, cudaStream_t stream);
// Sets the kernel's shared-memory attributes (call before launching or
// capturing); returns the resident CTAs per SM and, for cluster > 1, the
// clusters of that size that can be resident at once (0: none).
int batch_prepare(bool c64, int cluster, int* max_clusters);

// Inner products for expectation values (observable_kernels.cu): per block
// Re<x, y>, Im<x, y>, |y|^2 (FP64-class), partials[grid][3].
cudaError_t launch_dot3(const void* x, const void* y, int64_t dim, bool c64, double* partials, int grid,
                        cudaStream_t stream);

// Pulse gradient and overlap (gradient_kernels.cu).
// out_b = w(b) conj(in_b), w(b) = sum_q w_bits[q] b_q (bit order; NULL: 1).
cudaError_t launch_conj_weight(const void* in, void* out, int64_t dim, bool c64, int n, const double* w_bits,
                               int grid, cudaStream_t stream);
// acc[q][0..5] += weight * (S0_q, S1_q, D_q as re/im pairs) of (mu, nu); a
// grid of nchunks x n blocks; partials needs nchunks * n * 6 doubles.
cudaError_t launch_generator(const void* mu, const void* nu, int64_t dim, bool c64, int n, int nchunks,
                             double* partials, double weight, double* acc, cudaStream_t stream);
// Per block Re<a, b>, Im<a, b>, |a|^2, |b|^2 (FP64-class), partials[grid][4].
cudaError_t launch_overlap(const void* a, const void* b, int64_t dim, bool c64, double* partials, int grid,
                           cudaStream_t stream);

// Lindblad master equation on vec(rho) (lindblad_kernels.cu), complex128 or
// complex64 (FP32 products, FP64-class reductions).
constexpr int kLindbladMaxAtoms = 14;   // vec(rho) of 4^14 amplitudes
constexpr int kLindbladMaxKrylov = 64;  // Arnoldi basis vectors
struct LindbladParams {
  int n;
  // by bit q: <0|h_q|1> = Omega_q/2 e^{+i phi_q} (re, im), dephasing and decay rates (1/us)
  double hre[kLindbladMaxAtoms], him[kLindbladMaxAtoms];
  double gd[kLindbladMaxAtoms], gr[kLindbladMaxAtoms];
};
// y = L(x); E: [2^n] diagonal energies by bit-order index, in the working
// precision (float for c64, double for c128).
cudaError_t launch_lindblad_apply(const void* x, void* y, const void* E, const LindbladParams& p, bool c64, int grid,
                                  cudaStream_t stream);
// out[2k], out[2k+1] = Re, Im <V_k, w> for k < nvec (device array of nvec
// device pointers); partials needs nchunks * nvec * 2 doubles.
cudaError_t launch_multi_dot(const void* const* V, int nvec, const void* w, int64_t total, bool c64, int nchunks,
                             double* partials, double* out, cudaStream_t stream);
// w = (overwrite ? 0 : w) - sum_k (coef[2k] + i coef[2k+1]) V_k; *norm2_out = |w|^2
// (device); partials needs grid doubles.
cudaError_t launch_multi_axpy(const void* const* V, const double* coef, int nvec, void* w, int64_t total, bool c64,
                              bool overwrite, int grid, double* partials, double* norm2_out, cudaStream_t stream);

// Bounded-wait error path (wait_check_kernels.cu): sets *err after a wait on
// a barrier that nothing completes gives up.
cudaError_t launch_wait_check(int* err, cudaStream_t stream);

// Sampling (sample_kernels.cu): chunks of kSampleChunk amplitudes.
constexpr int64_t kSampleChunk = 256;
cudaError_t launch_block_sums(const void* psi, int64_t dim, bool c64, int64_t chunk, double* sums, cudaStream_t stream);
cudaError_t launch_sample(const void* psi, int64_t dim, bool c64, int64_t chunk, const double* chunk_cdf, int64_t nchunks,
                          double total, int64_t shots, uint64_t seed, uint64_t* out, cudaStream_t stream);

}  // namespace rsv
