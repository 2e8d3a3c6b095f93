/*
 * rsv — state-vector emulation of Rydberg atom arrays on NVIDIA B300 (sm_103a).
 *
 * C ABI of the time-evolution hot path described in arXiv 2510.09813
 * ("Efficient Emulation of Neutral Atom Quantum Hardware"), Sec. II-III:
 *
 *   H(t) = sum_i Omega_i(t)/2 (cos phi_i X_i - sin phi_i Y_i) - sum_i delta_i(t) n_i
 *          + sum_{i<j} C6 / |r_i - r_j|^6 n_i n_j                  (Eq. (3), plus a phase)
 *   psi_{k+1} = exp(-i H_k dt) psi_k                               (Eq. (6))
 *
 * with H_k taken at the midpoint of step k from pulses sampled every 1 ns
 * (Sec. III) and exp(-i H_k dt) psi_k evaluated by Lanczos (Sec. III.A).
 *
 * Conventions used by every call:
 *   - Basis order (Eq. (4), row-major N-index tensor): atom 0 is the most
 *     significant bit; amplitude index b = sum_i b_i 2^(N-1-i). Sampled
 *     bitstrings use the same packing.
 *   - Units: positions in micrometres, Omega and delta in rad/us, phi in rad,
 *     time in ns (integers) or us (doubles, named *_us), C6 in rad*um^6/us.
 *   - Precision RSV_C128: complex128 state, FP64 arithmetic. RSV_C64: complex64
 *     state and FP32 matvec; Krylov inner products/norms are accumulated to
 *     FP64-class accuracy, the tridiagonal exponential and the pair energies
 *     are FP64.
 *   - Amplitude arrays are interleaved (re, im) pairs: 16 bytes per amplitude
 *     for RSV_C128, 8 bytes for RSV_C64.
 *   - Errors: every call returns an rsv_status; nothing throws across the ABI.
 *     rsv_last_error() gives a human-readable message for the calling thread.
 *   - Streams: all device work of a context is ordered on the context's
 *     stream (given at creation, or created by the library).
 */
#ifndef RSV_H
#define RSV_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RSV_API __attribute__((visibility("default")))
#else
#define RSV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rsv_status;
#define RSV_OK 0
#define RSV_ERR_INVALID_ARG (-1)      /* bad pointer, size, shape or option */
#define RSV_ERR_OUT_OF_MEMORY (-2)    /* request exceeds the context's device arena */
#define RSV_ERR_NOT_CONVERGED (-3)    /* Krylov step needed more than max_substeps restarts */
#define RSV_ERR_TIMEOUT (-4)          /* a wait ran out (rsv_poll) */
#define RSV_ERR_CUDA (-5)             /* a CUDA runtime call failed */
#define RSV_ERR_COINCIDENT_ATOMS (-6) /* two atoms at the same position */
#define RSV_ERR_NOT_FOUND (-7)        /* unknown ticket */

#define RSV_C128 0
#define RSV_C64 1

/* rsv_config.flags */
#define RSV_FLAG_CONTROL_LAUNCH 1 /* run each Krylov control step (the reduction of alpha_j and
                                     beta_{j+1} and the convergence test of Sec. III.A.1) as a launch of
                                     its own after the iteration's last pass, instead of in the last CTA
                                     to finish that pass; same arithmetic and results, one more launch */

typedef struct rsv_ctx rsv_ctx;
typedef struct rsv_solver rsv_solver;
typedef struct rsv_result rsv_result;
typedef struct rsv_batch rsv_batch;
typedef struct rsv_server rsv_server;
typedef struct rsv_hamiltonian rsv_hamiltonian;

/* One emulation problem in the paper's terms (Sec. II.A, Sec. III). All
 * pointers are host pointers owned by the caller; the library copies what it
 * needs before the call returns. */
typedef struct {
  int32_t n_atoms;             /* 1 .. 30 (RSV_C64) / 1 .. 29 (RSV_C128), bounded by memory */
  int32_t dim;                 /* 2 or 3: coordinates per atom */
  const double* positions_um;  /* [n_atoms][dim] */
  double c6;                   /* interaction constant C of Eq. (3) */
  int32_t t_ns;                /* number of 1-ns samples = sequence duration in ns */
  int32_t omega_rows;          /* 1 (same pulse for every atom) or n_atoms */
  int32_t delta_rows;          /* 1 or n_atoms */
  int32_t phi_rows;            /* 0 (no phase), 1 or n_atoms */
  const double* omega;         /* [omega_rows][t_ns], sample n at t = n ns */
  const double* delta;         /* [delta_rows][t_ns] */
  const double* phi;           /* [phi_rows][t_ns] or NULL when phi_rows == 0 */
  const void* initial_state;   /* NULL: |0...0> (the QPU's initial state, Sec. II.B); else
                                  2^n_atoms amplitudes in the config's precision (host) */
} rsv_problem;

/* Solver options. Zero fields take the documented default. */
typedef struct {
  int32_t dt_ns;        /* step dt, an integer number of ns (Sec. III); required, >= 1 */
  int32_t precision;    /* RSV_C128 or RSV_C64 */
  double krylov_tol;    /* precision parameter p of Sec. III.A.1: a Krylov space is accepted
                           when beta_m |[exp(-i tau T_m) e_1]_{m-1}| <= p. Default 1e-12 (C128),
                           1e-7 (C64) */
  int32_t m_max;        /* Krylov dimension cap, 2 .. 64. Default 30. When reached without
                           convergence the step is split (Krylov restart on a shorter time) */
  int32_t max_substeps; /* restarts allowed per time step before RSV_ERR_NOT_CONVERGED; default 64 */
  int32_t obs_stride;   /* record <n_i> every obs_stride steps; 0 records only t = 0 and the end */
  int32_t flags;        /* 0 or RSV_FLAG_CONTROL_LAUNCH; other bits: RSV_ERR_INVALID_ARG */
} rsv_config;

typedef struct {
  int64_t steps;              /* time steps taken */
  int64_t krylov_iterations;  /* matvecs (Lanczos iterations) */
  int64_t substeps;           /* Krylov restarts beyond one per step */
  double max_error_estimate;  /* largest accepted a-posteriori Krylov error estimate */
  double seconds;             /* wall time of the solve on the host */
  int64_t kernel_launches;    /* library kernels launched so far */
  int32_t tile_passes;        /* streaming passes per matvec (1 or 2) */
  int32_t segment_bits;       /* strided pass: contiguous amplitude bits per segment (autotuned) */
  int32_t l2_partner_bits;    /* strided pass: bits whose flip partners are read through L2 */
  int32_t tile_order_bits;    /* strided pass: segment-index bits varied fastest across tiles (autotuned) */
  int32_t krylov_dim_max;     /* Krylov dimension cap in use (m_max; autotuned for batches created with m_max < 0) */
  int32_t strided_tile_bits;  /* strided pass: log2 amplitudes of its shared-memory tile (x-only tiles: 13 for
                                 complex64, 12 for complex128; tiles staging x and z: 12 / 11); 0 = one pass */
  int64_t phase_gauge_steps;  /* time steps with a laser phase run in the gauge frame: psi <- U^dagger psi,
                                 real-coefficient passes, psi <- U psi, U = exp(-i sum_i phi_i n_i) */
} rsv_stats;

/* Kernel classes of the time step, for rsv_solver_kernel_times. */
#define RSV_KERNEL_PASS_FIRST 0  /* contiguous-tile pass: diagonal + low flips (+ the whole matvec if N is small) */
#define RSV_KERNEL_PASS_SECOND 1 /* strided-tile pass: high flips + Lanczos reductions */
#define RSV_KERNEL_CONTROL 2     /* Krylov control step as a launch of its own (RSV_FLAG_CONTROL_LAUNCH;
                                    fused into the second pass otherwise) */
#define RSV_KERNEL_COMBINE 3     /* psi = |psi| sum_k u_k v_k fused with <n_i> */
#define RSV_KERNEL_SETUP 4       /* per step and restart: diagonal tables, Krylov restart (begin) */
#define RSV_KERNEL_KINDS 5

typedef struct {
  double ms[RSV_KERNEL_KINDS];        /* summed device time, CUDA events on the launch stream */
  int64_t launches[RSV_KERNEL_KINDS];
  double bytes[RSV_KERNEL_KINDS];     /* summed algorithmic HBM bytes (each operand read or written once) */
  /* The Krylov control step wherever it runs (fused into the second pass or
   * launched), timed on the device (%globaltimer, first to last instruction of
   * the step; the fused tail's arrival count is outside): all steps, and those
   * that evaluated the small exponential (convergence test, partial step). */
  double control_step_ms;
  int64_t control_steps;
  double control_check_ms;
  int64_t control_checks;
} rsv_kernel_times;

/* ---- context -------------------------------------------------------------- */

/* Creates a context on CUDA device `device`. arena_bytes > 0 caps the device
 * memory the context may hold (solvers beyond it fail with
 * RSV_ERR_OUT_OF_MEMORY); 0 means no cap. `cuda_stream` (a cudaStream_t) is the
 * stream all of the context's work is ordered on; pass cudaStreamLegacy
 * ((cudaStream_t)0x1) to share the legacy default stream with other code.
 * NULL makes the context create and own a non-blocking stream, which does NOT
 * wait for work other libraries queue on the default stream: callers that
 * hand in device buffers written elsewhere must then synchronise themselves. */
RSV_API rsv_status rsv_create(rsv_ctx** out, int32_t device, size_t arena_bytes, void* cuda_stream);
/* Destroys a context after its stream drains. Solvers and results still open
 * on it are freed first; their handles become invalid. */
RSV_API void rsv_destroy(rsv_ctx* ctx);
/* Message of the calling thread's last failed call ("" if none). Valid until
 * the thread's next rsv_* call. */
RSV_API const char* rsv_last_error(void);
/* Library version string. */
RSV_API const char* rsv_version(void);

/* Device bytes a solve of n_atoms at `precision` with Krylov cap m_max holds
 * apart from its sequence: the state, m_max basis vectors, two work vectors,
 * the per-tile diagonal rows and 2 MiB of tables and partial sums. A solver
 * adds its per-step parameters and recorded occupation rows (the admission
 * checks count those too). Sec. III.A.1 gives the same accounting for the
 * paper's complex128 emulator (16 * 2^N bytes per vector). */
RSV_API size_t rsv_footprint_bytes(int32_t n_atoms, int32_t precision, int32_t m_max);

/* ---- host-side preparation (Sec. II.A, Sec. III) ---------------------------- */

/* Pair energies V[i][j] = C6 / |r_i - r_j|^6 (i != j), V[i][i] = 0, FP64,
 * written to v_out[n_atoms * n_atoms] (atom order). RSV_ERR_COINCIDENT_ATOMS
 * if two atoms coincide. */
RSV_API rsv_status rsv_pair_energies(int32_t n_atoms, int32_t dim, const double* positions_um, double c6, double* v_out);

/* Number of time steps for a sequence of t_ns samples and step dt_ns: the
 * steps cover [0, t_ns] ns; a last step shorter than dt_ns covers the rest. */
RSV_API int32_t rsv_num_steps(int32_t t_ns, int32_t dt_ns);

/* Midpoint parameters of every step (Sec. III): for step k starting at s_k with
 * length l_k (ns), m = s_k + l_k / 2 and the value is (x[floor m] + x[ceil m]) / 2
 * (sample indices clamped to t_ns - 1). Outputs are [steps][n_atoms] (atom
 * order) plus tau_us[steps] = l_k / 1000; phi_out may be NULL. */
RSV_API rsv_status rsv_midpoint_parameters(const rsv_problem* problem, int32_t dt_ns, double* omega_out, double* delta_out,
                                   double* phi_out, double* tau_us_out);

/* ---- operator-level calls on device buffers ---------------------------------- */

/* y = H x for one constant Hamiltonian of Eq. (3): the fused structured matvec
 * (diagonal + bit-flip permutations, Sec. III.A). v_pairs is the host
 * [n_atoms][n_atoms] pair-energy matrix (atom order); omega, delta and phi
 * (phi may be NULL) are host [n_atoms] arrays. x_dev and y_dev are device
 * buffers of 2^n_atoms amplitudes in `precision`, caller-owned, 16-byte
 * aligned, not overlapping. Runs on the context stream; returns after launch. */
RSV_API rsv_status rsv_apply_hamiltonian(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const double* v_pairs,
                                 const double* omega, const double* delta, const double* phi, const void* x_dev,
                                 void* y_dev);

/* A prepared Hamiltonian (Eq. (3), same arguments as rsv_apply_hamiltonian)
 * for repeated products: the parameter tables and the per-tile diagonal rows
 * are built once on the device (context arena). */
RSV_API rsv_status rsv_hamiltonian_create(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const double* v_pairs,
                                          const double* omega, const double* delta, const double* phi,
                                          rsv_hamiltonian** out);
/* y = H x on caller-owned device buffers (2^n_atoms amplitudes, 16-byte
 * aligned, not overlapping). Only enqueues the streaming passes on the context
 * stream; nothing is allocated or synchronised. */
RSV_API rsv_status rsv_hamiltonian_apply(rsv_hamiltonian* h, const void* x_dev, void* y_dev);
/* Waits for the operator's enqueued products; RSV_ERR_TIMEOUT if a kernel's
 * bounded wait gave up. */
RSV_API rsv_status rsv_hamiltonian_sync(rsv_hamiltonian* h);
RSV_API void rsv_hamiltonian_destroy(rsv_hamiltonian* h);
/* Energy moments of a device state psi (2^n amplitudes, the operator's
 * precision, unnormalised): out[0] + i out[1] = <psi|H|psi>, out[2] =
 * <psi|H^2|psi> = |H psi|^2, accumulated to FP64-class accuracy (host array of
 * 3). Uses one vector of context-arena scratch; synchronises the context
 * stream. */
RSV_API rsv_status rsv_hamiltonian_expectation(rsv_hamiltonian* h, const void* psi_dev, double* out);

/* |psi|^2 and <n_i> = sum_b |psi_b|^2 b_i (atom order) of a device state,
 * accumulated to FP64; results copied to the host arrays (occ may be NULL).
 * Synchronises the context stream. */
RSV_API rsv_status rsv_observe(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const void* psi_dev, double* norm2_out,
                       double* occ_out);

/* Pair correlations C[i][j] = sum_b |psi_b|^2 b_i b_j (atom order; C[i][i] =
 * <n_i> unnormalised) of a device state, accumulated to FP64, written to the
 * host array out[n_atoms][n_atoms]. One observation pass per atom: the pass
 * for atom i counts only amplitudes with b_i = 1. Synchronises the context
 * stream. */
RSV_API rsv_status rsv_correlations(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const void* psi_dev, double* out);

/* `shots` basis indices drawn from |psi_b|^2 / |psi|^2 of a device state by
 * inverse CDF (FP64 running sums). Shot s uses Philox4x32-10 with counter
 * (s mod 2^32, s >> 32, 0, 0) and key (seed mod 2^32, seed >> 32):
 * u = ((x0 << 21) | (x1 >> 11)) * 2^-53, b = min{b : cdf(b) > u * cdf(D-1)}.
 * Written to the host array out[shots]. Synchronises the context stream. */
RSV_API rsv_status rsv_sample(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const void* psi_dev, int64_t shots,
                      uint64_t seed, uint64_t* out);

/* rsv_observe without a context and without allocating. The paper has no
 * counterpart: it is a service entry, not a step of the method.
 *
 * For callers that hold a device state but must not allocate: a monitor that
 * inspects a running job's state without changing its device footprint (once
 * the job's arena and a framework's caching allocator hold HBM, a new
 * allocation can fail, and it would escape the arena's admission accounting),
 * and host loops that may not block (this call only enqueues work; rsv_observe
 * allocates a context and synchronises).
 *
 * Writes out_dev[0] = |psi|^2 and out_dev[1 + i] = <n_i> = sum_b |psi_b|^2 b_i
 * (atom order), FP64, into the caller's device array of n_atoms + 1 doubles
 * (8-byte aligned). psi_dev: device state of 2^n_atoms amplitudes in
 * `precision`, 16-byte aligned, caller-owned, only read. Both must be on the
 * calling thread's current device. Work is enqueued on cuda_stream
 * (NULL = the legacy default stream) and the call returns without waiting.
 *
 * Scratch: a fixed device array inside the library, 256 KiB of partial sums
 * plus one status block (264,448 bytes), one copy per device. No scratch word
 * has to start at zero (each word read is written earlier in the same call).
 * n_atoms above 31 is rejected with RSV_ERR_INVALID_ARG and a message naming
 * the limit. The first call on each device does the set-up (looks up the
 * array's device address and the SM count, with that device current; this can
 * load the library's device code): make it before any stream capture. Calls
 * that overlap on one device (other threads or streams, before the previous
 * call's work has finished) share the array and race: order them on one
 * stream or serialise them. The looked-up address is kept for the life of the
 * process: do not use this entry on a device after cudaDeviceReset (or any
 * other re-creation of its primary context), whose array then lives at a new
 * address. psi_dev or out_dev that is not device memory of the current device
 * is rejected with RSV_ERR_INVALID_ARG (checked with
 * cudaPointerGetAttributes, which allocates nothing). */
RSV_API rsv_status rsv_observe_static(int32_t n_atoms, int32_t precision, const void* psi_dev, double* out_dev,
                                      void* cuda_stream);

/* ---- solver: a problem resident on the device --------------------------------- */

/* Prepares a problem: pair energies, per-step midpoint parameters, the Krylov
 * basis and the state (|0...0> or problem->initial_state) on the device. */
RSV_API rsv_status rsv_solver_create(rsv_ctx* ctx, const rsv_problem* problem, const rsv_config* config, rsv_solver** out);
RSV_API void rsv_solver_destroy(rsv_solver* s);
/* Advances up to n_steps time steps (stops at the end of the sequence).
 * Each step is one Lanczos evaluation of exp(-i H_k dt) psi (Eq. (6)), split
 * into Krylov restarts when m_max is reached. Records <n_i> per obs_stride.
 * Returns after the last step's work is complete on the device. */
RSV_API rsv_status rsv_solver_step(rsv_solver* s, int32_t n_steps);
/* Returns to t = 0: the state is reset to the problem's initial state, the
 * step counter and the recorded occupations to empty (row 0 is re-recorded).
 * Statistics keep accumulating. */
RSV_API rsv_status rsv_solver_rewind(rsv_solver* s);
/* Steps done so far and steps in the sequence. */
RSV_API rsv_status rsv_solver_progress(const rsv_solver* s, int32_t* done, int32_t* total);
/* Borrowed device pointer to the current state (2^n amplitudes), valid until
 * the solver is destroyed; bytes may be NULL. */
RSV_API rsv_status rsv_solver_state_device(rsv_solver* s, void** dev_ptr, size_t* bytes);
/* Copies the current state to host memory (bytes must be the state size). */
RSV_API rsv_status rsv_solver_get_state(rsv_solver* s, void* host_dst, size_t bytes);
/* Replaces the current state from host memory (does not reset the step counter). */
RSV_API rsv_status rsv_solver_set_state(rsv_solver* s, const void* host_src, size_t bytes);
/* Replaces the current state from a device buffer (copied on the context stream,
 * after work already queued there). */
RSV_API rsv_status rsv_solver_set_state_device(rsv_solver* s, const void* dev_src, size_t bytes);
/* Recorded occupations so far: rows of n_atoms doubles (row 0 = t = 0). If dst
 * is NULL only *n_rows is set; otherwise up to capacity_rows rows are copied. */
RSV_API rsv_status rsv_solver_occupations(rsv_solver* s, double* dst, int32_t capacity_rows, int32_t* n_rows);
RSV_API rsv_status rsv_solver_stats(const rsv_solver* s, rsv_stats* out);
/* Turns per-launch timing on (1) or off (0). While on, every kernel launch of
 * rsv_solver_step is bracketed by CUDA events on the context stream and its
 * duration and algorithmic bytes are accumulated by kernel class; turning it
 * on also clears the accumulators. Costs two event records per launch. */
RSV_API rsv_status rsv_solver_set_profiling(rsv_solver* s, int32_t on);
RSV_API rsv_status rsv_solver_kernel_times(const rsv_solver* s, rsv_kernel_times* out);

/* ---- whole solve ----------------------------------------------------------- */

/* Runs the whole sequence: creates a solver, steps to the end, and returns a
 * result that owns the final state and the recorded occupations. */
RSV_API rsv_status rsv_run(rsv_ctx* ctx, const rsv_problem* problem, const rsv_config* config, rsv_result** out);
/* Final state copied to host memory; bytes = 2^n * (16 or 8). */
RSV_API rsv_status rsv_result_state(const rsv_result* r, void* host_dst, size_t bytes);
/* Borrowed device pointer to the final state, valid until rsv_result_free. */
RSV_API rsv_status rsv_result_state_device(const rsv_result* r, void** dev_ptr, size_t* bytes);
/* Recorded occupations [rows][n_atoms]; dst NULL queries *n_rows. */
RSV_API rsv_status rsv_result_occupations(const rsv_result* r, double* dst, int32_t capacity_rows, int32_t* n_rows);
/* Samples of the final state (see rsv_sample). */
RSV_API rsv_status rsv_result_sample(const rsv_result* r, int64_t shots, uint64_t seed, uint64_t* out);
RSV_API rsv_status rsv_result_stats(const rsv_result* r, rsv_stats* out);
/* Served requests: seconds from submission to admission (wait) and from
 * admission to completion (service). rsv_run results: wait 0, service = the
 * solve's wall time. */
RSV_API rsv_status rsv_result_times(const rsv_result* r, double* wait_s, double* service_s);
RSV_API void rsv_result_free(rsv_result* r);

/* ---- batch: many independent registers in one persistent launch --------------- */

/* Prepares `count` independent problems (each its own register, pulses and
 * optional initial state) for batched evolution with one shared config
 * (config->m_max < 0: the Krylov depth is autotuned on a sample of the
 * registers among 12..40, see rsv_stats.krylov_dim_max). Each
 * register has at most 20 atoms. Device memory: the states, a copy of the
 * initial states, the per-step parameters, and per resident CTA a Krylov
 * workspace of (m_max + 1) * 2^(largest n_atoms) amplitudes; all from the
 * context arena (RSV_ERR_OUT_OF_MEMORY beyond its cap). The launch is captured
 * once into a CUDA graph on a stream the batch owns. */
RSV_API rsv_status rsv_batch_create(rsv_ctx* ctx, const rsv_problem* problems, int32_t count, const rsv_config* config,
                                    rsv_batch** out);
/* Resets every state to its initial state and evolves all registers over their
 * whole pulse sequences (Eq. (6) per register, Sec. III.A) in one persistent
 * kernel launch (graph replay): each CTA takes registers largest-first from a
 * device work counter and runs a register's every step, Lanczos iteration,
 * convergence test and substep on the device. Ordered after the context
 * stream's earlier work; returns when done. RSV_ERR_NOT_CONVERGED if a
 * register needed more than max_substeps substeps in a step. */
RSV_API rsv_status rsv_batch_run(rsv_batch* b);
/* Final state of register `index` (2^n amplitudes in the batch precision). */
RSV_API rsv_status rsv_batch_state(const rsv_batch* b, int32_t index, void* host_dst, size_t bytes);
/* Borrowed device pointer to that state, valid until rsv_batch_destroy. */
RSV_API rsv_status rsv_batch_state_device(const rsv_batch* b, int32_t index, void** dev_ptr, size_t* bytes);
/* Occupation rows [rows][n_atoms] of register `index`: t = 0, every obs_stride
 * steps, and the end (as rsv_solver_occupations); dst NULL queries *n_rows. */
RSV_API rsv_status rsv_batch_occupations(const rsv_batch* b, int32_t index, double* dst, int32_t capacity_rows,
                                         int32_t* n_rows);
/* Statistics of register `index`, or of the whole batch for index = -1
 * (seconds = device time of the last run, kernel_launches = runs so far,
 * tile_passes = resident CTAs of the launch). */
RSV_API rsv_status rsv_batch_stats(const rsv_batch* b, int32_t index, rsv_stats* out);
RSV_API void rsv_batch_destroy(rsv_batch* b);

/* ---- shot-to-shot noise: averages over perturbed copies of one problem --------- */

/* Evolves `shots` copies of `problem`, copy s with Omega scaled by
 * omega_scale[s], delta shifted by delta_shift[s] (rad/us) and, if
 * pos_shift_um is not NULL, atom i displaced by pos_shift_um[(s * n_atoms + i)
 * * dim + k] (um), and writes the mean of their occupation rows to occ_mean
 * [rows][n_atoms] (host; the rows of rsv_solver_occupations). Sec. III.A names
 * shot-to-shot variation of the Hamiltonian parameters as one way the emulator
 * models noise; the random draws are the caller's inputs. Copies of at most 20
 * atoms run as one batched launch (rsv_batch_*), larger ones one by one. NULL
 * occ_mean queries *n_rows. */
RSV_API rsv_status rsv_run_shots(rsv_ctx* ctx, const rsv_problem* problem, const rsv_config* config, int32_t shots,
                                 const double* omega_scale, const double* delta_shift, const double* pos_shift_um,
                                 double* occ_mean, int32_t capacity_rows, int32_t* n_rows);

/* Solves `count` problems with one config (each the evolution of Eq. (6),
 * Sec. III) and returns one result per problem in outs[count] (each freed
 * with rsv_result_free). Problems of at
 * most 20 atoms are evolved together by one batched persistent launch
 * (rsv_batch_*; their results share it, and it is freed with the last of
 * them). Larger problems run on the streaming solver one after another, with
 * m_max < 0 read as the default there. On error every result made so far is
 * freed and outs[] is NULL. Synchronises the context stream. */
RSV_API rsv_status rsv_run_batch(rsv_ctx* ctx, const rsv_problem* problems, int32_t count, const rsv_config* config,
                                 rsv_result** outs);

/* ---- fidelity and gradients ------------------------------------------------ */

/* Overlap of two device states (Sec. III results: fidelity with a target):
 * out[0] + i out[1] = <a|b> = sum_b conj(a_b) b_b, out[2] = |a|^2,
 * out[3] = |b|^2, accumulated to FP64-class accuracy (host array of 4). The
 * fidelity is (out[0]^2 + out[1]^2) / (out[2] out[3]). a_dev, b_dev: 2^n_atoms
 * amplitudes in `precision`, 16-byte aligned, caller-owned, only read.
 * Synchronises the context stream. */
RSV_API rsv_status rsv_overlap(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const void* a_dev,
                               const void* b_dev, double* out);
/* Fidelity of two device states (Sec. III results: fidelity with a target):
 * *out = |<a|b>|^2 / (|a|^2 |b|^2), from the sums of rsv_overlap (host
 * double). Arguments as for rsv_overlap; RSV_ERR_INVALID_ARG if either state
 * has zero norm. Synchronises the context stream. */
RSV_API rsv_status rsv_fidelity(rsv_ctx* ctx, int32_t n_atoms, int32_t precision, const void* a_dev,
                                const void* b_dev, double* out);

/* Value and gradient of an occupation observable at the end of the sequence,
 * <O>(T) = <psi_K| sum_i weights[i] n_i |psi_K> (psi_K unnormalised, as
 * evolved), with respect to every pulse sample (Sec. V: the emulator's
 * expectation values are differentiable with respect to the pulse tensors).
 *
 * Exact for the piecewise-constant evolution of Eq. (6) up to the Krylov
 * tolerance and a quadrature error below 1e-13 relative: adjoint method, the
 * costate and the state evolved backwards (as conjugated forward Lanczos
 * steps under the phase-negated Hamiltonian) through each step, the Duhamel
 * integral of each step by composite 8-point Gauss-Legendre.
 *
 * weights: [n_atoms] host array (atom order). panels: Gauss-Legendre panels
 * per step, 0 = automatic (ceil(W tau / 4) with W the Gershgorin bound of the
 * step's spectral width sum_{i<j} V_ij + sum |delta_i| + sum |Omega_i|), else
 * 1 .. 4096 for every step. Outputs (host, overwritten): *value_out;
 * d_omega [omega_rows][t_ns], d_delta [delta_rows][t_ns] and, when non-NULL
 * and phi_rows > 0, d_phi [phi_rows][t_ns], shaped like the problem's pulse
 * arrays (a one-row array is shared by all atoms, so its gradient sums over
 * them; samples the midpoint rule never reads get 0). *nodes_out (nullable):
 * quadrature nodes used; *stats_out (nullable): Krylov iterations and
 * launches of the forward and backward sweeps.
 *
 * Device memory from the context arena: the t_ns / dt_ns + 1 forward states
 * (checkpoints) plus three solvers' footprints (the forward solver is freed
 * before the two backward ones are made); RSV_ERR_OUT_OF_MEMORY when that
 * does not fit. config->obs_stride is ignored. Synchronises the context
 * stream. */
RSV_API rsv_status rsv_gradient(rsv_ctx* ctx, const rsv_problem* problem, const rsv_config* config,
                                const double* weights, int32_t panels, double* value_out, double* d_omega,
                                double* d_delta, double* d_phi, int64_t* nodes_out, rsv_stats* stats_out);

/* ---- diagnostics ------------------------------------------------------------ */

/* Runs the error path of the library's bounded device waits: one kernel waits
 * (with the same bounded wait the streaming passes use, limit 2 s) on a
 * barrier that nothing completes, gives up, and sets an error word. Returns
 * RSV_ERR_TIMEOUT with the message the solvers give for an aborted kernel; the
 * context stays usable. RSV_OK would mean the wait did not give up. No fault
 * or trap is raised. Synchronises the context stream (about 2 s). */
RSV_API rsv_status rsv_check_bounded_wait(rsv_ctx* ctx);

/* ---- open-system dynamics --------------------------------------------------- */

/* The Lindblad master equation (Sec. III.A: open-system dynamics),
 *     d rho/dt = -i [H(t), rho] + sum_L (L rho L^dag - {L^dag L, rho} / 2),
 * with H of Eq. (3) (and the phase) held at its midpoint value over each step
 * of config->dt_ns (Sec. III), and per atom i two channels (the paper names
 * noise channels without operators): Rydberg dephasing L = sqrt(g_dephasing[i])
 * n_i and spontaneous decay L = sqrt(g_relaxation[i]) |0><1|_i, rates in 1/us
 * (either array may be NULL = all zero).
 *
 * rho is a 2^n x 2^n matrix, row-major (basis order as for states), held on
 * the device as a vector of 4^n amplitudes in config->precision; n_atoms <= 14.
 * RSV_C128 computes in FP64; RSV_C64 keeps rho and the Krylov basis in FP32
 * with FP32 products and FP64-class inner products and norms. Each step is a
 * Krylov exponential of the Liouvillian: Arnoldi (the Liouvillian is not
 * Hermitian) with classical Gram-Schmidt twice, accepted when
 * h_{m+1,m} |[exp(tau H_m) e_1]_{m-1}| <= krylov_tol (default 1e-12 for
 * RSV_C128, 1e-7 for RSV_C64), and a step split by halving when m_max
 * (default 30, at most 64) is reached. problem->initial_state must be NULL.
 *
 * rho0: host [2^n][2^n] initial density matrix in config->precision, or NULL
 * for |0...0><0...0|. rho_out (nullable): host [2^n][2^n] in
 * config->precision, the final rho. occ_out (nullable): host [rows][n_atoms] of tr(rho n_i) at t = 0,
 * after every obs_stride-th step and at the end; at most capacity_rows rows
 * are written and *n_rows receives the count. With rho_out and occ_out both
 * NULL, only *n_rows is set. Device memory from the context arena:
 * (m_max + 2) vectors of 4^n amplitudes (16 or 8 bytes each). Synchronises the context stream. */
RSV_API rsv_status rsv_lindblad_run(rsv_ctx* ctx, const rsv_problem* problem, const rsv_config* config,
                                    const double* g_dephasing, const double* g_relaxation, const void* rho0,
                                    void* rho_out, double* occ_out, int32_t capacity_rows, int32_t* n_rows,
                                    rsv_stats* stats_out);

/* ---- serving: continuous admission of solves by device-memory footprint ------- */

typedef struct {
  int32_t slots;        /* solves in flight at once, each on its own CUDA stream; default 4 */
  int32_t batch_atoms;  /* 0: off. Else a complex64 request of at most this many atoms (<= 20) is solved
                           together with the queued complex64 requests of at most that many atoms and
                           the same config (dt, tolerances, m_max, obs_stride; any size and duration)
                           that fit, up to 64, by one batched launch (rsv_batch_*). A request with no
                           such companion in the queue, and every complex128 request, runs on the
                           streaming solver */
  size_t memory_bytes;  /* device bytes admitted solves may hold together. 0: the context arena's
                           free bytes at creation (capped context), else 90% of the device's free
                           memory */
  double max_bypass_s;  /* a queued request that does not fit may be passed by later requests that
                           do only while it has waited less than this; 0 = default 0.5 s,
                           negative = strict arrival order */
} rsv_server_config;

/* Starts a request server on a context. Worker threads take queued requests
 * in arrival order whenever the request's device footprint (state, Krylov
 * basis, work vectors, tables: the bytes its solver allocates) fits next to
 * the solves already running, so requests arriving while others run are
 * admitted as slots and memory free up, and their work overlaps on the device.
 * Each request runs the streaming solver on its own stream, or joins a
 * batched launch (config->batch_atoms). A capped context arena is
 * recommended: its allocations need no device-wide synchronisation. */
RSV_API rsv_status rsv_server_create(rsv_ctx* ctx, const rsv_server_config* config, rsv_server** out);
/* Queues one solve (the problem and config are copied; the call does not
 * wait). RSV_ERR_OUT_OF_MEMORY if its footprint exceeds the server's memory. */
RSV_API rsv_status rsv_submit(rsv_server* srv, const rsv_problem* problem, const rsv_config* config, uint64_t* ticket);
/* Waits up to timeout_ms (negative: no limit; 0: just check) for a ticket.
 * RSV_OK with *out = its result (the caller frees it; the ticket is then
 * retired), RSV_ERR_TIMEOUT if still queued or running, RSV_ERR_NOT_FOUND for
 * an unknown or retired ticket, or the solve's own error code. */
RSV_API rsv_status rsv_poll(rsv_server* srv, uint64_t ticket, int32_t timeout_ms, rsv_result** out);
/* The device footprint a server charges for one request (Sec. III.A.1 memory
 * accounting): the bytes its solver allocates (state, m_max Krylov vectors,
 * two work vectors, per-tile diagonal rows, tables, per-step parameters and
 * occupation rows), with the config's defaults applied. Host-only. */
RSV_API rsv_status rsv_request_bytes(const rsv_problem* problem, const rsv_config* config, size_t* out);
/* Current load: queued and running requests, and the device bytes charged to
 * the server's memory: the footprints of running solves plus what finished,
 * unfreed results still hold. A finished streaming solve keeps only its state
 * (2^n amplitudes; the rest goes back at once) until rsv_result_free; a
 * batched group keeps its whole footprint until its last result is freed.
 * Results held unfreed therefore delay later admissions, never overrun the
 * memory. */
RSV_API rsv_status rsv_server_load(rsv_server* srv, int32_t* queued, int32_t* running, size_t* bytes_in_use);
/* Cancels queued requests, waits for running ones, frees unclaimed results. */
RSV_API void rsv_server_destroy(rsv_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* RSV_H */
