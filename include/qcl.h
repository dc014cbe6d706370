/*
 * qcl.h -- C ABI of the GB300 engine for momentum-jump-free mixed
 * quantum-classical Liouville (QCL) dynamics.
 *
 * The engine estimates the density matrix of Eq. 1 (paper Sec. II A),
 *   d/dt rho_ab = -i w_ab rho_ab - (P/M) sum_g (d_ag rho_gb - rho_ag d_gb)
 *                 - (P/M) d rho_ab/dR - 1/2 (F_a + F_b) d rho_ab/dP ,
 * with a fixed, pre-allocated ensemble of walkers (Sec. II B: no spawning).
 * Each walker carries nuclear (R, P), an adiabatic index pair (a, b) and a
 * complex weight m exp(-i phi).  One step is: velocity Verlet on the mean force
 * -1/2 (F_a + F_b) (no momentum jump), the phase -i w_ab by the trapezoid rule,
 * and one stochastic index transition drawn from the coupling term of Eq. 1
 * with weight correction.  Outputs are ensemble averages of the diabatic and
 * adiabatic density matrices (the adiabatic excited-state population P_ad of
 * Sec. III is one of them).
 *
 * Conventions shared by every call:
 *  - Every call returns a qcl_status; QCL_OK is 0.  No C++ exception crosses
 *    the boundary.  qcl_last_error() gives a message for the calling thread.
 *  - "Device" pointers are CUDA global-memory addresses on the current device;
 *    "host" pointers are ordinary CPU memory.  The caller owns every device
 *    buffer passed in (ensemble and observation buffers); the library owns only
 *    the model's constant block (allocated by qcl_create_model).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls that take a stream only enqueue work and return; results
 *    are valid after the stream is synchronised.  Calls without a stream that
 *    return data to the host (qcl_reduce_observables, qcl_ensemble_status)
 *    synchronise the stream they are given.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed low
 *    word, seed high word), counter = (c0, traj low word, traj high word,
 *    purpose), traj = traj_id_offset + walker index.  Purpose 1 (initial
 *    sample): c0 = j gives the Box-Muller pair of mode j, c0 = N gives word 0
 *    for the index pair.  Purpose 2 (transition of step n): c0 = n >> 2, word
 *    n & 3.  A walker's stream depends only on (seed, traj, step), so results
 *    do not depend on launch shape, chunking or sharding.
 */
#ifndef QCL_H
#define QCL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t qcl_status;
#define QCL_OK 0
#define QCL_ERR_INVALID_ARG 1  /* a size, pointer or parameter is out of range */
#define QCL_ERR_UNSUPPORTED 2  /* valid but not built: n_states > 8, n_modes > 256, ... */
#define QCL_ERR_OUT_OF_MEMORY 3 /* a buffer is smaller than the size query asks for,
                                   or the server's arena is full */
#define QCL_ERR_CUDA 4         /* a CUDA runtime call failed (message has the name) */
#define QCL_ERR_TIMEOUT 5      /* a bounded wait ran out */
#define QCL_ERR_NUMERICAL 6    /* a non-finite value or a degenerate gap was seen */
#define QCL_ERR_BUSY 7         /* the server queue is full */
#define QCL_ERR_NOT_FOUND 8    /* unknown request id */

/* Working precision of an ensemble. */
#define QCL_PREC_FP64 0        /* everything in FP64: one kernel launch per step (comparator) */
#define QCL_PREC_FP32_BULK 1   /* FP32 Verlet/force/coupling, phase and weight carried as
                                  compensated FP32 pairs, FP64 ensemble reduction;
                                  persistent register-resident kernel */

#define QCL_MAX_STATES 8
#define QCL_MAX_MODES 256

/* Linear vibronic-coupling model (the spin-boson and vibronic systems of Sec.
 * II C are instances): V(R) = 1/2 sum_j M_j w_j^2 R_j^2 + W(R),
 * W(R) = E + sum_j R_j K_j; E and each K_j are real symmetric
 * n_states x n_states, row-major; K is [n_modes][n_states * n_states].  All
 * arrays are host memory, copied by qcl_create_model.  hop_scale (kappa, in
 * [2^-16, 2^16]) and p_max (in (0, 1 - 2^-16]) shape the transition
 * probabilities p_e = min(kappa |A_e|, p_max), scaled down together when their
 * sum exceeds p_max; 0 selects the defaults 1 and 0.5.  (The bounds keep a
 * step's weight factor -- 1/(1 - sum p), or |A_e|/p_e after a transition --
 * within [2^-16, 2^17] except where |A_e| itself is large; values outside them
 * are rejected with QCL_ERR_INVALID_ARG.) */
typedef struct {
  int32_t n_states;
  int32_t n_modes;
  double hbar;
  const double* mass;
  const double* omega;
  const double* E;
  const double* K;
  double hop_scale;
  double p_max;
  int32_t repr;     /* QCL_REPR_ADIABATIC (0, Eq. 1 as printed) or QCL_REPR_DIABATIC */
  int32_t reserved; /* must be 0 */
} qcl_model_desc;

/* Electronic basis of the walkers' index pairs.
 *
 * QCL_REPR_ADIABATIC: Eq. 1 (Sec. II A) as printed -- pairs of eigenstates of
 *   W(R), phase from e_a - e_b, mean Hellmann-Feynman force, transitions from
 *   the nonadiabatic coupling d_ab . P/M.
 * QCL_REPR_DIABATIC: the same equation in the R-independent basis of W, where
 *   d = 0 and the coupling is the off-diagonal potential: phase from
 *   V_aa - V_bb, mean force -1/2 (dV_aa/dR + dV_bb/dR), transitions a -> g with
 *   amplitude -i V_ga dt/hbar and b -> g with +i V_bg dt/hbar.  The imaginary
 *   unit is carried as a per-walker count of quarter turns (weight
 *   m exp(-i phi) i^q).  Any N_s and mode count in both precisions.
 *   Trajectory spawning takes either representation.  The
 *   observables keep their layout: diabatic rho_ij (the
 *   walkers' own pairs) and adiabatic rho_ab (rotated at the walker's R by its
 *   eigenvectors, each with its largest-magnitude component positive). */
#define QCL_REPR_ADIABATIC 0
#define QCL_REPR_DIABATIC 1

typedef struct qcl_model qcl_model; /* opaque */

/* Identity of an ensemble: walker count, Philox seed, global id of walker 0
 * (for sharding) and working precision.  The same descriptor must be given to
 * every call on the same ensemble buffer. */
typedef struct {
  int64_t n_traj;
  uint64_t seed;
  uint64_t traj_id_offset;
  int32_t precision;
  int32_t reserved;
} qcl_ensemble_desc;

/* Initial condition (host memory): diabatic electronic density rho_el0
 * (real symmetric [n_states * n_states], not all zero); each mode's Wigner
 * distribution of the harmonic thermal state at inverse temperature beta
 * (INFINITY = ground state), centred at (R0_j, P0_j):
 *   var R_j = hbar/(2 M_j w_j) coth(beta hbar w_j/2), var P_j = hbar M_j w_j/2 coth(...).
 * wigner = 0 starts every walker exactly at (R0, P0).  The index pair is drawn
 * from |rho_ad_ab| / sum |rho_ad| with rho_ad = U(R)^T rho_el0 U(R) at the
 * walker's own R (probabilities quantised to 2^-24), and m0 = rho_ad_ab / p_ab. */
typedef struct {
  const double* rho_el0;
  const double* R0;
  const double* P0;
  double beta;
  int32_t wigner;
  int32_t reserved;
} qcl_init_desc;

/* Status words kept in the ensemble buffer's header. */
typedef struct {
  int64_t step;          /* absolute step the ensemble has reached */
  uint32_t flags;        /* bit 0: non-finite value, bit 1: degenerate gap,
                            bit 2: step0 did not match the ensemble's step */
  uint32_t reserved;
  uint64_t n_degenerate; /* walker-steps that met a degenerate gap (coupling set to 0) */
  uint64_t n_nonfinite;  /* walkers that produced a non-finite value */
} qcl_ens_status;

#define QCL_FLAG_NONFINITE 1u
#define QCL_FLAG_DEGENERATE 2u
#define QCL_FLAG_STEP_MISMATCH 4u
#define QCL_FLAG_SPAWN_OVERFLOW 8u

/* Message for the last failing call on this thread ("" if none). */
const char* qcl_last_error(void);

/* Library version string. */
const char* qcl_version(void);

/* Validates the model (sizes, symmetry, finiteness, positive masses and
 * frequencies), derives its constants and copies them to a device block owned
 * by the returned handle (on the current device).  *out is NULL on failure. */
qcl_status qcl_create_model(const qcl_model_desc* d, qcl_model** out);

/* Frees the handle and its device block.  NULL is accepted. */
qcl_status qcl_destroy_model(qcl_model* model);

/* Bytes of device memory the ensemble buffer needs (256-byte aligned SoA:
 * header, R and P as [n_modes][n_traj], weight, phase, index pair). */
qcl_status qcl_ensemble_bytes(const qcl_model* model, const qcl_ensemble_desc* ens,
                              size_t* bytes);

/* Bytes of device memory an observation buffer for n_out output times needs
 * (FP64 rows of sums, per-tile FP64 partials, finalised means). */
qcl_status qcl_obs_bytes(const qcl_model* model, const qcl_ensemble_desc* ens, int64_t n_out,
                         size_t* bytes);

/* Initial sample (Sec. II B: walkers pre-allocated, state in contiguous
 * arrays).  Writes every walker and the header (step 0) of ens_buf. */
qcl_status qcl_sample_initial(const qcl_model* model, const qcl_ensemble_desc* ens,
                              const qcl_init_desc* init, void* ens_buf, size_t ens_bytes,
                              void* stream);

/* Advances every walker from absolute step step0 (must equal the ensemble's
 * step, else QCL_FLAG_STEP_MISMATCH is set and nothing moves) by n_steps of
 * length dt.  At each absolute step s with s % out_stride == 0 and
 * step0 < s <= step0 + n_steps (and at s = 0 when step0 == 0) it writes output
 * row k = s / out_stride (k < n_out) of obs_buf: the FP64 sums over walkers of
 * every observable contribution and of its square, added in a fixed tree
 * (32-walker groups, tiles of qcl_shard_tile_walkers walkers, tiles in index
 * order), so that results do not depend on the launch shape and two calls give
 * the same bits as one.  FP64 ensembles launch one kernel per step; FP32-bulk
 * ensembles run a persistent kernel over the tiles with state held in
 * registers (two-state models of 33..256 modes split each walker's modes over
 * 2 or 4 warps, so their tiles hold 128 or 64 walkers).  N_s-state models
 * keep R and P in registers or, with the same arithmetic and results, in the
 * ensemble buffer, read twice per step (once for the diabatic representation):
 * beyond the register limit (32 modes for N_s <= 4, 8 beyond) always, below it
 * where that form measured faster (QCL_OPT_MODES_IN_MEMORY). */
qcl_status qcl_propagate(const qcl_model* model, const qcl_ensemble_desc* ens, void* ens_buf,
                         size_t ens_bytes, int64_t step0, int64_t n_steps, double dt,
                         int32_t out_stride, void* obs_buf, size_t obs_bytes, int64_t n_out,
                         void* stream);

/* Ensemble averages (divide by n_traj) of the output rows [k0, k0 + n_rows),
 * computed on the device and copied to host_out (synchronises `stream`): the
 * diabatic and adiabatic density matrices whose averages the paper reduces
 * (Sec. II B) and plots (P_ad, Sec. III).  QCL_ERR_INVALID_ARG for a NULL
 * pointer, an invalid ensemble descriptor, rows outside [0, n_out) or host_len
 * below n_rows (2Q + 3); QCL_ERR_OUT_OF_MEMORY when obs_bytes is below
 * qcl_obs_bytes for this ensemble and n_out.
 * Per row, with NS = n_states and Q = 4 NS^2 quantities:
 *   [0, Q)      means: q = 2(i NS + j) + c, diabatic rho_ij (c = 0 real, 1 imag);
 *               q = 2 NS^2 + 2(a NS + b) + c, adiabatic rho_ab
 *   [Q, 2Q)     standard errors sqrt((S2 - S^2/N) / (N (N - 1))) of the same
 *   2Q, 2Q+1    trace of the diabatic matrix (real, imaginary)
 *   2Q + 2      walker count N
 * host_len must be at least n_rows * (2Q + 3). */
qcl_status qcl_reduce_observables(const qcl_model* model, const qcl_ensemble_desc* ens,
                                  const void* obs_buf, size_t obs_bytes, int64_t n_out,
                                  int64_t k0, int64_t n_rows, double* host_out, size_t host_len,
                                  void* stream);

/* The same rows as qcl_reduce_observables, written to device memory dev_out
 * (dev_len doubles, at least n_rows * (2Q + 3); caller-owned) by a kernel
 * enqueued on `stream`, without synchronising or copying to the host: for
 * pipelines that keep results on the device or read them later.  The same
 * argument checks and error codes as qcl_reduce_observables (dev_len in place
 * of host_len). */
qcl_status qcl_finalize_observables(const qcl_model* model, const qcl_ensemble_desc* ens,
                                    const void* obs_buf, size_t obs_bytes, int64_t n_out,
                                    int64_t k0, int64_t n_rows, double* dev_out, size_t dev_len,
                                    void* stream);

/* Copies the raw FP64 sum rows [k0, k0 + n_rows) (2Q doubles each: sums, then
 * sums of squares) to host memory (synchronises `stream`); used to combine
 * shards. */
qcl_status qcl_read_sums(const qcl_model* model, const qcl_ensemble_desc* ens,
                         const void* obs_buf, size_t obs_bytes, int64_t n_out, int64_t k0,
                         int64_t n_rows, double* host_out, size_t host_len, void* stream);

/* Byte offsets of the ensemble buffer's arrays: [0] R, [1] P, [2] weight
 * (FP64 value, or FP32 high part), [3] FP32 weight low part, [4] phase (FP64, or
 * FP32 high part), [5] FP32 phase low part, [6] index pair (uint16: a | b << 8),
 * [7] total bytes, [8] FP32 weight exponent (int32: weight = (hi + lo) 2^e),
 * [9] eigenvectors U [n_states^2][n_traj] (U[i][a] at row i*NS + a; models with
 * more than two states), [10] FP32 eigenvalues [n_states][n_traj] (FP32-bulk
 * models with more than two states).  R and P are [n_modes][n_traj]; element
 * size 8 (FP64) or 4 (FP32 bulk). */
qcl_status qcl_ensemble_layout(const qcl_model* model, const qcl_ensemble_desc* ens,
                               size_t offsets[11]);

/* Checkpoint restore (no counterpart in the paper): makes ens_buf an
 * ensemble at absolute step `step` from walker arrays the caller has written
 * into it at the offsets of qcl_ensemble_layout -- the arrays of a saved
 * ensemble of the same model, walker count and precision, or another
 * precision's state converted by the caller (FP32 bulk: R, P rounded to FP32,
 * weight as (hi + lo) 2^e, phase as hi + lo).  Writes the header (identity and
 * step; status flags and counters cleared) by a kernel enqueued on `stream`;
 * the walker arrays are not read or changed.  The next qcl_propagate passes
 * step0 = step and continues each walker's random stream at that step, so a
 * restored ensemble advances exactly as the saved one would have.
 * QCL_ERR_INVALID_ARG for a NULL or unaligned buffer, an invalid descriptor or
 * step < 0; QCL_ERR_OUT_OF_MEMORY when ens_bytes is below
 * qcl_ensemble_bytes. */
qcl_status qcl_ensemble_restore(const qcl_model* model, const qcl_ensemble_desc* ens,
                                void* ens_buf, size_t ens_bytes, int64_t step, void* stream);

/* Reads the ensemble header's status words (synchronises `stream`). */
qcl_status qcl_ensemble_status(const qcl_model* model, const qcl_ensemble_desc* ens,
                               const void* ens_buf, size_t ens_bytes, qcl_ens_status* out,
                               void* stream);

/* ------------------------------------------- propagation without allocation
 * The paper has no counterpart to this entry point.  It is qcl_propagate for
 * FP32-bulk ensembles, for callers that cannot allocate device memory when
 * they propagate: for example a service that reserved all of its device memory
 * at start-up and may not call cudaMalloc or cudaFree afterwards (those calls
 * can wait on the whole device), or a plug-in that is only handed buffers by
 * its host application.  The caller still passes the ensemble (input and
 * output) and `rows`, a device array of n_out x 8 NS^2 doubles that receives
 * the same FP64 output rows as qcl_propagate writes into its observation
 * buffer (sums, then sums of squares; the same bits).  The per-tile partial
 * sums that qcl_propagate keeps in the observation buffer live instead in one
 * static device array of QCL_NOALLOC_SCRATCH_BYTES inside the library: every
 * GPU that loads the library holds it until the process exits.
 *  - The call allocates nothing (no cudaMalloc, no cudaFree, no host heap).
 *  - The first call on each device looks up the array's device address with
 *    that device current (cudaGetSymbolAddress); make that first call before
 *    any stream capture on the device.  The address is kept for the device's
 *    primary context (the one the CUDA runtime uses): calls under another
 *    context, or after cudaDeviceReset, are not supported.
 *  - All calls share the one array and it keeps the last call's contents; no
 *    part of it needs to start at zero (every value a call reads, the same
 *    call wrote first).  Calls that overlap on the GPU (other streams or other
 *    host threads) race on the array: serialise them.
 *  - One output time needs ceil(n_traj / tile) x 256 bytes of the array, with
 *    tile = qcl_shard_tile_walkers (256 walkers for models of at most 32
 *    modes, 128 for 33-64 modes, 64 for 65-256 modes); a walker count that
 *    does not fit even one output time -- about 33 million walkers up to 32
 *    modes, 16.7 million for 33-64 modes, 8.3 million beyond -- is rejected
 *    with QCL_ERR_UNSUPPORTED and a message giving the limit.  Smaller counts
 *    fit more output times per launch (at most 32).
 *  - The argument checks and their error codes are those of qcl_propagate
 *    (in the same order); after them, ensembles that are not FP32 bulk, models
 *    of more than two states and walker counts beyond the array are rejected
 *    with QCL_ERR_UNSUPPORTED.  The QCL_OPT_GRID_CAP option and the model's
 *    launch shape apply as for qcl_propagate. */
#define QCL_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
qcl_status qcl_propagate_noalloc(const qcl_model* model, const qcl_ensemble_desc* ens,
                                 void* ens_buf, size_t ens_bytes, int64_t step0, int64_t n_steps,
                                 double dt, int32_t out_stride, double* rows, size_t rows_bytes,
                                 int64_t n_out, void* stream);

/* ------------------------------------------------------------------ shards
 * Walkers are independent and each draws its random numbers from its global id,
 * so an ensemble can be split into shards of contiguous walkers (one per GPU),
 * each propagated with traj_id_offset = its first walker.  The output sums of a
 * shard of 2^k tiles (tiles of qcl_shard_tile_walkers walkers) aligned to a
 * multiple of 2^k tiles are a subtree of the single-ensemble reduction tree;
 * combining the shards' sums by the same zero-padded binary tree gives the same
 * bits as one unsharded run (no counterpart in the paper, which uses one GPU). */

/* Walkers per reduction tile of an FP32-bulk (or FP64) ensemble of this model. */
qcl_status qcl_shard_tile_walkers(const qcl_model* model, int32_t precision, int64_t* walkers);

/* Host-side combine: out[i] = binary tree over s (zero-padded to a power of
 * two) of shard_sums[s * n_elems + i], shards in walker order.  Applied to
 * the chunk sums of all shards (qcl_read_chunk_sums, chunks in walker order)
 * it gives the unsharded rows bit for bit. */
qcl_status qcl_combine_shards(const double* shard_sums, int32_t n_shards, int64_t n_elems,
                              double* out);

/* Balanced shards.  Walkers per chunk: 1024 reduction tiles (the first level
 * of the tile fold, an aligned subtree of the reduction tree).  A shard that
 * starts at a multiple of this count (its traj_id_offset) and ends there or at
 * the ensemble's end computes its chunks' sums exactly as the unsharded run
 * does, so ranks can take contiguous runs of floor(C / world) or
 * ceil(C / world) of the C chunks, within one chunk of each other. */
qcl_status qcl_shard_chunk_walkers(const qcl_model* model, int32_t precision, int64_t* walkers);

/* The per-chunk FP64 sums of output rows [k0, k0 + n_rows) of an ensemble
 * propagated by qcl_propagate: host_out[(k - k0) C q2 + c q2 + i] for chunk c
 * (of *n_chunks = C, in walker order) and entry i of the row's 2Q sums (sums,
 * then sums of squares; q2 = 8 NS^2).  With one chunk these are the rows
 * themselves.  host_out = NULL only sets *n_chunks.  Synchronises `stream`.
 * Not kept by qcl_propagate_noalloc or for spawning ensembles. */
qcl_status qcl_read_chunk_sums(const qcl_model* model, const qcl_ensemble_desc* ens,
                               const void* obs_buf, size_t obs_bytes, int64_t n_out, int64_t k0,
                               int64_t n_rows, double* host_out, size_t host_len,
                               int64_t* n_chunks, void* stream);

/* Measured multiply-add throughput of the current device (no counterpart in
 * the paper; the roofline denominators): which = 0 FP32 FFMA, 1 FP64 DFMA.
 * Runs a fixed microbenchmark (independent FMA chains on every SM, timed with
 * CUDA events on `stream`, about 10-100 ms) and returns flops per second
 * (2 per FMA).  Synchronises the stream. */
qcl_status qcl_measure_peak(int32_t which, double* flops_per_s, void* stream);

/* ---------------------------------------------------------------------------
 * Launch shape and autotuning of the FP32-bulk persistent kernels (no
 * counterpart in the paper).  Three knobs, none of which changes a bit of any
 * result (each walker's arithmetic and each reduction tile are the same
 * whatever the shape):
 *   walkers_per_thread  1 or 2 (0 = default: 2 for two-state models of at most
 *                       4 modes or of 65..100 modes, else 1).  With 2 a thread
 *                       advances one walker of each of two consecutive tiles
 *                       as the two lanes of packed FP32x2 instructions; 2 is
 *                       available for two-state models of at most 8 modes or
 *                       of 65..100 modes (a walker's modes over four warps),
 *                       otherwise 1 is used.  A launch whose tiles do not
 *                       outnumber the resident block slots also runs 1, so
 *                       that every slot gets a tile.
 *   blocks_per_sm       resident blocks per SM of the persistent grid (0 = the
 *                       kernel's occupancy limit; larger values are clamped).
 *   outputs_per_launch  output times per persistent launch, 1..32 (0 = 32): a
 *                       propagate call is cut into launches at output steps.
 * Threads per block are fixed at 256: a block's threads hold one reduction
 * tile (or two, with two walkers per thread), whose size defines the
 * summation tree of every observable.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t walkers_per_thread;
  int32_t blocks_per_sm;
  double walker_steps_per_s; /* rate measured by qcl_autotune for this shape (0 if set by hand) */
  int32_t outputs_per_launch;
  int32_t reserved;          /* must be 0 */
} qcl_launch_shape;

/* Sets the shape every later FP32-bulk launch for this model uses.
 * QCL_ERR_INVALID_ARG for walkers_per_thread outside {0, 1, 2}, negative
 * blocks_per_sm or outputs_per_launch outside [0, 32]. */
qcl_status qcl_set_launch_shape(qcl_model* model, const qcl_launch_shape* shape);
qcl_status qcl_get_launch_shape(const qcl_model* model, qcl_launch_shape* shape);

/* Scratch bytes qcl_autotune needs for a probe ensemble of probe_walkers
 * walkers advanced n_steps steps with the given output stride. */
qcl_status qcl_autotune_bytes(const qcl_model* model, int64_t probe_walkers, int64_t n_steps,
                              int32_t out_stride, size_t* bytes);

/* Times every candidate shape (walkers per thread 1 and, where available, 2;
 * blocks per SM from 1 to the occupancy limit) on a probe ensemble sampled in
 * `scratch` (ground-state Wigner walkers at R = 0 in state 0, FP32 bulk),
 * each over n_steps steps of dt with outputs every out_stride steps after one
 * warm-up run; then, with the fastest of those, 8, 16 and 32 output times per
 * launch over max(n_steps, 64 out_stride) steps.  Stores the fastest shape in
 * the model (as qcl_set_launch_shape); *best receives it with its measured
 * rate.  qcl_autotune_bytes sizes the scratch for the longer probe.
 * Synchronises the stream. */
qcl_status qcl_autotune(qcl_model* model, int64_t probe_walkers, int64_t n_steps, double dt,
                        int32_t out_stride, void* scratch, size_t scratch_bytes,
                        qcl_launch_shape* best, void* stream);

/* ---------------------------------------------------------------------------
 * Trajectory spawning (either representation, any N_s and mode count, FP64 or
 * FP32 bulk).
 *
 * The scheme of the CPU code that the paper's GPU version replaces (Sec. II B:
 * there a new trajectory was started each time a transition test fired, so
 * the walker count was not fixed).  Each step a walker runs the same
 * deterministic step and
 * transition test as in qcl_propagate, but a fired test does not move it: it
 * keeps its pair and weight and spawns a child at the event's target pair
 * with weight m A_e / p_hat_e (diabatic: with the event's quarter turns) and
 * the parent's (R, P, phi); no 1/(1 - sum p_hat) factor is applied.  Children
 * are inserted right after their parents (deterministic count / scan /
 * scatter), so results are reproducible bit for bit and the walkers descending
 * from one initial walker (its family) stay contiguous.  A child's random
 * stream is keyed by words 0-1 of Philox block (c0 = step, parent id, purpose
 * 3) with bit 63 set.
 *
 * ens->n_traj is the number n0 of initial walkers (families) and
 * ens->precision the arithmetic (QCL_PREC_FP64, or QCL_PREC_FP32_BULK: the
 * FP32-bulk walker arithmetic -- compensated phase and weight pairs with a
 * carried exponent -- one step per launch with the state in HBM); capacity is
 * the walker slots the buffer holds (n0 <= capacity <= 2^36).  The observation
 * buffer is sized by qcl_obs_bytes(model, ens, n_out) as for any FP64
 * ensemble; its rows hold, per output, the sums over families of the family
 * sums X_k of the walker contributions and of X_k^2, so qcl_reduce_observables
 * gives means over n0 and standard errors over independent families.  When a
 * step's children would exceed capacity they are dropped and
 * QCL_FLAG_SPAWN_OVERFLOW is set in the status: every later result of that
 * ensemble is invalid.  Buffers are caller-owned and 256-byte aligned.
 * ------------------------------------------------------------------------ */

/* Bytes of a spawning ensemble buffer (header, two walker sets of capacity
 * slots, per-parent staging, scan scratch, family starts). */
qcl_status qcl_spawn_bytes(const qcl_model* model, const qcl_ensemble_desc* ens, int64_t capacity,
                           size_t* bytes);

/* Byte offsets within the buffer of walker set `set` (0 or 1; the current set
 * is the ensemble's step & 1): offsets[0..6] = R [n_modes][capacity], P (same),
 * m, phi (double in FP64, float in FP32), index pair (uint16: a | q << 4 |
 * b << 8), random-stream id (uint64), family (uint32); offsets[7] = total
 * bytes; FP32 only (0 in FP64): offsets[8] = m_lo (float), [9] = m_exp
 * (int32; the weight is (m + m_lo) 2^m_exp), [10] = phi_lo (float); N_s > 2
 * only (else 0): offsets[11] = the carried eigenvectors U [N_s * N_s][capacity]
 * (double; element (i, a) at row i * N_s + a). */
qcl_status qcl_spawn_layout(const qcl_model* model, const qcl_ensemble_desc* ens, int64_t capacity,
                            int32_t set, size_t offsets[12]);

/* Samples the n0 initial walkers into set 0 (as qcl_sample_initial; ids
 * traj_id_offset + i, family i). */
qcl_status qcl_spawn_sample(const qcl_model* model, const qcl_ensemble_desc* ens,
                            const qcl_init_desc* init, int64_t capacity, void* buf, size_t bytes,
                            void* stream);

/* Advances the spawning ensemble by n_steps from absolute step step0 (< 2^32
 * in total), observing at every absolute step that is a multiple of
 * out_stride (and at step 0 when step0 == 0).  Arguments as qcl_propagate. */
qcl_status qcl_spawn_propagate(const qcl_model* model, const qcl_ensemble_desc* ens,
                               int64_t capacity, void* buf, size_t bytes, int64_t step0,
                               int64_t n_steps, double dt, int32_t out_stride, void* obs_buf,
                               size_t obs_bytes, int64_t n_out, void* stream);

/* Live walkers of the current set (synchronises the stream). */
qcl_status qcl_spawn_live(const qcl_model* model, const qcl_ensemble_desc* ens, int64_t capacity,
                          const void* buf, int64_t* n_live, void* stream);

/* ---------------------------------------------------------------- serving
 * A request loop for many solves of different models, walker counts and step
 * counts arriving over time (continuous batching; no counterpart in the paper,
 * which runs one solve at a time).  The server admits queued requests in
 * arrival order while the caller's device arena has room for their ensemble
 * and observation buffers and fewer than max_active are running; it advances
 * all admitted requests together in rounds of at most quantum_steps steps
 * each (a packed request also at most 32 output times), packing adiabatic
 * two-state requests of up to 8
 * modes into shared persistent launches (a CUDA graph replayed every round
 * when use_graphs is set) unless their walkers fill the GPU by themselves
 * (at least 6 x SMs tiles of 256 walkers), which, like the other requests,
 * get persistent launches of their own; requests arriving meanwhile join at
 * the next round.  A
 * request's results do not depend on what it is batched with.  Requests run
 * in FP32-bulk precision.  The server owns one CUDA stream (plus eight side
 * streams on which requests with launches of their own run side by side) and
 * a worker thread; the caller owns the arena (device memory, 256-byte aligned), which
 * must stay valid until qcl_server_destroy returns. */
typedef struct qcl_server qcl_server; /* opaque */

typedef struct {
  void* arena;            /* device memory the server sub-allocates */
  size_t arena_bytes;
  int32_t max_active;     /* requests propagating at the same time (>= 1) */
  int32_t quantum_steps;  /* steps a request advances per round (>= 1) */
  int32_t use_graphs;     /* 1: replay the packed launches as a CUDA graph */
  int32_t max_queue;      /* queued requests beyond which submit returns BUSY (0: no limit) */
  double round_timeout_s; /* a round not finished after this long fails its requests (0: 600 s) */
  double round_flops;     /* work budget per round in algorithmic flops (walkers x steps x
                             flops per walker-step: 10 per mode + 26 for two-state models, 12
                             per mode + 26 in their general form, 25 N_s^2 with more states).
                             0: every active request advances quantum_steps each round.  > 0:
                             requests advance in ascending order of remaining work (shortest
                             first; one skipped 16 rounds in a row goes first) until the budget
                             is spent, the last one by part of its quantum (at least one step),
                             the others wait for a later round.  Results do not depend on it. */
} qcl_server_desc;

typedef struct {
  const qcl_model_desc* model; /* copied at submit */
  const qcl_init_desc* init;   /* copied at submit */
  int64_t n_traj;
  uint64_t seed;
  uint64_t traj_id_offset;
  int64_t n_steps;
  double dt;
  int32_t out_stride;
  int32_t reserved;
} qcl_request_desc;

#define QCL_REQ_QUEUED 0
#define QCL_REQ_RUNNING 1
#define QCL_REQ_DONE 2
#define QCL_REQ_ERROR 3

typedef struct {
  int64_t n_submitted, n_done, n_error, n_active, n_queued;
  int64_t rounds, graph_replays;
  size_t arena_used;
  double traj_steps_done;   /* sum over finished requests of n_traj x n_steps */
  double latency_p50_s;     /* finish - submit, over finished requests */
  double latency_p99_s;
  double latency_mean_s;
  double span_s;            /* first submit to last finish */
  double throughput;        /* traj_steps_done / span_s */
  double device_busy_s;     /* device time of the busy periods: CUDA events on the
                               server's stream from the work of the first admission
                               after an idle spell (sampling included) to the end of
                               the work that retires the last active request */
  double device_throughput; /* traj_steps_done / device_busy_s */
} qcl_server_statistics;

qcl_status qcl_server_create(const qcl_server_desc* d, qcl_server** out);

/* Copies the request and queues it; *id identifies it.  QCL_ERR_OUT_OF_MEMORY
 * if it could never fit the arena, QCL_ERR_BUSY if the queue is full. */
qcl_status qcl_server_submit(qcl_server* s, const qcl_request_desc* r, int64_t* id);

/* State of a request (QCL_REQ_*) and, once done, its observables: n_rows rows
 * laid out as qcl_reduce_observables writes them, copied to host_out when it is
 * not NULL (host_len doubles at least).  A failed request returns
 * QCL_ERR_NUMERICAL with its message. */
qcl_status qcl_server_poll(qcl_server* s, int64_t id, int32_t* state, double* host_out,
                           size_t host_len, int64_t* n_rows);

/* Blocks until the request is done or failed, or timeout_s passes
 * (QCL_ERR_TIMEOUT). */
qcl_status qcl_server_wait(qcl_server* s, int64_t id, double timeout_s, int32_t* state);

qcl_status qcl_server_stats(qcl_server* s, qcl_server_statistics* out);

/* Stops the worker after its current round and releases the server's
 * resources (not the arena).  NULL is accepted. */
qcl_status qcl_server_destroy(qcl_server* s);

/* ----------------------------------------------------------- instrumentation
 * Process-wide options:
 *   QCL_OPT_GRID_CAP  cap on the persistent grid (0: SMs x resident blocks);
 *                     results do not depend on it (fixed reduction tree)
 *   QCL_OPT_TIMING    1: record a CUDA event pair on the launching stream around
 *                     every persistent-kernel and FP64 step-kernel launch
 *   QCL_OPT_MODES_IN_MEMORY  where the FP32-bulk N_s-state kernels (N_s > 2)
 *                     and the FP32 spawning steps keep R and P: 0 (default)
 *                     the faster form as measured for the model's N_s, mode
 *                     count and representation; 1 in the ensemble buffer for
 *                     every mode count; 2 in registers wherever a register
 *                     form exists (N_s-state: up to 32 modes for N_s <= 4, 8
 *                     beyond; two-state spawning: up to 32).  Every choice
 *                     gives the same bits. */
#define QCL_OPT_GRID_CAP 1
#define QCL_OPT_TIMING 2
#define QCL_OPT_MODES_IN_MEMORY 3
qcl_status qcl_set_option(int32_t key, int64_t value);

/* Kernel launches made by the library since the last reset; resets the counter
 * when reset != 0. */
qcl_status qcl_launch_count(int64_t* count, int32_t reset);

/* Device time recorded under QCL_OPT_TIMING for kernel class `which`
 * (0: FP32-bulk persistent kernel, 1: FP64 step kernel): total milliseconds and
 * launch count.  Synchronises the recorded events, then clears them. */
qcl_status qcl_kernel_time(int32_t which, double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* QCL_H */
