/*
 * libdcs -- dynamic-circuit MPS simulation on one B300 (sm_103a): C ABI.
 *
 * The operations follow the paper "Tensor Network Simulation of Dynamic Circuits":
 *   - branch state {(p_gamma, c_gamma, psi_gamma)}     (Def. "State of a dynamic circuit")
 *   - InitializeState |0...0>, c = 0, p = 1, F = 1      (Alg. 1 / Alg. 2, initialisation)
 *   - CompressionStep of one unitary chunk, F *= f      (Sec. "Simulating unitary quantum
 *                                                        circuits with DMRG", Defs. "Unitary
 *                                                        chunk", "Compression step")
 *   - MeasureProb / Measure / Collapse                  (Sec. "Mid-circuit measurements")
 *   - classically controlled operations                 (Sec. "Classically controlled
 *                                                        operations")
 *   - reset = measure + conditional X                   (Sec. "Reset operations")
 *   - chunk construction                                (Sec. "Handling unitary chunks in
 *                                                        dynamic circuits")
 *   - single-path and multi-path strategies, TopK       (Alg. 1, Alg. 2)
 *
 * Conventions
 *   - Every call returns dcs_status_t; dcs_last_error(ctx) describes the last failure.
 *   - Device work is enqueued on the stream given to dcs_create and is asynchronous unless
 *     a call says it synchronises (the ones that fill host buffers).
 *   - The caller owns the device arena (at least dcs_arena_bytes() bytes, 256-byte aligned)
 *     and all host buffers.  The library allocates no device memory; it keeps host
 *     metadata and a pinned host staging buffer per context.
 *   - Qubit q is MPS site q; two-qubit gates act on neighbouring qubits.
 *   - Slots: in single-path mode a slot is one shot (independent run of Alg. 1); in
 *     multi-path mode slots hold the branches of the list L of Alg. 2.
 *   - Complex numbers are stored as (re, im) pairs; tensors on the device are complex64,
 *     probabilities and fidelities float64.
 */
#ifndef DCS_H
#define DCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* dcs_stream_t; /* a cudaStream_t */

typedef enum {
  DCS_OK = 0,
  DCS_ERR_INVALID = 1,     /* bad argument or configuration */
  DCS_ERR_OOM = 2,         /* arena or slot pool too small */
  DCS_ERR_ZERO_PROB = 3,   /* collapse onto an outcome with p_m <= 1e-12 (per-slot flag) */
  DCS_ERR_NUMERICAL = 4,   /* NaN/Inf in a norm, probability or fidelity (per-slot flag) */
  DCS_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  DCS_ERR_CUDA = 6,        /* a CUDA runtime call failed */
  DCS_ERR_UNSUPPORTED = 7  /* valid request outside what this build implements */
} dcs_status_t;

/* classical register: up to 64 * DCS_CWORDS bits per slot */
#define DCS_CWORDS 8
/* largest number of qubits (MPS sites) */
#define DCS_MAX_QUBITS 128
/* largest bond dimension held in shared memory; above it the tiles live in a per-slot
 * global work area */
#define DCS_MAX_CHI_FUSED 32
/* largest bond dimension */
#define DCS_MAX_CHI 1024
#define DCS_MAX_CHUNK_LAYERS 4 /* gate layers one chunk may hold (chunk_layers) */

typedef enum {
  DCS_COND_NONE = 0,
  DCS_COND_XOR = 1,
  DCS_COND_AND = 2,
  DCS_COND_OR = 3,
  DCS_COND_TABLE = 4
} dcs_cond_op;

/* phi(c) of a classically controlled operation (Sec. "Classically controlled operations":
 * a Boolean function of the classical register).  XOR (parity), AND or OR of the bits set in
 * mask, compared with value (0 or 1); DCS_COND_TABLE: any Boolean function of at most 5
 * bits, given by its truth table -- the bits set in mask, in ascending bit order, form the
 * index i (the smallest bit is bit 0 of i) and phi = bit i of (uint32_t)value.
 * op == DCS_COND_NONE: always true.  A TABLE condition with more than 5 bits in mask is
 * refused with DCS_ERR_INVALID. */
typedef struct {
  uint64_t mask[DCS_CWORDS];
  int32_t op;
  int32_t value;
} dcs_cond;

typedef enum {
  DCS_OP_GATE1 = 1,   /* 2x2 unitary on q0 */
  DCS_OP_GATE2 = 2,   /* 4x4 unitary on (q0, q1), |q0 - q1| = 1, basis |s_q0 s_q1> */
  DCS_OP_MEASURE = 3, /* measure q0 into cbit */
  DCS_OP_RESET = 4    /* reset q0 through cbit (measure into cbit, X if cbit == 1) */
} dcs_op_kind;

/* One circuit operation.  m holds the gate matrix row-major as (re, im) pairs:
 * m[2*(r*d + c)] = Re U[r][c], m[2*(r*d + c) + 1] = Im U[r][c], d = 2 or 4. */
typedef struct {
  int32_t kind;
  int32_t q0;
  int32_t q1;
  int32_t cbit;
  double m[32];
  dcs_cond cond;
} dcs_op;

/* Arithmetic of the large-bond contractions (chi_max > 32 or DCS_PATH_GLOBAL):
 * DCS_PREC_FP32: FP32 CUDA-core GEMMs; DCS_PREC_TF32X3: tcgen05 tensor-core GEMMs with TF32
 * inputs split in three products (x = hi + lo) and FP32 accumulation for the initial guess,
 * the environment cache and every sweep but the last, which runs in FP32 as refinement (its
 * f is the reported partial fidelity); DCS_PREC_BF16X3: the same with BF16 hi / lo parts
 * (kind::f16 MMAs, about 2^-16 relative per product instead of 2^-22, half the tensor-pipe
 * time), the last sweep again FP32.  The shared-memory kernels (chi_max <= 32) always use
 * FP32 CUDA cores. */
typedef enum { DCS_PREC_FP32 = 0, DCS_PREC_TF32X3 = 1, DCS_PREC_BF16X3 = 2 } dcs_precision;

typedef enum {
  DCS_PATH_AUTO = 0,    /* shared-memory tiles up to chi_max = 32, global tiles above */
  DCS_PATH_SHARED = 1,  /* shared-memory tiles (chi_max <= 32) */
  DCS_PATH_GLOBAL = 2   /* per-slot global work area, tiled GEMM contractions */
} dcs_kernel_path;

typedef struct {
  int32_t n_qubits;     /* 1 .. DCS_MAX_QUBITS */
  int32_t chi_max;      /* bond-dimension cap (the paper's chi) */
  double tol;           /* relative discarded weight allowed per truncation */
  int32_t sweeps;       /* one-site sweeps per compression step (the paper's s), >= 1 */
  int32_t chunk_k;      /* maximum operations per chunk (the paper's k); 0 = no limit */
  int32_t chunk_layers; /* maximum gate layers per chunk, 0 .. DCS_MAX_CHUNK_LAYERS (0 and 1:
                           one layer, MPO bond <= 4); a chunk of L layers is compressed in one
                           step against their composed MPO (bond <= 4^L), its guess taken
                           layer by layer; L > 1 runs on the global work area only */
  int32_t precision;    /* dcs_precision */
  int32_t kernel_path;  /* dcs_kernel_path */
  int32_t n_cbits;      /* classical register size m, <= 64 * DCS_CWORDS */
  int32_t n_slots;      /* shots (single-path) or branch-pool capacity (multi-path) */
  uint64_t seed;        /* key of the counter-based outcome sampler */
} dcs_config;

/* Per-slot result flags (dcs_get_results). */
#define DCS_FLAG_DRAW_NEAR_THRESHOLD 1u /* some draw had |u - p_0| < 1e-6 */
#define DCS_FLAG_ZERO_PROB 2u           /* a collapse was refused (p_m <= 1e-12) */
#define DCS_FLAG_NUMERICAL 4u           /* NaN/Inf met in a norm or probability */
#define DCS_FLAG_TOPK_NEAR_TIE 8u       /* TopK cut through keys within one bucket */

typedef struct dcs_ctx_s* dcs_ctx_t;

/* Bytes of device arena dcs_create needs for cfg (all slots, MPS pair, environment
 * caches, per-slot state, circuit program).  0 if cfg is invalid. */
size_t dcs_arena_bytes(const dcs_config* cfg);

/* InitializeTN: bind a context to the caller's device arena and stream.  Carves the arena;
 * does not touch device memory.  cfg is copied.  Fails with DCS_ERR_OOM if arena_bytes <
 * dcs_arena_bytes(cfg), DCS_ERR_UNSUPPORTED if chi_max > DCS_MAX_CHI (or chi_max >
 * DCS_MAX_CHI_FUSED with DCS_PATH_SHARED).
 * Arena layout: per slot two MPS buffers and one environment cache, sized by the bond
 * capacities cap_b = min(C, 2^min(b, n-b)) (C >= chi_max the bond cap of the kernel path):
 * site j holds cap_j x 2 x cap_{j+1} complex64, bond b's environment cap_b x D x cap_b with
 * D = 4^max(1, chunk_layers) the MPO bond cap. */
dcs_status_t dcs_create(dcs_ctx_t* ctx, const dcs_config* cfg, void* dev_arena,
                        size_t arena_bytes, dcs_stream_t stream);

/* Releases host resources of ctx; the arena stays the caller's. */
dcs_status_t dcs_destroy(dcs_ctx_t ctx);

/* Message of the last failing call on ctx (never NULL). */
const char* dcs_last_error(dcs_ctx_t ctx);

/* InitializeState (Alg. 1 / Alg. 2 first line): every slot of the first n_active gets
 * |0...0>, c = 0, p = 1, F = 1, centre 0.  multipath = 0: n_active shots, shot id of slot
 * i = shot0 + i (the sampler's counter); multipath = 1: one branch (n_active must be 1),
 * the rest of the pool free. */
dcs_status_t dcs_init_state(dcs_ctx_t ctx, int n_active, int multipath, uint64_t shot0);

/* Hybrid single-path start (Sec. "Dynamic procedure for GHZ state preparation": multi-path
 * evaluates the part of the circuit before the first measurement once, while independent
 * single-path runs repeat it): after dcs_init_state(ctx, 1, 0, shot0) and the
 * measurement-free prefix of the circuit run on that one shot, copies its state, register, p and F into list positions 1 .. n_active - 1, each
 * shot keeping its own sampler counter shot0 + position, so that the list holds n_active
 * shots exactly as if all of them had run the prefix.  Asynchronous.  The device checks that
 * the list held one shot; otherwise nothing changes and dcs_get_results returns
 * DCS_ERR_INVALID until the next dcs_init_state.  DCS_ERR_INVALID on the host for a
 * multi-path context or n_active outside [1, n_slots]. */
dcs_status_t dcs_fork_shots(dcs_ctx_t ctx, int n_active);

/* CompressionStep for one chunk on every active slot.  gates: n_gates GATE1/GATE2 ops that
 * form one chunk: cut into sub-layers where a two-qubit gate meets a qubit that already
 * carries one of the current sub-layer, at most max(1, chunk_layers) of them (each a layer
 * of disjoint nearest-neighbour blocks);
 * conditions are evaluated per slot on its register, and a slot on which every gate is
 * skipped is left unchanged (no compression, f = 1).  Otherwise the ket is replaced by
 * the compressed bra and F *= f.  fid_out: optional DEVICE pointer to n_slots doubles
 * receiving f per slot (1 for skipped slots).  Returns DCS_ERR_INVALID if the gates need
 * more sub-layers than that. */
dcs_status_t dcs_apply_layer(dcs_ctx_t ctx, const dcs_op* gates, int n_gates,
                             double* fid_out);

/* MeasureProb: p_0 = <psi|P_0|psi> / <psi|psi> of qubit for every active slot (moves the
 * orthogonality centre to qubit).  p0_out: DEVICE pointer to n_slots doubles (inactive
 * slots untouched). */
dcs_status_t dcs_measure_prob(dcs_ctx_t ctx, int qubit, double* p0_out);

/* Single-path Measure (Alg. 1): per shot, u = Philox4x32-10(key = seed, counter =
 * (meas_idx, 0, shot id)) as a 53-bit double, m = 0 iff u < p_0, Collapse onto m
 * (P_m / sqrt(p_m)), p *= p_m, c[cbit] = m.  Draws with |u - p_0| < 1e-6 set
 * DCS_FLAG_DRAW_NEAR_THRESHOLD; p_m <= 1e-12 sets DCS_FLAG_ZERO_PROB and leaves the slot
 * uncollapsed. */
dcs_status_t dcs_measure_sample(dcs_ctx_t ctx, int qubit, int cbit, uint64_t meas_idx);

/* Collapse onto given outcomes (tests, replay of a recorded path): outcome is a HOST
 * array of n_slots bytes (0/1).  p *= p_m, c[cbit] = m, same error flags. */
dcs_status_t dcs_collapse(dcs_ctx_t ctx, int qubit, int cbit, const uint8_t* outcome);

/* Multi-path measurement (Alg. 2): every active branch gamma spawns the children gamma m,
 * m in {0, 1} with p_m > eps, in list order (children of earlier branches first, m = 0
 * before m = 1): p_{gamma m} = p_gamma p_m, c[cbit] = m, F copied, MPS = Collapse(m).
 * Fails with DCS_ERR_OOM (state unchanged) if the children exceed the pool. */
dcs_status_t dcs_branch_split(dcs_ctx_t ctx, int qubit, int cbit, double eps);

/* Adaptive pruning of the branch ensemble (the paper's conclusion names pruning strategies
 * beyond top-M as future work).  With p_min > 0, every later branch split (dcs_branch_split,
 * and the measurements of dcs_run_circuit in multi-path mode) drops the children whose path
 * probability p_gamma p_m is below p_min, after the top-M rule; the child that comes first in
 * the key order of dcs_branch_topk always stays, so the ensemble never empties.  The dropped
 * mass is missing from the sum of p, as with top-M.  p_min = 0 (the default) turns it off;
 * p_min outside [0, 1) is refused with DCS_ERR_INVALID.  Host-only, takes effect at once. */
dcs_status_t dcs_set_pruning(dcs_ctx_t ctx, double p_min);

/* TopKByWeight (Alg. 2): if more than M branches are active keep the M with the largest
 * p_gamma, compared through the key round(p / (1e-5 * max p)); equal keys keep list order.
 * The retained branches keep their relative order; p is not renormalised. */
dcs_status_t dcs_branch_topk(dcs_ctx_t ctx, int M);

/* Branch compaction by an explicit selection: entry i of the active list (the order of
 * dcs_get_results) stays iff keep[i] != 0; the kept branches keep their relative order, the
 * dropped slots are free for the next split; p is not renormalised.  keep is a HOST array of
 * n bytes, staged through the context's pinned buffer; n must equal the active count, which
 * the device checks: a different count leaves the list unchanged, and dcs_get_results
 * returns DCS_ERR_INVALID from then until the next dcs_init_state.  This is the last step of
 * TopKByWeight (Alg. 2) when the ensemble is sharded over several contexts (one per GPU):
 * each rank gathers every rank's p, selects with dcs_topk_select_global, and keeps its own
 * slice.  DCS_ERR_INVALID for a null mask, n < 0, n > n_slots or a single-path context. */
dcs_status_t dcs_branch_keep(dcs_ctx_t ctx, const uint8_t* keep, int n);

/* Host-only, needs no context or device: TopKByWeight (Alg. 2) and adaptive pruning over
 * an ensemble spread across ranks.  p holds the n path probabilities of every rank's active
 * branches, concatenated in rank order (each rank's list in the order of dcs_get_results),
 * which is the list order of the whole ensemble.  keep (n bytes) receives 1 for the
 * retained branches: if n > M the M largest by the key round(p / (1e-5 * max p)) of
 * dcs_branch_topk, the maximum taken over all n, equal keys keeping list order; then, when
 * p_min > 0, every retained branch with p < p_min is dropped except the first of the key
 * order (the rule of dcs_set_pruning).  The result equals what one context holding the whole
 * list would keep.  DCS_ERR_INVALID for n < 0, M < 1, null pointers with n > 0, p_min outside
 * [0, 1), or a p that is negative or not finite. */
dcs_status_t dcs_topk_select_global(const double* p, int n, int M, double p_min, uint8_t* keep);

/* Synchronises and copies results to HOST buffers (each may be NULL, each sized for
 * n_slots entries): for the active slots in list order, p (n doubles), F (n doubles), the
 * register (n * DCS_CWORDS words), flags (n bytes), and the number n of active slots.  The
 * data comes down through the context's pinned host staging buffer, which grows (one
 * cudaMallocHost) the first time it is too small.  DCS_ERR_OOM if the branch pool ran out
 * during the circuit, DCS_ERR_TIMEOUT if a bounded wait of the tensor-core pipeline gave up
 * (that step's results are not to be trusted), DCS_ERR_INVALID after a dcs_branch_keep or
 * dcs_fork_shots that found a list of the wrong length, DCS_ERR_CUDA on a copy or earlier
 * asynchronous error, or when the device's active count or slot list lies outside the pool
 * (corrupted device state; nothing is written to the buffers then).  The buffers are
 * written before the device status is reported; the status stays set until the next
 * dcs_init_state. */
dcs_status_t dcs_get_results(dcs_ctx_t ctx, double* p, double* fid, uint64_t* cbits,
                             int* n_active, uint8_t* flags);

/* Synchronises and copies the bond dimensions of every active slot, in list order, to the
 * HOST buffer bonds (n_slots x (n_qubits + 1) int32, row i = slot i of the list: chi_0 ..
 * chi_n of its current MPS); *n_active receives the number of rows written.  DCS_ERR_CUDA
 * if a copy fails or the device's slot list lies outside the pool. */
dcs_status_t dcs_get_bonds(dcs_ctx_t ctx, int32_t* bonds, int* n_active);

/* Checkpoint: synchronises and writes the MPS of active slot `slot` (list position) to a
 * HOST buffer: int32 n, int32 bonds[n+1], int32 centre, then the site tensors
 * [chi_l][2][chi_r] as complex64.  *bytes is the capacity on input and the size written
 * on output; host_buf == NULL only queries the size. */
dcs_status_t dcs_export_mps(dcs_ctx_t ctx, int slot, void* host_buf, size_t* bytes);

/* Restore a slot's MPS from the dcs_export_mps format.  Bond b must lie in 1 .. cap_b
 * (see dcs_create), bonds 0 and n must be 1; otherwise DCS_ERR_INVALID.  Synchronises the
 * device. */
dcs_status_t dcs_import_mps(dcs_ctx_t ctx, int slot, const void* host_buf, size_t bytes);

/* Appends one branch at the end of the active list of a multi-path context, in a free slot:
 * its MPS from a HOST buffer in the dcs_export_mps format (bond b in 1 .. cap_b, bonds 0 and
 * n equal to 1), its path probability p, fidelity estimate F, register (DCS_CWORDS words)
 * and flags.  This is how a branch moves between ranks of an ensemble split over several
 * contexts (Alg. 2; the sender exports it, reads p, F, register and flags with
 * dcs_get_results, and drops it with dcs_branch_keep).  Synchronises the device.
 * DCS_ERR_OOM if every slot is active; DCS_ERR_INVALID for null pointers, a single-path
 * context, a malformed buffer, p negative or not finite, or F not finite. */
dcs_status_t dcs_branch_append(dcs_ctx_t ctx, const void* host_buf, size_t bytes, double p,
                               double F, const uint64_t* cwords, uint8_t flags);

/* Runs a whole dynamic circuit (ops in order) from the current state: resets are lowered
 * to measurement + conditional X; operations are grouped into chunks (a chunk closes at a
 * measurement, at chunk_k operations, and before a two-qubit gate touching a qubit that
 * already carries one in the chunk's current sub-layer once the chunk holds
 * max(1, chunk_layers) sub-layers; below that the gate opens the next sub-layer); each
 * chunk is one dcs_apply_layer; runs of
 * measurements are sampled (single-path, measurement ordinals counted from meas_idx0) or
 * split and pruned to M branches (multi-path, M = max_branches; 0 = no pruning).  The
 * circuit's tables are copied to the device once per call.  Asynchronous. */
dcs_status_t dcs_run_circuit(dcs_ctx_t ctx, const dcs_op* ops, int n_ops, uint64_t meas_idx0,
                             int max_branches);

/* Number of kernels this context launched since it was created (a host-side count). */
uint64_t dcs_kernel_launches(dcs_ctx_t ctx);

/* Bytes this context copied host -> device (circuit tables, forced outcomes) since it was
 * created. */
uint64_t dcs_bytes_uploaded(dcs_ctx_t ctx);

/* Synchronises and reads the device counters since the last dcs_init_state: compression
 * steps run (summed over slots) and one-site sweeps run.  A compression step whose initial
 * guess is exact (no truncation beyond tol) runs no sweep: the guess is then the target
 * W|A> itself, which every one-site update would return unchanged. */
dcs_status_t dcs_get_counters(dcs_ctx_t ctx, uint64_t* compressions, uint64_t* sweeps);

/* Complex GEMM, the contraction primitive of the large-bond compression kernels (every
 * environment and site product of the compression step is one): for each of `batch`
 * problems b, C_b[m, n] = sum_k opA(m, k) opB(k, n), m < M, n < N, k < K, with
 * opA(m, k) = A[b sab + m sam + k sak] (conjugated if conjA), opB(k, n) =
 * B[b sbb + k sbk + n sbn] (conjugated if conjB), written to C[b scb + m scm + n scn].
 * A, B, C are DEVICE complex64 arrays, strides in elements (each below 2^31).
 * mode DCS_GEMM_SIMT: FP32 CUDA-core GEMM with shared-memory tiles.
 * mode DCS_GEMM_TENSOR: tcgen05 tensor-core GEMM (TF32 inputs, FP32 accumulators in tensor
 * memory) with each operand split as x = hi + lo (3 products): about 2^-22 relative per
 * product, plus the rounding of the tensor core's FP32 accumulation, which grows with K
 * (relative Frobenius error of random products measured at 1.4e-6 for K = 64 and 1.5e-5 for
 * K = 1024, against 2e-7 and 8e-7 for DCS_GEMM_SIMT);
 * mode DCS_GEMM_TENSOR_BF16X3: the same with BF16 parts (kind::f16), about 2^-16 relative;
 * err_dev: DEVICE int set to 1 if a bounded completion wait gave up (result invalid).
 * One CTA per problem; asynchronous on `stream`. */
#define DCS_GEMM_SIMT 0
#define DCS_GEMM_TENSOR 1
#define DCS_GEMM_TENSOR_BF16X3 2
dcs_status_t dcs_cgemm(int32_t mode, int32_t batch, int32_t M, int32_t N, int32_t K,
                       const void* A, int64_t sam, int64_t sak, int64_t sab, int32_t conjA,
                       const void* B, int64_t sbk, int64_t sbn, int64_t sbb, int32_t conjB,
                       void* C, int64_t scm, int64_t scn, int64_t scb, int32_t* err_dev,
                       dcs_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * Allocation-free compression (the paper has no counterpart to this call).
 *
 * For callers that cannot allocate device memory -- code running under a framework that
 * owns the whole GPU through its own pool, or inside a section where cudaMalloc would
 * synchronise the device or is not allowed -- this one call runs the same compression step
 * as dcs_apply_layer on a single MPS without a context and without allocating anything.
 * Its working memory is a fixed device array of DCS_NOALLOC_SCRATCH_BYTES inside the
 * library, which every GPU that loads the library holds until the process exits.
 *
 *   n_qubits <= DCS_NOALLOC_MAX_QUBITS, chi_max <= DCS_NOALLOC_MAX_CHI and
 *   n_gates <= DCS_NOALLOC_MAX_GATES; larger requests return DCS_ERR_OOM (too big for the
 *   fixed scratch), malformed ones DCS_ERR_INVALID.
 *   gates: one chunk, as for dcs_apply_layer (HOST array).
 *   creg: HOST pointer to DCS_CWORDS words of the classical register that the gates'
 *   conditions read, or NULL for all zeros.
 *   ket: DEVICE buffer of the input MPS, site j at complex64 offset j * 2 * Cc^2, Cc = 4 if
 *   chi_max <= 4 else 8, each site packed row-major as [chi_l][2][chi_r]; ket_bonds: DEVICE
 *   int32[n_qubits + 1] with ket_bonds[0] = ket_bonds[n] = 1 and every bond in 1 .. Cc;
 *   ket_centre: its orthogonality centre (host int).  Read only.
 *   bra, bra_bonds, bra_centre (may be NULL), f: DEVICE outputs in the same layout; f is one
 *   double.  If every gate is skipped by its condition, the ket is copied through, f = 1.
 *   Failures found on the device are reported in the outputs (the call itself has returned
 *   DCS_OK by then): ket bonds outside the rule above give bra_bonds[0] = 0, bra_centre = -1
 *   and f = NaN, with no tensor read or written; a NaN/Inf met in the step or a bounded
 *   device wait that gave up gives f = NaN.
 *
 * The first call on a device looks up the scratch array's device address for that device
 * (with the device current).  Calls share
 * the scratch and it keeps the last call's contents, so calls that overlap on the GPU (on
 * different streams) race.  The call copies the chunk's tables from static host storage and
 * returns after they have been staged, which waits for earlier work on the stream.
 * --------------------------------------------------------------------------------------- */
#define DCS_NOALLOC_MAX_QUBITS 64
#define DCS_NOALLOC_MAX_CHI 8
#define DCS_NOALLOC_MAX_GATES 256
#define DCS_NOALLOC_SCRATCH_BYTES (512u * 1024u)

dcs_status_t dcs_compress_noalloc(int32_t n_qubits, int32_t chi_max, double tol, int32_t sweeps,
                                  const dcs_op* gates, int32_t n_gates, const uint64_t* creg,
                                  const void* ket, const int32_t* ket_bonds, int32_t ket_centre,
                                  void* bra, int32_t* bra_bonds, int32_t* bra_centre, double* f,
                                  dcs_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* DCS_H */
