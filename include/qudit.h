/*
 * qudit.h -- C ABI of libqudit.so: GB300 (sm_103a) block simulation of
 * mixed-radix (qubit-qudit hybrid) state vectors.
 *
 * Method: Velmurugan et al., "Fast classical simulation of qubit-qudit hybrid
 * systems" (arXiv 2410.17876).  A gate is applied directly to the state
 * vector, never by building the circuit unitary (section "Proposed
 * Methodology").  For a gate on wire q_i of dimension d_i, the amplitudes
 * that differ only in digit i form an equivalence class of d_i members
 * spaced b_i = d_0 * ... * d_{i-1} apart (section "Superposition gates",
 * table of equivalent classes); each class is multiplied by the d_i x d_i
 * matrix.  Phase gates scale blocks (section "Phase Gates"), permutation
 * gates rotate them (section "Permutation Gates"), and controlled gates act
 * only on classes whose control digits match (section "Controlled and
 * Multi-Controlled Gates").
 *
 * Conventions shared by every call:
 *   - Wire q_0 is the least significant digit of a basis index; the digit
 *     of wire w in index j is floor(j / b_w) mod d_w.
 *   - Amplitudes are complex; host arrays are interleaved (re, im) IEEE
 *     binary64, so a state of D amplitudes is 2*D doubles.
 *   - Gate matrices are host arrays of P*P complex binary64, row-major,
 *     interleaved (2*P*P doubles); row index = output basis state.  For a
 *     gate on several wires the local index lists the first wire as least
 *     significant.  A complex64 state rounds the matrix to binary32 once.
 *   - Every call returns a qd_status; on failure it writes nothing to its
 *     out-parameters and qd_last_error() holds a message (per thread).
 *     No C++ exception crosses this boundary.
 *   - Apply calls are asynchronous on the state's CUDA stream; input arrays
 *     are copied before the call returns, so the caller may reuse them at
 *     once.  Readouts to host memory synchronise the stream.
 *   - A state is used by one host thread at a time.
 */
#ifndef QUDIT_H
#define QUDIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qd_state qd_state;

typedef int32_t qd_status;
#define QD_OK 0
#define QD_ERR_ARG 1         /* invalid argument (range, duplicate wire, null pointer) */
#define QD_ERR_OOM 2         /* device or host allocation failed */
#define QD_ERR_CUDA 3        /* a CUDA runtime call or kernel launch failed */
#define QD_ERR_TIMEOUT 4     /* a bounded device-side wait gave up */
#define QD_ERR_UNSUPPORTED 5 /* valid request outside the library's limits */
#define QD_ERR_DEVICE 6      /* a kernel reported an error through its status word */

/* Precision of the stored amplitudes. */
#define QD_C64 0  /* complex64: binary32 re/im, binary32 arithmetic */
#define QD_C128 1 /* complex128: binary64 re/im, binary64 arithmetic */

/* Limits of the library. */
#define QD_MAX_WIRES 48      /* wires per state */
#define QD_MAX_DIM 64        /* dimension of one wire */
#define QD_MAX_GATE_DIM 64   /* P = product of a gate's wire dimensions */
#define QD_MAX_CONTROLS 16   /* control wires per gate */

/* ------------------------------------------------------------------------
 * State lifetime (section "Proposed Methodology": the state is the vector
 * of D = d_0 * ... * d_{n-1} amplitudes; only that vector is stored).
 * --------------------------------------------------------------------- */

/* Create a state of n wires with dimensions dims[0..n-1] (each 2..QD_MAX_DIM)
 * in |0...0>, its amplitudes in device memory owned by the library.
 * stream: a cudaStream_t the state's work is issued on (NULL = legacy
 * default stream).  QD_ERR_ARG for a bad dimension or D overflow,
 * QD_ERR_OOM if the allocation fails. */
qd_status qd_state_create(const int32_t* dims, int32_t n, int32_t prec, void* stream,
                          qd_state** out);

/* Wrap caller-owned device memory (for example a torch tensor) as a state.
 * dev_ptr must be 16-byte aligned and hold at least D amplitudes of the
 * given precision (bytes >= D * 8 for QD_C64, D * 16 for QD_C128); its
 * contents are left as they are.  The caller keeps the memory alive until
 * qd_state_destroy.  The library still allocates a small reduction
 * workspace for the state. */
qd_status qd_state_wrap(void* dev_ptr, size_t bytes, const int32_t* dims, int32_t n,
                        int32_t prec, void* stream, qd_state** out);

/* Release the state (and its memory if the library owns it).  Waits for the
 * state's stream.  NULL is accepted. */
qd_status qd_state_destroy(qd_state* st);

/* Set the state to the basis state |0...0>.  Asynchronous: two kernels on
 * the state's stream (a fill of every amplitude with zero, then the one set
 * to 1), no runtime memset. */
qd_status qd_state_reset(qd_state* st);

/* Issue the state's later work on another cudaStream_t (NULL = default). */
qd_status qd_state_set_stream(qd_state* st, void* stream);

/* Number of amplitudes D, number of wires and precision. Any out pointer may be NULL. */
qd_status qd_state_info(const qd_state* st, int64_t* num_amplitudes, int32_t* num_wires,
                        int32_t* prec);

/* Device pointer of the amplitudes (interleaved re/im in the state's precision). */
qd_status qd_state_device_ptr(const qd_state* st, void** dev_ptr);

/* Copy 2*D host doubles (interleaved) into the state (rounded once to
 * binary32 for QD_C64).  Synchronous. */
qd_status qd_state_set_amplitudes(qd_state* st, const double* host_interleaved);

/* Copy the state to 2*D host doubles (widened exactly for QD_C64). Synchronous. */
qd_status qd_state_get_amplitudes(qd_state* st, double* host_interleaved);

/* Copy the raw amplitudes (2*D floats for QD_C64, 2*D doubles for QD_C128)
 * to host memory of `bytes` bytes.  Synchronous. */
qd_status qd_state_get_raw(qd_state* st, void* host, size_t bytes);

/* The same copy, enqueued on the state's stream; the call returns without
 * waiting for it.  Queued gates and the lazy frame are applied first, as
 * for qd_state_get_raw.  The host buffer belongs to the caller and may be
 * read after qd_synchronize on this state; it should be page-locked
 * (cudaHostAlloc, or pinned by the caller's framework), since the CUDA
 * runtime runs a copy into pageable memory through its own staging and
 * returns only once it has landed.  With two states on two streams, one
 * state's read-back then runs while the other state computes.  QD_ERR_ARG
 * for NULL arguments or a buffer smaller than the state; QD_ERR_CUDA if the
 * copy cannot be enqueued. */
qd_status qd_state_get_raw_async(qd_state* st, void* host, size_t bytes);

/* Checkpoint and resume (the paper has no counterpart).  qd_state_save
 * writes the state (after any queued gates and the lazy frame) to a file:
 * a 64-byte header (magic "QDSTATE1", precision, number of wires, D), the
 * wire dimensions as int32, then the raw amplitudes; qd_state_load reads
 * such a file into a state of the same dims and precision (QD_ERR_ARG
 * otherwise, the state unchanged if the header does not match).  Both copy
 * through a pinned staging buffer of at most 256 MiB and are synchronous.
 * QD_ERR_ARG for a path that cannot be opened or a short file; QD_ERR_OOM
 * if the staging buffer cannot be allocated. */
qd_status qd_state_save(qd_state* st, const char* path);
qd_status qd_state_load(qd_state* st, const char* path);

/* Data movement of the wire-swap exchange/* Data movement of the wire-swap exchange between the shards of a state
 * partitioned over several GPUs by its most significant wires (the paper
 * names distributed execution as future work, section "Conclusion").  With
 * lo = b_wire, d = d_wire and hi = D / (lo d), amplitude (h d + y) lo + l of
 * the state is amplitude (y hi + h) lo + l of the moved order: `wire`
 * becomes the most significant digit and the other wires keep their order,
 * so the d blocks that go to d different shards are contiguous.
 * qd_state_wire_to_top writes the moved order to dev_out; qd_state_wire_from_top
 * sets the state from dev_in holding the moved order (as
 * qd_state_set_amplitudes does: queued gates are dropped).  The device
 * buffer holds D amplitudes of the state's precision, is 16-byte aligned,
 * owned by the caller and must not overlap the state.  Asynchronous on the
 * state's stream.  QD_ERR_ARG for a NULL, misaligned or overlapping buffer
 * or a wire out of range. */
qd_status qd_state_wire_to_top(qd_state* st, int32_t wire, void* dev_out);
qd_status qd_state_wire_from_top(qd_state* st, int32_t wire, const void* dev_in);

/* ------------------------------------------------------------------------
 * Gates./* ------------------------------------------------------------------------
 * Gates.
 * --------------------------------------------------------------------- */

/* Apply a d x d matrix U (d = dims[target]) to wire `target`: every class
 * of d amplitudes spaced b_target apart is multiplied by U (section
 * "Superposition gates").  Diagonal matrices are applied as phase gates
 * (section "Phase Gates"; rows with an entry of exactly 1 are not touched)
 * and matrices with one non-zero per row and column as permutations
 * (section "Permutation Gates"); the result is the same as the dense
 * product.  The matrix is not checked for unitarity. */
qd_status qd_apply_gate(qd_state* st, int32_t target, const double* U);

/* Controlled form (section "Controlled and Multi-Controlled Gates"): the two
 * lists ctrl_wires[0..n_ctrl-1] and ctrl_vals[0..n_ctrl-1]; U acts only on
 * basis states whose digit on every control wire equals its value, all
 * other amplitudes are left unchanged.  Control wires must be distinct,
 * differ from the target, and each value must be < its wire's dimension.
 * Only the D / (d_target * prod d_c) matching classes are visited: the
 * control digits are inserted into the enumeration instead of testing
 * every index. n_ctrl = 0 is qd_apply_gate. */
qd_status qd_apply_controlled(qd_state* st, int32_t target, const double* U,
                              const int32_t* ctrl_wires, const int32_t* ctrl_vals,
                              int32_t n_ctrl);

/* The same controlled gate in the paper's formulation, for comparison with
 * qd_apply_controlled (section "Controlled and Multi-Controlled Gates": the
 * control condition floor(i / b_k) mod d_k = v_k is checked index by index,
 * O(D M) tests for M controls): every one of the D / d_target classes of the
 * target wire is visited and its M control digits are tested; matching
 * classes get the update qd_apply_controlled gives them, bit for bit.
 * Arguments and validation as qd_apply_controlled; single wires of
 * dimension <= 8 only (QD_ERR_UNSUPPORTED otherwise).  Asynchronous. */
qd_status qd_apply_controlled_scan(qd_state* st, int32_t target, const double* U,
                                   const int32_t* ctrl_wires, const int32_t* ctrl_vals,
                                   int32_t n_ctrl);

/* Multi-wire gate: a P x P matrix on k distinct wires wires[0..k-1]
 * (P = prod dims[wires[m]] <= QD_MAX_GATE_DIM; local index with wires[0]
 * least significant), optionally controlled as in qd_apply_controlled
 * (ctrl_wires/ctrl_vals may be NULL when n_ctrl = 0).  The paper treats
 * multi-qudit gates in its problem statement (section "Proposed
 * Methodology") and through controls; the class structure generalises to
 * the P amplitudes that differ only in the digits of the gate's wires. */
qd_status qd_apply_multi(qd_state* st, const int32_t* wires, int32_t k, const double* U,
                         const int32_t* ctrl_wires, const int32_t* ctrl_vals, int32_t n_ctrl);

/* ------------------------------------------------------------------------
 * Circuits and gate fusion.  The paper executes gates one after another
 * (section "Experimental Analysis": runtime grows with the N gates executed
 * sequentially) and leaves parallelism across blocks as future scope
 * (end of section "Example Circuit").  A circuit call may run several
 * consecutive gates per pass over the state: a tile holds every amplitude
 * whose digits outside a cached wire set S are fixed (S = the lowest wires,
 * for contiguous rows, plus the high wires the pass's gates act on); each
 * tile is read once, all the pass's gates are applied to it in on-chip
 * memory, and it is written back once.  Gates are reordered only across
 * gates they commute with (disjoint written wires; controls and diagonal
 * gates commute with each other), so the result equals the sequential one
 * up to rounding.
 * --------------------------------------------------------------------- */
#define QD_MAX_GATE_WIRES 6

/* One gate of a circuit: n_wires target wires (local index with wires[0]
 * least significant), n_ctrl controls with values, and the offset, in
 * complex entries, of its P x P row-major matrix inside the `matrices`
 * array passed with the circuit (2 doubles per entry). */
typedef struct qd_gate_desc {
    int32_t n_wires;
    int32_t n_ctrl;
    int32_t wires[QD_MAX_GATE_WIRES];
    int32_t ctrl_wires[QD_MAX_CONTROLS];
    int32_t ctrl_vals[QD_MAX_CONTROLS];
    int64_t matrix_offset;
} qd_gate_desc;

#define QD_FUSE_OFF 0   /* one kernel pass per gate */
#define QD_FUSE_TILE 1  /* shared-memory tile passes over cached wire sets */
#define QD_FUSE_BLOCK 2 /* the circuit is grouped into blocks of at most block_dim (default 64 for
                           complex64, 8 for complex128) dimensions, each composed in binary64 and
                           applied in one pass over the state; complex64 blocks of 17 or more
                           dimensions (with QD_TC_BF16X3 and no controls: 9 or more) run as set
                           by tc_mode */

/* Arithmetic of complex64 blocks and multi-wire gates of 17..64 dimensions,
 * and with QD_TC_BF16X3 of those of 9..16 dimensions without controls too
 * (qd_fusion_opts.tc_mode, qd_set_fusion).  The block is applied as the real
 * contraction [Re Y; Im Y] = [[Re M, -Im M], [Im M, Re M]] [Re X; Im X].
 * The tensor-core modes split both operands, a = a_hi + a_lo, and accumulate
 * A_hi X_hi + A_hi X_lo + A_lo X_hi in FP32 in tensor memory. */
#define QD_TC_TF32X3 0 /* tensor cores, TF32 parts (about 2^-21 relative per block); the default */
#define QD_TC_BF16X3 1 /* tensor cores, BF16 parts (about 2^-16 relative per block); blocks without
                          controls (9..64 dimensions) stream the state through a ring of
                          shared-memory tiles (the classes of a tile as tensor-memory rows of
                          the MMA's A operand) */
#define QD_TC_OFF 2    /* FP32 CUDA cores (binary32 FMA, no split) */

typedef struct qd_fusion_opts {
    int32_t mode;          /* QD_FUSE_OFF or QD_FUSE_TILE */
    int32_t max_tile_amps; /* amplitudes per tile, 0 = default (8192 complex64, 4096 complex128) */
    int32_t min_gates;     /* passes with fewer gates run gate by gate; 0 = default (2) */
    int32_t min_row;       /* contiguous amplitudes per tile row, 0 = default (16 c64, 8 c128) */
    int32_t block_dim;     /* inside a pass, runs of gates on a few wires are composed (binary64,
                              on the host) into one P x P block with P <= block_dim (at most 16);
                              0 = default (16), 1 = no composition */
    int32_t tc_mode;       /* QD_TC_TF32X3 (0, default), QD_TC_BF16X3 or QD_TC_OFF */
} qd_fusion_opts;

/* Apply n_gates gates in order.  Each gate is validated as in
 * qd_apply_multi before anything is launched (QD_ERR_ARG / UNSUPPORTED:
 * nothing applied).  opts = NULL means QD_FUSE_OFF.  Asynchronous; the
 * arrays may be reused when the call returns. */
qd_status qd_apply_circuit(qd_state* st, const qd_gate_desc* gates, int32_t n_gates,
                           const double* matrices, const qd_fusion_opts* opts);

/* Deferred fusion of the single-gate calls.  After qd_set_fusion with
 * max_block_dim >= 2, qd_apply_gate / qd_apply_controlled / qd_apply_multi
 * validate their gate and copy it into a host queue instead of launching;
 * the queue runs as one qd_apply_circuit call in QD_FUSE_BLOCK mode
 * (block_dim = max_block_dim, at most 64; tc_mode as above) at qd_flush,
 * before every readout, qd_state_get_amplitudes / get_raw / device_ptr /
 * set_stream / qd_synchronize, and whenever it holds 4096 gates.
 * qd_state_set_amplitudes and qd_state_reset discard the queue (the state
 * is overwritten).  max_block_dim <= 1 flushes and returns to one launch
 * per call; tc_mode also selects the arithmetic of unfused complex64
 * multi-wire gates of 17..64 dimensions (BF16X3 without controls: 9..64).  QD_ERR_ARG for an unknown
 * tc_mode. */
qd_status qd_set_fusion(qd_state* st, int32_t max_block_dim, int32_t tc_mode);

/* Lazy permutations and phases for the single-gate calls (off by default).
 * With enable = 1 an uncontrolled single-wire gate whose matrix has exactly
 * one entry of modulus 1 per row and column (X_{+a}, Z_d, S, T and their
 * products) launches nothing: it is folded into a per-wire digit relabeling
 * and phase vector kept on the host.  Every other gate runs with its
 * control values and matrix rewritten for that frame (the wire's pending
 * phases folded into the matrix; a controlled gate applies its target
 * wires' pending phases first, as one diagonal launch per wire, since its
 * unmatched classes keep them).  qd_norm and qd_marginal need no extra
 * work; amplitude readouts, probabilities, qd_state_device_ptr,
 * qd_apply_circuit, qd_set_fusion and qd_set_lazy(st, 0) first apply the
 * frame (one pass per touched wire); set_amplitudes and reset clear it.
 * Deferred fusion (qd_set_fusion >= 2) takes precedence: its queued gates
 * are not folded. */
qd_status qd_set_lazy(qd_state* st, int32_t enable);

/* Run the gates queued by deferred fusion (no-op when none are queued). */
qd_status qd_flush(qd_state* st);

/* The execution plan of qd_apply_circuit without a GPU: exec_order[i] is the
 * index of the i-th gate executed, pass_of[i] its pass, pass_tile_amps[p]
 * the tile size of pass p (0 = a per-gate kernel pass), pass_flops[p] the
 * arithmetic of pass p over the whole state (real floating-point operations:
 * 8 P per amplitude for a dense P x P block or gate, 6 per changed amplitude
 * for a diagonal or phased-permutation one, 0 for a pure permutation; for a
 * complex64 run of gates applied one by one in registers, 8 d per amplitude
 * of the classes each d x d gate's controls admit), and
 * *n_passes the number of passes.  Every array has n_gates entries;
 * pass_tile_amps and pass_flops may be NULL. */
qd_status qd_plan_circuit(const int32_t* dims, int32_t n, int32_t prec, const qd_gate_desc* gates,
                          int32_t n_gates, const double* matrices, const qd_fusion_opts* opts,
                          int32_t* exec_order, int32_t* pass_of, int64_t* pass_tile_amps,
                          double* pass_flops, int32_t* n_passes);

/* ------------------------------------------------------------------------
 * Sparse states (the paper's sparse variant: only the non-zero amplitudes
 * are stored, and a unitary is applied by inspecting their indices; end of
 * section "Example Circuit", GHZ runs of section "Experimental Analysis").
 * complex128 amplitudes; single-wire gates on wires of dimension 2..8,
 * optionally controlled.  Basis states are 128-bit keys, so the basis
 * may be far larger than 2^64 (the paper's keys are 64-bit): the wires'
 * bit widths ceil(log2 d) must sum to at most 128 and D must stay below
 * 2^128.  A whole circuit runs in one launch on one CTA with the
 * amplitudes in shared memory while the support stays within
 * QD_SPARSE_MAX_NNZ non-zero amplitudes after every gate; after
 * qd_sparse_reserve, larger supports run gate by gate on the whole GPU.
 * --------------------------------------------------------------------- */
#define QD_SPARSE_MAX_NNZ 512
#define QD_SPARSE_MAX_WIRES 128
#define QD_SPARSE_MAX_RESERVE (1 << 22)

typedef struct qd_sparse qd_sparse;

/* A sparse state in |0...0> on n wires (dims[w] in 2..8).  stream: the
 * cudaStream_t its work runs on (NULL = legacy default stream).
 * QD_ERR_ARG for a dimension out of range or a basis beyond 128 bits. */
qd_status qd_sparse_create(const int32_t* dims, int32_t n, void* stream, qd_sparse** out);
qd_status qd_sparse_destroy(qd_sparse* s);

/* Allow supports of up to max_nnz non-zero amplitudes (QD_SPARSE_MAX_NNZ <
 * max_nnz <= QD_SPARSE_MAX_RESERVE; never shrinks).  Calls whose support
 * stays within QD_SPARSE_MAX_NNZ keep running in one launch on one CTA;
 * a call that goes beyond it runs gate by gate on the whole GPU: entries in
 * global memory, dense gates through a global hash table of classes (370
 * to 640 bytes of device memory per entry of capacity: three entry buffers
 * and a table of 2 to 4 slots per entry).  QD_ERR_ARG for
 * max_nnz out of range, QD_ERR_OOM if the buffers cannot be allocated (the
 * state and its capacity unchanged). */
qd_status qd_sparse_reserve(qd_sparse* s, int64_t max_nnz);

/* Apply n_gates single-wire gates (qd_gate_desc with n_wires = 1, controls
 * allowed; matrices as in qd_apply_circuit) in order.  Synchronous.  Exact
 * zeros are dropped.  QD_ERR_UNSUPPORTED (state left as before the call)
 * if a gate has more than one wire or the support exceeds QD_SPARSE_MAX_NNZ
 * (or the capacity set by qd_sparse_reserve). */
qd_status qd_sparse_run(qd_sparse* s, const qd_gate_desc* gates, int32_t n_gates, const double* matrices);

/* Number of stored (non-zero) amplitudes. */
qd_status qd_sparse_nnz(const qd_sparse* s, int64_t* nnz);

/* The stored amplitudes in ascending basis-index order: index i =
 * index_lo[i] + 2^64 index_hi[i] (mixed-radix, q_0 least significant),
 * amplitude (amps[2i], amps[2i+1]).  max = room in each array
 * (QD_ERR_ARG if it is below the count); *n_out = count. */
qd_status qd_sparse_get(qd_sparse* s, uint64_t* index_lo, uint64_t* index_hi, double* amps_interleaved,
                        int64_t max, int64_t* n_out);

/* ------------------------------------------------------------------------
 * Batches of independent circuits.  Each circuit starts from its own
 * |0...0> state; the states of one run live side by side in one device
 * buffer owned by the batch.  The paper simulates one circuit at a time;
 * independent circuits share nothing, so they run concurrently:
 *   - a circuit whose state fits one CTA's shared memory (D <=
 *     small_max_amps) and whose gates are all single-wire with d <= 5 and
 *     at most 7 controls runs whole inside one CTA -- all such circuits in
 *     one launch, the state written to HBM once at the end;
 *   - every other circuit runs as a (fused) circuit program, round-robin on
 *     n_streams auxiliary streams joined back to the batch stream;
 *   - with use_graph, the whole run is captured in a CUDA graph, launched,
 *     and kept for qd_batch_relaunch.
 * Every circuit's squared norm is reduced on the GPU after its last gate.
 * --------------------------------------------------------------------- */
typedef struct qd_batch qd_batch;

typedef struct qd_circuit {
    int32_t n_wires;
    const int32_t* dims;        /* n_wires dimensions, q_0 first */
    int32_t n_gates;
    const qd_gate_desc* gates;  /* as for qd_apply_circuit */
    const double* matrices;
} qd_circuit;

typedef struct qd_batch_opts {
    int32_t small_max_amps;  /* 0 = default (8192 complex64, 4096 complex128) */
    int32_t n_streams;       /* 0 = default (8), at most 64 */
    int32_t use_graph;       /* capture the run in a CUDA graph */
    int32_t path;            /* 0 (default): circuits whose passes are all tile passes run through the
                                device-side layer queue; 1: every such circuit as its own program on
                                the auxiliary streams */
    qd_fusion_opts fusion;   /* for circuits outside the one-CTA path */
} qd_batch_opts;

/* Create an empty batch whose work is issued on `stream` (NULL = default). */
qd_status qd_batch_create(int32_t prec, void* stream, qd_batch** out);

/* Validate all n circuits (nothing runs if one is invalid: QD_ERR_ARG or
 * QD_ERR_UNSUPPORTED naming the circuit), lay out their states, and issue
 * the run asynchronously.  opts = NULL: defaults with tile fusion.  The
 * arrays may be reused when the call returns.  A batch is used by one host
 * thread at a time; a new run replaces the previous run's states. */
qd_status qd_batch_run(qd_batch* b, const qd_circuit* circuits, int32_t n, const qd_batch_opts* opts);

/* Launch the graph captured by the last qd_batch_run again (same circuits,
 * recomputed from |0...0>).  QD_ERR_ARG if that run was not captured. */
qd_status qd_batch_relaunch(qd_batch* b);

/* Device pointer and amplitude count of circuit i's state after the run. */
qd_status qd_batch_state(qd_batch* b, int32_t i, void** dev_ptr, int64_t* num_amplitudes);

/* Circuit i's final state as 2*D host doubles (widened exactly for
 * QD_C64).  Synchronous. */
qd_status qd_batch_get_amplitudes(qd_batch* b, int32_t i, double* host_interleaved);

/* The n squared norms of the last run into host_out.  Synchronous. */
qd_status qd_batch_norms(qd_batch* b, double* host_out);

qd_status qd_batch_synchronize(qd_batch* b);
qd_status qd_batch_destroy(qd_batch* b);

/* ------------------------------------------------------------------------
 * Serving.  Requests (circuits, each from |0...0>) arrive over time; a
 * worker thread admits them in arrival order while the state bytes fit the
 * server's device-memory budget and an execution slot is free, runs them
 * concurrently with the requests already on the GPU (continuous batching:
 * small states admitted in the same step share one one-CTA-per-circuit
 * launch, larger ones run as fused circuit programs on their own streams),
 * reduces each final state's squared norm, frees its memory (unless kept)
 * and publishes the result with arrival / admission / completion times on
 * the server's clock (seconds since creation).  A request's kernels depend
 * only on its own circuit: its result is the same alone and in any mix.
 * --------------------------------------------------------------------- */
typedef struct qd_server qd_server;

typedef struct qd_server_opts {
    uint64_t hbm_budget_bytes; /* device memory for resident states, 0 = 8 GiB */
    int32_t max_slots;         /* concurrent larger requests, 0 = 16 */
    int32_t small_max_amps;    /* one-CTA path threshold, 0 = default */
    int32_t max_group;         /* small requests per launch, 0 = 1024 */
    int32_t reserved;
    qd_fusion_opts fusion;     /* for larger requests (mode QD_FUSE_OFF = per gate) */
} qd_server_opts;

typedef struct qd_request_result {
    uint64_t id;
    int32_t status;          /* QD_OK or the error of this request */
    int32_t kept;            /* state kept until qd_server_release */
    int64_t num_amplitudes;
    double norm;             /* squared norm of the final state */
    double t_arrival, t_admit, t_done;
} qd_request_result;

/* Create a server (allocates the state budget, starts the worker thread). */
qd_status qd_server_create(int32_t prec, const qd_server_opts* opts, qd_server** out);

/* Submit a circuit now (copied before return).  keep_state: keep the final
 * state on the device until qd_server_release.  QD_ERR_ARG for an invalid
 * circuit, QD_ERR_UNSUPPORTED if its state exceeds the whole budget. */
qd_status qd_server_submit(qd_server* s, const qd_circuit* c, int32_t keep_state, uint64_t* id_out);

/* Submit a circuit that arrives at server time release_time (an open-loop
 * load generator can submit a whole trace ahead of time). */
qd_status qd_server_submit_at(qd_server* s, const qd_circuit* c, int32_t keep_state, double release_time,
                              uint64_t* id_out);

/* Move up to max finished results into out (oldest first); *n_out = count. */
qd_status qd_server_poll(qd_server* s, qd_request_result* out, int32_t max, int32_t* n_out);

/* Wait until every submitted request has finished (QD_ERR_TIMEOUT otherwise). */
qd_status qd_server_drain(qd_server* s, double timeout_s);

/* Current server time in seconds. */
qd_status qd_server_now(qd_server* s, double* t);

/* A finished, kept request's state as 2*D host doubles.  Synchronous. */
qd_status qd_server_get_amplitudes(qd_server* s, uint64_t id, double* host_interleaved);

/* Return a kept state's memory to the budget. */
qd_status qd_server_release(qd_server* s, uint64_t id);

/* Stop the worker after all submitted requests finished, free everything. */
qd_status qd_server_destroy(qd_server* s);

/* ------------------------------------------------------------------------
 * Readouts.  Sums run in binary64 with compensated (Neumaier) summation in
 * a fixed order, so results are deterministic for a given state size.
 * The paper defines no readout; these are the standard Born-rule
 * quantities of the state vector.
 * --------------------------------------------------------------------- */

/* sum_j |psi_j|^2 into *out (host).  Synchronous. */
qd_status qd_norm(qd_state* st, double* out);

/* |psi_j|^2 for all j into host_out[0..D-1].  Synchronous. */
qd_status qd_probabilities(qd_state* st, double* host_out);

/* |psi_j|^2 into device memory dev_out[0..D-1] (8-byte aligned).  Asynchronous. */
qd_status qd_probabilities_device(qd_state* st, double* dev_out);

/* Marginal of one wire: host_out[x] = sum over j with digit_wire(j) = x of
 * |psi_j|^2, for x < dims[wire].  Synchronous. */
qd_status qd_marginal(qd_state* st, int32_t wire, double* host_out);

/* Wait for all work issued on the state's stream. */
qd_status qd_synchronize(qd_state* st);

/* ------------------------------------------------------------------------
 * Norm without allocation.  The paper has no counterpart to this call; it
 * exists for callers that cannot allocate device memory: a framework whose
 * caching allocator owns all device memory and forbids allocations beside
 * it, or a latency-critical loop that must not stall on the device-wide
 * synchronisation an allocation can cause.  qd_norm needs a qd_state, and
 * creating a state allocates its reduction workspace; this call allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine).
 *
 * dev_amps: num_amplitudes interleaved amplitudes in device memory (float
 *   pairs for QD_C64, 8-byte aligned; double pairs for QD_C128, 16-byte
 *   aligned), owned by the caller and only read.
 * dev_out: one double in device memory (8-byte aligned) that receives
 *   sum_j |psi_j|^2, computed exactly as qd_norm does (binary64, Neumaier
 *   compensation, fixed order), so the two agree bit for bit on the same
 *   amplitudes, whichever the alignment of dev_amps (an 8-byte-aligned
 *   complex64 pointer reads each pair of amplitudes with two loads instead
 *   of one, in the same order).
 * stream: the cudaStream_t the two kernels are issued on (NULL = default);
 *   the call is asynchronous, read dev_out after synchronising the stream.
 *
 * Scratch: the partial sums live in a fixed device array inside the library,
 * QD_NORM_NOALLOC_BLOCKS pairs of doubles (16 KiB), which every GPU that
 * loads the library keeps until the process exits.  The first call on each
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture.
 * Calls share the array and it keeps the last call's contents (each call
 * writes every entry it reads before reading it, so nothing needs
 * clearing); calls whose kernels overlap on the GPU -- on different streams
 * or different host threads without ordering -- race on it and give wrong
 * results.  Order them on one stream or with events.  The looked-up address
 * is kept for the life of the process: after cudaDeviceReset (or anything
 * else that destroys a device's primary context) it is stale, so do not
 * call qd_norm_noalloc on that device again in the same process.
 *
 * Errors: QD_ERR_ARG for NULL or misaligned pointers, an unknown precision,
 * or num_amplitudes outside [1, QD_NORM_NOALLOC_MAX_AMPLITUDES];
 * QD_ERR_UNSUPPORTED for a device ordinal of 64 or above (the library keeps
 * one looked-up address per device for ordinals 0..63);
 * QD_ERR_CUDA if the set-up or a launch fails.
 * --------------------------------------------------------------------- */
#define QD_NORM_NOALLOC_BLOCKS 1024
#define QD_NORM_NOALLOC_MAX_AMPLITUDES ((int64_t)1 << 44)
qd_status qd_norm_noalloc(const void* dev_amps, int64_t num_amplitudes, int32_t prec, void* stream,
                          double* dev_out);

/* ------------------------------------------------------------------------
 * Introspection (host only; no GPU needed).
 * --------------------------------------------------------------------- */

/* Message of the last failed call on this thread ("" if none). */
const char* qd_last_error(void);

/* Number of kernels this library has launched in the process so far. */
uint64_t qd_launch_count(void);

/* Bytes of gate data this library has copied from host to device memory in
 * the process so far: circuit descriptors (with composed block matrices and
 * tensor-core operands) and single-gate matrices.  Amplitude uploads
 * (qd_state_set_amplitudes, qd_state_load) and the batch and sparse paths'
 * own uploads are not counted. */
uint64_t qd_bytes_uploaded(void);

/* Library version string. */
const char* qd_version(void);

/* Plan of a gate without a GPU: which kernel family would run it
 * (0 = per-class register kernel, 1 = shared-memory tile kernel),
 * the number of classes visited, the vector width in amplitudes and the
 * kind the matrix was classified as (0 dense, 1 diagonal, 2 permutation).
 * Arguments as in qd_apply_multi plus the state's dims/prec. */
typedef struct qd_plan_info {
    int32_t family;
    int32_t kind;
    int32_t vec;
    int32_t touched_rows; /* rows of each class that are written */
    int64_t classes;      /* classes visited */
    int64_t run;          /* contiguous run of the class enumeration, in amplitudes */
} qd_plan_info;
qd_status qd_plan_gate(const int32_t* dims, int32_t n, int32_t prec, const int32_t* wires,
                       int32_t k, const double* U, const int32_t* ctrl_wires,
                       const int32_t* ctrl_vals, int32_t n_ctrl, qd_plan_info* out);

/* Testing hook of the bounded waits in the tensor-core block kernels (complex64
 * blocks of 17..64 dimensions: qd_apply_multi, QD_FUSE_BLOCK passes, deferred
 * fusion; the register-staged kernel and the BF16x3 tile-ring kernel).  The paper has no counterpart; it exists so that the timeout path
 * can be exercised without a GPU fault.  Every mbarrier wait of that kernel
 * gives up after spin_limit polls (0 = the default, 2^26); the kernel then
 * records QD_ERR_TIMEOUT in its status word, issues no further work, writes
 * no output, releases its tensor memory and returns, and the next readout
 * of the state (qd_norm, qd_probabilities, ...) returns QD_ERR_TIMEOUT.
 * stall_producers != 0 makes the kernel's producer (or loader) warps publish
 * nothing, so the first waits run out and the pass leaves the state as it was.  The
 * setting is process-wide and applies to launches issued after the call;
 * (0, 0) restores the defaults.  Always QD_OK. */
qd_status qd_test_set_tc_wait(uint32_t spin_limit, int32_t stall_producers);

/* Testing hook: launches of the BF16x3 tile-ring kernel since the library was
 * loaded (process-wide), so that a test can tell which tensor-core kernel
 * ran a block.  Always QD_OK; out may not be NULL. */
qd_status qd_test_tc_ring_launches(int64_t* out);

/* Bounds-checked build (compiled with QD_BOUNDS=1: a debug build of the
 * library in place of a memory sanitizer; the paper has no counterpart).
 * Its gate kernels -- per-class register kernel, multi-wire tile kernel,
 * fused tile passes, the batch layer queue and the tensor-core block kernel
 * -- check every global index they form against the size of the buffer it
 * indexes; an index outside is recorded (the first one) and that access is
 * skipped, with no trap or assert.  qd_bounds_status reads and clears the
 * record: QD_OK and *first_bad_index = -1 if nothing was recorded,
 * QD_ERR_DEVICE and the index otherwise.  *checks_compiled is 1 in the
 * bounds-checked build, 0 in the regular one (where the record stays empty).
 * Either out pointer may be NULL. */
qd_status qd_bounds_status(int64_t* first_bad_index, int32_t* checks_compiled);

/* Testing hook of the bounds-checked build: the per-class register kernel
 * and the multi-wire tile kernel are told that their state is `amplitudes`
 * shorter than it is, so that accesses to its last amplitudes are reported
 * (and skipped) -- the check exercised without any access outside a buffer.
 * 0 restores the default.  QD_ERR_ARG for a negative value. */
qd_status qd_test_set_bounds_shrink(int64_t amplitudes);

/* Host self-test of the index arithmetic (division by invariant integers
 * and the class enumeration) against plain integer division on
 * `trials` random cases.  QD_OK if every case agrees. */
qd_status qd_selftest_host(int32_t trials);

#ifdef __cplusplus
}
#endif

#endif /* QUDIT_H */
