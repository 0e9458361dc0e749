/*
 * qsim.h -- C ABI of the GB300 state-vector library (sm_103a).
 *
 * The library applies parameterised gates to 2^n-amplitude complex state
 * vectors on one GPU and computes the reversible-adjoint gradient, following
 * the register / instruction-set statement of Yao.jl (arXiv 1912.10877):
 * Sec. "Instructions on Quantum Registers" (instruct!, measure, measure!),
 * Sec. "Representing Quantum Circuits" (apply! of a chain), Sec. "Forward
 * Mode" (expect of sums of Pauli strings), Sec. "Reverse Mode" (expect',
 * Eqs. apply-back and outer-product) and Sec. "Batched Quantum Registers".
 *
 * Conventions shared by every entry point
 *  - Qubit order is little-endian: qubit loc l (0-based) is bit l of the basis
 *    index; the paper's 1-based qubit q is loc q-1.
 *  - A k-qubit gate on locs (l_0, ..., l_{k-1}) has matrix index bit j <->
 *    qubit l_j; matrices are row-major 2^k x 2^k with interleaved (re, im)
 *    doubles and are always passed in FP64 (the library rounds them once to
 *    FP32 for complex64 states).
 *  - Controls: ctrl value 1 = control on |1>, 0 = inverse control on |0>.
 *  - Amplitudes are interleaved (re, im): QS_C64 = 2 x float per amplitude,
 *    QS_C128 = 2 x double.  A batch of registers is stored back to back,
 *    register r at element offset offsets[r] (offsets are prefix sums of
 *    2^{n_r}); each register is contiguous.
 *  - Pointers named dev_* are device pointers; host_* are host pointers.
 *    Every call is asynchronous on the state's stream except those that write
 *    host outputs, which synchronise that stream before returning.
 *  - Every entry point returns QS_OK (0) or a negative status; no exception
 *    crosses the ABI.  qs_last_error() gives a message for the calling thread.
 *  - Handles are not thread-safe; use one handle per host thread or serialise.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define QS_OK 0
#define QS_EINVAL (-1)        /* bad argument: size, loc, duplicate qubit, null pointer */
#define QS_ENOMEM (-2)        /* device or host allocation failed */
#define QS_EDEVICE (-3)       /* a CUDA call or kernel failed */
#define QS_ETIMEDOUT (-4)     /* a bounded device-side wait gave up */
#define QS_EUNSUPPORTED (-5)  /* valid request the library does not implement */

/* amplitude types */
#define QS_C64 0   /* complex64: FP32 math and accumulation for gate application */
#define QS_C128 1  /* complex128: FP64 */

#define QS_MAXK 5        /* largest gate arity (targets) */
#define QS_MAXQ 40       /* largest register (qubits) */

/* gate kinds (App. "Builtin Block Types"; R_S(theta) = exp(-i S theta / 2),
 * Sec. "Forward Mode"; shift(theta) = diag(1, e^{i theta}), listing
 * "inspecting gates"; phase(theta) = e^{i theta} on the target) */
enum qs_gate_kind {
  QS_GATE_I = 0, QS_GATE_X, QS_GATE_Y, QS_GATE_Z, QS_GATE_H, QS_GATE_S, QS_GATE_SDG,
  QS_GATE_T, QS_GATE_TDG, QS_GATE_RX, QS_GATE_RY, QS_GATE_RZ, QS_GATE_SHIFT,
  QS_GATE_PHASE, QS_GATE_SWAP, QS_GATE_ROT, QS_GATE_MATRIX
};

/* One entry of a flat gate list (the paper's put / control / chain blocks,
 * flattened).  QS_GATE_ROT is exp(-i theta/2 * sigma_{paulis[0]} (x) ...) on
 * locs; QS_GATE_MATRIX reads 2^k x 2^k entries at mat_offset of the matrix
 * pool given to qs_circuit_create. */
typedef struct qs_gate_desc {
  int32_t kind;              /* enum qs_gate_kind */
  int32_t nlocs;             /* k, 1..QS_MAXK (SWAP: 2) */
  int32_t locs[QS_MAXK];     /* target qubits */
  int32_t paulis[QS_MAXK];   /* ROT: 1 = X, 2 = Y, 3 = Z per target */
  int32_t param;             /* index into the parameter vector, -1 = use theta */
  int32_t reserved;
  uint64_t ctrl_mask;        /* bit q set: qubit q is a control */
  uint64_t ctrl_vals;        /* bit q: required value of control q */
  int64_t mat_offset;        /* MATRIX: offset in complex entries into the pool */
  double theta;              /* fixed angle when param < 0 */
} qs_gate_desc;

/* One Pauli string with a real coefficient: qubit q carries X if only bit q of
 * x_mask is set, Z if only bit q of z_mask is set, Y if both. */
typedef struct qs_pauli_term {
  double coeff;
  uint64_t x_mask;
  uint64_t z_mask;
} qs_pauli_term;

typedef struct qs_state qs_state;
typedef struct qs_circuit qs_circuit;
typedef struct qs_observable qs_observable;

/* Message describing the last failure on the calling thread ("" if none). */
const char* qs_last_error(void);

/* ---------------------------------------------------------------- states */

/* Bytes of amplitude storage for nreg registers of nqubits[r] qubits. */
int qs_state_bytes(int nreg, const int32_t* host_nqubits, int dtype, size_t* out_bytes);

/* A register (nbatch = 1) or a uniform batch of nbatch registers of nqubits
 * qubits (Sec. "Batched Quantum Registers").  dev_buf, if not NULL, must hold
 * qs_state_bytes() bytes, 256-byte aligned, and stays owned by the caller for
 * the life of the handle; if NULL the library allocates and frees it.  The
 * amplitudes are NOT initialised: call qs_state_reset or qs_state_upload.
 * stream is a cudaStream_t (NULL = legacy default stream). */
int qs_state_create(int nqubits, int dtype, int nbatch, void* dev_buf, void* stream,
                    qs_state** out);

/* A batch of nreg registers of uneven sizes host_nqubits[r] (1..QS_MAXQ). */
int qs_batch_create(int nreg, const int32_t* host_nqubits, int dtype, void* dev_buf,
                    void* stream, qs_state** out);

int qs_state_destroy(qs_state* s);
int qs_state_set_stream(qs_state* s, void* stream);

/* Device pointer of the amplitudes, total bytes, and element offsets of the
 * registers (host_offsets may be NULL; else it receives nreg + 1 values). */
int qs_state_data(const qs_state* s, void** dev_ptr, size_t* bytes, int64_t* host_offsets);

/* |x_r> on every register r: host_basis[r] is the basis index (NULL = |0...0>). */
int qs_state_reset(qs_state* s, const uint64_t* host_basis);

/* Copy all amplitudes from / to host memory (pageable or pinned), in the
 * state's dtype and layout.  Both synchronise the stream. */
int qs_state_upload(qs_state* s, const void* host_amps);
int qs_state_download(const qs_state* s, void* host_amps);

/* Wait for every operation queued on the state's stream.  Returns
 * QS_ETIMEDOUT if, since the last call, a tensor-core kernel's bounded wait
 * for its own MMA completion gave up (its tile was then left unwritten); the
 * word is device-wide and is cleared by this call.  Other errors as
 * QS_EDEVICE. */
int qs_state_sync(qs_state* s);

/* ---------------------------------------------------------------- level-1 operations
 *
 * The pieces of the reversible adjoint (Sec. "Reverse Mode", Eq. apply-back)
 * for a caller that walks a circuit gate by gate itself, e.g. over a state
 * split into pieces across processes: the gradient of U = exp(-i theta c H) is
 * 2 c Im<lambda|H psi>, an inner product; lambda = O psi is a sum of Pauli
 * strings applied to copies of psi.  a/b, dst/src and x/y must have the same
 * dtype and register sizes (QS_EINVAL otherwise). */

/* dst <- src, asynchronous on dst's stream (order src's earlier work before
 * it: same stream or an event).  The dtypes may differ (same register sizes):
 * complex64 -> complex128 widens exactly, complex128 -> complex64 rounds to
 * nearest. */
int qs_state_copy(qs_state* dst, const qs_state* src);

/* <a_r|b_r> = sum_i conj(a_r,i) b_r,i per register r into host_out[2 nreg]
 * (re, im): products and sums in FP64, per-block partial sums folded in block
 * order (the same result on every run).  Runs on a's stream and synchronises
 * it. */
int qs_state_inner(qs_state* a, const qs_state* b, double* host_out);

/* y <- y + alpha x in the states' precision (alpha rounded to FP32 for
 * complex64), asynchronous on y's stream.  x and y must be distinct. */
int qs_state_axpy(qs_state* y, double alpha_re, double alpha_im, const qs_state* x);

/* One gate of the reversible adjoint walk (Sec. "Reverse Mode", Eq.
 * apply-back) on two complex128 single registers psi and lambda of the same
 * size, for a caller that walks a circuit itself with other work in between
 * (a register split over processes exchanges shard halves between gates).
 * g's targets and controls are qubits of these registers.  A parameterised
 * gate U = exp(-i theta c H) (RX, RY, RZ, SHIFT, PHASE, ROT on at most 3
 * targets; QS_EUNSUPPORTED beyond) first adds
 * 2 c Im<lambda|(P_ctrl (x) H)|psi> to dev_grad[g->param] (device memory,
 * FP64, added in stream order: no synchronisation), P_ctrl the projector onto
 * the control values; then psi <- U^dag psi and lambda <- U^dag lambda in
 * FP64; any other gate is only uncomputed.  host_mats: interleaved complex
 * doubles a MATRIX gate reads at mat_offset (else may be NULL); host_params:
 * the parameter vector (theta = host_params[g->param]).  Asynchronous on
 * psi's stream (lambda must be ordered with it). */
int qs_adjoint_step(qs_state* psi, qs_state* lam, const qs_gate_desc* g, const double* host_mats,
                    const double* host_params, double* dev_grad);

/* Host-side matrices of one gate record (no device work; callable without a
 * GPU): host_U (may be NULL) receives U, or U^dag if dagger_u != 0 (2^k x 2^k,
 * row-major, interleaved re/im, index bit j <-> locs[j], controls not
 * included); host_G / host_cfac (may be NULL) the generator H on the targets
 * and c with U = exp(-i theta c H) (QS_EINVAL for a gate without a
 * parameter).  host_mats / host_params as for qs_adjoint_step. */
int qs_gate_desc_matrices(const qs_gate_desc* g, const double* host_mats, const double* host_params, int dagger_u,
                          double* host_U, double* host_G, double* host_cfac);

/* The first level of a measurement over a register split into nshards
 * pieces (host only): with the pieces' weights P_s = <psi_s|psi_s>, each shot
 * picks a piece by qs_measure's walk (T = left fold of the weights, t = u T,
 * the first piece whose running sum exceeds t, else the last positive one)
 * and the uniform u' = (t - prefix) / P_s (kept below 1) that the piece's own
 * sampler then takes.  QS_EINVAL for a uniform outside [0, 1). */
int qs_sample_shards(int nshards, const double* host_weights, int nshots, const double* host_u,
                     int32_t* host_shard, double* host_u_in_shard);

/* ---------------------------------------------------------------- options */

/* Process-wide switches (not thread-safe against concurrent launches).
 * QS_OPT_TENSOR_CORES: which kernel applies dense 4- and 5-qubit gates to
 * complex64 states.  2: always the tensor cores (complex product as a real
 * 3xTF32 GEMM, FP32 accuracy); 0: always the CUDA cores; 1 (default): the
 * tensor cores for the target placements where they measured faster: targets
 * q..q+k-1 without controls (read by TMA tensor copies), other 5-qubit blocks
 * unless every target is at qubit 5 or above, other 4-qubit blocks on qubit 0. */
#define QS_OPT_TENSOR_CORES 1
int qs_set_option(int option, int value);
int qs_get_option(int option, int* value);

/* ---------------------------------------------------------------- faithful gradients */

/* Sec. "Forward Mode: Faithful Quantum Gradients".  Shot-based <O> on every
 * register of s: the terms are split into groups that share a measurement
 * basis on every qubit (qubit-wise commuting, in order of first appearance;
 * qs_observable_groups gives their count G).  Per group, a copy of the state
 * (dev_work: s's size) is rotated to the group's basis (X: H; Y: S^dag then
 * H), nshots indices are sampled per register with the deterministic sampler
 * (see qs_measure) from host_u[g][r][0..nshots-1] in [0, 1), and each term
 * counts (-1)^(ones of the sample on its qubits); host_out[r] = sum over
 * groups and terms of coeff * count / nshots, plus the identity terms'
 * coefficients.  Synchronises the stream. */
int qs_observable_groups(const qs_observable* o, int* ngroups);
int qs_shot_expect(qs_state* s, const qs_observable* o, const double* host_u, int nshots, void* dev_work,
                   double* host_out);

/* Eq. shiftrule for every parameter: d<O>/dtheta_k = (<O>(theta_k + pi/2) -
 * <O>(theta_k - pi/2)) / 2 from |0...0>.  Every parameter must be used by
 * exactly one uncontrolled Pauli rotation (RX, RY, RZ, ROT; QS_EUNSUPPORTED
 * otherwise).  The 2 P shifted circuits run as one batch in dev_states (2 P
 * registers of the circuit's size in dtype, register 2k: +pi/2, 2k+1: -pi/2;
 * complex64 circuits that fit the batched engine run in one persistent
 * launch).  nshots = 0: exact <O>; else shot-based as qs_shot_expect with
 * host_u[g][2P][nshots] and dev_work of dev_states' size.  stream: a
 * cudaStream_t.  host_grad: P doubles.  Synchronises the stream. */
int qs_faithful_gradient(const qs_circuit* c, const double* host_params, const qs_observable* o, int dtype,
                         int nshots, const double* host_u, void* dev_states, void* dev_work, void* stream,
                         double* host_grad);

/* MMD loss of the Born machine p = |circuit |0...0>|^2 against the target
 * distribution host_target (2^n doubles), Sec. "Forward Mode" (Listing mmd):
 * L = E_{x,x'~p} K - 2 E_{x~p,y~q} K + E_{y,y'~q} K with the Gaussian kernel
 * K(x, y) = exp(-(x - y)^2 / (2 sigma^2)) on basis indices, and
 * dL/dtheta_k = (p_+ - p_-)^T K (p - q) from the circuits at theta_k +- pi/2
 * (same parameter conditions as qs_faithful_gradient).  dev_states holds
 * 2P + 1 registers (2k: +pi/2, 2k+1: -pi/2, 2P: unshifted).  nshots = 0:
 * exact distributions; else the empirical distributions of nshots samples per
 * register drawn with host_u[2P + 1][nshots] (plug-in estimates).  n <= 16.
 * host_grad: P doubles; host_loss: L (may be NULL).  Synchronises the stream. */
int qs_mmd_gradient(const qs_circuit* c, const double* host_params, const double* host_target, double sigma,
                    int dtype, int nshots, const double* host_u, void* dev_states, void* stream,
                    double* host_grad, double* host_loss);

/* ---------------------------------------------------------------- sparse matrices */

/* CSR matrix of a Pauli sum on nqubits qubits (Sec. "Matrix Representation",
 * App. "Matrix Types"; mat(heisenberg(20)) in Sec. "Matrix Representation and
 * AD Performance"), in two device passes.  qs_observable_csr_rows writes the
 * row pointers (dev_rowptr: 2^n + 1 int64) using dev_scratch (2^n / 1024 + 2
 * int64) and returns the nonzero count in *host_nnz (synchronises);
 * qs_observable_csr_fill then writes the column indices (dev_cols: nnz int64,
 * ascending within a row) and values (dev_vals: nnz interleaved complex
 * doubles).  Entry (i, j) = sum of the terms with x_mask = i ^ j of
 * coeff * i^{popcount(x&z)} * (-1)^{popcount(j&z)} (the action qs_expect
 * uses); entries that sum to exactly zero are not stored.  At most 64
 * distinct x masks and 256 terms (QS_EUNSUPPORTED otherwise); nqubits <= 34.
 * stream: a cudaStream_t. */
int qs_observable_csr_rows(const qs_observable* o, int nqubits, int64_t* dev_rowptr, int64_t* dev_scratch,
                           int64_t* host_nnz, void* stream);
int qs_observable_csr_fill(const qs_observable* o, int nqubits, const int64_t* dev_rowptr, int64_t* dev_cols,
                           double* dev_vals, void* stream);

/* Failure-path self-test (no counterpart in the paper): one device thread waits
 * on an mbarrier phase that nothing completes, through the bounded wait the
 * tensor-core kernels use, with a limit of limit_ms (0 < limit_ms <= 1000).
 * host_result[0] = 1 if the wait (wrongly) succeeded, [1] = the abort flag it
 * raised, [2] = microseconds waited.  Returns QS_ETIMEDOUT when the wait gave
 * up and the device status word reported it (the expected outcome), and clears
 * the word.  Synchronises the device. */
int qs_selftest_bounded_wait(double limit_ms, int* host_result);

/* ---------------------------------------------------------------- gates */

/* instruct!(reg, U, locs, ctrl_locs, ctrl_vals) on every register of s
 * (Sec. "Instructions on Quantum Registers"; the general multi-control,
 * multi-qubit, arbitrary-location instruction of Sec. "Performance").
 * host_mat: 2^k x 2^k row-major interleaved complex doubles (not checked for
 * unitarity).  locs and ctrl_locs must be distinct and < every register's n.
 * The library picks a diagonal, permutation or dense kernel from the matrix's
 * non-zero pattern (App. "Matrix Types"); dense k = 4, 5 on complex64 states
 * may run on the tensor cores (QS_OPT_TENSOR_CORES; targets < 32). */
int qs_apply_gate(qs_state* s, const double* host_mat, int k, const int32_t* host_locs,
                  int nctrl, const int32_t* host_ctrl_locs, const int32_t* host_ctrl_vals);

/* The same for a named gate (enum qs_gate_kind other than MATRIX) at angle
 * theta; host_paulis is read only for QS_GATE_ROT. */
int qs_apply_named(qs_state* s, int kind, int k, const int32_t* host_locs,
                   const int32_t* host_paulis, int nctrl, const int32_t* host_ctrl_locs,
                   const int32_t* host_ctrl_vals, double theta);

/* ---------------------------------------------------------------- circuits */

/* Immutable gate list of nqubits qubits with nparams parameters.
 * host_mats: pool of interleaved complex doubles for MATRIX gates (may be
 * NULL if none), nmat complex entries.  Everything is copied. */
int qs_circuit_create(int nqubits, const qs_gate_desc* host_gates, int ngates,
                      const double* host_mats, int64_t nmat, int nparams, qs_circuit** out);
int qs_circuit_destroy(qs_circuit* c);
int qs_circuit_info(const qs_circuit* c, int* nqubits, int* ngates, int* nparams);

/* Host-side view of gate `index` of c (no device work; callable without a
 * GPU): host_desc (may be NULL) receives its descriptor; host_U (may be NULL)
 * its 2^k x 2^k matrix at host_params (App. "Builtin Block Types"; row-major,
 * interleaved re/im, index bit j <-> locs[j], controls not included);
 * host_G / host_cfac (may be NULL) the generator H on the targets and the
 * factor c with U = exp(-i theta c H) (Sec. "Reverse Mode"; rotations: Pauli
 * string, c = 1/2; shift: P1, c = -1; phase: identity, c = -1).  Asking for
 * H or c of a gate without a parameter is QS_EINVAL. */
int qs_circuit_gate_matrices(const qs_circuit* c, int index, const double* host_params,
                             qs_gate_desc* host_desc, double* host_U, double* host_G,
                             double* host_cfac);

/* Passes and phases of the circuit's tile-engine schedule for tiles of
 * tile_qubits qubits (0 = 13); builds and caches the schedule (device
 * tables) if needed.  QS_EUNSUPPORTED if the circuit does not fit the engine. */
int qs_circuit_schedule_info(const qs_circuit* c, int tile_qubits, int* npasses, int* nphases);

/* The order in which the tile engine applies the circuit's gates for tiles of
 * tile_qubits qubits (0 = 13), host only (no device work).  The engine first
 * rewrites each SWAP(a, b) as X(b) controlled by a, X(a) controlled by b, X(b)
 * controlled by a (each also carrying the SWAP's controls); host_order[i] is
 * the index, in that expanded list, of the i-th gate applied and host_pass[i]
 * its pass.  Inside a pass the engine may still fuse runs of gates on one
 * qubit and apply commuting diagonal gates together; the order here is the
 * scheduler's (Sec. "Representing Quantum Circuits": reordering is valid only
 * between gates on disjoint qubits).  *ngates receives the expanded gate count;
 * call with NULL arrays to size them.  QS_EUNSUPPORTED if the circuit does not
 * fit the engine (fewer than 5 or more than 32 qubits, multi-target gates
 * other than SWAP). */
int qs_circuit_tile_order(const qs_circuit* c, int tile_qubits, int* ngates, int32_t* host_order,
                          int32_t* host_pass);

/* apply!(reg, chain): gates in list order on every register of s (Sec.
 * "Representing Quantum Circuits").  host_params: nparams doubles shared by
 * all registers, or nbatch * nparams (register-major) with
 * QS_APPLY_PER_REGISTER.  By default consecutive single-qubit gates on one
 * qubit (no gate on that qubit in between) are multiplied on the host and
 * applied as one pass; QS_APPLY_UNFUSED launches one kernel per gate.
 * complex64 registers of the circuit's size with at least 256 tiles of 2^13
 * amplitudes (n >= 21, or batches) run the tile engine instead: the gate
 * list is scheduled into passes over 13-qubit tiles (gates move earlier only
 * past gates on other qubits), one HBM round trip of the state per pass, with
 * every gate of a pass applied in shared memory / registers.  It takes
 * single-target gates (their controls, tested per amplitude, may sit on any
 * qubit) plus SWAPs (as three CNOTs) on registers of 5..32 qubits; other
 * circuits use the per-gate path.  QS_APPLY_TILES forces the tile engine
 * (QS_EUNSUPPORTED if the circuit does not fit) and QS_APPLY_TILE_QUBITS(m)
 * sets the tile size (9..13; registers smaller than the tile form one tile).  A circuit keeps its
 * schedule and a parameter buffer between calls, so applies of one circuit
 * (and qs_backward_tiled, which shares them) must not overlap on different
 * streams: the caller serialises them.  The schedule's tables are memory of the
 * device that was current when it was built; an apply with another device
 * current rebuilds them there (a circuit used on two devices in turn pays
 * that rebuild at each switch).
 * QS_APPLY_BLOCKS fuses the gates into blocks of at most k qubits
 * (QS_APPLY_BLOCK_QUBITS(k), 1..5, default 5; targets and controls both
 * count) and applies each block as one k-qubit instruction with the product
 * matrix of its gates; dense 4- and 5-qubit blocks of complex64 states may run
 * on the tensor cores (QS_OPT_TENSOR_CORES).  Gates wider than k stay single.
 * QS_APPLY_PRECISE (complex64; the per-gate path, or with QS_APPLY_BLOCKS the
 * block path; QS_EINVAL with QS_APPLY_TILES): every gate or block in a
 * dense, diagonal or phased-permutation form of up to 5 qubits (fused 1-qubit
 * runs included, controls allowed) is applied with its FP64 matrix held as
 * FP32 hi + lo and each output amplitude summed in double-float and rounded to
 * FP32 once, on the CUDA cores, so the only error left is the storage rounding
 * of the amplitudes (the plain path also rounds the matrix, an error coherent
 * over the whole state; the tensor-core blocks are not used). */
#define QS_APPLY_PER_REGISTER 1
#define QS_APPLY_UNFUSED 2
#define QS_APPLY_TILES 4
#define QS_APPLY_BLOCKS 8
#define QS_APPLY_PRECISE 32
#define QS_APPLY_TILE_QUBITS(m) ((m) << 8)
#define QS_APPLY_BLOCK_QUBITS(k) ((k) << 16)
int qs_apply_circuit(qs_state* s, const qs_circuit* c, const double* host_params, int flags);

/* A whole circuit on one small register (n <= 24) in ONE kernel launch, for
 * registers whose gate-by-gate launches cost more than their arithmetic: the
 * circuit's blocks of at most kmax qubits (qs_circuit_blocks: dense matrices,
 * controls inside the block) run back to back in a cooperative launch of
 * grid_ctas CTAs (0 = one per SM), each block reading the state from one
 * buffer and writing the other (every output amplitude of a tuple is a work
 * item), with a grid barrier between blocks; complex128 in FP64, complex64 in
 * FP32.  If o is not NULL (diagonal observables only: Z strings, at most 64
 * terms) <O> is evaluated in the same launch (pairwise FP64 sums) into
 * dev_out[0] (device).  Every grid-barrier wait is bounded; a wait that gives
 * up leaves the state unspecified and makes the next qs_state_sync return
 * QS_ETIMEDOUT.  Asynchronous on s's stream; uses s's scratch (a second state
 * buffer and the block tables). */
int qs_run_circuit_one_launch(qs_state* s, const qs_circuit* c, const double* host_params, int kmax,
                              const qs_observable* o, int grid_ctas, double* dev_out);

/* The k-qubit blocks QS_APPLY_BLOCKS applies (host only, no device work).
 * *nblocks receives their count.  If not NULL: host_widths[b] = block b's
 * qubit count; host_locs[b * QS_MAXK + j] = its qubits, ascending, padded
 * with -1; host_mats[b * 2 * 4^QS_MAXK ...] = its 2^w x 2^w matrix (row-major
 * interleaved complex doubles, bit j of an index <-> host_locs[b][j], zero
 * padded) for the parameters host_params.  Call once with NULL arrays for the
 * count.  Blocks are listed in application order. */
int qs_circuit_blocks(const qs_circuit* c, const double* host_params, int kmax, int* nblocks,
                      int32_t* host_widths, int32_t* host_locs, double* host_mats);

/* Autotuner for one circuit on one state shape: applies the circuit with each
 * candidate flag set (per-gate without fusion, the default, blocks of 2..5
 * qubits, and for complex64 registers of the circuit's size the tile engine
 * with 10..13-qubit tiles), 1 warm-up + reps timed applies each (wall clock
 * around a synchronised stream), and returns the fastest in *best_flags.
 * If ncand is not NULL it holds the capacity of host_cand_flags / host_cand_ms
 * on entry and the number of candidates on return (ms = -1: not applicable).
 * The state's amplitudes are used as scratch: they are overwritten. */
int qs_autotune_circuit(qs_state* s, const qs_circuit* c, const double* host_params, int reps,
                        int* best_flags, int* ncand, int32_t* host_cand_flags, double* host_cand_ms);

/* As qs_apply_circuit on a single register (per gate, complex64 1-qubit gates
 * compensated as with QS_APPLY_PRECISE), also saving forward checkpoints:
 * after gate index g (0-based) with (g + 1) % ckpt_every == 0 and g + 1 <
 * ngates, the state is copied to slot (g + 1) / ckpt_every - 1 of dev_ckpts,
 * which must hold qs_checkpoint_count() states of the state's dtype. */
int qs_checkpoint_count(const qs_circuit* c, int ckpt_every, int* count);
int qs_apply_circuit_ckpt(qs_state* s, const qs_circuit* c, const double* host_params,
                          int ckpt_every, void* dev_ckpts);

/* ---------------------------------------------------------------- observables */

/* O = sum_t coeff_t P_t (Sec. "Forward Mode", expect; Listing "Heisenberg
 * Hamiltonian" for sums of Pauli strings).  Strings must be Hermitian as
 * given (any X/Y/Z pattern is). */
int qs_observable_create(const qs_pauli_term* host_terms, int nterms, qs_observable** out);
int qs_observable_destroy(qs_observable* o);

/* <psi_r|O|psi_r> for every register r into host_out[nreg] (FP64 reduction). */
int qs_expect(qs_state* s, const qs_observable* o, double* host_out);

/* The same expectation values for callers that cannot allocate device memory:
 * host frameworks that own all device memory through their own allocator,
 * latency-critical loops that must not call cudaMalloc or cudaFree (which can
 * synchronise the device), and processes under a fixed device-memory budget.
 * The paper has no counterpart; this is a property of this library only.
 * Allocates nothing and needs no handle: dev_amps holds nreg registers of
 * nqubits qubits back to back (dtype QS_C64 or QS_C128), host_terms the
 * observable, dev_out nreg doubles the caller allocated; asynchronous on
 * stream (a cudaStream_t, NULL = legacy default stream).  Its reduction
 * scratch is one fixed 512 KiB array of 65536 FP64 partial sums that every GPU
 * loading the library keeps until the process exits; a request needing more
 * than that (nreg * nterms > 65536) or more than 64 terms, or nreg > 65535,
 * is rejected with QS_EINVAL.  All calls share the array and every call
 * overwrites the part it reads, so nothing carries over from an earlier
 * call -- but calls whose kernels overlap on the GPU (different streams, or
 * different host threads) race on it and must be serialised by the caller.
 * The first call on each device resolves the array's device address
 * (cudaGetSymbolAddress, which may load the library's GPU module); make
 * that first call before any stream capture.  The address is kept for the
 * life of the process: it assumes the device's primary context lives that
 * long, so do not call this entry point after a cudaDeviceReset on that
 * device (a launch failure inside this call clears the cached address, and
 * the next call resolves it again). */
int qs_expect_static(const void* dev_amps, int dtype, int nqubits, int nreg,
                     const qs_pauli_term* host_terms, int nterms, double* dev_out, void* stream);

/* ---------------------------------------------------------------- gradient */

/* Device bytes of the work buffer qs_backward needs for an n-qubit register
 * (two complex128 states: psi and its adjoint lambda). */
int qs_backward_work_bytes(int nqubits, size_t* out_bytes);

/* expect'(O, reg => circuit) (Sec. "Reverse Mode"): s holds the circuit's
 * OUTPUT state psi_N of a single register (left unchanged).  With lambda =
 * O psi_N, gates are walked backwards; a gate U = exp(-i theta c H) adds
 * 2 c Im<lambda|H|psi> to host_grad[param] (rotations c = 1/2, H = Pauli;
 * shift c = -1, H = P1; phase c = -1, H = 1; H includes the control
 * projector), then psi <- U^dag psi and lambda <- U^dag lambda (Eq.
 * apply-back), in FP64 in dev_work.  If ckpt_every > 0, dev_ckpts holds the
 * checkpoints written by qs_apply_circuit_ckpt and psi restarts from them
 * (bounding uncompute drift).  host_grad receives nparams doubles (shared
 * parameters add up); host_loss, if not NULL, receives <psi_N|O|psi_N>. */
int qs_backward(qs_state* s, const qs_circuit* c, const double* host_params,
                const qs_observable* o, int ckpt_every, const void* dev_ckpts, void* dev_work,
                double* host_grad, double* host_loss);

/* Reversible backward over k-qubit blocks (QS_APPLY_BLOCKS with width kmax),
 * Sec. "Reverse Mode" with a fused block as the unit: walking the blocks from
 * last to first, one pass forms rho = sum_x psi_x lambda_x^dag over the
 * block's tuples (FP32 products per 128 tuples for complex64, FP64 sums), the
 * gradients of the block's gates follow on the host in FP64 as
 * 2 c Im Tr(E H E^dag rho) (E: the block's later gates, H: the generator with
 * its control projector), then psi and lambda are uncomputed by the block's
 * adjoint.  s holds the final state of a single register (complex64 or
 * complex128) and holds the uncomputed initial state on return.  dev_work:
 * qs_backward_blocks_work_bytes() bytes (lambda).  host_grad: nparams doubles
 * (written), host_loss: <O> (may be NULL).  Every block must span at most
 * QS_MAXK qubits (QS_EUNSUPPORTED otherwise).  Synchronises the stream. */
int qs_backward_blocks_work_bytes(int nqubits, int dtype, size_t* out_bytes);
int qs_backward_blocks(qs_state* s, const qs_circuit* c, const double* host_params,
                       const qs_observable* o, int kmax, void* dev_work, double* host_grad,
                       double* host_loss);

/* ---------------------------------------------------------------- batched registers */

/* A batch of registers of uneven sizes, each with its own circuit, parameter
 * vector and observable, run forward (and optionally through the reversible
 * backward pass) in ONE persistent launch (Sec. "Batched Quantum Registers";
 * Sec. "Reverse Mode").  complex64 states, FP32 gate arithmetic and
 * uncompute, FP64 accumulation of losses and gradients above the warp level.
 * Restrictions: every gate has one target (controls allowed; X, Y, Z, H, S,
 * SDG, T, TDG, RX, RY, RZ, SHIFT, PHASE, 1-qubit MATRIX), each register has
 * 5..30 qubits and at most 2048 parameters, observables are diagonal (sums
 * of Z strings).  circuits[r]->nqubits is register r's size.  Each circuit is
 * scheduled into fused passes over tiles of tile_qubits qubits (0 = 13) and
 * 4-qubit register phases; the program holds device tables and the backward
 * work buffers (two complex64 copies of every register larger than a tile). */
typedef struct qs_batch_program qs_batch_program;

#define QS_BATCH_RESET 1  /* start every register from |0...0> (else from the state's content) */
#define QS_BATCH_GRAD 2   /* also run the backward pass and write gradients */

int qs_batch_program_create(int nreg, const qs_circuit* const* circuits,
                            const qs_observable* const* observables, int tile_qubits,
                            qs_batch_program** out);

/* The same with the fusion width and the precision chosen by the caller.
 * phase_qubits (2..4, 0 = the widest the path takes: 4, or 3 with
 * QS_BATCH_PRECISE): register qubits per phase, i.e. every gate on
 * those qubits inside a phase is applied to 2^phase_qubits amplitudes held in
 * one thread's registers (the batched engine's k-qubit fusion); the tile then
 * holds at most 9 + phase_qubits qubits (512 threads x 2^phase_qubits
 * amplitudes), tile_qubits 0 = that maximum.
 * flags QS_BATCH_PRECISE (phase_qubits 2 or 3): the forward pass stays in
 * complex64 with FP32 arithmetic, but every gate matrix is applied with its
 * FP32 rounding error compensated (U = U_hi + U_lo, both FP32, U_lo = the
 * FP64 matrix minus U_hi) and each output amplitude is summed in
 * double-float and rounded to FP32 once (this removes the coherent error of
 * rounding the same matrix for every amplitude); the
 * reversible uncompute of psi and lambda (Sec. "Reverse Mode", Eq. apply-back)
 * runs in double-float arithmetic (each real a pair hi + lo of FP32 values,
 * about 48 significant bits: FP64-class accuracy on the FP32 units; psi and
 * lambda of registers larger than the tile stream through double-float work
 * buffers, 16 bytes per amplitude each); gradient contributions are FP32
 * products of the hi parts summed in FP32 over a thread's pairs and a warp,
 * then in FP64.  The program's shape is read back with qs_batch_program_shape. */
#define QS_BATCH_PRECISE 1
int qs_batch_program_create_ex(int nreg, const qs_circuit* const* circuits,
                               const qs_observable* const* observables, int tile_qubits,
                               int phase_qubits, int flags, qs_batch_program** out);
int qs_batch_program_shape(const qs_batch_program* p, int* tile_qubits, int* phase_qubits, int* flags);
int qs_batch_program_destroy(qs_batch_program* p);

/* Register count, total parameters, parameter offsets (nreg + 1, host) and
 * amplitude offsets (nreg + 1, host) of the program (NULL outputs skipped). */
int qs_batch_program_info(const qs_batch_program* p, int* nreg, int64_t* nparams_total,
                          int64_t* host_param_offsets, int64_t* host_amp_offsets);

/* One persistent launch on s's stream (s: a qs_batch_create state of the
 * same register sizes, QS_C64).  The device current at
 * qs_batch_program_create holds the program's tables and must be current here
 * (QS_EINVAL otherwise); runs of one program must not overlap on the GPU (they
 * share its work buffers and work counter).  dev_params: the registers' parameter
 * vectors back to back (device, FP64); dev_loss[nreg] receives <O_r>;
 * with QS_BATCH_GRAD, dev_grad (same layout as dev_params) receives the
 * gradients.  The final states psi_N are left in s. */
int qs_batch_run(qs_state* s, const qs_batch_program* p, const double* dev_params, double* dev_loss,
                 double* dev_grad, int flags);

/* Autotuner of the batched engine's tile shape: builds the program for every
 * tile size from 13 down to 11 qubits (tile_qubits of qs_batch_program_create;
 * registers larger than the tile stream tiles of that size, smaller ones stay
 * resident), runs it on s with dev_params once as warm-up and reps times
 * timed with CUDA events (forward + gradient when dev_grad is not NULL), and
 * returns the fastest in *best_tile (pass it to qs_batch_program_create).
 * If ncand is not NULL it holds the capacity of host_tiles / host_ms on entry
 * and the candidate count on return (ms = -1: the size does not fit).  s's
 * amplitudes and dev_loss / dev_grad are overwritten.  Synchronises. */
int qs_batch_autotune(int nreg, const qs_circuit* const* circuits, const qs_observable* const* observables,
                      qs_state* s, const double* dev_params, double* dev_loss, double* dev_grad, int reps,
                      int* best_tile, int* ncand, int32_t* host_tiles, double* host_ms);

/* Autotuner of the fusion width and the tile shape together: for every phase
 * width from 4 (3 with QS_BATCH_PRECISE) down to 2 and the three largest tile
 * sizes that width allows, builds the program with flags, runs it as
 * qs_batch_autotune does, and returns the fastest in *best_tile and
 * *best_phase (pass them to qs_batch_program_create_ex).  host_tiles /
 * host_phases / host_ms list the candidates as in qs_batch_autotune. */
int qs_batch_autotune_ex(int nreg, const qs_circuit* const* circuits, const qs_observable* const* observables,
                         int flags, qs_state* s, const double* dev_params, double* dev_loss, double* dev_grad,
                         int reps, int* best_tile, int* best_phase, int* ncand, int32_t* host_tiles,
                         int32_t* host_phases, double* host_ms);

/* Device bytes of the work buffer of qs_backward_tiled (two complex64
 * copies: psi and lambda). */
int qs_backward_tiled_work_bytes(int nqubits, size_t* out_bytes);

/* expect'(O, reg => circuit) for large complex64 registers (Sec. "Reverse
 * Mode", Eq. apply-back): the same walk as qs_backward on the tile engine's
 * schedule (passes in reverse, gates in reverse inside each phase), with the
 * uncompute of psi and lambda in FP32 in dev_work and every gradient
 * contribution accumulated in FP64 from the warp level up (per-CTA partials
 * folded in CTA order, so the result is reproducible).  s holds psi_N (left
 * unchanged); tile_qubits 0 = 13.  Gates and parameter kinds as for the tile
 * engine of qs_apply_circuit (QS_EUNSUPPORTED otherwise); at most 64
 * observable terms and about 11000 parameters. */
int qs_backward_tiled(qs_state* s, const qs_circuit* c, const double* host_params,
                      const qs_observable* o, int tile_qubits, void* dev_work, double* host_grad,
                      double* host_loss);

/* ---------------------------------------------------------------- measurement */

/* measure / measure! on all qubits (Sec. "Instructions on Quantum
 * Registers"), nshots samples per register from |psi|^2 using the caller's
 * uniform numbers host_u[nreg][nshots] in [0, 1) into host_out[nreg][nshots].
 * Deterministic contract: p_i = re*re + im*im (separately rounded FP64
 * multiply and add; complex64 amplitudes are promoted exactly); level-0
 * blocks of 1024 consecutive p_i and level-1 blocks of 1024 level-0 sums are
 * left folds; total T is the left fold of the level-1 sums; for t = u * T
 * each level walks its values from the carried prefix, takes the first
 * value whose running sum exceeds t (else the last positive value, else the
 * last) and carries its exclusive prefix down.  collapse != 0 (requires
 * nshots == 1) projects each register onto its sample and renormalises.
 * QS_EINVAL for nshots < 1, a uniform outside [0, 1) or collapse with
 * nshots != 1.  Synchronises the stream (host_out is written on return). */
int qs_measure(qs_state* s, const double* host_u, int nshots, int64_t* host_out, int collapse);

/* qs_measure with its uniforms generated on the device from a seed, so that a
 * seed alone fixes the sampled indices (bit for bit, whatever the caller's
 * random source).  The paper fixes no random source; this library's is
 * SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): draw k (k >= 1) is the
 * 64-bit finaliser (x ^= x >> 30, x *= 0xBF58476D1CE4E5B9, x ^= x >> 27,
 * x *= 0x94D049BB133111EB, x ^= x >> 31) of x = seed + k * 0x9E3779B97F4A7C15
 * (mod 2^64), and u = (x >> 11) * 2^-53.  Register r's shot j takes draw
 * k = r * nshots + j + 1; the walk from u is qs_measure's.  Same arguments,
 * errors and synchronisation as qs_measure. */
int qs_measure_seeded(qs_state* s, uint64_t seed, int nshots, int64_t* host_out, int collapse);

#ifdef __cplusplus
}
#endif

#endif /* QSIM_H */
