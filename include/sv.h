/*
 * libsv -- C-ABI of the GB300 statevector engine.
 *
 * The library applies a circuit's gate list to a 2^n complex statevector held
 * in the GPU's HBM: the full-circuit execution path the paper compares
 * (Sec. III-B, Listing 3: circuit in, full probability vector out), which also
 * simulates every cut-subcircuit instance of the CutQC Evaluator (Sec. IV-A,
 * "Evaluator"; Fig. 1).  Every step of the path runs in the library's own
 * sm_103a kernels; there is no CPU fallback.
 *
 * Conventions (all entry points)
 *   - Amplitude i of an n-qubit state is stored at element i; index bit q is
 *     qubit q (little-endian, as the Statevector.probabilities call of
 *     Listings 2 and 3).  Amplitudes are interleaved (re, im):
 *     SV_C64 = 2 x float32 (8 bytes), SV_C128 = 2 x float64 (16 bytes), so a
 *     state takes 2^n * 8 or 2^n * 16 bytes (Table III lists the latter).
 *   - Every call returns SV_OK (0) or a negative sv_status; no C++ exception
 *     crosses this boundary.  sv_status_str() maps a code to a static string.
 *   - Pointers named *_host are host memory; pointers with an *_is_device flag
 *     may be either.  The caller owns every buffer it passes and must keep it
 *     valid for the duration of the call only: calls are synchronous unless
 *     stated otherwise.
 *   - A handle must not be used from two host threads at once.
 */
#ifndef LIBSV_SV_H
#define LIBSV_SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SV_OK = 0,
    SV_ERR_ARG = -1,      /* null pointer, bad enum value, non-finite angle  */
    SV_ERR_QUBIT = -2,    /* qubit index out of range or repeated operands   */
    SV_ERR_OOM = -3,      /* device allocation failed / does not fit in HBM  */
    SV_ERR_SIZE = -4,     /* output length or byte count does not match 2^n  */
    SV_ERR_CUDA = -5,     /* a CUDA runtime call failed                      */
    SV_ERR_TIMEOUT = -6,  /* a bounded device-side wait ran out              */
    SV_ERR_STATE = -7     /* handle used after a failure left it undefined   */
} sv_status;

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_dtype;

/* Gate set of the engine.  Matrices follow Qiskit's conventions (the paper
 * runs Qiskit 1.0.2 and Aer 0.14, Sec. V-A), global phases included:
 *   H = [[1,1],[1,-1]]/sqrt2   X   Y = [[0,-i],[i,0]]   Z = diag(1,-1)
 *   S = diag(1,i)   T = diag(1,e^{i pi/4})
 *   RX(t) = [[c,-is],[-is,c]]   RY(t) = [[c,-s],[s,c]]   RZ(t) = diag(e^{-it/2}, e^{it/2})
 *   U3(t,p,l) = [[c, -e^{il} s], [e^{ip} s, e^{i(p+l)} c]]     (c = cos t/2, s = sin t/2)
 * Two-qubit gates act on the local index b(q0) + 2 b(q1):
 *   CX (q0 = control, q1 = target)   CZ = diag(1,1,1,-1)
 *   RZZ(t) = diag(e^{-it/2}, e^{it/2}, e^{it/2}, e^{-it/2})   SWAP              */
typedef enum {
    SV_H = 0, SV_X, SV_Y, SV_Z, SV_S, SV_T, SV_RX, SV_RY, SV_RZ, SV_U3,
    SV_CX, SV_CZ, SV_RZZ, SV_SWAP, SV_NUM_OPS
} sv_op;

/* One gate: q1 = -1 for one-qubit gates; theta/phi/lambda unused by fixed
 * gates.  40 bytes: int32 x 3, 4 bytes padding, float64 x 3. */
typedef struct {
    int32_t op, q0, q1;
    double theta, phi, lambda;
} sv_gate;

/* Arithmetic used for complex128 states.
 *   SV_ARITH_NATIVE: IEEE float64 multiply-adds on the FP64 units.
 *   SV_ARITH_DF64:   float64 storage, gate arithmetic in double-float pairs on
 *                    the FP32 units (error-free TwoProd / TwoSum transforms,
 *                    Dekker 1971; Joldes, Muller, Popescu 2017), about 47
 *                    significant bits per operation.
 *   SV_ARITH_TC:     float64 storage; inside a call the state is held in Q56
 *                    fixed point (x * 2^56 in an int64 per component, also in
 *                    HBM between the call's passes) and fused-block products
 *                    run on the tensor cores (tcgen05.mma, accumulators in
 *                    tensor memory) with an exact split of both operands into
 *                    seven balanced 8-bit digits held as float16: exact digit
 *                    products, exact float32 sums per digit level, levels 0..6
 *                    re-assembled in 64-bit integers (error below 2^-50 per
 *                    component and block product, an absolute bound: about
 *                    2^-35 relative to a 30-qubit amplitude of typical size
 *                    2^-15).  Precondition: every component of every state the
 *                    call passes through lies in [-1, 1], which a state of norm
 *                    at most 1 guarantees (the blocks are unitary).  States
 *                    evolved from a basis state satisfy it; for caller-supplied
 *                    amplitudes (sv_set_amplitudes, sv_create_on) the first
 *                    call measures the norm exactly and uses SV_ARITH_DF64 if it
 *                    exceeds 1 + 2^-40.  A block whose digit sums could leave
 *                    the exact float32 range (none of the unitary blocks seen)
 *                    also falls back to SV_ARITH_DF64.
 *   SV_ARITH_TC_SYNC: the same digit products on the warp-level mma.sync
 *                    path (unsigned lower digits), kept as the measured
 *                    baseline of the tensor-memory kernel.
 *   SV_ARITH_AUTO:   SV_ARITH_TC for states of 20 or more qubits, else
 *                    SV_ARITH_DF64 (measured crossover; on GB300 the FP64
 *                    pipe runs at about 1/70 of the FP32 pipe, so native
 *                    FP64 is never the automatic choice).  SV_ARITH_TC and
 *                    SV_ARITH_TC_SYNC fall back to SV_ARITH_DF64 below 8
 *                    qubits.
 * complex64 states: SV_ARITH_NATIVE (and SV_ARITH_DF64 / SV_ARITH_TC_SYNC)
 * compute in float32 FMAs; SV_ARITH_TC splits every float32 component into
 * three bfloat16 parts and forms the six part products of float32 accuracy
 * on the tensor cores (tcgen05.mma, float32 accumulation in tensor memory);
 * SV_ARITH_AUTO takes SV_ARITH_TC from 23 qubits on.  No magnitude limit. */
typedef enum {
    SV_ARITH_AUTO = 0,
    SV_ARITH_NATIVE = 1,
    SV_ARITH_DF64 = 2,
    SV_ARITH_TC = 3,
    SV_ARITH_TC_SYNC = 4
} sv_arith;

/* Run options; a null pointer or 0 fields mean "auto".
 *   max_fuse_k:   largest fused block, 1..5 qubits; 1 = no fusion (each gate
 *                 is applied on its own).
 *   tile_qubits:  qubits per shared-memory tile (cache blocking, the
 *                 single-GPU counterpart of the chunk size nc, Sec. III-B).
 *   arith:        sv_arith for complex128 states.
 *   debug_checks: bit 0 (1): check the plan's invariants before launching
 *                 (SV_ERR_STATE if one fails).  bit 1 (2): failure-detection
 *                 test hook for SV_ARITH_TC: the call's first dense block
 *                 issues no MMAs, so the kernel's bounded wait (one second)
 *                 runs out; the call returns SV_ERR_TIMEOUT and leaves the
 *                 state undefined until sv_reset / sv_set_amplitudes.
 *   timing:       nonzero = record CUDA events around every kernel launch on
 *                 the handle's stream and report the durations in
 *                 sv_apply_stats (kernel_ms, max_kernel_ms).               */
typedef struct {
    int32_t max_fuse_k;
    int32_t tile_qubits;
    int32_t arith;
    int32_t debug_checks;
    int32_t timing;
} sv_run_opts;

typedef struct sv_state sv_state;

/* Bytes of a state: 2^n * 8 (SV_C64) or 2^n * 16 (SV_C128); 0 if n is not in
 * 1..34 or dt is not a sv_dtype.  Host-only; the memory column of Table III
 * (complex128: 2^n x 16 bytes, 30 qubits = 17.18 GB). */
size_t sv_state_bytes(int n_qubits, int dt);

/* Creates an n-qubit state (1 <= n <= 34) in a device buffer the library
 * allocates and owns, initialised to |0...0>, on the current CUDA device and
 * a stream the library creates.  SV_ERR_OOM if it does not fit.  The
 * statevector a simulation starts from (Sec. III-B: 2^n complex amplitudes,
 * memory doubling per qubit; Listing 3 runs the circuit on one such state,
 * the device chosen at run time); 34 qubits is the largest width the paper
 * simulates (Sec. V-B, Table III). */
int sv_create(int n_qubits, int dt, sv_state** out);

/* Wraps a caller-owned device buffer (for example a torch tensor) of
 * exactly sv_state_bytes(n, dt) bytes, 16-byte aligned, as a state.  The
 * buffer's contents are taken as the state (no initialisation).  Work is
 * issued on cuda_stream (a cudaStream_t; NULL = the legacy default stream).
 * The caller keeps the buffer alive until sv_destroy. */
int sv_create_on(void* dev_ptr, size_t bytes, int n_qubits, int dt,
                 void* cuda_stream, sv_state** out);

/* Frees the handle and, unless created by sv_create_on, its buffer.  The
 * paper has no counterpart (Aer frees its state when the run ends,
 * Listing 3); the caller decides here how long a state stays resident. */
void sv_destroy(sv_state* s);

/* Points a handle made by sv_create_on at another caller-owned buffer (same
 * rules as sv_create_on; the stream is kept), reusing its workspaces. */
int sv_rebind(sv_state* s, void* dev_ptr, size_t bytes, int n_qubits, int dt);

int sv_num_qubits(const sv_state* s);
int sv_dtype_of(const sv_state* s);
/* Device pointer of the amplitudes (for zero-copy interop). */
void* sv_device_ptr(const sv_state* s);

/* Sets the state to the basis state |basis_index> (< 2^n): the initial
 * state of a run (|0...0>, Listing 3) or a cut-subcircuit variant's
 * computational-basis input (the Evaluator's initialisations, Sec. III-A,
 * Eqs. 3.5-3.6).  SV_ERR_ARG if basis_index >= 2^n. */
int sv_reset(sv_state* s, uint64_t basis_index);

/* Applies gates[0..n_gates) in list order (validated first: SV_ERR_ARG for an
 * unknown opcode or a non-finite angle, SV_ERR_QUBIT for a qubit outside
 * 0..n-1 or a two-qubit gate with q0 == q1; nothing is applied then).
 * The gates are fused into blocks of up to max_fuse_k qubits and grouped into
 * tile passes (one HBM read and write of the state per pass).  Returns after
 * the kernels have finished. */
int sv_apply_circuit(sv_state* s, const sv_gate* gates, size_t n_gates,
                     const sv_run_opts* opts);

/* p_i = |a_i|^2 for all 2^n amplitudes, computed and written as float64
 * (complex64 amplitudes are squared exactly, without first rounding to
 * float32).  out_len must equal 2^n (else SV_ERR_SIZE).  out is host memory
 * unless out_is_device.  Page-locked host memory (cudaHostAlloc, or
 * registered and mapped) is written by the kernel directly over the host
 * link; pageable host memory goes through a 128 MiB device staging buffer.
 * Listing 3's probabilities() call. */
int sv_probabilities(sv_state* s, double* out, size_t out_len, int out_is_device);

/* Marginal distribution over the qubits set in qubit_mask: out[k] is the sum
 * of p_i over every i whose masked bits, packed in ascending qubit order,
 * equal k.  out_len must equal 2^popcount(mask).  The CutQC Builder's
 * reconstruction over chosen qubits (Sec. IV-A, "Builder and Verifier"). */
int sv_marginal_probabilities(sv_state* s, uint64_t qubit_mask, double* out,
                              size_t out_len, int out_is_device);

/* Marginal distribution as sv_marginal_probabilities, for callers that cannot
 * let a library allocate device memory: processes whose device memory is
 * fully reserved by another allocator, and latency-critical loops where a
 * cudaFree (which waits for the whole device) would stall other streams.  The
 * paper has no counterpart; this is an interface convenience.
 *   amplitudes: the state's device pointer (16-byte aligned, 2^n amplitudes
 *               of dtype dt), read only; no handle is needed.
 *   out:        2^popcount(mask) float64, host memory unless out_is_device.
 *   cuda_stream: the cudaStream_t to run on (NULL = legacy default stream);
 *               the call synchronises that stream and returns after the
 *               result is in out, so it cannot be recorded into a CUDA graph.
 * It allocates nothing: its scratch is a static 1.5 MiB device array inside
 * the library (held on every GPU that loads the library until exit), so the
 * mask may select at most 16 qubits (SV_ERR_SIZE beyond).  The first call on
 * each device looks the array up (with that device current); make that first
 * call before any stream capture.  All calls share the array and clear what
 * they use, so calls that overlap on the GPU race: serialise them. */
int sv_marginal_probabilities_noalloc(const void* amplitudes, int n_qubits, int dt,
                                      uint64_t qubit_mask, double* out, size_t out_len,
                                      int out_is_device, void* cuda_stream);

/* Copies the amplitudes (sv_state_bytes bytes, in the state's dtype) out, or
 * in (sv_set_amplitudes: checkpoint restore).  The full statevector output a
 * simulation can return beside the probabilities (Sec. III-B; the paper's
 * per-circuit results are written to disk for later steps, Sec. IV-A).
 * bytes must equal sv_state_bytes (else SV_ERR_SIZE); the buffer is host
 * memory unless *_is_device.  Amplitudes set from outside are checked as
 * SV_ARITH_TC describes before the next tensor-core call. */
int sv_amplitudes(sv_state* s, void* out, size_t bytes, int out_is_device);
int sv_set_amplitudes(sv_state* s, const void* in, size_t bytes, int in_is_device);

/* sum_i |a_i|^2, accumulated exactly in 128-bit fixed point on the device
 * (order-independent, so bitwise reproducible) and rounded once to float64.
 * The sum of the probability vector Listing 3 returns (1 for a normalised
 * state; Sec. III-A's reconstruction assumes normalised subcircuit
 * distributions).  Valid for sums below 16 (SV_ARITH_TC states have norm 1). */
int sv_norm(sv_state* s, double* out);

/* Statistics of the last sv_apply_circuit on this handle. */
typedef struct {
    int32_t n_blocks;        /* fused blocks                                */
    int32_t n_passes;        /* tile passes = HBM read+write sweeps         */
    int32_t fuse_k;          /* fusion width used                           */
    int32_t tile_qubits;     /* tile qubits used                            */
    int32_t arith;           /* sv_arith used                               */
    int32_t n_launches;      /* kernels launched                            */
    double  flops;           /* modelled arithmetic, real flops             */
    double  hbm_bytes;       /* passes x 2 x state bytes                    */
    double  plan_ms;         /* host planning time                          */
    double  kernel_ms;       /* sum of kernel durations (opts->timing only) */
    double  max_kernel_ms;   /* longest single launch (opts->timing only)   */
    double  upload_bytes;    /* descriptors + coefficients copied host->device */
    double  alu_ops;         /* modelled ALU lane operations of the passes:
                                FP32 ops (complex64, df64) or FP64 ops (native) */
    double  tensor_flops;    /* SV_ARITH_TC: bfloat16 MMA flops of the digit products */
} sv_apply_stats;
int sv_last_stats(const sv_state* s, sv_apply_stats* out);

/* Batched form -- the CutQC Evaluator's subcircuit instances (Sec. IV-A,
 * "Evaluator"; three measurement and four initialisation variants per cut,
 * Fig. 1), run together instead of by a pool of worker processes (Listing 4).
 * Every item is simulated from |0...0> (each its own width and dtype) and its
 * full probability vector (2^n float64) is written to probs_out (device or
 * host memory, kept valid by the caller until the batch is destroyed).  The
 * items' states live in one pooled device arena; each item is planned on its
 * own (its result does not depend on the other items), and pass i of every
 * item runs in one multi-state tile-pass launch.  The whole sequence (init,
 * passes, probabilities) is captured once in a CUDA graph that
 * sv_batch_execute replays, on a stream of the highest priority (its
 * launches are scheduled ahead of pending launches on other streams; running
 * kernels are not preempted).  item_status[i] receives each item's sv_status
 * (may be NULL); invalid items are skipped, the others still run. */
typedef struct {
    int32_t n_qubits;
    int32_t dt;
    const sv_gate* gates;
    size_t n_gates;
    double* probs_out;
    int32_t probs_on_device;
} sv_batch_item;
int sv_batch_run(const sv_batch_item* items, size_t n_items,
                 const sv_run_opts* opts, int* item_status);

/* The same in three steps, for replaying one batch many times: create (plan,
 * allocate, upload, capture the graph), execute (replay and wait; copies
 * host-side outputs), destroy.  sv_batch_create returns SV_ERR_OOM when the
 * arena does not fit in free device memory. */
typedef struct sv_batch sv_batch;
int sv_batch_create(const sv_batch_item* items, size_t n_items,
                    const sv_run_opts* opts, int* item_status, sv_batch** out);
int sv_batch_execute(sv_batch* b);
void sv_batch_destroy(sv_batch* b);

/* Arena variant for callers that manage device memory themselves (a serving
 * loop on a caching allocator: freeing device memory with cudaFree stalls the
 * whole device).  sv_batch_arena_bytes reports the bytes a batch of these
 * items needs; sv_batch_create_in builds the batch inside the caller's
 * device buffer (256-byte aligned, at least that many bytes), which the
 * caller keeps alive until sv_batch_destroy and frees afterwards. */
int sv_batch_arena_bytes(const sv_batch_item* items, size_t n_items,
                         const sv_run_opts* opts, size_t* bytes);
int sv_batch_create_in(const sv_batch_item* items, size_t n_items,
                       const sv_run_opts* opts, int* item_status,
                       void* arena, size_t arena_bytes, sv_batch** out);

/* Counts of a batch: launches in its graph, device bytes it holds, and the
 * duration of the last sv_batch_execute measured with CUDA events. */
typedef struct {
    int32_t n_items, n_launches;
    double arena_bytes, last_ms;
} sv_batch_info;
int sv_batch_stats(const sv_batch* b, sv_batch_info* out);

/* CutQC reconstruction of the uncut distribution from the subcircuit-variant
 * probabilities (Sec. III-A, Eqs. 3.2-3.7; the Builder's reconstruction, with
 * its partial mode over chosen qubits, Sec. IV-A "Builder and Verifier").
 *   up_probs:   3^K device pointers: the upstream circuit's distribution over
 *               its width_a qubits for measurement variant v = sum_j m_j 3^j
 *               (m_j: 0 = I/Z, 1 = X, 2 = Y on cut j).
 *   down_probs: 4^K device pointers: the downstream distribution over its
 *               width_b qubits for initialisation s = sum_j s_j 4^j
 *               (s_j: 0 = |0>, 1 = |1>, 2 = |+>, 3 = |+i> on cut j).
 *   cut_pos_a:  K upstream qubit indices of the cut wires.
 *   keep_mask_a / keep_mask_b: qubits kept in the output (upstream mask must
 *               exclude the cut qubits); the rest are summed out.
 *   out:        2^(kept_a + kept_b) float64; index = kept upstream bits
 *               (ascending) then kept downstream bits above them.
 * Term sums are exact (signed 128-bit fixed point); 1 <= K <= 6.  The pointer
 * tables are host arrays; the call allocates device scratch and returns after
 * the result is in out. */
int sv_cut_reconstruct(const double* const* up_probs, const double* const* down_probs,
                       int n_cuts, int width_a, const int32_t* cut_pos_a, int width_b,
                       uint64_t keep_mask_a, uint64_t keep_mask_b,
                       double* out, size_t out_len, int out_is_device);

/* Cut-subcircuit variants with shared work (the Evaluator's instances,
 * Sec. IV-A, Fig. 1), producing the same outputs as running every variant
 * through sv_batch_run, within the tolerance of the arithmetic:
 *   upstream: body_a (width_a qubits) is simulated once from |0..0>; variant
 *     v = sum_j m_j 3^j appends the basis change of cut j (m_j: 0 = I/Z none,
 *     1 = X: H, 2 = Y: S^dagger then H) on qubit cut_pos_a[j] to a copy;
 *     its probabilities go to up_out[v] (2^width_a float64).
 *   downstream: body_b (width_b qubits) is simulated from each computational
 *     basis state of the cut qubits cut_pos_b[] (2^K runs); variant
 *     s = sum_j s_j 4^j (s_j: 0 = |0>, 1 = |1>, 2 = |+>, 3 = |+i>) is formed as
 *     a linear combination of those states (the body is linear); its
 *     probabilities go to down_out[s] (2^width_b float64).
 * 1 + 2^K body simulations replace 3^K + 4^K.  Outputs are host memory
 * unless outs_on_device; 1 <= K <= 6. */
int sv_cut_variants(int dt, const sv_gate* body_a, size_t n_a, int width_a,
                    const int32_t* cut_pos_a, const sv_gate* body_b, size_t n_b,
                    int width_b, const int32_t* cut_pos_b, int n_cuts,
                    double* const* up_out, double* const* down_out,
                    int outs_on_device, const sv_run_opts* opts);

/* Measured autotuner (the paper's analogue: Aer's blocking_qubits and the
 * Evaluator's worker count, both set by trial, Sec. IV-A, Listing 4).  The
 * planner picks the fusion width and the fusion variant for each circuit by
 * a cost model; by default an analytic one, or, once sv_set_costs installed
 * a table for the (dtype, arithmetic) pair, these costs measured on the
 * device.  All figures are picoseconds per amplitude of the state (so a 2^n
 * state pays 2^n times each):
 *   pass_ps       one tile pass that applies nothing (the tile's HBM read
 *                 and write and its conversions);
 *   dense_ps[k]   one dense block of k qubits (k = 1..5; 0 unused); the
 *                 tensor-core modes pad blocks below 3 qubits to 3, and the
 *                 complex128 digit mode has no 5-qubit blocks (0 there);
 *   diag_ps       one diagonal block with general phases;
 *   sign_ps       one diagonal block of signs only (CZ / Z);
 *   perm_ps[k]    one permutation block of k qubits with quarter phases.
 * A Kronecker block costs k dense_ps[1] outside the tensor-core modes and
 * dense_ps[k] in them; a permutation block with other phases adds diag_ps. */
typedef struct {
    int32_t dt, arith;           /* the pair measured (arith resolved, not AUTO) */
    int32_t n_qubits, tile_qubits;  /* the calibration state and its tiles     */
    double pass_ps;
    double dense_ps[6];
    double diag_ps, sign_ps;
    double perm_ps[6];
} sv_costs;

/* Measures the table on the current device: single-pass synthetic plans on
 * a 24-qubit (complex128) or 25-qubit (complex64) state, timed with CUDA
 * events, each the fastest of three runs.  arith is resolved as for a
 * 24-qubit state (SV_ARITH_AUTO gives the tensor-core modes).  Allocates the
 * state and frees it before returning; SV_ERR_OOM if it does not fit. */
int sv_calibrate(int dt, int arith, sv_costs* out);

/* Installs (or, with costs = NULL, removes) the measured table for the pair
 * (dt, arith), where arith is the resolved mode the table was measured for
 * (SV_ARITH_NATIVE, SV_ARITH_DF64 or SV_ARITH_TC).  Process-wide; host only
 * (no device call).  Plans made afterwards for that pair use it. */
int sv_set_costs(int dt, int arith, const sv_costs* costs);

/* Static description of a status code. */
const char* sv_status_str(int status);

/* Library version string. */
const char* sv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LIBSV_SV_H */
