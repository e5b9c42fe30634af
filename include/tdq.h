/*
 * tdq.h -- C ABI of the GB300 tensor-network circuit contraction library.
 *
 * The calls follow the workflow of TeD-Q's tensor-network mode (Sec. 3.2):
 *   (a) build the circuit and convert it to a tensor network   tdq_circuit_*, tdq_network_build
 *   (c) find a contraction path, (d) slice it                    tdq_plan_find
 *   (e) contract it, many times, for values and gradients        tdq_plan_compile, tdq_execute
 * and the reusable mechanism of Sec. 1 / Sec. 2: a compiled plan is built once
 * and executed for every new parameter set.
 *
 * Conventions (fixed here because amplitudes are phase-sensitive):
 *   - qubit 0 is the most significant bit of a basis index (Sec. 5.1.1);
 *   - RY(t) = [[cos t/2, -sin t/2], [sin t/2, cos t/2]] as printed in Sec. 3.2.1;
 *     RX(t) = exp(-i t X/2), RZ(t) = diag(e^{-it/2}, e^{it/2}),
 *     RZZ(t) = exp(-i t Z(x)Z/2), U3(t,f,l) = [[c, -e^{il} s], [e^{if} s, e^{i(f+l)} c]];
 *   - two-qubit gates list (control, target) for CNOT; CNOT is the reading of
 *     the tensor printed in Sec. 3.2.1: E[e,f,c,d] = [e == c][f == c xor d].
 *
 * Memory: the library owns its handles and every workspace it needs, which it
 * allocates in tdq_plan_compile; tdq_execute allocates nothing.  Parameter,
 * input and output buffers belong to the caller; on tdq_execute they are
 * device pointers (CUDA global memory of the exec's device), used on the
 * caller's stream.
 *
 * Errors: every call returns a tdq_status; tdq_last_error() gives a message
 * for the calling thread.  No C++ exception crosses this boundary.  Argument
 * and structure errors are found on the host.  Errors found by a kernel
 * (non-finite parameters, a wait that timed out) are recorded in a device
 * status word of the exec and returned by tdq_exec_status().
 */
#ifndef TDQ_ABI_H_
#define TDQ_ABI_H_

#ifndef __CUDACC_RTC__ /* run-time compiled device code defines the fixed-width types itself */
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tdq_status {
  TDQ_OK = 0,
  TDQ_ERR_ARG = 1,         /* invalid argument or handle */
  TDQ_ERR_OOM = 2,         /* device or host allocation failed, or over budget */
  TDQ_ERR_CUDA = 3,        /* a CUDA runtime/driver call failed */
  TDQ_ERR_TIMEOUT = 4,     /* a bounded device wait ran out */
  TDQ_ERR_NONFINITE = 5,   /* a parameter or input was NaN or infinite */
  TDQ_ERR_UNSUPPORTED = 6, /* valid request this build does not handle */
  TDQ_ERR_STATE = 7        /* call out of order (e.g. empty circuit) */
} tdq_status;

/* Gate kinds (Sec. 2, Sec. 3.2.1, Sec. 5.2 listings). */
typedef enum tdq_gate {
  TDQ_H = 0, TDQ_X = 1, TDQ_Y = 2, TDQ_Z = 3,
  TDQ_RX = 4, TDQ_RY = 5, TDQ_RZ = 6, TDQ_U3 = 7,
  TDQ_CNOT = 8, TDQ_CZ = 9, TDQ_RZZ = 10
} tdq_gate;

/* Angle sources for tdq_circuit_gate: j >= 0 is parameter column j;
 * TDQ_INPUT(j) is input feature j (angle encoding, Sec. 5.3, Eq. 11);
 * TDQ_FIXED takes the constant from the `fixed` array. */
#define TDQ_FIXED (-1)
#define TDQ_INPUT(j) (-2 - (j))

typedef struct tdq_circuit tdq_circuit;
typedef struct tdq_network tdq_network;
typedef struct tdq_plan tdq_plan;
typedef struct tdq_exec tdq_exec;

/* Message describing the last failed call on this thread ("" if none).
 * Owned by the library, valid until the next call on the thread. */
const char* tdq_last_error(void);

/* ABI version (major * 100 + minor). */
int tdq_version(void);

/* ------------------------------------------------------------ circuit (Sec. 2)
 * A circuit is an ordered list of gates on n_qubits (1..64) qubits, a list of
 * Pauli-Z product observable terms and a list of amplitude bitstrings. */

/* Create an empty circuit.  *out owned by the caller; free with
 * tdq_circuit_destroy.  ERR_ARG if n_qubits is outside 1..64. */
tdq_status tdq_circuit_create(int n_qubits, tdq_circuit** out);

/* Append gate `kind` on qubits[0..nq) (nq = 1 or 2, distinct, in range).
 * angle_src[i] (i < number of angles of the gate: 1 for RX RY RZ RZZ, 3 for
 * U3, 0 otherwise) is a parameter column, TDQ_INPUT(j) or TDQ_FIXED, in which
 * case fixed[i] is the angle.  angle_src / fixed may be NULL for gates without
 * angles.  ERR_ARG on a bad kind, qubit or source. */
tdq_status tdq_circuit_gate(tdq_circuit* c, int kind, const int* qubits, int nq,
                            const int* angle_src, const double* fixed);

/* Add the observable term coeff * prod_{q in z_qubits} Z_q to output group
 * `group` (>= 0).  The value of a group is the sum of its terms' expectation
 * values <0|U^dagger Z.. U|0> (Sec. 4, Eq. 9; the list of measurements of
 * Sec. 2).  nz = 0 is the identity term. */
tdq_status tdq_circuit_observable(tdq_circuit* c, const int* z_qubits, int nz, double coeff,
                                  int group);

/* Request the amplitude <x|U|0...0> for bits[q] = x_q in {0,1}, q < n_qubits
 * (Sec. 3.2.1: the probability amplitude of a given final state). */
tdq_status tdq_circuit_amplitude(tdq_circuit* c, const uint8_t* bits);

/* Sizes: number of gates, parameter columns, input features, output groups,
 * observable terms and amplitude requests.  Any pointer may be NULL. */
tdq_status tdq_circuit_info(const tdq_circuit* c, int* n_gates, int* n_params, int* n_inputs,
                            int* n_groups, int* n_terms, int* n_amplitudes);

tdq_status tdq_circuit_destroy(tdq_circuit* c);

/* ------------------------------------------------ tensor network (Sec. 3.2 (a))
 * The network of one output: for an expectation term, the ket network (|0>
 * per qubit, one tensor per gate with indices (outputs..., inputs...)), Z
 * tensors on the term's qubits and the complex-conjugate network closing it
 * (Sec. 3.2.1); for an amplitude, the ket network closed by <x_q| on every
 * qubit.  All index dimensions are 2. */

typedef struct tdq_net_opts {
  int output;    /* TDQ_OUT_EXPVAL (one observable term) or TDQ_OUT_AMPLITUDE */
  int index;     /* which term (tdq_circuit_observable order) or amplitude request */
  int lightcone; /* expectation networks: keep only the backward causal cone of
                    the term's qubits (the other gates cancel with their
                    conjugates); ignored for amplitudes */
  int split_2q;  /* structural simplification (Sec. 3.2.1): a two-qubit gate
                    that is block diagonal in its first qubit, G = sum_s
                    |s><s| (x) V_s (CNOT, CZ, RZZ), becomes two rank-3 tensors
                    joined by a bond of dimension 2 -- exact, and the bond
                    is one index where the gate was two across a cut */
  int hyper;     /* structural simplification (Sec. 3.2.1, diagonal reduction):
                    diagonal gates (Z, RZ, CZ, RZZ) and Z observables become
                    tensors of their diagonals on the wires' existing indices,
                    and CNOT keeps its control wire's index (a rank-3 tensor
                    [out == in xor control]); those indices are then shared by
                    more than two tensors (hyperedges: a contraction keeps an
                    index while another tensor still holds it).  Anti-diagonal
                    reduction: X and Y keep the wire's index too, which every
                    later tensor on the wire reads complemented
                    (tdq_network_tensor_flips); Y leaves the phases (i, -i) of
                    its input value as a one-index tensor.  Takes precedence
                    over split_2q for CNOT, CZ and RZZ */
} tdq_net_opts;

/* Build the network.  The network keeps its own copy of the circuit.
 * ERR_ARG for a missing term / amplitude.  Free with tdq_network_destroy. */
tdq_status tdq_network_build(const tdq_circuit* c, const tdq_net_opts* opts, tdq_network** out);

/* Tensor count, index count, qubits and gates kept (after the light cone). */
tdq_status tdq_network_info(const tdq_network* n, int* n_tensors, int* n_indices, int* n_qubits,
                            int* n_gates);

/* Describe tensor i: kind (0 |0>, 1 gate, 2 Z observable, 3 <bit|), circuit
 * gate index (kind 1), conj flag (bra side), bit value (kind 3), rank and its
 * index ids in storage order (idx[0] most significant); idx needs rank slots. */
tdq_status tdq_network_tensor(const tdq_network* n, int i, int* kind, int* gate, int* conj, int* bit,
                              int* rank, int* idx);

/* Complemented indices of tensor i (hyper networks, anti-diagonal
 * reduction): bit a of *flip set means index a is read complemented -- the
 * entry at value v of that index is the plain tensor's entry at v ^ 1.  The
 * plain tensor of a Y reduction (kind 6 with a Y gate) holds Y[1 - i][i]. */
tdq_status tdq_network_tensor_flips(const tdq_network* n, int i, int* flip);

tdq_status tdq_network_destroy(tdq_network* n);

/* ------------------------------------- contraction path and slicing (Sec. 3.2 (c), (d)) */

typedef enum tdq_path_method {
  TDQ_PATH_GREEDY = 0,        /* greedy (Sec. 3.2.2 default finder): pair with the least
                                 result-minus-operand entries first; ties by FLOPs
                                 p(2q-1) (Eq. 5), result size, lower tensor ids */
  TDQ_PATH_RANDOM_GREEDY = 1, /* Boltzmann sampling among the 8 best pairs, weight
                                 exp(-(cost - best) / (temperature * max(1, |best|))) */
  TDQ_PATH_PARTITION = 2      /* contraction tree by recursive bipartition of the
                                 network's hypergraph (Sec. 3.2.2, the hypergraph
                                 pathfinder): each node's tensors split to minimise the
                                 indices cut plus w |outer(A) - outer(B)| (outer indices
                                 spread evenly over the children), sides at most
                                 (1 + eps) / 2 of the node; small nodes finish greedy.
                                 Each trial draws eps, w and the cutoff from its seed */
} tdq_path_method;

typedef struct tdq_plan_opts {
  int method;         /* tdq_path_method */
  uint64_t seed;      /* random-greedy sampling and slice tie-breaking */
  double temperature; /* random-greedy only; <= 0 means 1 */
  int target_log2;    /* slice until every tensor has at most 2^target_log2
                         entries (Sec. 3.2.3 greedy); 0 = no slicing */
  int repeats;        /* random-greedy and partition: trials with seeds seed,
                         seed+1, ... (run on the host's cores); the plan with
                         the fewest FLOPs over all slices wins (the repeats of
                         Sec. 3.2.4); <= 1 means one */
  int slice_trials;   /* two-phase slicing-aware search (Sec. 3.2.3), phase 1:
                         randomised greedy slicings per trial tree, the tree
                         scored by its best; 0 = the single greedy slicing */
  int slice_final;    /* phase 2: further randomised slicings of the winning
                         tree (the paper's default is 1024); 0 = none.  Both
                         in [0, 2^20]; they act only when target_log2 > 0 */
  int rank_simplify;  /* 1: rank simplification before the search (Sec. 3.2.1,
                         the local processing of the network): while two
                         tensors share an index and their contraction has no
                         more indices than the larger of them, contract the
                         pair with the smallest result; these steps open the
                         path and the finder searches the tensors left.  0 =
                         off.  Other values: ERR_ARG */
} tdq_plan_opts;

/* Find a pairwise path (SSA: ids < n_tensors are the network's tensors, id
 * n_tensors + s is the result of step s) and a set of sliced indices. */
tdq_status tdq_plan_find(const tdq_network* n, const tdq_plan_opts* opts, tdq_plan** out);

/* Plan from a caller-given path (pairs[2 s], pairs[2 s + 1], n_tensors - 1
 * steps, every id used once) and sliced index ids. */
tdq_status tdq_plan_from_path(const tdq_network* n, const int* pairs, int n_steps, const int* sliced,
                              int n_sliced, tdq_plan** out);

typedef struct tdq_stats {
  double log2_flops_per_slice; /* log2 of sum over steps of p(2q-1) */
  double flops;                /* all slices */
  int max_log2_width;          /* largest tensor of one slice, log2 entries */
  int n_sliced;                /* number of sliced indices (2^n_sliced slices) */
  int n_steps;
  double log2_bytes_per_slice; /* log2 of complex64 bytes read + written by all steps */
} tdq_stats;

tdq_status tdq_plan_stats(const tdq_plan* p, tdq_stats* s);

/* Launch units a compiled tree plan would run for `batch` rows within a
 * workspace budget (0: 64 GiB), in the order of tdq_exec_timings, and their
 * features (12 floats per unit; see the design notes): feats [n_units][12]
 * or NULL to query *n_units.  *repeats = batches of slices per execute.
 * Host only: no device work. */
tdq_status tdq_plan_features(const tdq_plan* p, int batch, int64_t workspace_bytes, float* feats, int max_units,
                             int* n_units, int* repeats);

/* Copy out the path (2 * n_steps ints) and the sliced ids (n_sliced ints). */
tdq_status tdq_plan_path(const tdq_plan* p, int* pairs, int* sliced);

tdq_status tdq_plan_destroy(tdq_plan* p);

/* ------------------------------------------------- compile and execute (Sec. 3.2 (e))
 * The state-sweep path: the ket network (|0> tensors and gate tensors) is
 * contracted in circuit order -- the |0>'s into one rank-n tensor, then each
 * gate tensor absorbed into it -- and the result closed with the observable
 * and the conjugate ket (the expectation network of Sec. 3.2.1), or with <x|
 * for amplitudes.  Gradients are the reverse sweep of that path (Sec. 4.1)
 * or the parameter-shift rule (Sec. 4.2, Eq. 10). */

typedef enum tdq_output {
  TDQ_OUT_EXPVAL = 0,    /* values[b][g]: the circuit's output groups */
  TDQ_OUT_AMPLITUDE = 1, /* values[b][a][2]: (re, im) of each amplitude request */
  TDQ_OUT_STATE = 2,     /* state sweep only: values[b][x][2], the final state
                            vector U|psi0> (Sec. 3.1: the state-vector mode's
                            state()); x = sum_q bit_q 2^(n-1-q) */
  TDQ_OUT_PROBS = 3      /* state sweep only: values[b][x] = |<x|U|psi0>|^2
                            (Sec. 3.1: probabilities) */
} tdq_output;

typedef enum tdq_grad {
  TDQ_GRAD_NONE = 0,
  TDQ_GRAD_ADJOINT = 1,    /* reverse sweep with un-computation (Sec. 4.1) */
  TDQ_GRAD_PARAM_SHIFT = 2 /* 2 shifted evaluations per angle, batched (Sec. 4.2) */
} tdq_grad;

typedef struct tdq_compile_opts {
  int batch;       /* rows B per tdq_execute (>= 1) */
  int output;      /* tdq_output */
  int grad;        /* tdq_grad (expectation outputs only) */
  int device;      /* CUDA device ordinal */
  int max_smem_qubits; /* 0 = default (13 with adjoint gradients, else 14): largest
                          n whose state one CTA holds whole in shared memory */
  int tile_qubits;     /* 0 = default (12): bits per shared-memory tile of the
                          HBM-resident sweep, 5..13 */
  int plain;           /* tree plans: 1 = one kernel launch per pairwise step
                          (no fusion of the path into one launch) */
  int64_t workspace_bytes; /* tree plans: HBM budget for batched slices
                              (0 = half the free memory, at most 64 GiB) */
  int record_timings;  /* tree plans: time every launch unit of the first slice
                          batch; tiled state sweeps: every tile-pass launch of
                          the first row chunk; with CUDA events (see
                          tdq_exec_timings, tdq_exec_launch_work) */
  int interpret;       /* state sweep: 1 = run the gate program through the
                          generic kernels, which decode it at run time; 0 =
                          compile a kernel specialised to this circuit (NVRTC,
                          at compile time; cached per process) */
  int fwd_reg_bits;    /* state sweep, specialised programs: state bits held in
                          registers per forward register pass (1..4; 0 =
                          default: 2 whole-state, 4 tiled) */
  int rev_reg_bits;    /* ... per reverse register pass (1..4; 0 = default:
                          2 whole-state, 4 tiled; generic kernels 3) */
  int subtree_log2;    /* tree plans: steps whose operands and result all have at
                          most 2^subtree_log2 entries run inside the fused
                          subtree launch (one CTA per subtree); larger ones get a
                          launch each.  0 = default (11); 1..13 */
  int autotune;        /* sweeps and multi-circuit launches: 1 = compile candidate
                          launch configurations and keep the fastest on this
                          circuit and batch (timed with CUDA events on synthetic
                          parameters at compile time): whole-state kernels CTA
                          size 128/256/512 x register bits 2/3, tiled sweeps tile
                          bits 10..13 (see tdq_compile_multi for its candidates);
                          requires interpret, register bits and tile_qubits 0 */
  int tc_min_log2;     /* tree plans: large steps of at least 2^tc_min_log2 complex
                          multiply-adds (and a shape the tiles fit) run on the
                          tensor cores, smaller ones on the SIMT kernels (the
                          tensor-core launch has a fixed cost).  0 = default;
                          1 = whenever the shape fits; 64 = never */
} tdq_compile_opts;

/* Compile the circuit's state-sweep contraction for repeated execution.
 * Allocates the device program and every workspace (HBM ~ B * 2^n * 8 bytes
 * per state kept, x2 with gradients) on opts->device.  ERR_UNSUPPORTED if
 * n_qubits > 30 (use a tensor-network plan).  *out freed by tdq_exec_destroy.
 * Expectation outputs: the parameter-free CNOT, CZ, X, Y and Z gates that
 * commute to the end of the circuit (every later gate acts on other qubits)
 * are contracted with the observable first -- each maps a Z-product term to
 * a Z-product term (CNOT(c -> t): Z_t -> Z_c Z_t; X, Y: Z -> -Z) -- an exact
 * change of contraction order (Sec. 3.2.1), so the sweep never applies them
 * to the state. */
tdq_status tdq_compile_sweep(const tdq_circuit* c, const tdq_compile_opts* opts, tdq_exec** out);

/* The CUDA source tdq_compile_sweep compiles (NVRTC) for circuit c unless
 * opts->interpret is set: its register passes written out gate by gate, bits
 * and table rows as constants.  tile_qubits = 0: the whole-state kernel (one
 * CTA per row; n <= 14); 5..13: the tiled kernels of each tile pass of that
 * many bits (the state in HBM; n <= 30).  grad: TDQ_GRAD_NONE or
 * TDQ_GRAD_ADJOINT (with the reverse programs).  For a circuit with
 * observables it is the expectation program: parameter-free CNOT, CZ, X, Y
 * and Z gates that commute to the end of the circuit are folded into the
 * Z-product terms instead (see tdq_compile_sweep).  The source includes the
 * library's device headers (tdq.h, sweep_common.cuh, engine.cuh, k1_body.cuh,
 * k2_body.cuh).  Writes the NUL-terminated source to buf if cap allows;
 * *len = bytes needed (buf may be NULL to query it).  Host only: no device
 * call.  ERR_ARG on a bad grad, tile size or short buffer; ERR_UNSUPPORTED
 * beyond the qubit limits. */
tdq_status tdq_sweep_source(const tdq_circuit* c, int grad, int tile_qubits, char* buf, size_t cap, size_t* len);

/* Many circuits of uneven qubit counts and depths in one persistent launch of
 * the whole-state kernel (Sec. 3.1 sweep per row, the forward, observable and
 * reverse sweeps of K2): circuit c runs batch[c] rows -- its data samples and,
 * with TDQ_GRAD_PARAM_SHIFT, the 2 P_c + 1 shifted copies of each sample as
 * further rows of the same launch.  Persistent CTAs take (circuit, row) items
 * from a device counter, the costliest circuits first; every circuit's program
 * is specialised (straight-line code, compiled at run time) into one kernel.
 * Requires n_c <= 13 with adjoint gradients, else <= 14, and expectation
 * outputs (opts->output = TDQ_OUT_EXPVAL; opts->batch is ignored, batch[]
 * gives the rows; opts->interpret must be 0).  Threads per CTA and register
 * bits: opts->fwd_reg_bits / rev_reg_bits (0 = 2), 256 threads (fewer if
 * every state is small); opts->autotune = 1 instead times CTA sizes 128, 256,
 * 512 with register bits 2 and 3 on this workload and keeps the fastest.
 * tdq_execute then takes packed buffers (params_stride must be 0): circuit c's
 * rows of parameters and gradients [batch[c]][P_c], inputs [batch[c]][F_c],
 * values and weights [batch[c]][n_groups_c] at the offsets tdq_multi_layout
 * reports; the call is one kernel launch (plus the shift-rule combine), and a
 * call repeating the previous call's pointers is replayed as a CUDA graph.
 * ERR_ARG for bad arguments (checked before any device call), ERR_UNSUPPORTED
 * for a circuit too large for one CTA. */
tdq_status tdq_compile_multi(const tdq_circuit* const* circuits, const int* batch, int n_circuits,
                             const tdq_compile_opts* opts, tdq_exec** out);

/* Launch configuration of a sweep or multi-circuit exec (the one the
 * autotuner kept, or the defaults): config[4] = {threads per CTA, forward
 * register bits, reverse register bits, tile bits of a tiled sweep (0 for the
 * whole-state kernel) or the persistent CTAs of a multi-circuit launch}.
 * Tree plans: {reverse tree (0 none, 1 fused in one CTA, 2 every value kept,
 * 3 values recomputed region by region from checkpoints -- chosen when keeping
 * every value does not fit the workspace budget), recompute regions, slices
 * per launch, workspace entries (complex64) per batch entry}. */
tdq_status tdq_exec_config(const tdq_exec* e, int* config);

/* Host only: the CUDA source of the persistent multi-circuit kernel for these
 * circuits (what tdq_compile_multi compiles with the same threads and register
 * bits; grad: tdq_grad), written like tdq_sweep_source: modules, each after a
 * line "// ==== tdq module <i>" -- module 0 the kernel, module c + 1 circuit
 * c's row function -- compiled separately as relocatable device code (in
 * parallel) and linked into one kernel. */
tdq_status tdq_multi_source(const tdq_circuit* const* circuits, int n_circuits, int grad, int threads,
                            int fwd_reg_bits, int rev_reg_bits, char* buf, size_t cap, size_t* len);

/* Circuit c's element offsets in the packed buffers of a multi-circuit exec
 * (params and grads, inputs, values and weights; any pointer may be NULL) and
 * the launch configuration config[4] = {threads per CTA, forward register
 * bits, reverse register bits, persistent CTAs} (NULL to skip). */
tdq_status tdq_multi_layout(const tdq_exec* e, int c, int64_t* params_off, int64_t* inputs_off, int64_t* values_off,
                            int* config);

/* Execute once for B rows on `stream` (a cudaStream_t; NULL = legacy default).
 *   d_params      float [B][params_stride] row-major, parameter column j of row
 *                 b at d_params[b * params_stride + j]; params_stride = 0
 *                 shares one row across the batch.  May be NULL if P == 0.
 *   d_inputs      float [B][F] input features, or NULL if F == 0.
 *   d_values      double output, [B][n_groups] (expectations) or
 *                 [B][n_amplitudes][2] (amplitudes).
 *   d_grad_w      double [B][n_groups] weights w of F_b = sum_g w[b][g] f_g(b),
 *                 the function whose gradient is taken; NULL = all ones.
 *   d_grads       float [B][P]: dF_b / d params[b][j]; required iff the exec
 *                 was compiled with a gradient mode, else must be NULL.
 * Asynchronous: returns after enqueueing.  Device errors are reported by
 * tdq_exec_status.  Not thread-safe per exec (one stream at a time). */
tdq_status tdq_execute(tdq_exec* e, const float* d_params, int64_t params_stride,
                       const float* d_inputs, double* d_values, const double* d_grad_w,
                       float* d_grads, void* stream);

/* Synchronise the exec's last stream and return (then clear) the device
 * status word: TDQ_OK, TDQ_ERR_NONFINITE or TDQ_ERR_TIMEOUT. */
tdq_status tdq_exec_status(tdq_exec* e);

/* Initial state psi0 of every later tdq_execute of a state-sweep exec, in
 * place of |0...0> (Sec. 3.1: a user-given initial state vector).
 *   d_psi0      device, complex64 as (re, im) float pairs, [rows][2^n]; row b
 *               at d_psi0 + 2 * b * row_stride floats; basis index x as for
 *               TDQ_OUT_STATE.  Used as given (not normalised).  NULL restores
 *               |0...0>.
 *   row_stride  complex elements between rows: 0 (one state for every row) or
 *               >= 2^n.
 * The pointer is kept, not copied: the caller keeps the buffer alive and
 * unchanged while execs that use it run.  Gradients (adjoint and parameter
 * shift) and every output kind take it into account.  ERR_ARG on a bad
 * stride; ERR_UNSUPPORTED for tensor-network plans (they contract <x| or
 * Z-terms against |0...0>). */
tdq_status tdq_exec_set_initial_state(tdq_exec* e, const float* d_psi0, int64_t row_stride);

/* Compile a tensor-network plan (Sec. 3.2 (e)): every pairwise step of the
 * path, batched over rows and slices, with the slices' results summed in
 * FP64.  opts->output is taken from the network.  tdq_execute then writes
 * values[b][0] = the term's coefficient times the expectation (expectation
 * networks) or values[b][0..1] = (re, im) of the amplitude.
 * opts->grad = TDQ_GRAD_ADJOINT (expectation networks): the reverse tree of
 * the path (backpropagation, Sec. 4.1) -- each step C = A.B passes its
 * cotangent to A and B, the leaves' cotangents give dF/dtheta = Re sum
 * Lbar * dL/dtheta, summed over slices in FP64 -- written to grads [B][P]
 * for F = w[b] * value (d_grad_w [B], NULL = 1).  The whole network runs in
 * one CTA per (row, slice) when its values and cotangents fit in shared
 * memory, else every step (and its reverse) is its own launch with every
 * intermediate kept.  All workspaces are allocated here: a whole
 * path of one (row, slice) in one CTA's shared memory when it fits (fused),
 * else an HBM workspace of batched slices within opts->workspace_bytes.  When
 * keeping every value and cotangent of the per-step reverse tree does not fit
 * that budget, the forward pass keeps only checkpoints (the leaves and the
 * roots of regions of the tree) and the reverse pass recomputes each region's
 * values from them before running its reverse steps (about one extra forward
 * pass).  ERR_OOM if even that does not fit (slice further).
 * Values-only plans (not plain, not timed): the steps too large for the fused
 * subtree launch run concurrently where the tree allows -- independent branches
 * on up to four streams joined to the caller's, ordered by the operands and by
 * reuse of workspace -- and a tdq_execute call that repeats the previous call's
 * pointers, stride and stream is captured once as a CUDA graph and replayed
 * from then on (the buffers' contents are read at run time, so new parameters
 * in the same buffer need no new capture). */
tdq_status tdq_plan_compile(const tdq_plan* p, const tdq_compile_opts* opts, tdq_exec** out);

/* Contract only slices [first, first + count) of a tree exec's 2^n_sliced
 * slices (tdq_plan_stats) from the next tdq_execute on: values (and gradients)
 * are then the FP64 partial sums over that range.  The slicing identity of
 * Sec. 3.2.3 -- the full result is the sum over all slices, and the slices
 * are independent sub-networks of one shape -- lets ranks contract disjoint
 * ranges in parallel and add their partials with one sum.  count = 0 gives zero
 * partials.  Default: every slice.  ERR_ARG for a range outside
 * [0, 2^n_sliced); ERR_UNSUPPORTED for sweep and multi-circuit execs.  A
 * captured graph of the previous range is dropped. */
tdq_status tdq_exec_set_slice_range(tdq_exec* e, int64_t first, int64_t count);

/* Per-launch-unit device times (ms) of the last tdq_execute of an exec
 * compiled with record_timings.  Tree plans: unit 0 is the launch of all
 * small-step subtrees, unit 1 + i the i-th large step, for the first batch of
 * slices (the units repeat for every further batch).  Tiled state sweeps:
 * every tile-pass launch of the first row chunk (see tdq_exec_launch_work).  Synchronises the exec's
 * stream.  ms may be NULL to query *n.  ERR_STATE without record_timings. */
tdq_status tdq_exec_timings(tdq_exec* e, float* ms, int max, int* n);

/* Algorithmic work of each launch unit that tdq_exec_timings times, for a
 * tiled state sweep (the state in HBM): flops[u] (FP32 operations by the
 * counting rule of tdq_exec_work), bytes[u] (its HBM traffic model: the
 * state read and written once per pass, psi and lambda in reverse passes)
 * and kind[u] (0 forward tile pass, 1 last pass with the observable and its
 * reverse sweep fused, 2 reverse tile pass), for the rows of the first row
 * chunk; units in launch order.  Any array may be NULL; all NULL queries *n.
 * ERR_UNSUPPORTED for other exec kinds.  Host only. */
tdq_status tdq_exec_launch_work(const tdq_exec* e, double* flops, double* bytes, int* kind, int max, int* n);

/* Number of kernel launches the last tdq_execute enqueued. */
int tdq_exec_launches(const tdq_exec* e);

/* Static work counts of one execute per row: algorithmic FLOPs and bytes of
 * the dominant kernel's traffic model (see the design notes); any may be NULL. */
tdq_status tdq_exec_work(const tdq_exec* e, double* flops_per_row, double* bytes_per_row,
                         int* kernel_class);

tdq_status tdq_exec_destroy(tdq_exec* e);

/* ------------------------------------------------ learned cost model (K8)
 * Not in the paper, which ranks paths by FLOPs p(2q-1) (Sec. 3.2.2, Eq. 5):
 * a 3-layer perceptron n_features -> hidden -> hidden -> 1 (FP32, ReLU)
 * trained on the engine's own launch timings (tdq_exec_timings) against the
 * launch features (tdq_plan_features) to predict log time, used to rank
 * candidate plans by predicted device time.  Parameters are one packed FP32
 * vector W1 [H][F], b1 [H], W2 [H][H], b2 [H], W3 [H], b3; the loss is the
 * mean squared error.  All device pointers; calls are asynchronous on
 * `stream` except tdq_costmodel_params. */
typedef struct tdq_costmodel tdq_costmodel;

/* He-uniform weights from `seed`, zero biases; 1 <= n_features <= 32,
 * hidden 32 or 64.  Device memory for parameters, gradient, Adam moments. */
tdq_status tdq_costmodel_create(int n_features, int hidden, uint64_t seed, int device, tdq_costmodel** out);

/* Copy the packed parameters to (set = 0) or from (set = 1, which also resets
 * Adam) host memory; host may be NULL to query *n_params. */
tdq_status tdq_costmodel_params(tdq_costmodel* m, float* host, int* n_params, int set);

/* Loss and gradient for rows X [N][F], targets t [N]; the gradient is kept
 * for the next Adam step and copied to d_grads [n_params] if given;
 * d_loss [1] if given. */
tdq_status tdq_costmodel_loss_grad(tdq_costmodel* m, const float* d_X, const float* d_t, int N, float* d_loss,
                                   float* d_grads, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the kept gradient. */
tdq_status tdq_costmodel_adam_step(tdq_costmodel* m, float lr, void* stream);

/* `epochs` full-batch steps (loss_grad + adam_step); d_losses [epochs] or NULL. */
tdq_status tdq_costmodel_train(tdq_costmodel* m, const float* d_X, const float* d_t, int N, int epochs, float lr,
                               float* d_losses, void* stream);

/* y [N] = model(X [N][F]). */
tdq_status tdq_costmodel_predict(tdq_costmodel* m, const float* d_X, int N, float* d_y, void* stream);

tdq_status tdq_costmodel_destroy(tdq_costmodel* m);

/* ------------------------------------------------ kernel-level entry points
 * The tensor-core product used by the large pairwise steps of Sec. 3.2 (e)
 * (each step is C[m][n] = sum_k A[m][k] B[n][k] over the fused indices):
 *   D[b][i][j] = sum_k X[b][i][k] Y[b][j][k],   complex64 (interleaved re, im),
 * row-major, X [batch][I][K], Y [batch][J][K], D [batch][I][J], all device
 * pointers; 3xTF32 split precision with FP32 accumulation on tcgen05.
 * Requires I % 128 == 0, J % 64 == 0, K % 8 == 0, 1 <= batch <= 65535
 * (ERR_ARG otherwise).  d_status: a device int the kernel ORs
 * (1 << TDQ_ERR_TIMEOUT) into if a bounded wait ran out.  Asynchronous. */
tdq_status tdq_cgemm_nt(int batch, int I, int J, int K, const float* dX, const float* dY, float* dD,
                        int* d_status, void* stream);

/* tdq_cgemm_nt with a caller-set bound on the waits of its main loop (the
 * handshakes between the warps that stage operands, the thread that issues
 * the tensor-core products and the read-out of the accumulators): wait_ns of
 * the global timer, 0 .. 1e9 (tdq_cgemm_nt uses 1e9).  A wait that runs out
 * sets (1 << TDQ_ERR_TIMEOUT) in *d_status; the kernel then stops issuing,
 * waits (always with the 1 s bound) for the products it issued, frees its
 * tensor memory and returns, leaving D unspecified.  Failure detection
 * without a fault: a bound too short for the staging makes the first wait run
 * out before any product is issued (0: a wait that is not already complete
 * gives up at once).  ERR_ARG as tdq_cgemm_nt, or for wait_ns
 * outside the range. */
tdq_status tdq_cgemm_nt_bounded(int batch, int I, int J, int K, const float* dX, const float* dY, float* dD,
                                int* d_status, int64_t wait_ns, void* stream);

/* ------------------------------------------------ execution without allocation
 * No counterpart in the paper: an addition for callers that cannot call
 * cudaMalloc -- for example code running under a memory manager that owns
 * every device allocation, or a service that reserves its memory at start-up
 * and forbids cudaMalloc / cudaFree on the request path (those calls can
 * synchronise the device and fail under fragmentation).
 *
 * Executes the circuit's whole-state sweep once, with the values of the
 * output groups and the parameter-shift gradient of F = sum_g f_g, using
 * no allocation at all: every device table and the per-copy values of the
 * shift rule live in one fixed array of 8 MiB (8388608 bytes) that the
 * library declares in device memory (every GPU that loads the library holds
 * it until the process exits).  The caller passes device inputs and outputs:
 *   d_params  float [batch][params_stride] (stride 0: one row shared)
 *   d_inputs  float [batch][n_inputs] or NULL
 *   d_values  double [batch][n_groups]
 *   d_grads   float [batch][n_params]
 * Limits: n_qubits <= 13; the tables plus 8 * batch * (1 + 2 * angles)
 * bytes must fit in the 8 MiB, else ERR_ARG names the size needed.  The
 * first call on a device looks up the array's device address for that device.
 * Every call on a device shares the array, which keeps the last call's
 * contents: calls that overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  Errors found by the kernels are not reported (a NaN
 * parameter gives NaN outputs).  Asynchronous on `stream` (the host tables
 * are staged before the call returns). */
tdq_status tdq_execute_param_shift_noalloc(const tdq_circuit* c, int batch, const float* d_params,
                                           int64_t params_stride, const float* d_inputs, double* d_values,
                                           float* d_grads, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TDQ_ABI_H_ */
