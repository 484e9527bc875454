/*
 * qtc.h — C ABI of the GB300 tensor-network contraction engine for quantum
 * circuits (QAOA Max-Cut), after "qTorch: The quantum tensor contraction
 * handler" (arXiv 1709.03636).
 *
 * The problem (Section 1): given a circuit and an initial state, compute an
 * expectation value <psi|M|psi> (Section 3.3) or an amplitude.  The pipeline
 * follows Sections 2-3: circuit -> closed tensor network -> contraction
 * ordering (Algorithm 1 "LG" or Algorithm 2 "Stoch") -> a sequence of
 * pairwise contractions (Eq. 1) -> scalar.
 *
 * Conventions for every call:
 *  - All functions return a qtc_status; none aborts.  On failure the
 *    thread-local message from qtc_last_error() says why.
 *  - Host arrays passed in are copied before the call returns; the caller
 *    keeps ownership.  Output pointers are owned by the caller.
 *  - "device" pointers are CUDA global-memory addresses on the engine's
 *    device; "host" pointers are ordinary (pageable or pinned) host memory.
 *  - Device memory is never allocated by the library: every device buffer it
 *    uses lives in the arena the caller hands to qtc_engine_create.  The one
 *    allocation it makes is a small pinned, device-mapped host buffer per
 *    engine (allocated by the first host-pointer expectation call, freed by
 *    qtc_engine_destroy) through which such calls pass parameters and
 *    results without copies.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls with host outputs return once their results are in
 *    host memory (for qtc_qaoa_expectation on the shared-memory executor,
 *    before the launch has fully retired: later work on any stream that
 *    needs the launch gone should wait on the stream); calls with device
 *    outputs are asynchronous on it.
 *  - Handles are not thread-safe; use one engine per host thread.
 */
#ifndef QTC_H
#define QTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum qtc_status {
  QTC_OK = 0,
  QTC_ERR_INVALID = 1,     /* bad argument, graph, observable or handle      */
  QTC_ERR_ARENA = 2,       /* the plan needs more arena than was given        */
  QTC_ERR_TIMEOUT = 3,     /* a bounded device-side wait expired              */
  QTC_ERR_CUDA = 4,        /* a CUDA runtime call failed                      */
  QTC_ERR_UNSUPPORTED = 5  /* valid request this build does not implement     */
} qtc_status;

/* Element type of the contraction.  C128 = complex double; C64 = complex
 * float with FP32 accumulation; SPLIT_BF16 = C64, except that contraction
 * steps large enough to be dense GEMMs run on the tensor cores with each
 * FP32 operand split into two BF16 parts (hi + lo) and the three products
 * hi*hi + hi*lo + lo*hi accumulated in FP32. */
typedef enum qtc_dtype { QTC_C128 = 0, QTC_C64 = 1, QTC_SPLIT_BF16 = 2 } qtc_dtype;

/* Gates (Section 2: nodes of the network).  Angles follow
 * RX(t) = exp(-i t X/2), RZ(t) = exp(-i t Z/2), ZZ(t) = exp(-i t Z(x)Z/2);
 * the QAOA phase gate of Section 4.1 is ZZ(gamma) and the mixer
 * exp(-i beta X) is RX(2 beta). */
typedef enum qtc_gate {
  QTC_GATE_H = 0, QTC_GATE_X = 1, QTC_GATE_Y = 2, QTC_GATE_Z = 3,
  QTC_GATE_RX = 4, QTC_GATE_RZ = 5, QTC_GATE_ZZ = 6, QTC_GATE_CNOT = 7,
  /* One-qubit noise channels (Section 2's density-matrix form admits
   * operations that are not unitary): rho -> sum_k K_k rho K_k^dagger with
   * strength s = the gate's constant, 0 <= s <= 1, no parameter slot.
   * DEPOLARIZE: (1-s) rho + s/3 (X rho X + Y rho Y + Z rho Z);
   * DEPHASE: (1-s) rho + s Z rho Z;
   * AMPDAMP: K0 = [[1,0],[0,sqrt(1-s)]], K1 = [[0,sqrt(s)],[0,0]].
   * In the network a channel is one rank-4 tensor joining the ket and bra
   * wires of its qubit; it needs an expectation-value observable (not
   * QTC_OBS_AMPLITUDE). */
  QTC_GATE_DEPOLARIZE = 8, QTC_GATE_DEPHASE = 9, QTC_GATE_AMPDAMP = 10
} qtc_gate;

/* Observables (Section 3.3: <psi|M|psi> for a Pauli string M, or the
 * amplitude <x|psi> of one basis state). */
typedef enum qtc_obs_kind {
  QTC_OBS_ZZ = 0,         /* Z_u Z_v                                        */
  QTC_OBS_IDENTITY = 1,   /* the identity: <psi|psi> = 1 (needs lightcone=0) */
  QTC_OBS_PAULI = 2,      /* pauli[q] in {'I','X','Y','Z'} for q = 0..n-1    */
  QTC_OBS_AMPLITUDE = 3,  /* <x|psi>, x given by bits[q] in {0,1}            */
  QTC_OBS_PROJECTOR = 4   /* <psi| prod_q P_q |psi>: bits[q] = 0 or 1 projects
                           * qubit q on |0> or |1>, 2 leaves it unmeasured;
                           * the probability of the measured outcomes
                           * (Section 3.3).  Every qubit gets one closing
                           * tensor, so with lightcone = 0 all projector
                           * networks of a circuit share one structure
                           * (see qtc_plan_reuse).                           */
} qtc_obs_kind;

typedef struct qtc_observable {
  int kind;               /* qtc_obs_kind                                   */
  int u, v;               /* qubits of QTC_OBS_ZZ                           */
  const char* pauli;      /* QTC_OBS_PAULI: n characters, host              */
  const uint8_t* bits;    /* QTC_OBS_AMPLITUDE, _PROJECTOR: n bytes, host   */
} qtc_observable;

/* Contraction ordering (Section 3.1). */
typedef enum qtc_order_kind {
  QTC_ORDER_STOCH = 0,    /* Algorithm 2: random wire, rank-growth threshold */
  QTC_ORDER_LG = 1        /* Algorithm 1: elimination ordering of the line
                             graph, found by min-fill with random restarts   */
} qtc_order_kind;

typedef struct qtc_plan_opts {
  int kind;               /* qtc_order_kind                                 */
  uint64_t seed;          /* SplitMix64 seed of the random choices          */
  int max_rejections;     /* Stoch: MaxRejections (<= 0 means 10)           */
  int restarts;           /* LG: number of randomised min-fill runs (<=0: 8)*/
  double budget_ms;       /* LG: stop restarting after this long (<=0: none)*/
} qtc_plan_opts;

typedef struct qtc_plan_info {
  int n_tensors;          /* leaves of the network                          */
  int n_labels;           /* distinct indices (wires / hyperedges)          */
  int n_steps;            /* pairwise contractions (Eq. 1)                  */
  int max_rank;           /* largest intermediate rank (width + 1 bound)    */
  double cmacs;           /* complex multiply-adds: sum of 2^(b+x+y+z)      */
  double bytes_c64;       /* algorithmic bytes: sum 8*(|A|+|B|+|C|)         */
  double lg_width;        /* LG: width of the line-graph elimination order  */
} qtc_plan_info;

typedef struct qtc_batch_info {
  int n_networks;
  int n_params;
  int max_rank;           /* over all networks                              */
  int n_steps_total;
  double cmacs;           /* forward, all networks                          */
  double bytes_c64;       /* forward algorithmic bytes, all networks        */
  int n_smem_networks;    /* networks executed entirely in shared memory    */
  int n_global_networks;  /* networks with steps executed from global memory*/
  double grad_cmacs;      /* adjoint sweep only: two contractions per step  */
  double grad_bytes_c64;  /* adjoint sweep only, algorithmic bytes          */
} qtc_batch_info;

typedef struct qtc_program_info {
  int graph;              /* 1: graph executor (waves), 0: one shared-memory launch */
  int n_waves;            /* launches per evaluation                         */
  int n_tasks;            /* tasks over all waves                            */
  int n_global_steps;     /* global-memory contractions over all waves       */
  int n_smem_tasks;       /* shared-memory programs over all waves           */
  int smem_bytes;         /* dynamic shared memory per CTA                   */
  double work_bytes;      /* global work buffer (largest wave)               */
  double table_bytes;     /* device program tables, all waves                */
  int n_gemm_steps;       /* of which split-BF16 tensor-core GEMMs            */
  int warp_teams;         /* 1: shared-memory networks run one per warp      */
  int n_ops;              /* shared-memory ops over all networks (CTA teams) */
  int n_warp_steps;       /* warp steps over all networks (warp teams)       */
  int max_warp_steps;     /* warp steps of the longest network               */
  int n_solo_steps;       /* of the warp steps, those one op runs alone      */
  int stage_ops;          /* ops or warp steps a team stages at a time       */
  /* graph executor: global intermediates and adjoints summed over networks,
   * as placed (tensors whose live ranges do not meet share memory) and with
   * a region of their own per tensor (what reuse saves) */
  double net_global_bytes;
  double net_global_bytes_unshared;
  /* graph executor with the gradient: the most checkpoint segments of any
   * network (1: every forward value stored for the adjoint sweep; k > 1: the
   * network's stored values alone exceed the wave limit, so values used only
   * inside one of k segments are dropped and recomputed by the sweep) */
  int checkpoint_segments;
} qtc_program_info;

typedef struct qtc_engine qtc_engine;
typedef struct qtc_circuit qtc_circuit;
typedef struct qtc_network qtc_network;
typedef struct qtc_plan qtc_plan;
typedef struct qtc_batch qtc_batch;

/* Last error message of the calling thread ("" if none).  Valid until the
 * next failing call on this thread. */
const char* qtc_last_error(void);

/* ---- engine -------------------------------------------------------------
 * An engine binds one CUDA device and one caller-owned device arena
 * [arena, arena + arena_bytes), 256-byte aligned (an arena_bytes that is not
 * a multiple of 256 is rounded down to one).  Plans, intermediates,
 * counters and results are carved from it; the library never calls
 * cudaMalloc.  Program tables grow from the front; the global-memory
 * intermediates of the graph executor use one work buffer at the back,
 * shared by all programs of the engine, so calls on one engine must not
 * overlap on the GPU (issue them on one stream).  The arena must stay valid
 * until qtc_engine_destroy. */
qtc_status qtc_engine_create(int device, void* arena, size_t arena_bytes,
                             qtc_engine** out);
/* Frees the engine's host objects and its mapped host buffer, after waiting
 * for the engine's device to finish (a host-pointer call may return before
 * its launch has retired).  The arena stays the caller's. */
void qtc_engine_destroy(qtc_engine* e);
/* Forget every prepared program, making the whole arena free again. */
qtc_status qtc_engine_reset(qtc_engine* e);

/* ---- circuits (Section 2, Section 4.1) ---------------------------------
 * A circuit has n qubits starting in |0>, a list of gates, and n_params
 * real parameters.  A gate's angle is coeff * params[slot] + constant
 * (slot = -1: constant only). */
qtc_status qtc_circuit_create(int n, int n_params, qtc_circuit** out);
qtc_status qtc_circuit_add_gate(qtc_circuit* c, int gate, const int32_t* qubits,
                                int slot, double coeff, double constant);
/* QAOA Max-Cut circuit of Section 4.1 on the graph with m edges
 * edges[2i], edges[2i+1] (host): H on every qubit, then for k = 1..p the
 * phase gates ZZ(gamma_k) on every edge and RX(2 beta_k) on every qubit.
 * Parameters: slot k-1 = gamma_k, slot p+k-1 = beta_k.  The edge list is
 * kept as the default set of ZZ observables of qtc_batch_create. */
qtc_status qtc_circuit_qaoa(int n, const int32_t* edges, int m, int p,
                            qtc_circuit** out);
/* The same circuit with the channel `channel` (QTC_GATE_DEPOLARIZE, _DEPHASE
 * or _AMPDAMP) of strength `strength` on every qubit after each layer's
 * mixer: the noisy QAOA model.  Parameters and observables as above. */
qtc_status qtc_circuit_qaoa_noisy(int n, const int32_t* edges, int m, int p, int channel,
                                  double strength, qtc_circuit** out);
void qtc_circuit_destroy(qtc_circuit* c);

/* ---- networks (Section 2) ----------------------------------------------
 * Builds the closed network of <psi|M|psi> as a ket network, its complex
 * conjugate (bra) and the observable between them, with bond dimension 2
 * (Section 2 uses dimension-4 superoperator wires; fusing each ket/bra wire
 * pair gives that form back).  lightcone != 0 keeps only the gates in the
 * reverse light cone of the observable.  diag_mode != 0 attaches diagonal
 * gates (ZZ, RZ, Z) to the wire they act on, so one index may be shared by
 * more than two tensors, and gives CNOT its sparse form: the control wire
 * passes through and the target gets a rank-3 tensor t_out = t_in xor c
 * (the gate sparsity Sections 5-6 name as missing); diag_mode = 0 gives
 * every gate its own input and output wires (rank-4 ZZ and CNOT tensors).
 * A leading H on |0> is folded into the state |+>. */
qtc_status qtc_network_build(const qtc_circuit* c, const qtc_observable* obs,
                             int lightcone, int diag_mode, qtc_network** out);
/* Leaves of a network, for inspection.  counts: host, 2 ints
 * (n_leaves, n_labels).  Each array may be NULL; otherwise it holds n_leaves
 * entries (labels: 4 per leaf, unused slots -1), host:
 * kind (LeafKind code, see device_program.h), conj (1 = bra side, values
 * complex-conjugated), slot/coeff/constant (angle = coeff*params[slot] +
 * constant), labels in storage order (label k = bit k of the element index). */
/* Leaf `leaf` of a network evaluated on the host at `params` (host,
 * n_params doubles): the tensor of the gate, state, observable or channel of
 * Section 2 that the executors build, 2^rank complex elements as interleaved
 * (re, im) doubles in val (host), and d/dparams[slot] of each in der (host,
 * nullable; zeros for a leaf without a parameter).  Element index bit k is
 * label k of qtc_network_leaves.  QTC_ERR_INVALID for a leaf out of range. */
qtc_status qtc_network_leaf_values(const qtc_network* n, int leaf, const double* params,
                                   double* val, double* der);
qtc_status qtc_network_leaves(const qtc_network* n, int32_t* counts, int32_t* kind,
                              int32_t* conj, int32_t* slot, double* coeff,
                              double* constant, int32_t* labels);
void qtc_network_destroy(qtc_network* n);

/* ---- plans (Section 3.1, Algorithms 1 and 2) ---------------------------- */
qtc_status qtc_plan_create(const qtc_network* n, const qtc_plan_opts* opts,
                           qtc_plan** out);
/* A plan for network n with the contraction tree of `like`, without a new
 * ordering search: n must have the same structure (leaf count, and every
 * leaf's labels) as like's network; only the tensor values may differ (e.g.
 * the projector networks of one circuit, Section 3.3's sequence of
 * contractions reusing one ordering).  QTC_ERR_INVALID otherwise. */
qtc_status qtc_plan_reuse(const qtc_plan* like, const qtc_network* n, qtc_plan** out);
qtc_status qtc_plan_stats(const qtc_plan* p, qtc_plan_info* info);
/* Writes the contraction tree: for step s, operands (lhs[s], rhs[s]) are
 * tensor ids (0..n_tensors-1 leaves, n_tensors+t the result of step t).
 * Arrays hold n_steps entries (host). */
qtc_status qtc_plan_steps(const qtc_plan* p, int32_t* lhs, int32_t* rhs);
/* Every step as Eq. 1's index classes (the step lowering of Section 3.1's
 * pairwise contractions): shapes[4s .. 4s+3] = (b, x, y, z), the numbers of
 * batch labels (held by both operands and kept), free labels of the first
 * operand, summed labels, and free labels of the second operand, so that
 * rank A = b + x + y, rank B = b + y + z, rank C = b + x + z and the step
 * costs 2^(b+x+y+z) complex multiply-adds.  shapes: host, 4 * n_steps ints. */
qtc_status qtc_plan_step_shapes(const qtc_plan* p, int32_t* shapes);
void qtc_plan_destroy(qtc_plan* p);

/* Contract one network on the GPU (Eq. 1 applied step by step).
 * params: host, n_params values.  out_re_im: host, 2 doubles (the scalar
 * <psi|M|psi> or <x|psi>).  grad_re_im: host, nullable, 2*n_params doubles:
 * d(scalar)/d(params[k]) as (re, im) pairs, by the adjoint sweep. */
qtc_status qtc_contract(qtc_engine* e, const qtc_plan* p, const double* params,
                        int dtype, void* stream, double* out_re_im,
                        double* grad_re_im);

/* ---- QAOA batches (all edge networks of one graph) ---------------------
 * One <Z_u Z_v> network per observable edge obs_edges[2i], [2i+1] (host;
 * NULL = the circuit's QAOA edges), each with its own plan. */
qtc_status qtc_batch_create(const qtc_circuit* c, const int32_t* obs_edges,
                            int m, int lightcone, int diag_mode,
                            const qtc_plan_opts* opts, qtc_batch** out);
qtc_status qtc_batch_stats(const qtc_batch* b, qtc_batch_info* info);
void qtc_batch_destroy(qtc_batch* b);

/* Edge networks are independent (the objective of Section 4.1 is a sum over
 * edges), so one graph shards over devices or processes with a single sum of
 * the 1 + 2p results at the end.  qtc_batch_partition assigns each network of
 * b to one of n_parts parts by longest processing time first on its
 * algorithmic bytes (forward, plus the adjoint sweep when want_grad): the
 * costliest remaining network goes to the part with the least work so far.
 * part_of_net: host, n_networks ints (0..n_parts-1) out; part_cost: host,
 * nullable, n_parts doubles out (bytes per part).  Host only, deterministic:
 * every process computes the same partition without communication. */
qtc_status qtc_batch_partition(const qtc_batch* b, int n_parts, int want_grad,
                               int32_t* part_of_net, double* part_cost);
/* A new batch holding networks nets[0..k-1] of b (host, k ints), with their
 * observables, weights and plans as they are in b (no new ordering search), so
 * that a part's results are those of the same networks in the whole batch.
 * Its expectation calls return the part's share: <C> and the gradient summed
 * over its networks only. */
qtc_status qtc_batch_subset(const qtc_batch* b, const int32_t* nets, int k, qtc_batch** out);

/* Builds, validates and describes the batch's device program on the host
 * only (no GPU call): every access range, counter and dependency order of a
 * graph program is checked against its buffers.  force_graph, small_rank and
 * max_wave_bytes as in qtc_engine_set_graph_options / qtc_engine_set_limits;
 * smem_limit: shared memory per CTA to plan for (0: 227 KiB). */
qtc_status qtc_batch_program_info(qtc_batch* b, int dtype, int want_grad, int force_graph,
                                  int small_rank, size_t max_wave_bytes, size_t smem_limit,
                                  qtc_program_info* info);

/* Launch configuration of the batch's prepared program on this engine
 * (prepares it when needed): grid and block size, dynamic shared memory per
 * CTA, CTAs resident per SM, launches per evaluation, tensor-memory columns
 * per CTA (0: no tensor-core tasks).  out: host, 6 ints. */
qtc_status qtc_batch_launch_info(qtc_engine* e, qtc_batch* b, int dtype, int want_grad,
                                 int32_t* out);

/* Upload the batch's device program for (dtype, want_grad) into the arena.
 * Optional: the expectation calls below prepare on first use. */
qtc_status qtc_batch_prepare(qtc_engine* e, qtc_batch* b, int dtype,
                             int want_grad, void* stream);

/* <C> = sum_i (1 - <Z_u Z_v>_i)/2 over the batch's edges (Eqs. for the
 * Max-Cut objective and its clauses, Section 4.1), and its gradient.
 * gammas, betas: host, p values each.  C_out: host, 1 double.
 * per_edge_out: host, nullable, m doubles <Z_u Z_v>_i.
 * grad_out: host, nullable (needs want_grad), 2p doubles
 * d<C>/d(gamma_1..p, beta_1..p).  One launch per wave: the kernel reads the
 * parameters from and writes the results to the engine's mapped host buffer.
 * With the shared-memory executor the kernel then stores a per-call sequence
 * number there after a system-scope fence, and the call returns when it reads
 * that number (or when `stream` is idle); the graph executor synchronises
 * `stream`.  A launch or kernel error is returned either way.  <C> and the
 * gradient are FP64 sums over the edge networks; with the shared-memory
 * executor the terms are added in no fixed order (atomics), so repeated
 * calls can differ in the last bits. */
qtc_status qtc_qaoa_expectation(qtc_engine* e, qtc_batch* b,
                                const double* gammas, const double* betas,
                                int dtype, int want_grad, void* stream,
                                double* C_out, double* per_edge_out,
                                double* grad_out);

/* Same computation with device-resident inputs and outputs, asynchronous
 * on `stream` (no host synchronisation; capturable in a CUDA graph once the
 * batch is prepared).  params_dev: device, 2p doubles (gammas then betas).
 * out_dev: device, 2 + 2p + m doubles: [<C>, d<C>/dtheta (2p, zeros when
 * want_grad = 0), <Z_u Z_v> per edge (m), status] where status is 0, or
 * QTC_ERR_TIMEOUT (3) when a bounded device-side dependency wait expired
 * (the values are then invalid).  One kernel launch per wave: batches whose
 * networks all fit one CTA's shared memory run in one launch; larger ones
 * run in waves whose global intermediates stay under the engine's limit. */
qtc_status qtc_qaoa_expectation_device(qtc_engine* e, qtc_batch* b,
                                       const double* params_dev, int dtype,
                                       int want_grad, void* stream,
                                       double* out_dev);

/* Number of kernel launches the last expectation or contract call on this
 * engine issued (for launch accounting). */
int qtc_engine_last_launches(const qtc_engine* e);

/* Limits of the graph executor (networks too large for one CTA's shared
 * memory): max_wave_bytes bounds the global-memory intermediates of the
 * networks contracted in one launch (default 8 GiB; a network needing more
 * returns QTC_ERR_ARENA), wait_limit_ms bounds every device-side wait for a
 * producer task (default 10000 ms; on expiry the launch stops early and the
 * status reads QTC_ERR_TIMEOUT).  Invalidates prepared programs. */
qtc_status qtc_engine_set_limits(qtc_engine* e, size_t max_wave_bytes, double wait_limit_ms);

/* Program formation (tests and tuning): force_graph != 0 runs every
 * network through the graph executor even when it fits one CTA's shared
 * memory; small_rank > 0 moves every tensor of higher rank to global memory
 * (default 10).  Invalidates prepared programs. */
qtc_status qtc_engine_set_graph_options(qtc_engine* e, int force_graph, int small_rank);

/* Task shapes (tuning; see the autotuner of the Python package): a chunk
 * task of a global step of the graph executor covers about
 * 2^task_terms_log2 multiply-adds (12..20, default 16); a shared-memory
 * subtree task holds at most subtree_bytes of values (4096..32768, default
 * 32768); warp_teams: 0 keeps the shared-memory executor at one network per
 * CTA, 1 (default) runs one network per warp where the network's program
 * fits, 2 does so with the warp steps always read from global memory
 * (complex64 only); graph_hi_occupancy != 0 runs complex64 graph programs
 * without tensor-core tasks on a kernel build capped for five CTAs per SM
 * (default 0: four).  Invalidates prepared programs.  QTC_ERR_INVALID
 * outside those ranges. */
qtc_status qtc_engine_set_task_options(qtc_engine* e, int task_terms_log2, int subtree_bytes,
                                       int warp_teams, int graph_hi_occupancy);

/* Tile form of the graph executor's global steps (tuning and tests): 0
 * (default) keeps every step on the row and split chunk paths; 1 stages the
 * steps with both operands in global memory, and the long reductions,
 * through shared memory in tiles (16-byte copies of each operand's tile,
 * contraction in shared memory and registers); 2 does so for every step that
 * tiles; 3 reads the operands of steps summing at least three labels in
 * place (tile decomposition without staging copies) and 4 does so for every
 * step that tiles.
 * Invalidates prepared programs.  QTC_ERR_INVALID outside 0..4. */
qtc_status qtc_engine_set_tile_mode(qtc_engine* e, int mode);

/* Host-only check of the tile lowering (no GPU call): builds the batch's
 * graph program with force_graph, small_rank and tile_mode as above and, for
 * every tile step with at most 2^max_bits multiply-adds, emulates its tile
 * copies, thread decomposition and reductions on seeded random operands and
 * compares the result with the plain contraction over the step's bit maps.
 * Steps whose rows go four at a time sharing operand elements are emulated
 * the same way (row order, the group's distinct elements).
 * max_err: host, 1 double (largest absolute difference); n_checked: host,
 * 1 int (steps compared). */
qtc_status qtc_selftest_tile_steps(qtc_batch* b, int dtype, int want_grad, int force_graph,
                                   int small_rank, int tile_mode, int max_bits,
                                   double* max_err, int32_t* n_checked);

/* Launches a one-task program whose task waits for a counter nothing ever
 * signals, so that the bounded wait expires after the engine's wait limit and
 * the kernel returns normally.  Returns QTC_ERR_TIMEOUT when the bound works
 * (anything else is a failure).  Used by the failure-detection tests. */
qtc_status qtc_selftest_wait_timeout(qtc_engine* e, void* stream);

/* ---- answer strings (Section 3.3) ----------------------------------------
 * The sequential estimate of a likely output string: for q = 0..n-1,
 * contract <psi| prod P |psi> with qubits 0..q-1 projected on the values
 * already chosen, qubit q on |0> and the others traced out (n contractions of
 * networks that share one structure, so the first plan's contraction tree,
 * ordered by `opts`, is reused for all), compare P(prefix, x_q = 0) with
 * P(prefix) - P(prefix, x_q = 0) and keep the likelier value; an exact tie
 * is broken by a SplitMix64 stream seeded with tie_seed.  params: host,
 * n_params values (nullable when the circuit has none); opts: host, nullable
 * (LG defaults).  bits_out: host, n bytes (0 or 1); probs_out: host, n
 * doubles, the probability of each chosen prefix.  Synchronous; the circuit
 * may hold noise channels (density-matrix marginals). */
qtc_status qtc_answer_string(qtc_engine* e, const qtc_circuit* c, const double* params,
                             int dtype, const qtc_plan_opts* opts, uint64_t tie_seed,
                             void* stream, uint8_t* bits_out, double* probs_out);

/* ---- full-Hilbert-space reference (Section 5's comparison method) ---------
 * <C> of a QAOA circuit (qtc_circuit_qaoa) from the 2^n state vector on the
 * GPU: |+>^n, per layer the diagonal phase and the RX mixer, moved through
 * shared memory in tiles of up to 12 qubits per pass.  n <= 32, m <= 512; the
 * state lives in the engine's work buffer (2^n * 8 or 16 bytes).  per_edge
 * != 0 also computes <Z_a Z_b> per edge (extra passes).  dtype C128 or C64.
 * Host form: gammas, betas (p each) in, C_out (1) and per_edge_out
 * (nullable, m) out, synchronous.  Device form: params_dev (2p doubles),
 * out_dev (1 + m doubles: <C>, then <Z_a Z_b> per edge when per_edge),
 * asynchronous on `stream`. */
qtc_status qtc_statevector_qaoa(qtc_engine* e, const qtc_circuit* c, const double* gammas,
                                const double* betas, int dtype, int per_edge, void* stream,
                                double* C_out, double* per_edge_out);
qtc_status qtc_statevector_qaoa_device(qtc_engine* e, const qtc_circuit* c,
                                       const double* params_dev, int dtype, int per_edge,
                                       void* stream, double* out_dev);

/* ---- evaluation without device allocation --------------------------------
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory at all (code running inside another
 * framework's memory pool, or a plugin whose host forbids cudaMalloc), so
 * they cannot hand the library an arena either.  It computes exactly what
 * qtc_qaoa_expectation_device computes, on the caller's current device,
 * with the same inputs and outputs: params_dev (device, 2p doubles) and
 * out_dev (device, 2 + 2p + m doubles, same layout), for batches whose
 * networks all fit one CTA's shared memory (others: QTC_ERR_UNSUPPORTED).
 *
 * Its scratch (program tables, per-network result rows, counters) is a
 * fixed file-scope device array of QTC_STATIC_SCRATCH_BYTES, which every GPU
 * that loads the library keeps until the process exits.  The call allocates
 * no device memory and calls no allocating CUDA or library routine; a batch
 * whose program does not fit returns QTC_ERR_ARENA with the size it needs.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, no allocation); the first call on a device also
 * loads the library's device code there, so make it before any stream
 * capture.  The host-side program is built once per batch and cached; when a
 * call brings a batch other than the previous call's, it first copies that
 * batch's program tables into the array from pageable host memory on
 * `stream`, so run every batch through this call once before any stream
 * capture that contains it.
 * Every call shares the one array and leaves its contents behind (the call
 * clears the counters it needs zeroed), so calls whose executions overlap on
 * the GPU — from two streams or two host threads — race and must not be
 * issued.  Asynchronous on `stream`. */
#define QTC_STATIC_SCRATCH_BYTES (16u << 20)
qtc_status qtc_qaoa_expectation_static(qtc_batch* b, const double* params_dev, int dtype,
                                       int want_grad, void* stream, double* out_dev);

#ifdef __cplusplus
}
#endif
#endif /* QTC_H */
