/*
 * qn.h -- C ABI of libqnoise: stochastic noisy-QAOA trajectory ensembles on one
 * GB300 (sm_103a).
 *
 * Method (arXiv 2210.15874, Sec. "Stochastic Noise Implementation"): every
 * member of an ensemble of K circuits re-applies the ideal circuit's gates in
 * order; after each gate a uniform number per noise channel picks a Kraus
 * operator, which is applied to the state.  The output probability vector of
 * each member, phi = |psi|^2, is averaged: sigma_approx = sum_k phi_k / K.
 * The expectation of the MaxCut cost C (Sec. "Quantum Approximate Optimization
 * Algorithm") is averaged the same way.
 *
 * Conventions fixed by this library (the paper leaves them open):
 *   - Circuit: H on every qubit, then for l = 1..p: for every edge (i, j) in the
 *     given order the phase gate diag(1, e^{-i gamma_l}, e^{-i gamma_l}, 1) on
 *     (i, j), then exp(-i beta_l X) on qubits 0..n-1 in order.
 *     Basis index bit q is qubit q.  C(x) = #edges (i, j) with x_i != x_j.
 *   - Noise after every gate (the H layer included), in the order: gate, one
 *     depolarizing Pauli on the gate's qubits, amplitude damping on the first
 *     qubit, amplitude damping on the second qubit.
 *   - Pauli codes: 1q 0..3 = I, X, Y, Z; 2q 4a+b with a on the edge's first
 *     qubit.  Code k is the first with w0 < floor(2^32 * (P_0 + .. + P_k)) (sums in
 *     FP64, in code order); the last code takes the rest.
 *   - Randomness: Philox4x32-10 with key (seed_lo, seed_hi), counter
 *     (gate index, 0, t_lo, t_hi) for global trajectory id t.  Word 0 picks the
 *     Pauli; words 1 and 2 are the damping draws u = (w + 0.5) * 2^-32 of the
 *     gate's first and second qubit.  Results of trajectory t therefore do not
 *     depend on the launch batch size or on which batch t falls in.
 *   - Damping (textbook Kraus pair K0 = diag(1, sqrt(1-gamma)),
 *     K1 = sqrt(gamma) |0><1|): K1 is chosen when u < gamma * P(qubit = 1); the
 *     state is renormalised after each site.
 *
 * Status and threading: every call returns a qn_status and never throws.  A
 * handle is not thread-safe; distinct handles are independent.  Work is queued
 * on the handle's stream; qn_expectation, qn_probs, qn_traj_debug, qn_grad and
 * qn_profile_read synchronise that stream.  On any non-OK status,
 * qn_last_error() returns a thread-local message describing it.
 */
#ifndef QN_H
#define QN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QN_OK = 0,
    QN_EINVAL = 1,   /* invalid argument; nothing was launched */
    QN_ENOMEM = 2,   /* device allocation failed or the footprint exceeds free memory */
    QN_ECUDA = 3,    /* a CUDA runtime call failed (message has the CUDA error string) */
    QN_ETIMEOUT = 4, /* reserved: a bounded device-side wait gave up */
    QN_ESTATE = 5    /* wrong call order (e.g. results before a run) or a kernel flagged a
                        non-finite or zero norm */
} qn_status;

/* Opaque handle.  Owns its device memory (or memory from the allocator set below). */
typedef struct qn_batch qn_batch;

/* Problem graph, host memory, read during qn_run_qaoa only.
 *   n          number of vertices = qubits, 1 <= n <= 30
 *   num_edges  number of edges, >= 0
 *   edges      2*num_edges int32: edge e is (edges[2e], edges[2e+1]); 0 <= v < n,
 *              endpoints distinct, no duplicate edge.  The order is the order in
 *              which the phase gates are applied. */
typedef struct {
    int32_t n;
    int32_t num_edges;
    const int32_t *edges;
} qn_graph;

/* Noise model (Sec. "Modeling Noise"; depolarizing Kraus set of that section).
 *   p1, p2     depolarizing strength after 1q and 2q gates.
 *              param = 0: p is the total non-identity probability; each 1q Pauli
 *              has p/3, each 2q non-II Pauli p/15 (p1 <= 1, p2 <= 1).
 *              param = 1: the paper's lambda, K0 = sqrt(1 - 3 lambda/4) I, so the
 *              1q Pauli total is 3 lambda/4 (lambda <= 4/3) and the 2q total is
 *              15 lambda/16 (lambda <= 16/15).
 *   damping    amplitude-damping gamma in [0, 1] after every gate on each of its
 *              qubits (0 disables damping).
 *   twoq_mode  0: 15-Pauli two-qubit depolarizing channel after a 2q gate;
 *              1: independent 1q channels of strength p2 on both qubits (Fig. 2's
 *              per-qubit noise on a 2q gate). */
typedef struct {
    double p1, p2, damping;
    int32_t twoq_mode;
    int32_t param;
} qn_noise;

/* Create a handle for n qubits (1..30) and an ensemble of `trajectories` (>= 1)
 * members drawn from `seed`.  No device memory is allocated until the first
 * run.  *out receives the handle (caller frees with qn_batch_destroy). */
qn_status qn_batch_create(int32_t n, int64_t trajectories, uint64_t seed, qn_batch **out);

/* Set the CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream;
 * NULL = legacy default stream) on which all later work of the handle is queued. */
qn_status qn_batch_set_stream(qn_batch *h, void *cuda_stream);

/* Route device allocations through alloc(bytes, ctx) / free(ptr, ctx) (e.g. the
 * PyTorch caching allocator).  Must be called before the first run.  alloc must
 * return memory aligned to at least 256 bytes, or NULL on failure. */
qn_status qn_batch_set_allocator(qn_batch *h, void *(*alloc)(size_t, void *),
                                 void (*free_fn)(void *, void *), void *ctx);

/* Trajectories evolved per launch (B).  0 (the default) picks
 * B = min(trajectories, max(1, 512 MiB / (8 * 2^n))).  Statevectors take
 * 8 * 2^n * B bytes of HBM (complex64). */
qn_status qn_batch_set_launch_batch(qn_batch *h, int64_t B);

/* Fused layers (on = 1, the default; 0 = one sweep per gate).  With Pauli-only
 * noise (damping == 0) no branch depends on the state, so each QAOA layer is
 * applied as a few sweeps instead of E + n: the cost layer (every phase gate
 * and every Pauli's Z part) is one diagonal factor folded into a mixer sweep,
 * and the mixer rotations are applied in windows of consecutive qubits -- for
 * n >= 10 a first window of qubits 0-11 where that makes fewer windows than
 * qubits 0-7 does (n = 16-19, 23-26, 30), then windows of at most 7 over the
 * rest (2 sweeps per layer at n = 16, 3 at n = 20-26, 4 at n = 30); below 10
 * qubits five per sweep.  Needs
 * at most 64 edges; otherwise gates are swept one by one.  With damping == 0
 * fusion takes precedence over shared-prefix mode.  With damping, fusion acts
 * in shared-prefix mode only: consecutive phase gates of a layer on at most 10
 * qubits form a group whose damping branches are all drawn from one joint
 * distribution of those qubits, and the group is applied in one sweep; for
 * n >= 12 the mixer rotations go in blocks -- qubits 0-7 (the sweep of the
 * layer's last phase group rotates qubits 0-3, the block's own sweep qubits
 * 4-7), then four qubits per sweep -- each block's damping drawn from the joint
 * of its qubits after its rotations (the same Kraus draws as gate by gate; the
 * state differs by FP32 rounding).  Without shared-prefix
 * mode damping runs are swept gate by gate. */
qn_status qn_batch_set_fusion(qn_batch *h, int32_t on);

/* Arithmetic of the fused layers (Pauli-only noise, fusion on, n >= 11):
 *   0  FP32 on the CUDA cores, the windows of qn_batch_set_fusion (the default);
 *   1  TF32 tensor cores: the mixer rotations of five qubits per sweep as two
 *      GEMMs with the +-1 Hadamard matrix (exp(-i beta X) = H diag(e^{-i beta},
 *      e^{i beta}) H), TF32 operands, FP32 accumulation (ceil(n / 5) sweeps per
 *      layer);
 *   2  the same with BF16x3 operands: each FP32 value split exactly into three
 *      bf16 terms, whose products with the +-1 matrix are exact (FP32
 *      accumulation: about FP32 accuracy).
 * A choice of arithmetic with no counterpart in the paper: every mode draws the
 * same Kraus operators (Sec. "Stochastic Noise Implementation") and differs only
 * by rounding.  Other runs ignore the setting.  QN_EINVAL for another mode. */
qn_status qn_batch_set_precision(qn_batch *h, int32_t mode);

/* Shared-prefix mode (on = 1; default 0).  Trajectories whose Kraus strings
 * agree so far share one statevector; when a trajectory's own Pauli or damping
 * draw differs from the shared branch it forks into a copy.  Every trajectory
 * sees exactly the draws it would see alone; with fusion off results equal the
 * default mode's up to FP summation order, with fusion on (phase-gate groups,
 * see qn_batch_set_fusion) up to FP32 rounding of the states.  Only the work on
 * common prefixes is done once.  A launch batch then holds up to B distinct states
 * (default B: a quarter of the free device memory, capped by trajectories).
 * qn_traj_debug and qn_grad are unaffected (they re-simulate trajectories one by
 * one). */
qn_status qn_batch_set_sharing(qn_batch *h, int32_t on);

/* How the launches of a shared-prefix run are sized (an execution choice with no
 * counterpart in the paper; results are the same in every mode up to the order of
 * FP64 sums, and the Kraus strings, states and <C>_t bit-identical):
 *   0  on the host: after every decide the host reads the live-slot count and sizes
 *      the next sweep's grid from it (the default);
 *   1  on the device: every sweep is a persistent launch whose blocks stride over the
 *      slots the device counts, every decide kernel reads the live count on the
 *      device, and the sigma pass takes its slot order and row blocks from device
 *      steps; the host reads nothing until the run is over (one wait at its end
 *      instead of one per group of gates);
 *   2  as 1, with the run after the noisy H layer captured in a CUDA graph on the
 *      handle's first run of a circuit and replayed by later runs whose circuit,
 *      noise, launch batch and buffers are the same (any seed, offset or trajectory
 *      count that keeps the launch batch); a run of another circuit captures again
 *      and updates the instantiated graph in place when its launches have the same
 *      shape.  Profiling (qn_batch_set_profiling) does not see replayed launches.
 * Other runs ignore the setting.  QN_EINVAL for another mode. */
qn_status qn_batch_set_launch_mode(qn_batch *h, int32_t mode);

/* Graph use of a handle in launch mode 2: runs that captured (and instantiated or
 * updated) a graph, runs that replayed one, and captures that updated the existing
 * graph in place.  Any pointer may be NULL. */
qn_status qn_graph_info(const qn_batch *h, int64_t *captures, int64_t *replays, int64_t *updates);

/* Global id of the handle's first trajectory (default 0): the handle evolves
 * trajectories first_trajectory .. first_trajectory + trajectories - 1, so
 * disjoint ranges on several handles or GPUs are shards of one ensemble whose
 * results do not depend on the sharding.  Resets the last run's results. */
qn_status qn_batch_set_offset(qn_batch *h, int64_t first_trajectory);

/* Evolve the whole ensemble through the noisy QAOA circuit of depth p with
 * angles gammas[p], betas[p] (host, radians) and accumulate, in FP64, the
 * ensemble sums of <C>_t, <C>_t^2 and |psi_t|^2 (Sec. "Stochastic Noise
 * Implementation": phi, sigma_approx).  p >= 0.  Asynchronous on the handle's
 * stream; previous results of the handle are replaced. */
qn_status qn_run_qaoa(qn_batch *h, const qn_graph *graph, int32_t p, const double *gammas,
                      const double *betas, const qn_noise *noise);

/* Ensemble mean of C, sum_t <C>_t / K, and its standard error
 * sqrt((S2/K - mean^2) / K).  Host outputs; blocks on the stream. */
qn_status qn_expectation(const qn_batch *h, double *mean, double *std_err);

/* sigma_approx = sum_t |psi_t|^2 / K (Sec. "Stochastic Noise Implementation")
 * into the caller's host buffer out[len], len == 2^n, each psi_t normalised.
 * The norms are exact to FP32 rounding of the states (a shared-prefix run that
 * ends on a full mixer block takes them from the joint the block was drawn
 * from), so the ensemble sum has mass K to that accuracy; it is scaled to unit
 * mass exactly.  QN_ESTATE if the mass is not positive and finite.  Blocks on
 * the stream. */
qn_status qn_probs(const qn_batch *h, double *out, int64_t len);

/* Ensemble gradient d<C>/d gamma_l and d<C>/d beta_l (host outputs, p values
 * each) of the last run's circuit.  Every trajectory is unitary when the noise
 * is Pauli-only, so the gradient is taken per trajectory by the adjoint method
 * and averaged.  Requires a previous qn_run_qaoa with damping == 0, else
 * QN_EINVAL.  Blocks on the stream. */
qn_status qn_grad(qn_batch *h, double *dgamma, double *dbeta);

/* Per-trajectory gradient of <C>_t for trajectories t0..t0+count-1 (0-based within the handle) of
 * the last run (damping == 0): dgamma[count*p], dbeta[count*p], row-major by
 * trajectory.  Host outputs; blocks on the stream. */
qn_status qn_grad_traj(qn_batch *h, int64_t t0, int64_t count, double *dgamma, double *dbeta);

/* Re-simulate trajectories t0..t0+count-1 (0-based within the handle) of the last run (same seed,
 * graph, angles, noise) and return, into caller-owned host buffers (any may be
 * NULL):
 *   amps        count * 2^n * 2 floats: final normalised statevector, (re, im)
 *               interleaved, basis index x (bit q = qubit q);
 *   branches    count * G bytes, G = n + p (E + n): per gate, Pauli code in bits
 *               0..3, K1 on the first qubit in bit 4, on the second in bit 5;
 *   c_per_traj  count doubles: <C>_t = sum_x |psi_t,x|^2 C(x).
 * The ensemble results of the last run are left unchanged.  Blocks. */
qn_status qn_traj_debug(qn_batch *h, int64_t t0, int64_t count, float *amps, uint8_t *branches,
                        double *c_per_traj);

/* The per-trajectory results of the last run in shared-prefix mode, read from
 * the states and draws that run itself made (Sec. "Stochastic Noise
 * Implementation": each member's Kraus string and its phi = |psi|^2) -- no
 * re-simulation, unlike qn_traj_debug.  Trajectories t0..t0+count-1 (0-based
 * within the handle) must lie in the run's last prefix tree (with the default
 * launch batch, the whole ensemble).  Into caller-owned host buffers (any may
 * be NULL), laid out as for qn_traj_debug:
 *   amps        count * 2^n * 2 floats: the final normalised state of each
 *               trajectory's slot, in the true basis with the trajectory's
 *               global phase; when the circuit's last mixer block was left
 *               pending (its sweep formed only the norms and the sigma pass
 *               applied it), the block is applied here to the slot's state (a
 *               slot forked at the block: its parent's) with the drawn factors;
 *   branches    count * G bytes: the Kraus string the run drew for each
 *               trajectory (Pauli code in bits 0..3, damping jumps in bits 4, 5);
 *               with phase groups and mixer blocks, the group decide's draws;
 *   c_per_traj  count doubles: <C>_t as the sigma pass formed it.
 * QN_ESTATE when the last run did not evolve shared prefixes, or when
 * qn_traj_debug, qn_grad or qn_grad_traj has run since (they reuse its
 * buffers); QN_EINVAL for a range outside the last prefix tree.  Blocks. */
qn_status qn_shared_readout(qn_batch *h, int64_t t0, int64_t count, float *amps, uint8_t *branches,
                            double *c_per_traj);

/* Error = 1 - (sum_x sqrt(sa_x se_x))^2 (Sec. "Stochastic Noise Implementation",
 * Eq. 1): fidelity distance between two host probability vectors of length
 * len.  Host-only; any negative entry gives QN_EINVAL. */
qn_status qn_fidelity_error(const double *sa, const double *se, int64_t len, double *out);

/* Counts of the last run: G gates per circuit, the library kernel launches it
 * queued, the statevector bytes its gate sweeps read and wrote (algorithmic:
 * 16 B per amplitude per sweep), and the number of distinct statevectors it
 * evolved (= trajectories, or the distinct Kraus strings in shared-prefix
 * mode).  Any output may be NULL. */
qn_status qn_run_info(const qn_batch *h, int64_t *gates, int64_t *launches, double *sweep_bytes, int64_t *states);

/* The gate groups of shared-prefix mode with damping and fusion on -- a view
 * of the schedule qn_run_qaoa uses (no counterpart in the paper; host only,
 * no device memory).  For an n-qubit graph and depth p, writes up to
 * `capacity` groups in circuit order: kind (0 = consecutive phase gates of a
 * layer on at most 10 qubits, at most 12 gates; 1 = a block of consecutive
 * mixer rotations, present when n >= 12), first gate (the noisy H layer is
 * gates 0 .. n-1), number of gates, and the group's qubits as a bit mask.
 * *count is the number of groups, also when it exceeds capacity.  Output
 * arrays may be NULL when capacity is 0.  QN_EINVAL on an invalid graph or
 * p < 0. */
qn_status qn_group_plan(int32_t n, const qn_graph *graph, int32_t p, int32_t capacity, int32_t *kind,
                        int32_t *first_gate, int32_t *gates, uint32_t *qubit_mask, int32_t *count);

/* The window schedule of the fused layers with Pauli-only noise -- a view of
 * the schedule qn_run_qaoa and qn_grad use (no counterpart in the paper; host
 * only, no device memory).  reverse = 0: the FP32 forward windows of one
 * layer, each one sweep with the cost diagonal folded into a sweep (below 10
 * qubits five per window; from 10 on qubits 0-11 or 0-7 first, the one that
 * leaves fewer windows, then balanced windows of at most 7).  reverse = 1: the
 * mixer windows of the fused adjoint of one layer (from 12 qubits on qubits
 * 0-9, then balanced windows of at most 6, the last of which also undoes the
 * cost diagonal; below 12 qubits 0 .. min(4, n)-1, then windows of two or
 * three, followed by a sweep of its own for the diagonal).  Writes up to
 * `capacity` windows (first qubit, qubits) in sweep order; *count is the
 * number of windows, also when it exceeds capacity.  The output arrays may be
 * NULL when capacity is 0.  QN_EINVAL unless 2 <= n <= 30 and reverse is 0 or
 * 1. */
qn_status qn_fused_windows(int32_t n, int32_t reverse, int32_t capacity, int32_t *q_lo, int32_t *qubits,
                           int32_t *count);

/* Tile map of the sweep of the mixer block on qubits q_lo .. q_lo + m - 1
 * whose next block has m_next qubits (q_lo + m .. q_lo + m + m_next - 1; 0:
 * no next block) -- exposed for tests (no counterpart in the paper; host
 * only).  A float4 index f holds amplitudes 2f and 2f + 1, so f bit b is
 * amplitude bit b + 1 and qubit 0 is inside the float4.  Writes the f bits
 * that go to lanes (lane_bits[3]), that hold the block's qubits (a_bits[4],
 * padded with free bits), the next block's (b_bits[4], padded), and the
 * remaining ones that number tiles (tile_bits[32], *ntile of them).
 * QN_EINVAL unless 12 <= n <= 30, 1 <= m <= 4, 0 <= m_next <= 4 and the qubits
 * fit below n. */
qn_status qn_mix_tile_map(int32_t n, int32_t q_lo, int32_t m, int32_t m_next, int8_t *lane_bits, int8_t *a_bits,
                          int8_t *b_bits, int8_t *tile_bits, int32_t *ntile);

/* Kernel timing with CUDA events recorded on the handle's stream: period = 0
 * (default) records none; period = k >= 1 brackets every k-th gate-sweep
 * launch and every init / observable launch with an event pair.  An event pair
 * stops the next sweep from overlapping the previous one's tail, so a period
 * above 1 keeps the timed stream representative. */
qn_status qn_batch_set_profiling(qn_batch *h, int32_t period);

/* Totals since the last read, for kernel family `kind` (0 = gate sweeps, 1 =
 * state init, 2 = ensemble accumulation, 3 = phase-group sweeps of
 * shared-prefix mode: joint passes and apply sweeps, 4 = mixer-block sweeps of
 * shared-prefix mode): launches, summed event milliseconds and algorithmic
 * bytes.  Kinds 0, 3 and 4 share one sampling counter.  Synchronises the
 * stream, then resets the totals. */
qn_status qn_profile_read(qn_batch *h, int32_t kind, int64_t *launches, double *ms, double *bytes);

/* Allocation-free variant of qn_run_qaoa for one batch (no counterpart in the
 * paper).  For callers that must not allocate device memory -- memory owned by
 * another runtime or pool, a fixed budget carved at start-up, or loops that
 * cannot take the synchronisation of cudaMalloc/cudaFree.  The library
 * allocates nothing: the caller passes the statevector workspace and the
 * outputs, and all other scratch comes from one static 8 MiB device array per
 * GPU (held until process exit).
 *   n, graph, p, gammas, betas, noise   as for qn_batch_create and qn_run_qaoa (host)
 *   seed, first_trajectory, count       trajectories first_trajectory ..
 *                                       first_trajectory + count - 1 of the
 *                                       ensemble drawn from seed (count <= 65535)
 *   psi        device, count * 2^n * 8 bytes, 16-byte aligned: workspace; on
 *              return it holds the final states in the library's internal form
 *   c_out      device, count doubles: <C>_t of each trajectory
 *   probs_out  device, 2^n doubles: overwritten with sum_t |psi_t,x|^2 over the
 *              batch (divide by count for sigma_approx)
 *   cuda_stream  cudaStream_t to queue on (NULL = legacy default stream)
 * Results equal those of a handle with the same seed.  Returns QN_EINVAL when
 * the batch needs more scratch than the 8 MiB array (lower count or n), and,
 * before anything is queued, when psi, c_out or probs_out is not device (or
 * managed) memory of the current device or the stream belongs to another
 * device.  The first call on each device looks up the array's device address
 * (again after the device's context was recreated); make it before any stream
 * capture.  Calls share the array: calls that overlap on the GPU race.  Blocks
 * until the batch is done. */
qn_status qn_run_qaoa_noalloc(int32_t n, const qn_graph *graph, int32_t p, const double *gammas,
                              const double *betas, const qn_noise *noise, uint64_t seed,
                              int64_t first_trajectory, int32_t count, void *psi, double *c_out,
                              double *probs_out, void *cuda_stream);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *qn_last_error(void);

/* Free the handle and its device memory (NULL is ignored).  Synchronises. */
void qn_batch_destroy(qn_batch *h);

#ifdef __cplusplus
}
#endif

#endif /* QN_H */
