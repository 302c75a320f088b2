// Internal interface between the host API (qn_api.cpp) and the device kernels
// (qn_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "qn.h"

namespace qn {

enum GateKind : int32_t { kGateH = 0, kGateZZ = 1, kGateRX = 2 };

// One circuit gate as the kernels see it.  For ZZ, (c, s) = (cos gamma, sin gamma)
// and the phase on differing bits is c - i s; for RX, exp(-i beta X) has
// (c, s) = (cos beta, sin beta).  q1 == q0 for 1q gates.
struct DevGate {
    int32_t kind;
    int32_t q0, q1;
    float c, s;
};

// Per-trajectory dynamic state, one per slot of a launch batch.
//   J     X-frame bits contributed by damping jumps already folded into the stored state
//   pend  X-frame bits of the jumps of the pending damping op (not yet applied)
//   pq0, pq1  qubits of the pending op (pq1 == pq0 for a 1q gate)
//   f     pending amplitude factors, indexed by (b0 | b1 << 1) with b0, b1 the
//         true bits of pq0, pq1 (for a 1q op only f[0] and f[3] are used)
struct __align__(16) TrajState {
    uint32_t J;
    uint32_t pend;
    int32_t pq0, pq1;
    float f[4];
};

// Launch-independent description of one batch of trajectories.
struct BatchView {
    float2 *psi;            // [b][2^n] stored (frame) state, complex64
    int32_t n;
    int32_t b;              // trajectories in this batch
    int64_t t0;             // global id of slot 0
    int32_t G;              // gates per circuit
    int32_t tiles;          // 2048-amplitude tiles per trajectory (init, observables)
    int32_t stiles;         // sweep blocks per trajectory (kSub tiles each)
    uint8_t *branch;        // [b][G]
    uint32_t *dwords;       // [b][G][2] damping words, or nullptr when damping == 0
    uint32_t *frame_x;      // [b][G+1] X-frame of the Pauli noise before gate g
    uint8_t *yphase;        // [b] number of Y Paulis mod 4
    float *hfac;            // [b][n][2] per-qubit factors of the noisy H layer
    TrajState *st;          // [b]
    double *partials;       // [b][tiles][4]
    double *inv_norm;       // [b] 1 / ||psi||^2 of the final state (set by k_observe)
    unsigned int *counters; // [b]
    int *status;            // device error word
    // Device-driven launches (shared-prefix mode): a sweep covers the slots
    // [*dyn_lo, *dyn_hi) (dyn_lo == nullptr: from 0), counts read on the device, as
    // dyn_tiles tiles per slot, handed out to a persistent grid in order from the
    // launch's counter *dyn_queue (zero at launch).  dyn_hi == nullptr: the grid was
    // sized on the host, one block per tile and slot.
    const int32_t *dyn_lo = nullptr;
    const int32_t *dyn_hi = nullptr;
    int32_t *dyn_queue = nullptr;
    int32_t dyn_tiles = 0;
};

// Shared-prefix mode: slots (distinct states) and their member trajectories.
struct SlotView {
    int32_t *members;    // [K] batch-local trajectory indices, grouped by slot
    int32_t *tmp;        // [K] partition scratch
    uint8_t *cls;        // [K] branch class of each member at the current gate
    int2 *range;         // [max_slots] (offset, count) of each slot in members
    int32_t *slot_count; // slots created so far
    int32_t *active;     // slots swept by the current gate
    int2 *forks;         // [max_slots] (parent, child) created at the current gate
    int32_t *fork_count;
    double *marg;        // [max_slots][4] damping marginal of each slot at the current gate
    int32_t max_slots;
    int32_t *prev_active = nullptr;  // live slots before the last decide (the slots from here
                                     // on were forked by it); set by the fork-finish kernel
    int32_t *live_log = nullptr;     // [1 + decides] decides so far, then the live-slot count
                                     // after each (device-driven runs: the host reads it after
                                     // the run for its byte accounting)
    int32_t dyn = 0;                 // device-driven: decide kernels read *active on the device
};

// Consecutive phase gates of one layer whose qubits S number at most 10 (shared-
// prefix mode with damping): their damping branches follow from the joint
// distribution of the true bits of S, because every op of the group is
// diagonal (phases, Z parts, K0) or a relabelling (X parts, K1) in the stored
// basis.
constexpr int kMaxGroupEdges = 12;
constexpr int kMaxGroupQubits = 10;
constexpr int kGroupBins = 1 << kMaxGroupQubits;

// A group of consecutive gates of one layer whose noise sites are all decided
// from one joint distribution of the true bits of the group's qubits S:
//   kind 0  phase gates (two damping sites each); the joint is taken before them
//   kind 1  mixer rotations on consecutive qubits (one site each); the joint is
//           that of the state after the rotations
struct GateGroup {
    int32_t g0, m, s;               // first gate, gates, qubits in S
    int32_t kind;
    int32_t sp[kMaxGroupQubits];    // qubits of S, ascending
    int32_t ei[kMaxGroupEdges];     // S index of each gate's first qubit
    int32_t ej[kMaxGroupEdges];     // S index of each gate's second qubit (== ei for a rotation)
    float c, sn;                    // cos, sin of the layer's gamma (kind 0) or beta (kind 1)
    uint16_t tab[4][256];           // index over S of the stored bits in each byte of y (kind 0)
};

// Mixer blocks: kMixQ consecutive qubits per sweep.  A block of the sweep
// takes tiles of 2048 float4 (11 f bits): kMixL bits L go to the lanes, kMixQ
// bits A hold the block's qubits, kMixQ bits B the next block's; A and B are
// filled up with low f bits left over.  In the first phase a thread holds the
// 2^kMixQ float4 along A (lane and warp from L and B), in the second those
// along B (lane and warp from L and A).  The other f bits number the tiles
// (ftile).  Qubit 0 is the pair inside a float4: a block holding it (has0) has
// its other qubits on A bits 0 ..; otherwise qubit q_lo + i sits on A bit i.
// The next block's qubit i sits on B bit i.
constexpr int kMixQ = 4;
constexpr int kMixL = 11 - 2 * kMixQ;
constexpr int kMixThreads = 2048 >> kMixQ;
struct MixMap {
    int8_t fL[5], fA[4], fB[4];
    int8_t ftile[32];
    int32_t ntile;    // tile bits
    int32_t M;        // qubits of this block
    int32_t has0;
    int32_t nN;       // qubits of the next block (0: no joint to accumulate)
    int32_t final_norm;  // last sweep of the circuit: also form 1 / ||psi||^2 per state
    int32_t tanf;     // |cos beta| >= |sin beta|: rotations in the tan form, else the cot form
    int32_t keep = 0;  // with final_norm: no sweep applies the block -- the sigma pass applies it
                       // on the fly and the group decide forms the norms (full blocks off qubit 0)
    // 8-qubit blocks (the factor table covers eight qubits, 256 entries):
    //  1  qubits 4-7 of the block over qubits 0-7 whose qubits 0-3 the sweep before rotated
    //     (L bits = qubits 1-3, A = qubits 4-7)
    //  2  the factors of the block over qubits 0-7, all of which the sweep before rotated
    //     (qubit 0 the float4 half, qubits 1-3 the L bits, qubits 4-7 the tile's f bits
    //     wsh .. wsh+3), with the rotations of A, the first half of the next (8-qubit) block,
    //     and that block's joint over A and B (B = its second half, rotated without being kept)
    //  3  the second half (A) of an 8-qubit block whose first half the sweep before rotated:
    //     that half sits on the tile's f bits wsh .. wsh+3, A is the high half of the index
    int32_t wide = 0;
    int32_t wsh = 0;
    int32_t full8 = 0;  // k_group_mix: rotate qubits 4-7 too and bin the stored values
};

// The circuit's last mixer block when its sweep kept the states (MixMap::keep):
// what the sigma pass needs to apply it to each state.
struct MixTail {
    const GateGroup *grp;   // device: the block (its angle)
    const float2 *T;        // [slots][kGroupBins] the block's drawn factors by stored bits
    const int32_t *parent;  // [slots] the parent of each slot forked at the block
    int32_t first_new;      // slots from this one on were forked at the block
    const int32_t *first_new_dev = nullptr;  // device-driven runs: first_new read on the device
};
constexpr int kMixSubs = 4;  // tiles per thread block (streamed through two shared buffers)

// Device view of one group step.  Per-slot arrays are indexed by slot; the
// per-member scratch arrays by the position of the member in SlotView::members.
// One outcome class of a slot in a group (written by the class step, read by the table step).
// A member's outcome string over a group: per gate 6 bits (Pauli code, then the
// two jump bits); gates 0-9 in x, gates 10-11 in y.  All zero: the shared path.
using GroupKey = ulonglong2;

struct GroupClass {
    GroupKey key;    // the class's outcome string
    int32_t slot;    // the slot the members were in
    int32_t target;  // the slot that holds them after the group (slot itself for class 0)
    int32_t start;   // first member position
    int32_t count;   // members
};

struct GroupView {
    const GateGroup *grp;    // group applied by this step
    const GateGroup *next;   // phase group whose joint the apply sweep accumulates, or nullptr
    const int32_t *src;      // per slot: the state a sweep reads (a forked slot's parent), or
                             // nullptr: every slot reads its own state
    int32_t slot_base;       // first slot of the launch (blockIdx.y + slot_base)
    int32_t pend;            // the gate before the group may have left a pending op
    int32_t *parent;         // [max_slots] decide writes each new slot's parent here
    float vc, vs;            // cos, sin of the mixer angle whose rotations of qubits 0-3 the
                             // layer's last phase-group sweep applies (k_group_mix)
    unsigned long long *Hcur;   // [max_slots][kGroupBins] joint of this group, fixed point 2^-60
    unsigned long long *Hnext;  // [max_slots][kGroupBins] joint of the next group (zero on entry)
    float2 *T;             // [max_slots][kGroupBins] amplitude factor by stored bits of S
    TrajState *st_prev;    // [max_slots] pending op of the gate before the group
    float *Htrue;          // [max_slots][kGroupBins] this group's joint by true bits (FP32)
    float *p1m;            // [max_slots][2 kMaxGroupEdges] shared path's gamma P(q=1) per site
    int32_t *pos_slot;     // [K] slot of each member position (then scratch of k_gd_classes)
    int32_t members;       // member positions in the prefix tree (K of this run)
    GroupKey *ekey;        // [K] outcome string of the member at each position (0: shared path)
    int32_t *evt;          // [K] per slot: member index of the k-th member with an event
    int32_t *rep;          // [K] per slot: first event with the same outcome string
    int32_t *lead;         // [K] per slot: events that open a class, in event order
    int32_t *lstart;       // [K] per slot: first position of each opened class
    int32_t *lcount;       // [K] per slot: members of each opened class
    GroupClass *cls;       // [max_slots] the classes of all slots
    int32_t *ncls;         // device counter of cls (reset by the fork-finish kernel)
    // The circuit's last mixer block, which no sweep applies (the sigma pass applies it to
    // each state on the fly): the table step also stores 1 / ||psi||^2 of every class's
    // final state, sum_b |T_b|^2 J_b over the joint J the block was drawn from.
    int32_t final_norm = 0;
};

// One QAOA layer for the fused (Pauli-only) sweeps.
struct LayerView {
    const uint64_t *ev;      // [4][256] edge-difference vectors by byte of y (bit e: endpoints of edge e differ)
    const float2 *phase;     // [E+1] e^{-i gamma k}
    const int2 *edges;       // [E]
    uint64_t *s;             // [b] edges whose endpoints' frame bits differ at their gate
    uint32_t *zm, *zc;       // [b] Z parts of the cost layer's Paulis: mask and frame parity
    uint32_t *mz, *mf;       // [b] mixer: Z part of each qubit's Pauli, frame bit at its gate
    float cb, sb;            // cos beta, sin beta of the layer
    int32_t num_edges;       // E (at most 64)
};

#if defined(__CUDACC__)
// The cost layer's diagonal factor at amplitude y (stored basis) for one
// trajectory: e^{-i gamma k} with k the number of edges whose stored endpoint
// bits differ from the frame's (EV byte tables xor s), times the sign of the
// Pauli Z parts (popc(y & zm) xor zc).
__device__ __forceinline__ float2 layer_phase(const LayerView &L, uint32_t y, uint64_t sv, uint32_t zm, uint32_t zc) {
    const uint64_t ev = __ldg(L.ev + (y & 255u)) ^ __ldg(L.ev + 256 + ((y >> 8) & 255u)) ^
                        __ldg(L.ev + 512 + ((y >> 16) & 255u)) ^ __ldg(L.ev + 768 + (y >> 24));
    const int k = __popcll(ev ^ sv);
    const float2 ph = __ldg(L.phase + k);
    const float sg = ((__popc(y & zm) ^ zc) & 1u) ? -1.0f : 1.0f;
    return make_float2(ph.x * sg, ph.y * sg);
}
#endif

// Arithmetic of the fused layers (Pauli-only noise): FP32 on the CUDA cores, or
// the mixer rotations as GEMMs on the tensor cores with TF32 operands or BF16x3
// split operands (FP32 accumulation either way).
enum Precision : int32_t { kPrecFP32 = 0, kPrecTF32 = 1, kPrecBF16x3 = 2 };

// One tensor-core sweep: the mixer rotations of the qubits `act` (bits of the
// window wl .. wl + 4) of one layer, dph[k] = e^{-i beta (popc(act) - 2k)} / 32.
struct TcSweep {
    int32_t wl;
    uint32_t act;
    float2 dph[6];
};

// Fused mixer windows (16 float4 per thread, the qubits beyond four on lane bits):
constexpr int kFuse0 = 8;      // the window that holds qubit 0 (n >= 10): qubit 0 in the float4,
                               // 1-3 on lane bits, 4-7 in registers
constexpr int kFuseTile = 12;  // the window of qubits 0-11 as one 2048-float4 tile in shared memory,
                               // taken where it saves a sweep per layer
constexpr int kFuse = 7;       // at most, each of the other windows (n >= 10)
constexpr int kFuseSmall = 5;  // n < 10: windows of five qubits, registers only
constexpr int kFuseChunks = 8;  // chunks of kThreads fibre-threads per fused-sweep block

struct NoiseDev {
    double gamma;              // damping (0 = off)
    uint64_t thr1[4];          // cumulative thresholds, 1q
    uint64_t thr2[16];         // cumulative thresholds, 2q
};

// The rule that splits a sigma pass over b states into row blocks (probs_parts):
// xb blocks per state, res resident blocks, at most pmax rows (kMaxProbParts and
// the sigma copies that fit); used = 0: the host chose the rows.
struct RowPlan {
    int64_t xb;
    int32_t res;
    int32_t pmax;
    int32_t used;
};
__host__ __device__ inline int row_parts(const RowPlan &r, int b) {
    // Every block of a row streams all of the row's states, so the launch takes about
    // ceil(xb P / res) rounds of b / P states each: take the P with the fewest
    // state-rounds (the smaller on a tie).  A row keeps at least one chunk of 32 states.
    const int64_t cap = ((int64_t)b + 31) / 32;
    const int pmax = (int)(cap < (int64_t)r.pmax ? (cap > 1 ? cap : 1) : r.pmax);
    int best = 1;
    double best_cost = 0.0;
    for (int p = 1; p <= pmax; ++p) {
        const double rounds = (double)((r.xb * p + r.res - 1) / r.res);
        const double cost = rounds * (double)(((int64_t)b + p - 1) / p);
        if (p == 1 || cost < best_cost * 0.995) {
            best = p;
            best_cost = cost;
        }
    }
    return best;
}

struct AccumView {
    int32_t num_edges;
    const int2 *edges;         // device
    const int32_t *order;      // shared-prefix mode: slot of position tt, or nullptr
    const double *weights;     // shared-prefix mode: trajectories per slot, or nullptr
    double *cpart;             // [b][xblocks] partial sums of |psi|^2 C(x)
    unsigned int *acc_counter; // 1
    double *c_out;             // [b] per-trajectory <C>_t
    double *probs;             // [2^n] ensemble sum, or nullptr
    double *sums;              // [2] S1, S2, or nullptr
    int32_t trivial_pending = 0;  // every state's pending op is the identity
    int32_t parts = 1;            // row blocks that split the states (k_probs grid y)
    double *spart = nullptr;      // [parts - 1][2^n] sigma terms of rows 1 .. parts-1
    // Device-driven runs: the state count b is *v.dyn_hi, read on the device, and the row
    // blocks are chosen there from it by the rule the host applies (row_plan); the grid's
    // y extent is the largest count, and rows beyond the chosen one leave at once.
    RowPlan rows{};
};

constexpr int kThreads = 256;        // threads per sweep block
constexpr int kF4PerThread = 4;      // float4 items per thread (8 amplitudes)
constexpr int kTileF4 = kThreads * kF4PerThread;  // float4 per tile (2048 amplitudes)

constexpr int kSub = 4;             // sub-tiles streamed by one sweep block (8192 amplitudes)

inline int64_t tiles_for(int n) {
    int64_t nf = (int64_t)1 << (n - 1 > 0 ? n - 1 : 0);
    return (nf + kTileF4 - 1) / kTileF4;
}

// Blocks per trajectory of a gate sweep (each streams kSub tiles).
inline int64_t sweep_tiles_for(int n) {
    int64_t nf = (int64_t)1 << (n - 1 > 0 ? n - 1 : 0);
    return (nf + (int64_t)kTileF4 * kSub - 1) / ((int64_t)kTileF4 * kSub);
}

// Kernel launch wrappers (qn_kernels.cu).  All return the launch's cudaError_t.
cudaError_t launch_prepare(const BatchView &v, const DevGate *gates, uint64_t seed, const NoiseDev &nz,
                           int damping_on, cudaStream_t s);
cudaError_t launch_init(const BatchView &v, cudaStream_t s);
cudaError_t launch_sweep(const BatchView &v, int g, const DevGate &gate, const NoiseDev &nz, int damping_on,
                         cudaStream_t s);
cudaError_t launch_observe(const BatchView &v, const AccumView &a, cudaStream_t s);
// Device-driven shared-prefix runs: order[0 .. slots) = the live slots by their first
// members (trajectory order), weights[slot] = its member count; pos is [K] scratch.
// Run once before a stream capture: the launch wrappers' one-time set-up (occupancy
// figures, shared-memory attributes), so that a captured run makes no such calls.
cudaError_t prewarm_dev_launches();
cudaError_t launch_slot_order(const SlotView &sv, int32_t *pos, int32_t *order, double *weights, int K, int *status,
                              cudaStream_t s);
cudaError_t launch_probs(const BatchView &v, const AccumView &a, cudaStream_t s);
// The sigma pass that applies the circuit's last mixer block on the fly (states
// kept by a MixMap::keep sweep); same outputs as launch_probs.
cudaError_t launch_probs_mix(const BatchView &v, const AccumView &a, const MixMap &mm, const MixTail &tl,
                             cudaStream_t s);
// Row blocks worth giving the sigma pass for b states (1 .. kMaxProbParts): k_probs
// with a pending op (kind 0) or without (1), or the pass of launch_probs_mix (2).
int probs_parts(int n, int b, int kind);
RowPlan probs_row_plan(int n, int kind);  // the inputs of that rule (row_parts) for n qubits
constexpr int kMaxProbParts = 16;
cudaError_t launch_readout(const BatchView &v, float2 *out, cudaStream_t s);
// What the readout of a shared-prefix run needs about the circuit's last mixer
// block when its sweep kept the states (MixMap::keep); keep = 0 otherwise.
struct ReadTail {
    int32_t keep;
    int32_t M;             // qubits of the block
    int32_t q[kMixQ];      // the block's qubits
    float c, s;            // cos beta, sin beta of the block's layer
    const float2 *T;       // [slots][kGroupBins] the block's drawn factors by stored bits
    const int32_t *parent; // [slots] parent of each slot forked at the block
    int32_t first_new;     // slots from this one on were forked at the block
};
// Final states of a shared-prefix run, one per output: out[o] = the normalised
// state of slot oslot[o] in the true basis, with trajectory otraj[o]'s global
// phase (device arrays of nout entries; out holds nout * 2^n amplitudes).
cudaError_t launch_slot_readout(const BatchView &v, const int32_t *oslot, const int32_t *otraj, int nout,
                                const ReadTail &rt, float2 *out, cudaStream_t s);
// Fused layers (Pauli-only): per-trajectory layer parameters from the branch
// tables, then sweeps applying the rotations of qubits [q_lo, q_lo + m) of
// layer Lr, with layer Lp's phase before them (pre) and layer Lq's after (post);
// norm (the circuit's last sweep, q_lo > 0): also 1/N_t, as launch_observe.
cudaError_t launch_layer_params(const BatchView &v, const LayerView &L, int g0, int E, cudaStream_t s);
cudaError_t launch_fused_sweep(const BatchView &v, const LayerView &Lp, const LayerView &Lr, const LayerView &Lq,
                               int q_lo, int m, bool pre, bool post, bool norm, cudaStream_t s);
cudaError_t launch_phase_sweep(const BatchView &v, const LayerView &L, cudaStream_t s);
// A fused window off qubit 0 of 4-7 qubits whose float4-index bits start at 11 - m or
// above: tiles of runs of consecutive float4 times the window's values, through shared
// memory; post: the next layer's phase (Lq) after the rotations; norm: the final norms
// (the circuit's last sweep).  fused_win_ok: the windows it takes (the others take
// launch_fused_sweep).
bool fused_win_ok(int n, int q_lo, int m, bool post, bool norm);
cudaError_t launch_fused_win(const BatchView &v, const LayerView &Lr, const LayerView &Lq, int q_lo, int m, bool post,
                             bool norm, cudaStream_t s);
// The first window of a fused layer for n >= 13: the rotations of qubits 0-11 of layer Lr
// in one sweep of 2048-float4 tiles (two phases through shared memory), with layer Lp's
// phase before them when pre.
cudaError_t launch_fused_tile12(const BatchView &v, const LayerView &Lp, const LayerView &Lr, bool pre,
                                cudaStream_t s);
// Tensor-core form of a fused sweep (n >= 11): the window's rotations as two
// GEMMs with the +-1 Hadamard matrix (qn_tc.cu), PRE / POST phases as for
// launch_fused_sweep.  kind: kPrecTF32 or kPrecBF16x3.
cudaError_t launch_tc_sweep(const BatchView &v, const LayerView &Lp, const LayerView &Lr, const LayerView &Lq,
                            const TcSweep &sw, bool pre, bool post, int kind, cudaStream_t s);
// Shared-prefix mode, gate g: sweep the `active` live slots; then draw each
// member's branch, fork the slots whose members drew other branches and copy
// the forked states (three launches; the new live-slot count is left in
// *sv.active).
cudaError_t launch_slot_sweep(const BatchView &v, const SlotView &sv, int active, int g, const DevGate &gate,
                              int damping_on, cudaStream_t s);
cudaError_t launch_slot_fork(const BatchView &v, const SlotView &sv, int active, int g, const DevGate &gate,
                             const NoiseDev &nz, int damping_on, cudaStream_t s);
// Shared-prefix mode, phase-gate groups: joint of the first group (read pass),
// per-slot decisions and forks of a group, and the apply sweep (which also
// accumulates the next group's joint).
cudaError_t launch_group_hist(const BatchView &v, const SlotView &sv, const GroupView &gv, int active, cudaStream_t s);
cudaError_t launch_group_decide(const BatchView &v, const SlotView &sv, const GroupView &gv, int ns, int active,
                                double gamma, cudaStream_t s);
cudaError_t launch_mix_sweep(const BatchView &v, const GroupView &gv, const MixMap &mm, int active, cudaStream_t s);
// The last phase group of a layer (gv.grp, its factors in gv.T) applied with the
// rotations of qubits 0-3 of the layer's first mixer block (angle gv.vc, gv.vs),
// which covers qubits 0-7: the sweep forms that block's joint in gv.Hnext after
// rotating qubits 4-7 as well (mm: the tile map of qubits 0-3 with next 4-7).
cudaError_t launch_group_mix(const BatchView &v, const GroupView &gv, const MixMap &mm, int active, cudaStream_t s);
cudaError_t launch_group_apply(const BatchView &v, const SlotView &sv, const GroupView &gv, int active, cudaStream_t s);
// Adjoint gradient: lambda = C psi_T, then one reverse sweep per gate g >= n
// adding d<C>_t / d theta_param into grad[t * nparam + param] (FP64).
cudaError_t launch_adj_init(const BatchView &v, float2 *lam, const AccumView &a, cudaStream_t s);
// Fused adjoint (Pauli-only noise, after a fused forward run that left the layer
// parameters of every layer): the reverse of the mixer rotations of qubits
// [q_lo, q_lo + m) of layer L on psi and lambda (m <= 4 with qubit 0, else <= 3),
// adding their terms to grad[t][param] (d<C>_t / d beta); and the reverse of layer
// L's cost diagonal, adding its term to grad[t][param] (d<C>_t / d gamma).
cudaError_t launch_adj_mixer(const BatchView &v, float2 *lam, const LayerView &L, int q_lo, int m, double *grad,
                             int param, int nparam, cudaStream_t s);
// The tiled reverse of one mixer window (n >= 12): qubits 0-9 (q_lo = 0, m = 10), or
// m = 2..6 qubits from q_lo >= 10; with phase also the layer's cost diagonal (the last
// window of the layer to be undone).  Terms to grad[t][pbeta] and, with phase,
// grad[t][pgamma].
cudaError_t launch_adj_win(const BatchView &v, float2 *lam, const LayerView &L, int q_lo, int m, bool phase,
                           double *grad, int pbeta, int pgamma, int nparam, cudaStream_t s);
cudaError_t launch_adj_phase(const BatchView &v, float2 *lam, const LayerView &L, double *grad, int param, int nparam,
                             cudaStream_t s);
cudaError_t launch_adj_sweep(const BatchView &v, float2 *lam, int g, const DevGate &gate, double *grad, int param,
                             int nparam, cudaStream_t s);
int64_t accumulate_xblocks(int n);

// Validated circuit and noise tables of one qn_run_qaoa call, built by the
// same host code the handle path uses (qn_api.cpp), for entry points that work
// without a handle.
struct QaoaPlan {
    std::vector<DevGate> gates;
    std::vector<int2> edges;
    NoiseDev nz;
    int damping_on;
};
qn_status plan_qaoa(int32_t n, const qn_graph *graph, int32_t p, const double *gammas, const double *betas,
                    const qn_noise *noise, QaoaPlan *out);
// Record `msg` as this thread's qn_last_error() and return `st`.
qn_status set_error(qn_status st, const char *msg);

}  // namespace qn
