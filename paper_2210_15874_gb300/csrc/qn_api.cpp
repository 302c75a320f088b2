// qn_api.cpp -- host side of the libqnoise C ABI (include/qn.h).
//
// Builds the QAOA gate list and the noise tables from the call's arguments,
// owns the device memory of a handle, and queues, per batch of B trajectories:
//   prepare     Philox draws, Pauli codes, X-frames, the noisy H layer
//   init        write-only sweep of the product state after the H layer
//   sweeps      one per remaining gate: gate, Pauli, damping draw
//   accumulate  phi = |psi|^2 into sigma_approx and <C>
//               (Sec. "Stochastic Noise Implementation")
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <unordered_map>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "qn.h"
#include "qn_internal.h"

using namespace qn;

namespace {

thread_local std::string g_last_error;

qn_status fail(qn_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

qn_status ok() {
    g_last_error.clear();
    return QN_OK;
}

#define QN_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return fail(QN_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define QN_TRY(expr)                       \
    do {                                   \
        qn_status s_ = (expr);             \
        if (s_ != QN_OK) return s_;        \
    } while (0)

struct HostGate {
    int32_t kind, q0, q1;
    double angle;
};

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    int kind = 0;
    double bytes = 0.0;
    // device-driven runs: bytes = per_state x the live count after `log_k` decides (known
    // once the run is over); -1: bytes is final
    int32_t log_k = -1;
    double per_state = 0.0;
};

// What a device-driven shared-prefix run leaves for the host to finish once it is over.
struct DevRun {
    std::vector<std::pair<int32_t, double>> acct;  // per sweep: (decides before it, bytes per live state)
    int64_t launches = 0;
    int32_t decides = 0;
    ReadTail read_tail{};  // first_new still to be read from the device
};

constexpr int kMaxQubits = 30;
constexpr int64_t kMaxGates = 1 << 20;
constexpr size_t kDefaultBatchBytes = (size_t)512 << 20;

// Page-locked host words into which shared-prefix runs read the live-slot count
// after each group (a copy into pageable memory returns only after a staged copy
// and wakes the host later).  One pool per process, allocated on first use and
// never freed -- cudaFreeHost would synchronise the device and stall other
// handles' streams; a handle takes one word and gives it back when destroyed.
// nullptr when the pool is spent or cannot be allocated (callers then use a
// pageable word).
constexpr int kPinnedWords = 4096;
struct PinnedWords {
    std::mutex mu;
    int32_t *base = nullptr;
    std::vector<int> free_list;
    bool tried = false;
};
PinnedWords &pinned_words() {
    static PinnedWords pool;
    return pool;
}
int32_t *pinned_word_take() {
    PinnedWords &p = pinned_words();
    std::lock_guard<std::mutex> lock(p.mu);
    if (!p.tried) {
        p.tried = true;
        void *ptr = nullptr;
        if (cudaHostAlloc(&ptr, kPinnedWords * sizeof(int32_t), cudaHostAllocPortable) == cudaSuccess) {
            p.base = static_cast<int32_t *>(ptr);
            for (int i = kPinnedWords - 1; i >= 0; --i) p.free_list.push_back(i);
        } else {
            cudaGetLastError();  // clear the error it left; callers fall back to pageable words
        }
    }
    if (!p.base || p.free_list.empty()) return nullptr;
    const int i = p.free_list.back();
    p.free_list.pop_back();
    return p.base + i;
}
void pinned_word_give(int32_t *w) {
    if (!w) return;
    PinnedWords &p = pinned_words();
    std::lock_guard<std::mutex> lock(p.mu);
    p.free_list.push_back((int)(w - p.base));
}

}  // namespace

struct qn_batch {
    int32_t *pinned_word = nullptr;  // page-locked word for the live-slot count (or nullptr)
    bool pinned_tried = false;
    int32_t n = 0;
    int64_t K = 0;
    uint64_t seed = 0;
    int64_t B_req = 0;
    int64_t offset = 0;
    cudaStream_t stream = nullptr;
    void *(*alloc_fn)(size_t, void *) = nullptr;
    void (*free_fn)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;

    // problem of the last run
    bool has_run = false;
    // the statevector buffer holds the final states of the whole ensemble (one launch batch,
    // one state per trajectory) as the last run left them: the adjoint can start from them
    bool final_states = false;
    std::vector<int32_t> edges;
    int32_t p = 0;
    std::vector<double> gammas, betas;
    qn_noise noise{};
    std::vector<HostGate> gates;
    std::vector<DevGate> dgates_host;
    std::vector<int2> edges_host;
    NoiseDev nz{};
    int damping_on = 0;
    int64_t B = 0;
    int64_t launches = 0;
    double sweep_bytes = 0.0;

    // device memory (all blocks listed in `blocks`)
    std::vector<void *> blocks;
    int64_t cap_B = 0;
    int32_t cap_G = -1;
    int32_t cap_E = -1;
    float2 *psi = nullptr;
    uint8_t *branch = nullptr;
    uint32_t *dwords = nullptr;
    uint32_t *frame_x = nullptr;
    uint8_t *yphase = nullptr;
    float *hfac = nullptr;
    TrajState *st = nullptr;
    double *partials = nullptr;
    unsigned int *counters = nullptr;
    double *inv_norm = nullptr;
    double *cpart = nullptr;
    unsigned int *acc_counter = nullptr;
    double *c_all = nullptr;
    double *c_dbg = nullptr;
    double *probs = nullptr;
    double *sums = nullptr;
    int *status = nullptr;
    DevGate *dgates = nullptr;
    int2 *dedges = nullptr;
    float2 *readout = nullptr;
    // fused layers (Pauli-only noise)
    int32_t fusion = 1;
    int32_t precision = kPrecFP32;  // arithmetic of the fused layers (qn_batch_set_precision)
    uint64_t *fl_ev = nullptr;    // [4][256]
    float2 *fl_phase = nullptr;   // [p][E+1]
    int2 *fl_edges = nullptr;     // [E]
    uint64_t *fl_s = nullptr;     // [p][B]
    uint32_t *fl_u = nullptr;     // [p][4][B]: zm, zc, mz, mf
    int32_t fl_cap_p = 0, fl_cap_E = -1;
    int64_t fl_cap_B = 0;
    std::vector<uint64_t> ev_host;
    std::vector<float2> phase_host;
    // shared-prefix mode
    int32_t sharing = 0;
    int32_t *sh_members = nullptr, *sh_tmp = nullptr, *sh_ctr = nullptr, *sh_order = nullptr;
    uint8_t *sh_cls = nullptr;
    int2 *sh_range = nullptr, *sh_forks = nullptr;
    double *sh_weights = nullptr;
    double *sh_marg = nullptr;
    int64_t sh_cap = 0;
    int64_t sh_slots = 0;  // slots of the last shared-prefix run (all chunks)
    // the last shared-prefix chunk as its run left it, for qn_shared_readout
    bool sh_valid = false;
    int64_t sh_last_t0 = 0;  // handle-local id of the chunk's first trajectory
    int32_t sh_last_kc = 0;  // trajectories in the chunk
    std::vector<int2> sh_range_host;       // [slots] member range of each final slot
    std::vector<int32_t> sh_members_host;  // [kc] batch-local trajectories grouped by slot
    std::vector<int32_t> sh_order_host;    // [slots] slot of each position of the sigma pass
    ReadTail sh_tail{};                    // the pending last mixer block, if its sweep kept the states
    float2 *sh_readbuf = nullptr;          // readout chunk of final states
    int32_t *sh_readidx = nullptr;         // [2][chunk] slot and trajectory of each output
    int64_t sh_readcap = 0;
    // phase-gate groups of shared-prefix mode with damping
    std::vector<GateGroup> groups;
    std::vector<int32_t> group_at;  // [G] index of the group that starts at gate g, or -1
    bool split8 = false;            // mixer blocks 0-7 and 8-15 rotated whole (see build_groups)
    GateGroup *gr_dev = nullptr;
    int64_t gr_cap = 0;
    unsigned long long *gv_H = nullptr;  // [2][gv_cap][256]
    float2 *gv_T = nullptr;
    TrajState *gv_stprev = nullptr;
    GroupKey *gv_ekey = nullptr;
    int32_t *gv_i32 = nullptr;  // [7][gv_cap]: evt, rep, lead, lstart, lcount, parent, pos_slot
    float *gv_htrue = nullptr;  // [gv_cap][kGroupBins]
    float *gv_p1m = nullptr;    // [gv_cap][2 kMaxGroupEdges]
    GroupClass *gv_cls = nullptr;
    int64_t gv_cap = 0;
    // device-driven launches (qn_batch_set_launch_mode): 0 = sized on the host from the
    // live-slot count read after every decide; 1 = persistent launches that read it on
    // the device; 2 = as 1, the run after its noisy H layer captured in a CUDA graph and
    // replayed while the circuit, noise and launch batch stay the same
    int32_t launch_mode = 0;
    int32_t *sh_log = nullptr;  // [1 + decides] the live-slot count after each decide
    int64_t sh_log_cap = 0;
    int32_t *sh_queue = nullptr;  // [sweep launches] work counters of the persistent sweeps
    int64_t sh_queue_cap = 0;
    cudaStream_t cap_stream = nullptr;  // private stream that graphs are captured on
    cudaGraphExec_t graph_exec = nullptr;
    std::string graph_sig;              // the launches the graph holds (kernels' arguments)
    int64_t graph_captures = 0, graph_replays = 0, graph_updates = 0;
    DevRun graph_run;                   // what the host finishes after a replay of the graph
    double *spart = nullptr;   // sigma terms of k_probs row blocks 1 .. parts-1
    int64_t spart_cap = 0;     // doubles
    float2 *lambda = nullptr;  // adjoint vectors (qn_grad), allocated on first use
    double *grad = nullptr;    // [K][2p] per-trajectory gradients
    int32_t grad_cap = 0;      // 2p the grad buffer was sized for

    // profiling: every `prof_period`-th gate-sweep launch (and every init /
    // observable launch) is bracketed by a CUDA event pair; 0 = off
    int32_t prof_period = 0;
    int64_t prof_counter = 0;
    std::vector<EventPair> events;
    std::vector<EventPair> spare;
    int64_t prof_launches[5] = {0, 0, 0, 0, 0};
    double prof_ms[5] = {0, 0, 0, 0, 0};
    double prof_bytes[5] = {0, 0, 0, 0, 0};
};

namespace {

qn_status dev_alloc(qn_batch *h, void **out, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    if (h->alloc_fn) {
        p = h->alloc_fn(bytes, h->alloc_ctx);
        if (!p) return fail(QN_ENOMEM, "allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(QN_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    h->blocks.push_back(p);
    *out = p;
    return QN_OK;
}

template <typename T>
qn_status alloc_t(qn_batch *h, T **out, size_t count) {
    void *p = nullptr;
    qn_status st = dev_alloc(h, &p, count * sizeof(T));
    *out = static_cast<T *>(p);
    return st;
}

void drop_graph(qn_batch *h) {
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
    h->graph_sig.clear();
}

void release_all(qn_batch *h) {
    if (!h->blocks.empty()) cudaStreamSynchronize(h->stream);
    drop_graph(h);
    for (void *p : h->blocks) {
        if (h->free_fn) h->free_fn(p, h->alloc_ctx);
        else cudaFree(p);
    }
    h->blocks.clear();
    h->psi = nullptr;
    h->readout = nullptr;
    h->lambda = nullptr;
    h->grad = nullptr;
    h->sh_members = h->sh_tmp = h->sh_ctr = h->sh_order = nullptr;
    h->sh_cls = nullptr;
    h->sh_range = h->sh_forks = nullptr;
    h->sh_weights = nullptr;
    h->sh_marg = nullptr;
    h->sh_cap = 0;
    h->sh_log = nullptr;
    h->sh_log_cap = 0;
    h->sh_queue = nullptr;
    h->sh_queue_cap = 0;
    h->sh_valid = false;
    h->sh_readbuf = nullptr;
    h->sh_readidx = nullptr;
    h->sh_readcap = 0;
    h->gr_dev = nullptr;
    h->gr_cap = 0;
    h->gv_H = nullptr;
    h->gv_T = nullptr;
    h->gv_stprev = nullptr;
    h->gv_ekey = nullptr;
    h->gv_i32 = nullptr;
    h->gv_htrue = nullptr;
    h->gv_p1m = nullptr;
    h->gv_cls = nullptr;
    h->gv_cap = 0;
    h->spart = nullptr;
    h->spart_cap = 0;
    h->fl_ev = nullptr;
    h->fl_phase = nullptr;
    h->fl_edges = nullptr;
    h->fl_s = nullptr;
    h->fl_u = nullptr;
    h->fl_cap_p = 0;
    h->fl_cap_E = -1;
    h->fl_cap_B = 0;
    h->grad_cap = 0;
    h->cap_B = 0;
    h->cap_G = -1;
    h->cap_E = -1;
}

size_t state_bytes(int n) { return (size_t)8 << n; }

// Every buffer a run of B trajectories per launch, G gates and E edges needs.
size_t footprint(int n, int64_t K, int64_t B, int32_t G, int32_t E) {
    const size_t tiles = (size_t)tiles_for(n);
    size_t s = (size_t)B * state_bytes(n);  // states (debug readout and adjoint vectors come on demand)
    s += (size_t)B * G * (1 + 8) + (size_t)B * (G + 1) * 4 + (size_t)B * (1 + 8 * n + sizeof(TrajState) + 4 + 8);
    s += (size_t)B * tiles * 32 + (size_t)B * 8 + (size_t)B * accumulate_xblocks(n) * 8 + (size_t)K * 8 +
         ((size_t)8 << n);
    s += (size_t)G * sizeof(DevGate) + (size_t)(E + 1) * 8 + 4096;
    return s;
}

qn_status ensure_buffers(qn_batch *h, int64_t B, int32_t G, int32_t E) {
    if (h->cap_B >= B && h->cap_G == G && h->cap_E >= E && !h->blocks.empty()) return QN_OK;
    release_all(h);
    const int n = h->n;
    size_t free_b = 0, total_b = 0;
    QN_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t need = footprint(n, h->K, B, G, E);
    if (!h->alloc_fn && need > free_b)
        return fail(QN_ENOMEM, "footprint %zu bytes exceeds free device memory %zu bytes", need, free_b);
    const size_t tiles = (size_t)tiles_for(n);
    QN_TRY(alloc_t(h, &h->psi, (size_t)B << n));
    QN_TRY(alloc_t(h, &h->branch, (size_t)B * G));
    QN_TRY(alloc_t(h, &h->dwords, (size_t)B * G * 2));
    QN_TRY(alloc_t(h, &h->frame_x, (size_t)B * (G + 1)));
    QN_TRY(alloc_t(h, &h->yphase, (size_t)B));
    QN_TRY(alloc_t(h, &h->hfac, (size_t)B * n * 2));
    QN_TRY(alloc_t(h, &h->st, (size_t)B));
    QN_TRY(alloc_t(h, &h->partials, (size_t)B * tiles * 4));
    QN_TRY(alloc_t(h, &h->counters, (size_t)B));
    QN_TRY(alloc_t(h, &h->inv_norm, (size_t)B));
    QN_TRY(alloc_t(h, &h->cpart, (size_t)B * accumulate_xblocks(n)));
    QN_TRY(alloc_t(h, &h->acc_counter, 1));
    QN_TRY(alloc_t(h, &h->c_all, (size_t)h->K));
    QN_TRY(alloc_t(h, &h->c_dbg, (size_t)B));
    QN_TRY(alloc_t(h, &h->probs, (size_t)1 << n));
    QN_TRY(alloc_t(h, &h->sums, 2));
    QN_TRY(alloc_t(h, &h->status, 1));
    QN_TRY(alloc_t(h, &h->dgates, (size_t)std::max(G, 1)));
    QN_TRY(alloc_t(h, &h->dedges, (size_t)std::max(E, 1)));
    QN_CUDA(cudaMemsetAsync(h->counters, 0, (size_t)B * sizeof(unsigned int), h->stream));
    QN_CUDA(cudaMemsetAsync(h->acc_counter, 0, sizeof(unsigned int), h->stream));
    h->cap_B = B;
    h->cap_G = G;
    h->cap_E = E;
    return QN_OK;
}

// ---------------------------------------------------------------------------
// Noise tables.  Pauli probabilities per code (Sec. "Modeling Noise": the
// depolarizing Kraus set; K0 weight 1 - 3 lambda / 4 for the paper's lambda)
// and the integer thresholds floor(2^32 * cumulative sum).
// ---------------------------------------------------------------------------
double total_1q(const qn_noise &nz, double x) { return nz.param == 1 ? 0.75 * x : x; }

void probs_1q(const qn_noise &nz, double out[4]) {
    const double p = total_1q(nz, nz.p1);
    out[0] = 1.0 - p;
    out[1] = out[2] = out[3] = p / 3.0;
}

void probs_2q(const qn_noise &nz, double out[16]) {
    if (nz.twoq_mode == 1) {
        const double p = total_1q(nz, nz.p2);
        const double s[4] = {1.0 - p, p / 3.0, p / 3.0, p / 3.0};
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) out[4 * a + b] = s[a] * s[b];
        return;
    }
    const double p = nz.param == 1 ? (15.0 / 16.0) * nz.p2 : nz.p2;
    out[0] = 1.0 - p;
    for (int k = 1; k < 16; ++k) out[k] = p / 15.0;
}

void thresholds(const double *pr, int count, uint64_t *thr) {
    double c = 0.0;
    for (int k = 0; k < count; ++k) {
        c += pr[k];
        double v = std::floor(c * 4294967296.0);
        v = std::min(std::max(v, 0.0), 4294967296.0);
        thr[k] = (uint64_t)v;
    }
}

qn_status validate_noise(const qn_noise *nz) {
    if (!nz) return fail(QN_EINVAL, "noise is NULL");
    if (nz->param != 0 && nz->param != 1) return fail(QN_EINVAL, "noise.param must be 0 or 1");
    if (nz->twoq_mode != 0 && nz->twoq_mode != 1) return fail(QN_EINVAL, "noise.twoq_mode must be 0 or 1");
    const double max1 = nz->param == 1 ? 4.0 / 3.0 : 1.0;
    const double max2 = nz->param == 1 ? (nz->twoq_mode == 1 ? 4.0 / 3.0 : 16.0 / 15.0) : 1.0;
    if (!(nz->p1 >= 0.0 && nz->p1 <= max1)) return fail(QN_EINVAL, "noise.p1 = %g outside [0, %g]", nz->p1, max1);
    if (!(nz->p2 >= 0.0 && nz->p2 <= max2)) return fail(QN_EINVAL, "noise.p2 = %g outside [0, %g]", nz->p2, max2);
    if (!(nz->damping >= 0.0 && nz->damping <= 1.0))
        return fail(QN_EINVAL, "noise.damping = %g outside [0, 1]", nz->damping);
    return QN_OK;
}

qn_status validate_graph(const qn_batch *h, const qn_graph *g) {
    if (!g) return fail(QN_EINVAL, "graph is NULL");
    if (g->n != h->n) return fail(QN_EINVAL, "graph.n = %d but the handle has n = %d", g->n, h->n);
    if (g->num_edges < 0) return fail(QN_EINVAL, "graph.num_edges < 0");
    if (g->num_edges > 0 && !g->edges) return fail(QN_EINVAL, "graph.edges is NULL");
    std::set<std::pair<int, int>> seen;
    for (int e = 0; e < g->num_edges; ++e) {
        const int a = g->edges[2 * e], b = g->edges[2 * e + 1];
        if (a < 0 || a >= g->n || b < 0 || b >= g->n)
            return fail(QN_EINVAL, "edge %d = (%d, %d) out of range [0, %d)", e, a, b, g->n);
        if (a == b) return fail(QN_EINVAL, "edge %d is a self-loop on %d", e, a);
        if (!seen.insert({std::min(a, b), std::max(a, b)}).second)
            return fail(QN_EINVAL, "edge %d = (%d, %d) is a duplicate", e, a, b);
    }
    return QN_OK;
}

void build_gates(qn_batch *h) {
    const int n = h->n, E = (int)h->edges.size() / 2;
    h->gates.clear();
    for (int q = 0; q < n; ++q) h->gates.push_back({kGateH, q, q, 0.0});
    for (int l = 0; l < h->p; ++l) {
        for (int e = 0; e < E; ++e) h->gates.push_back({kGateZZ, h->edges[2 * e], h->edges[2 * e + 1], h->gammas[l]});
        for (int q = 0; q < n; ++q) h->gates.push_back({kGateRX, q, q, h->betas[l]});
    }
    h->dgates_host.clear();
    for (const HostGate &g : h->gates) {
        DevGate d;
        d.kind = g.kind;
        d.q0 = g.q0;
        d.q1 = g.q1;
        d.c = (float)std::cos(g.angle);
        d.s = (float)std::sin(g.angle);
        h->dgates_host.push_back(d);
    }
    h->edges_host.clear();
    for (int e = 0; e < E; ++e) h->edges_host.push_back(make_int2(h->edges[2 * e], h->edges[2 * e + 1]));
}

// Mixer blocks need the block over qubits 0-7 and a full block after it, and a
// phase group before them (whose apply sweep forms the first block's joint).
bool mixer_blocks_fit(int n, int E) { return n >= 12 && E > 0; }
constexpr int kWideBlock = 2 * kMixQ;  // qubits of the layer's first mixer block
// Two 8-qubit blocks then full 4-qubit ones: the last phase group's sweep rotates
// qubits 0-7 whole, the next sweep applies their factors, rotates qubits 8-11 and
// forms the joint of 8-15 (12-15 rotated without being kept), the one after
// rotates 12-15: one sweep fewer per layer than blocks 0-7, 8-11, 12-15, ...
bool split8_fits(int n) { return n >= 20 && n % kMixQ == 0; }

// Phase-gate groups of every layer: greedy runs of consecutive ZZ gates whose
// qubits number at most kMaxGroupQubits (joints of 2^10 bins), at most
// kMaxGroupEdges gates (a member's outcome string takes 6 bits per gate in a
// two-word key).
void build_groups(qn_batch *h) {
    const int n = h->n, E = (int)h->edges.size() / 2;
    h->groups.clear();
    h->group_at.assign(h->gates.size(), -1);
    h->split8 = false;
    for (int l = 0; l < h->p; ++l) {
        const int base = n + l * (E + n);
        int g = base;
        while (g < base + E) {
            GateGroup z;
            std::memset(&z, 0, sizeof z);
            z.g0 = g;
            uint32_t S = 0;
            while (g < base + E && z.m < kMaxGroupEdges) {
                const uint32_t S2 = S | (1u << h->gates[g].q0) | (1u << h->gates[g].q1);
                if (__builtin_popcount(S2) > kMaxGroupQubits) break;
                S = S2;
                ++z.m;
                ++g;
            }
            int local[32];
            z.s = 0;
            for (int q = 0; q < n; ++q)
                if ((S >> q) & 1u) {
                    local[q] = z.s;
                    z.sp[z.s++] = q;
                }
            for (int e = 0; e < z.m; ++e) {
                z.ei[e] = local[h->gates[z.g0 + e].q0];
                z.ej[e] = local[h->gates[z.g0 + e].q1];
            }
            z.c = h->dgates_host[z.g0].c;
            z.sn = h->dgates_host[z.g0].s;
            for (int byte = 0; byte < 4; ++byte)
                for (int v = 0; v < 256; ++v) {
                    int bins = 0;
                    for (int bit = 0; bit < 8; ++bit) {
                        const int q = 8 * byte + bit;
                        if (((v >> bit) & 1) && q < n && ((S >> q) & 1u)) bins |= 1 << local[q];
                    }
                    z.tab[byte][v] = (uint16_t)bins;
                }
            h->group_at[z.g0] = (int32_t)h->groups.size();
            h->groups.push_back(z);
        }
        if (!mixer_blocks_fit(n, E)) continue;
        // mixer rotations in blocks of consecutive qubits: qubits 0-7 first (the sweep of the
        // layer's last phase group rotates qubits 0-3 and forms this block's joint, the block's
        // own sweep rotates qubits 4-7), then kMixQ at a time; with split8 qubits 0-7 and 8-15
        // (the sweep before rotates all of 0-7; blocks 8-15 split over two sweeps)
        h->split8 = split8_fits(n);
        for (int q = 0; q < n;) {
            const int w = q == 0 || (q == kWideBlock && h->split8) ? kWideBlock : kMixQ;
            GateGroup z;
            std::memset(&z, 0, sizeof z);
            z.kind = 1;
            z.g0 = base + E + q;
            z.m = z.s = std::min(w, n - q);
            for (int k = 0; k < z.m; ++k) {
                z.sp[k] = q + k;
                z.ei[k] = z.ej[k] = k;
            }
            q += w;
            z.c = h->dgates_host[z.g0].c;
            z.sn = h->dgates_host[z.g0].s;
            h->group_at[z.g0] = (int32_t)h->groups.size();
            h->groups.push_back(z);
        }
    }
}

// Tile map of the sweep of the mixer block on qubits q_lo .. q_lo + M - 1
// whose next block holds the qubits `next`: A bits = the block's f bits (qubit
// q sits on f bit q - 1; qubit 0 is the pair inside a float4), B bits = the
// next block's; L = the kMixL lowest f bits left (consecutive lanes read
// neighbouring float4 whenever the low f bits are free); then A and B are
// filled up to kMixQ with the lowest f bits left; every other f bit numbers
// tiles.
MixMap mix_map(int n, int q_lo, int M, const std::vector<int> &next) {
    MixMap mm;
    std::memset(&mm, 0, sizeof mm);
    const int nb = n - 1;  // f bits
    std::vector<bool> taken((size_t)std::max(nb, 1), false);
    auto lowest_free = [&]() {
        int f = 0;
        while (f < nb && taken[f]) ++f;
        taken[f] = true;
        return f;
    };
    mm.M = M;
    mm.has0 = q_lo == 0;
    mm.nN = (int)next.size();
    std::vector<int> A, B;
    for (int j = 0; j < M; ++j)
        if (q_lo + j > 0) {
            A.push_back(q_lo + j - 1);
            taken[q_lo + j - 1] = true;
        }
    for (int q : next) {
        B.push_back(q - 1);
        taken[q - 1] = true;
    }
    if (mm.has0) {
        // the block holding qubit 0 and a full next block cover f bits 0 .. 6; padding A
        // before L makes the tile the contiguous f bits 0 .. 10 (copied in address order)
        while ((int)A.size() < kMixQ) A.push_back(lowest_free());
        for (int i = 0; i < kMixL; ++i) mm.fL[i] = (int8_t)lowest_free();
    } else {
        for (int i = 0; i < kMixL; ++i) mm.fL[i] = (int8_t)lowest_free();
        while ((int)A.size() < kMixQ) A.push_back(lowest_free());
    }
    while ((int)B.size() < kMixQ) B.push_back(lowest_free());
    for (int i = 0; i < kMixQ; ++i) {
        mm.fA[i] = (int8_t)A[i];
        mm.fB[i] = (int8_t)B[i];
    }
    mm.ntile = 0;
    for (int f = 0; f < nb; ++f)
        if (!taken[f]) mm.ftile[mm.ntile++] = (int8_t)f;
    return mm;
}

bool use_groups(const qn_batch *h) { return h->fusion && h->damping_on && !h->groups.empty(); }

BatchView view_for(qn_batch *h, int64_t t0, int b) {
    BatchView v;
    v.psi = h->psi;
    v.n = h->n;
    v.b = b;
    v.t0 = t0;
    v.G = (int32_t)h->gates.size();
    v.tiles = (int32_t)tiles_for(h->n);
    v.stiles = (int32_t)sweep_tiles_for(h->n);
    v.branch = h->branch;
    v.dwords = h->dwords;
    v.frame_x = h->frame_x;
    v.yphase = h->yphase;
    v.hfac = h->hfac;
    v.st = h->st;
    v.partials = h->partials;
    v.inv_norm = h->inv_norm;
    v.counters = h->counters;
    v.status = h->status;
    return v;
}

qn_status check_status(const qn_batch *h);

// Row blocks for the sigma pass (probs_parts kind) over b states, with their sigma scratch.
qn_status probs_rows(qn_batch *h, int b, AccumView *a, int kind) {
    a->parts = a->probs ? probs_parts(h->n, b, kind) : 1;
    if (a->parts > 1) {
        const int64_t need = (int64_t)(a->parts - 1) << h->n;
        if (h->spart_cap < need) {
            QN_TRY(alloc_t(h, &h->spart, (size_t)need));
            h->spart_cap = need;
        }
        a->spart = h->spart;
    }
    return QN_OK;
}

// ---- profiling: one CUDA event pair per timed launch ----
bool prof_sampled(qn_batch *h, int kind) {
    if (h->prof_period <= 0) return false;
    if (kind == 1 || kind == 2) return true;
    return (h->prof_counter++ % h->prof_period) == 0;
}

qn_status prof_begin(qn_batch *h, EventPair *ep, int kind, double bytes) {
    ep->kind = -1;
    if (!prof_sampled(h, kind)) return QN_OK;
    if (!h->spare.empty()) {
        *ep = h->spare.back();
        h->spare.pop_back();
    } else {
        QN_CUDA(cudaEventCreate(&ep->a));
        QN_CUDA(cudaEventCreate(&ep->b));
    }
    ep->kind = kind;
    ep->bytes = bytes;
    QN_CUDA(cudaEventRecord(ep->a, h->stream));
    return QN_OK;
}

qn_status prof_end(qn_batch *h, EventPair *ep) {
    if (ep->kind < 0) return QN_OK;
    QN_CUDA(cudaEventRecord(ep->b, h->stream));
    h->events.push_back(*ep);
    return QN_OK;
}

qn_status prof_collect(qn_batch *h) {
    if (h->events.empty()) return QN_OK;
    QN_CUDA(cudaStreamSynchronize(h->stream));
    for (EventPair &ep : h->events) {
        float ms = 0.0f;
        QN_CUDA(cudaEventElapsedTime(&ms, ep.a, ep.b));
        h->prof_launches[ep.kind] += 1;
        h->prof_ms[ep.kind] += ms;
        h->prof_bytes[ep.kind] += ep.bytes;
        h->spare.push_back(ep);
    }
    h->events.clear();
    return QN_OK;
}

bool use_fusion(const qn_batch *h) {
    return h->fusion && !h->damping_on && h->edges.size() / 2 <= 64 && h->n >= 2;
}

// Graph tables of the fused cost layer: EV byte tables (bit e of EV(y) set when
// the endpoints of edge e differ in y) and e^{-i gamma_l k}, k = 0..E.
qn_status prepare_fusion(qn_batch *h) {
    const int E = (int)h->edges.size() / 2;
    const int p = h->p;
    const int64_t B = h->cap_B;
    if (h->fl_cap_p < p || h->fl_cap_E != E || h->fl_cap_B < B || !h->fl_ev) {
        QN_TRY(alloc_t(h, &h->fl_ev, 1024));
        QN_TRY(alloc_t(h, &h->fl_phase, (size_t)std::max(p, 1) * (E + 1)));
        QN_TRY(alloc_t(h, &h->fl_edges, (size_t)std::max(E, 1)));
        QN_TRY(alloc_t(h, &h->fl_s, (size_t)std::max(p, 1) * B));
        QN_TRY(alloc_t(h, &h->fl_u, (size_t)std::max(p, 1) * 4 * B));
        h->fl_cap_p = p;
        h->fl_cap_E = E;
        h->fl_cap_B = B;
    }
    std::vector<uint64_t> col((size_t)h->n, 0);
    for (int e = 0; e < E; ++e) {
        col[h->edges[2 * e]] ^= (uint64_t)1 << e;
        col[h->edges[2 * e + 1]] ^= (uint64_t)1 << e;
    }
    h->ev_host.assign(1024, 0);
    for (int b = 0; b < 4; ++b)
        for (int v = 0; v < 256; ++v) {
            uint64_t acc = 0;
            for (int k = 0; k < 8; ++k)
                if ((v >> k) & 1) {
                    const int q = 8 * b + k;
                    if (q < h->n) acc ^= col[q];
                }
            h->ev_host[(size_t)b * 256 + v] = acc;
        }
    h->phase_host.assign((size_t)std::max(p, 1) * (E + 1), make_float2(1.0f, 0.0f));
    for (int l = 0; l < p; ++l)
        for (int k = 0; k <= E; ++k)
            h->phase_host[(size_t)l * (E + 1) + k] =
                make_float2((float)std::cos(h->gammas[l] * k), (float)-std::sin(h->gammas[l] * k));
    QN_CUDA(cudaMemcpyAsync(h->fl_ev, h->ev_host.data(), 1024 * sizeof(uint64_t), cudaMemcpyHostToDevice, h->stream));
    QN_CUDA(cudaMemcpyAsync(h->fl_phase, h->phase_host.data(), h->phase_host.size() * sizeof(float2),
                            cudaMemcpyHostToDevice, h->stream));
    if (E > 0)
        QN_CUDA(cudaMemcpyAsync(h->fl_edges, h->edges_host.data(), (size_t)E * sizeof(int2), cudaMemcpyHostToDevice,
                                h->stream));
    return QN_OK;
}

LayerView layer_view(const qn_batch *h, int l) {
    const int E = (int)h->edges.size() / 2;
    const int64_t B = h->cap_B;
    LayerView L;
    L.ev = h->fl_ev;
    L.phase = h->fl_phase + (size_t)l * (E + 1);
    L.edges = h->fl_edges;
    L.s = h->fl_s + (size_t)l * B;
    L.zm = h->fl_u + ((size_t)l * 4 + 0) * B;
    L.zc = h->fl_u + ((size_t)l * 4 + 1) * B;
    L.mz = h->fl_u + ((size_t)l * 4 + 2) * B;
    L.mf = h->fl_u + ((size_t)l * 4 + 3) * B;
    L.cb = (float)std::cos(h->betas[l]);
    L.sb = (float)std::sin(h->betas[l]);
    L.num_edges = E;
    return L;
}

// The fused mixer windows (first qubit, qubits) of one layer.  n >= 10: the window
// that holds qubit 0, then ceil(rest / kFuse) windows of balanced sizes over the rest
// (at most kFuse, the larger ones first); the first window is qubits 0 .. kFuseTile-1
// (one tile in shared memory) where that makes fewer windows than qubits
// 0 .. kFuse0-1 (n = 16-19, 23-26, 30, ...).  n < 10: windows of kFuseSmall qubits.
std::vector<std::pair<int, int>> fused_windows(int n) {
    std::vector<std::pair<int, int>> w;
    if (n < 10) {
        for (int q_lo = 0; q_lo < n; q_lo += kFuseSmall) w.emplace_back(q_lo, std::min(kFuseSmall, n - q_lo));
        return w;
    }
    auto rest_windows = [&](int first) { return (n - first + kFuse - 1) / kFuse; };
    const int first = n > kFuseTile && rest_windows(kFuseTile) < rest_windows(kFuse0) ? kFuseTile : kFuse0;
    w.emplace_back(0, first);
    const int rest = n - first;
    const int count = rest_windows(first);
    int q_lo = first;
    for (int i = 0; i < count; ++i) {
        const int m = rest / count + (i < rest % count ? 1 : 0);
        w.emplace_back(q_lo, m);
        q_lo += m;
    }
    return w;
}

// All gates after the H layer as fused sweeps over the windows of fused_windows;
// the cost phase of layer 0 rides on the first sweep and that of layer l+1 on the
// last mixer sweep of layer l.  *norms: whether the circuit's last sweep also
// formed 1/N_t (FP32 windows, last window off qubit 0), so no norm pass follows.
qn_status run_fused_gates(qn_batch *h, const BatchView &v, double amp_bytes, bool ensemble, bool *norms) {
    *norms = false;
    const int n = h->n, p = h->p;
    const int E = (int)h->edges.size() / 2;
    for (int l = 0; l < p; ++l) {
        QN_CUDA(launch_layer_params(v, layer_view(h, l), n + l * (E + n), E, h->stream));
        h->launches += 1;
    }
    EventPair ep;
    if (h->precision != kPrecFP32 && n >= 11) {
        // tensor cores: windows of five qubits, ceil(n / 5) sweeps per layer; the last window
        // of a layer is the top five qubits with only the remaining ones rotated
        for (int l = 0; l < p; ++l) {
            for (int q_lo = 0; q_lo < n; q_lo += 5) {
                const int m = std::min(5, n - q_lo);
                TcSweep sw;
                sw.wl = std::min(q_lo, n - 5);
                sw.act = ((1u << m) - 1u) << (q_lo - sw.wl);
                for (int k = 0; k < 6; ++k) {
                    const double ang = h->betas[l] * (double)(m - 2 * k);
                    sw.dph[k] = make_float2((float)(std::cos(ang) / 32.0), (float)(-std::sin(ang) / 32.0));
                }
                const bool pre = l == 0 && q_lo == 0;
                const bool post = q_lo + m >= n && l + 1 < p;
                QN_TRY(prof_begin(h, &ep, 0, amp_bytes * 16.0));
                QN_CUDA(launch_tc_sweep(v, layer_view(h, l), layer_view(h, l), layer_view(h, post ? l + 1 : l), sw, pre,
                                        post, h->precision, h->stream));
                QN_TRY(prof_end(h, &ep));
                h->launches += 1;
                if (ensemble) h->sweep_bytes += amp_bytes * 16.0;
            }
        }
        return QN_OK;
    }
    const std::vector<std::pair<int, int>> windows = fused_windows(n);
    for (int l = 0; l < p; ++l) {
        for (const auto &wd : windows) {
            const int q_lo = wd.first, m = wd.second;
            const bool pre = l == 0 && q_lo == 0;
            const bool post = q_lo + m >= n && l + 1 < p;
            const bool norm = q_lo + m >= n && l + 1 == p && q_lo > 0;
            if (norm) *norms = true;
            QN_TRY(prof_begin(h, &ep, 0, amp_bytes * 16.0));
            if (m == kFuseTile)  // never the last window of a layer (n > kFuseTile)
                QN_CUDA(launch_fused_tile12(v, layer_view(h, l), layer_view(h, l), pre, h->stream));
            else if (fused_win_ok(n, q_lo, m, post, norm))
                QN_CUDA(launch_fused_win(v, layer_view(h, l), layer_view(h, post ? l + 1 : l), q_lo, m, post, norm,
                                         h->stream));
            else
                QN_CUDA(launch_fused_sweep(v, layer_view(h, l), layer_view(h, l), layer_view(h, post ? l + 1 : l),
                                           q_lo, m, pre, post, norm, h->stream));
            QN_TRY(prof_end(h, &ep));
            h->launches += 1;
            if (ensemble) h->sweep_bytes += amp_bytes * 16.0;
        }
    }
    return QN_OK;
}

// Queue the whole pipeline for the handle's trajectories t0 .. t0+b-1 (global ids
// offset + t0 ..; b <= cap_B).
// ensemble = true adds into probs / S1 / S2 and writes c_all; otherwise the
// per-trajectory <C>_t go to c_dbg only.
qn_status run_batch(qn_batch *h, int64_t t0, int b, bool ensemble) {
    const int n = h->n;
    const int G = (int)h->gates.size();
    BatchView v = view_for(h, h->offset + t0, b);
    const double amp_bytes = (double)b * (double)((size_t)1 << n);
    QN_CUDA(launch_prepare(v, h->dgates, h->seed, h->nz, h->damping_on, h->stream));
    h->launches += 1;
    EventPair ep;
    QN_TRY(prof_begin(h, &ep, 1, amp_bytes * 8.0));
    QN_CUDA(launch_init(v, h->stream));
    QN_TRY(prof_end(h, &ep));
    h->launches += 1;
    bool norms = false;
    if (use_fusion(h)) {
        QN_TRY(run_fused_gates(h, v, amp_bytes, ensemble, &norms));
    } else {
        for (int g = n; g < G; ++g) {
            QN_TRY(prof_begin(h, &ep, 0, amp_bytes * 16.0));
            QN_CUDA(launch_sweep(v, g, h->dgates_host[g], h->nz, h->damping_on, h->stream));
            QN_TRY(prof_end(h, &ep));
            h->launches += 1;
            if (ensemble) h->sweep_bytes += amp_bytes * 16.0;
        }
    }
    AccumView a;
    a.num_edges = (int32_t)h->edges_host.size();
    a.edges = h->dedges;
    a.order = nullptr;
    a.weights = nullptr;
    a.cpart = h->cpart;
    a.acc_counter = h->acc_counter;
    a.c_out = ensemble ? h->c_all + t0 : h->c_dbg;
    a.probs = ensemble ? h->probs : nullptr;
    a.sums = ensemble ? h->sums : nullptr;
    QN_TRY(probs_rows(h, b, &a, 0));
    if (!norms) {
        QN_TRY(prof_begin(h, &ep, 2, amp_bytes * 8.0));
        QN_CUDA(launch_observe(v, a, h->stream));
        QN_TRY(prof_end(h, &ep));
        h->launches += 1;
    }
    QN_TRY(prof_begin(h, &ep, 2, amp_bytes * 8.0));
    QN_CUDA(launch_probs(v, a, h->stream));
    QN_TRY(prof_end(h, &ep));
    h->launches += 1 + (a.parts > 1 ? 1 : 0);
    return QN_OK;
}

// Shared-prefix run of trajectories t0 .. t0 + kc - 1 (kc <= cap_B): one slot
// per distinct Kraus prefix, forked on the device as branches diverge.
// The device view of group gi (the group after it: nz, or nullptr) for a prefix tree of kc
// trajectories.
GroupView group_view(qn_batch *h, int gi, const GateGroup *nz, const SlotView &sv, int kc) {
    const GateGroup &z = h->groups[gi];
    GroupView gv;
    gv.grp = h->gr_dev + gi;
    gv.next = nz && nz->kind == 0 ? h->gr_dev + gi + 1 : nullptr;
    gv.vc = nz ? nz->c : 1.0f;
    gv.vs = nz ? nz->sn : 0.0f;
    gv.Hcur = h->gv_H + (size_t)(gi & 1) * h->gv_cap * kGroupBins;
    gv.Hnext = h->gv_H + (size_t)((gi + 1) & 1) * h->gv_cap * kGroupBins;
    gv.T = h->gv_T;
    gv.st_prev = h->gv_stprev;
    gv.ekey = h->gv_ekey;
    gv.evt = h->gv_i32;
    gv.rep = h->gv_i32 + h->gv_cap;
    gv.lead = h->gv_i32 + 2 * h->gv_cap;
    gv.lstart = h->gv_i32 + 3 * h->gv_cap;
    gv.lcount = h->gv_i32 + 4 * h->gv_cap;
    gv.parent = h->gv_i32 + 5 * h->gv_cap;
    gv.pos_slot = h->gv_i32 + 6 * h->gv_cap;
    gv.members = kc;
    gv.Htrue = h->gv_htrue;
    gv.p1m = h->gv_p1m;
    gv.cls = h->gv_cls;
    gv.ncls = sv.fork_count;  // reset by the fork-finish kernel
    gv.src = nullptr;
    gv.slot_base = 0;
    // a group right after the H layer or after another group finds no pending op
    // (decides leave none); one after a per-gate sweep may
    gv.pend = !(z.g0 == h->n || (gi > 0 && h->groups[gi - 1].g0 + h->groups[gi - 1].m == z.g0));
    return gv;
}

// The tile map of the sweep that applies group z (the group after it: nz): a mixer block's
// own map, or for the layer's last phase group (wide_next) the map of the rotations of
// qubits 0-3 that its sweep also applies.  keep: the circuit's last block, a full block off
// qubit 0 whose states the sigma pass reads anyway -- no sweep applies it: the sigma pass does.
MixMap group_mix_map(const qn_batch *h, const GateGroup &z, const GateGroup *nz, bool wide_next) {
    const int n = h->n;
    const int G = (int)h->gates.size();
    MixMap mm;
    if (wide_next) {
        mm = mix_map(n, 0, kMixQ, {4, 5, 6, 7});
        mm.tanf = std::fabs(nz->c) >= std::fabs(nz->sn);
        mm.full8 = h->split8;  // rotate qubits 4-7 as well
    }
    if (z.kind != 1) return mm;
    std::vector<int> next;
    if (nz && nz->kind == 1)
        for (int k = 0; k < nz->s; ++k) next.push_back(nz->sp[k]);
    const bool wide = z.s == kWideBlock;
    if (wide && z.sp[0] == 0 && h->split8) {
        // the factors of 0-7 (all rotated before), the rotations of 8-11 and the
        // joint of 8-15 (12-15 rotated without being kept)
        mm = mix_map(n, kWideBlock, kMixQ, {12, 13, 14, 15});
        mm.wide = 2;
        mm.wsh = 3;  // qubits 4-7: f bits 3-6
    } else if (wide && z.sp[0] == kWideBlock) {
        // the second half of 8-15: the rotations of 12-15, then the block's factors
        mm = mix_map(n, kWideBlock + kMixQ, kMixQ, next);
        mm.wide = 3;
        mm.wsh = kWideBlock - 1;  // qubits 8-11: f bits 7-10
    } else {
        // a block over 0-7 whose qubits 0-3 the sweep before rotated, or kMixQ qubits
        mm = wide ? mix_map(n, kMixQ, kMixQ, next) : mix_map(n, z.sp[0], z.s, next);
        mm.wide = wide ? 1 : 0;
    }
    mm.tanf = std::fabs(z.c) >= std::fabs(z.sn);
    mm.final_norm = z.g0 + z.m == G;  // the circuit's last sweep
    const bool next_phase = nz && nz->kind == 0;
    // its states are read once more by the sigma pass anyway: let that pass apply the block,
    // so no state is written and no sweep runs
    if (mm.final_norm && mm.M == kMixQ && !mm.has0 && mm.nN == 0 && !next_phase) mm.keep = 1;
    return mm;
}

// What the readout needs about the circuit's last mixer block z when its sweep kept the
// states (first_new: the slots from there on were forked at the block).
ReadTail keep_read_tail(const GateGroup &z, const GroupView &gv, int32_t first_new) {
    ReadTail rt{};
    rt.keep = 1;
    rt.M = z.s;
    for (int k = 0; k < kMixQ; ++k) rt.q[k] = k < z.s ? z.sp[k] : 0;
    rt.c = z.c;
    rt.s = z.sn;
    rt.T = gv.T;
    rt.parent = gv.parent;
    rt.first_new = first_new;
    return rt;
}

// The sigma pass's view of a shared-prefix run's accumulators (slot order and weights in
// sh_order, sh_weights); trivial_pending: the last sweep left no pending op.
AccumView shared_accum(qn_batch *h, bool trivial_pending) {
    AccumView a;
    a.num_edges = (int32_t)h->edges_host.size();
    a.edges = h->dedges;
    a.order = h->sh_order;
    a.weights = h->sh_weights;
    a.cpart = h->cpart;
    a.acc_counter = h->acc_counter;
    a.c_out = h->c_dbg;
    a.probs = h->probs;
    a.sums = h->sums;
    a.trivial_pending = trivial_pending ? 1 : 0;
    return a;
}


// The shared-prefix run after its noisy H layer with device-driven launches: every sweep
// is a persistent launch over the slots the device counts, every decide kernel reads the
// live-slot count on the device, the sigma pass takes its order and weights from a device
// step, and nothing is read back until the run is over.  The same launches (arguments and
// grids) come out whatever the draws, so a captured run replays for any seed and range of
// trajectories of the same circuit.  `st` is the handle's stream, or the capture stream.
qn_status enqueue_shared_dev(qn_batch *h, const BatchView &vh, const SlotView &svh, int kc, cudaStream_t st,
                             bool profile, DevRun *out) {
    const int n = h->n;
    const int G = (int)h->gates.size();
    const bool grouped = use_groups(h);
    DevRun &r = *out;
    BatchView v = vh;
    v.t0 = 0;  // only k_prepare reads the global ids
    v.b = kc;
    SlotView sv = svh;
    sv.dyn = 1;
    sv.prev_active = h->sh_ctr + 3;
    sv.live_log = h->sh_log;
    // a sweep over the slots [*lo, *hi) with a work counter of its own
    int64_t queues = 0;
    auto over = [&](const int32_t *lo, const int32_t *hi) {
        BatchView w = v;
        w.dyn_lo = lo;
        w.dyn_hi = hi;
        w.dyn_queue = h->sh_queue + std::min<int64_t>(queues++, h->sh_queue_cap - 1);
        return w;
    };
    auto v_all = [&]() { return over(nullptr, sv.active); };         // the live slots
    auto v_new = [&]() { return over(sv.prev_active, sv.active); };  // the slots forked by the last decide
    auto v_old = [&]() { return over(nullptr, sv.prev_active); };    // the slots live before it
    const double amp = (double)((size_t)1 << n);
    QN_CUDA(cudaMemsetAsync(h->sh_queue, 0, (size_t)h->sh_queue_cap * sizeof(int32_t), st));
    int32_t decides = 0;
    EventPair ep;
    auto begin = [&](int kind, double per_state) -> qn_status {
        ep.kind = -1;
        if (!profile) return QN_OK;
        QN_TRY(prof_begin(h, &ep, kind, 0.0));
        ep.log_k = decides;
        ep.per_state = per_state;
        return QN_OK;
    };
    auto end = [&]() -> qn_status { return profile ? prof_end(h, &ep) : QN_OK; };
    QN_CUDA(cudaMemsetAsync(h->sh_log, 0, sizeof(int32_t), st));
    QN_TRY(begin(1, 8.0 * amp));
    QN_CUDA(launch_init(over(nullptr, sv.slot_count), st));
    QN_TRY(end());
    r.launches += 1;
    bool final_norms = false, keep = false;
    MixMap keep_mm;
    MixTail keep_tail{};
    for (int g = n; g < G; ++g) {
        const int gi = grouped ? h->group_at[g] : -1;
        if (gi >= 0) {
            const GateGroup &z = h->groups[gi];
            const int ng = (int)h->groups.size();
            const GateGroup *nz = gi + 1 < ng && h->groups[gi + 1].g0 == z.g0 + z.m ? &h->groups[gi + 1] : nullptr;
            const bool first = z.kind == 0 && (gi == 0 || h->groups[gi - 1].g0 + h->groups[gi - 1].m != z.g0);
            const bool wide_next = z.kind == 0 && nz && nz->kind == 1 && nz->s == kWideBlock && nz->sp[0] == 0;
            GroupView gv = group_view(h, gi, nz, sv, kc);
            if (first) {
                QN_TRY(begin(3, 8.0 * amp));
                QN_CUDA(launch_group_hist(v_all(), sv, gv, kc, st));
                QN_TRY(end());
                r.acct.emplace_back(decides, 8.0 * amp);
                r.launches += 1;
            }
            const MixMap mm = group_mix_map(h, z, nz, wide_next);
            const bool last_block = z.kind == 1 && mm.keep;  // applied by the sigma pass, not swept
            gv.final_norm = last_block ? 1 : 0;
            QN_CUDA(launch_group_decide(v, sv, gv, z.s, kc, h->nz.gamma, st));
            ++decides;
            if (z.kind == 1) final_norms = final_norms || mm.final_norm;
            if (last_block) {
                keep = true;
                keep_mm = mm;
                keep_tail.grp = gv.grp;
                keep_tail.T = gv.T;
                keep_tail.parent = gv.parent;
                keep_tail.first_new_dev = sv.prev_active;
                r.read_tail = keep_read_tail(z, gv, 0);
                r.launches += 2;  // decide, finish
                g += z.m - 1;
                continue;
            }
            const double per_state = 16.0 * amp;
            QN_TRY(begin(z.kind == 0 ? 3 : 4, per_state));
            for (int part = 0; part < 2; ++part) {
                const BatchView vp = part == 0 ? v_new() : v_old();
                gv.src = part == 0 ? gv.parent : nullptr;
                gv.slot_base = 0;
                QN_CUDA(z.kind == 1 ? launch_mix_sweep(vp, gv, mm, kc, st)
                        : wide_next ? launch_group_mix(vp, gv, mm, kc, st)
                                    : launch_group_apply(vp, sv, gv, kc, st));
            }
            QN_TRY(end());
            r.acct.emplace_back(decides, per_state);
            r.launches += 4;  // decide, finish, the two sweeps
            g += z.m - 1;
            continue;
        }
        QN_TRY(begin(0, 16.0 * amp));
        QN_CUDA(launch_slot_sweep(v_all(), sv, kc, g, h->dgates_host[g], h->damping_on, st));
        QN_TRY(end());
        QN_CUDA(launch_slot_fork(v, sv, kc, g, h->dgates_host[g], h->nz, h->damping_on, st));
        r.acct.emplace_back(decides, 16.0 * amp);
        ++decides;
        r.launches += 4;
    }
    // the sigma pass over the final slots, in the order of their first members
    QN_CUDA(launch_slot_order(sv, sv.tmp, h->sh_order, h->sh_weights, kc, h->status, st));
    AccumView a = shared_accum(h, final_norms);
    const int kind = keep ? 2 : (final_norms ? 1 : 0);
    a.rows = probs_row_plan(n, kind);
    a.rows.used = 1;
    a.parts = a.rows.pmax;
    a.spart = a.parts > 1 ? h->spart : nullptr;
    QN_TRY(begin(2, (final_norms ? 8.0 : 16.0) * amp));
    if (!final_norms) QN_CUDA(launch_observe(v_all(), a, st));
    const BatchView vo = over(nullptr, sv.active);  // the sigma pass reads only the state count
    if (keep) QN_CUDA(launch_probs_mix(vo, a, keep_mm, keep_tail, st));
    else QN_CUDA(launch_probs(vo, a, st));
    if (queues > h->sh_queue_cap) return fail(QN_ESTATE, "device-driven run needs %lld work counters (%lld)",
                                              (long long)queues, (long long)h->sh_queue_cap);
    QN_TRY(end());
    r.launches += 3 + (final_norms ? 0 : 1) + (a.parts > 1 ? 1 : 0);  // order (2), observe, probs, combine
    r.decides = decides;
    return QN_OK;
}

// Bytes that fix every launch of a device-driven run (kernel arguments and grids): the
// handle's buffers, the circuit, the noise and the launch batch.  Equal signatures give
// the same launches, so a captured graph of one run serves the other.
std::string dev_signature(const qn_batch *h, const BatchView &v, const SlotView &sv, int kc) {
    std::string sig;
    auto put = [&](const void *p, size_t nb) { sig.append(reinterpret_cast<const char *>(p), nb); };
    // field by field: the structs' padding bytes are not initialised
    const void *vp[] = {v.psi, v.branch, v.dwords, v.frame_x, v.yphase, v.hfac, v.st, v.partials, v.inv_norm,
                        v.counters, v.status, sv.members, sv.tmp, sv.cls, sv.range, sv.slot_count, sv.active,
                        sv.forks, sv.fork_count, sv.marg};
    put(vp, sizeof vp);
    const int32_t vi[] = {v.n, v.b, v.G, v.tiles, v.stiles, sv.max_slots, kc};
    put(vi, sizeof vi);
    put(&h->nz.gamma, sizeof h->nz.gamma);
    put(h->nz.thr1, sizeof h->nz.thr1);
    put(h->nz.thr2, sizeof h->nz.thr2);
    put(&h->damping_on, sizeof h->damping_on);
    put(&h->fusion, sizeof h->fusion);
    const int32_t split = h->split8 ? 1 : 0;
    put(&split, sizeof split);
    for (const DevGate &g : h->dgates_host) {
        const int32_t gi[] = {g.kind, g.q0, g.q1};
        const float gf[] = {g.c, g.s};
        put(gi, sizeof gi);
        put(gf, sizeof gf);
    }
    static_assert(sizeof(GateGroup) == 4 * (4 + kMaxGroupQubits + 2 * kMaxGroupEdges + 2) + 2 * 4 * 256,
                  "GateGroup has no padding");
    if (!h->groups.empty()) put(h->groups.data(), h->groups.size() * sizeof(GateGroup));
    if (!h->group_at.empty()) put(h->group_at.data(), h->group_at.size() * sizeof(int32_t));
    const int32_t ne = (int32_t)h->edges_host.size();
    put(&ne, sizeof ne);
    const void *ptrs[] = {h->gr_dev, h->gv_H, h->gv_T, h->gv_stprev, h->gv_ekey, h->gv_i32, h->gv_htrue,
                          h->gv_p1m, h->gv_cls, h->sh_log, h->sh_queue, h->sh_order, h->sh_weights, h->cpart,
                          h->acc_counter,
                          h->c_dbg, h->probs, h->sums, h->dedges, h->spart};
    put(ptrs, sizeof ptrs);
    put(&h->gv_cap, sizeof h->gv_cap);
    put(&h->sh_queue_cap, sizeof h->sh_queue_cap);
    return sig;
}

// A shared-prefix run with device-driven launches (launch modes 1 and 2), after its noisy
// H layer was grouped into ns slots: enqueue (mode 1), or replay / capture and replay the
// CUDA graph of the run (mode 2); then, once it is over, read what the host keeps of it.
qn_status run_shared_dev(qn_batch *h, const BatchView &v, const SlotView &sv, int64_t t0, int kc, int ns) {
    const int n = h->n;
    DevRun run;
    if (h->launch_mode == 2) {
        std::string sig = dev_signature(h, v, sv, kc);
        if (!h->graph_exec || sig != h->graph_sig) {
            if (!h->cap_stream) QN_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
            QN_CUDA(prewarm_dev_launches());
            QN_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
            const qn_status st = enqueue_shared_dev(h, v, sv, kc, h->cap_stream, false, &run);
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &graph);
            if (st != QN_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (ec != cudaSuccess) return fail(QN_ECUDA, "capturing the run: %s", cudaGetErrorString(ec));
            cudaError_t e = cudaErrorUnknown;
            if (h->graph_exec) {
                // same launches in the same order (another circuit of the same shape): update in place
                cudaGraphExecUpdateResultInfo info{};
                e = cudaGraphExecUpdate(h->graph_exec, graph, &info);
                if (e == cudaSuccess) h->graph_updates += 1;
                else {
                    (void)cudaGetLastError();
                    cudaGraphExecDestroy(h->graph_exec);
                    h->graph_exec = nullptr;
                }
            }
            if (!h->graph_exec) e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                h->graph_exec = nullptr;
                h->graph_sig.clear();
                return fail(QN_ECUDA, "instantiating the run's graph: %s", cudaGetErrorString(e));
            }
            h->graph_sig = std::move(sig);
            h->graph_run = run;
            h->graph_captures += 1;
        } else {
            run = h->graph_run;
            h->graph_replays += 1;
        }
        QN_CUDA(cudaGraphLaunch(h->graph_exec, h->stream));
    } else {
        QN_TRY(enqueue_shared_dev(h, v, sv, kc, h->stream, true, &run));
    }
    h->launches += run.launches;
    // once the run is over: its status, the live-slot log, and the final slots
    QN_TRY(check_status(h));  // synchronises
    int32_t ctr[4] = {0, 0, 0, 0};
    QN_CUDA(cudaMemcpy(ctr, h->sh_ctr, sizeof ctr, cudaMemcpyDeviceToHost));
    std::vector<int32_t> log((size_t)run.decides + 1, 0);
    QN_CUDA(cudaMemcpy(log.data(), h->sh_log, log.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    const int nslots = ctr[1];
    if (ctr[0] > kc || nslots > kc || nslots < 1)
        return fail(QN_ESTATE, "shared-prefix run created %d slots for %d trajectories", ctr[0], kc);
    auto live_after = [&](int k) { return k == 0 ? ns : log[std::min<size_t>((size_t)k, log.size() - 1)]; };
    for (const auto &a : run.acct) h->sweep_bytes += (double)live_after(a.first) * a.second;
    for (EventPair &ep : h->events)
        if (ep.log_k >= 0) {
            ep.bytes = (double)live_after(ep.log_k) * ep.per_state;
            ep.log_k = -1;
        }
    std::vector<int2> fr((size_t)nslots);
    std::vector<int32_t> fm((size_t)kc), order((size_t)nslots);
    QN_CUDA(cudaMemcpy(fr.data(), h->sh_range, fr.size() * sizeof(int2), cudaMemcpyDeviceToHost));
    QN_CUDA(cudaMemcpy(fm.data(), h->sh_members, fm.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    QN_CUDA(cudaMemcpy(order.data(), h->sh_order, order.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    h->sh_slots += nslots;
    h->sh_valid = true;
    h->sh_last_t0 = t0;
    h->sh_last_kc = kc;
    h->sh_range_host = std::move(fr);
    h->sh_members_host = std::move(fm);
    h->sh_order_host = std::move(order);
    h->sh_tail = run.read_tail;
    h->sh_tail.first_new = ctr[3];  // the live slots before the last decide
    (void)n;
    return QN_OK;
}

qn_status run_shared(qn_batch *h, int64_t t0, int kc) {
    const int n = h->n;
    const int G = (int)h->gates.size();
    if (h->sh_cap < kc) {
        QN_TRY(alloc_t(h, &h->sh_members, (size_t)kc));
        QN_TRY(alloc_t(h, &h->sh_tmp, (size_t)kc));
        QN_TRY(alloc_t(h, &h->sh_cls, (size_t)kc));
        QN_TRY(alloc_t(h, &h->sh_range, (size_t)kc));
        QN_TRY(alloc_t(h, &h->sh_forks, (size_t)kc));
        QN_TRY(alloc_t(h, &h->sh_ctr, 4));
        QN_TRY(alloc_t(h, &h->sh_order, (size_t)kc));
        QN_TRY(alloc_t(h, &h->sh_weights, (size_t)kc));
        QN_TRY(alloc_t(h, &h->sh_marg, (size_t)kc * 4));
        h->sh_cap = kc;
    }
    const bool grouped = use_groups(h);
    if (grouped && h->gv_cap < kc) {
        QN_TRY(alloc_t(h, &h->gv_H, (size_t)2 * kc * kGroupBins));
        QN_TRY(alloc_t(h, &h->gv_T, (size_t)kc * kGroupBins));
        QN_TRY(alloc_t(h, &h->gv_stprev, (size_t)kc));
        QN_TRY(alloc_t(h, &h->gv_ekey, (size_t)kc));
        QN_TRY(alloc_t(h, &h->gv_i32, (size_t)7 * kc));
        QN_TRY(alloc_t(h, &h->gv_htrue, (size_t)kc * kGroupBins));
        QN_TRY(alloc_t(h, &h->gv_p1m, (size_t)kc * 2 * kMaxGroupEdges));
        QN_TRY(alloc_t(h, &h->gv_cls, (size_t)kc));
        h->gv_cap = kc;
    }
    if (grouped && h->gr_cap < (int64_t)h->groups.size()) {
        QN_TRY(alloc_t(h, &h->gr_dev, h->groups.size()));
        h->gr_cap = (int64_t)h->groups.size();
    }
    if (h->launch_mode != 0) {
        // device-driven: the live-slot log (one entry per decide), and sigma scratch for the
        // most row blocks the device may choose
        const int64_t need_log = (int64_t)G - n + 2;
        if (h->sh_log_cap < need_log) {
            QN_TRY(alloc_t(h, &h->sh_log, (size_t)need_log));
            h->sh_log_cap = need_log;
        }
        const int64_t need_queue = 3 * ((int64_t)G - n) + 8;  // at most three sweeps per gate, init, observe
        if (h->sh_queue_cap < need_queue) {
            QN_TRY(alloc_t(h, &h->sh_queue, (size_t)need_queue));
            h->sh_queue_cap = need_queue;
        }
        const int pmax = probs_row_plan(n, 0).pmax;
        const int64_t need = (int64_t)(pmax - 1) << n;
        if (pmax > 1 && h->spart_cap < need) {
            QN_TRY(alloc_t(h, &h->spart, (size_t)need));
            h->spart_cap = need;
        }
    }
    if (grouped) {
        QN_CUDA(cudaMemcpyAsync(h->gr_dev, h->groups.data(), h->groups.size() * sizeof(GateGroup),
                                cudaMemcpyHostToDevice, h->stream));
        QN_CUDA(cudaMemsetAsync(h->gv_H, 0, sizeof(unsigned long long) * 2 * (size_t)h->gv_cap * kGroupBins,
                                h->stream));
    }
    BatchView v = view_for(h, h->offset + t0, kc);
    QN_CUDA(launch_prepare(v, h->dgates, h->seed, h->nz, h->damping_on, h->stream));
    h->launches += 1;
    // group the trajectories by their noisy H-layer outcome (the first n branch bytes)
    std::vector<uint8_t> hbr((size_t)kc * n);
    std::vector<TrajState> tst((size_t)kc);
    std::vector<uint32_t> fx((size_t)kc);
    std::vector<float> hf((size_t)kc * n * 2);
    QN_CUDA(cudaMemcpy2DAsync(hbr.data(), n, h->branch, G, n, kc, cudaMemcpyDeviceToHost, h->stream));
    QN_CUDA(cudaMemcpyAsync(tst.data(), h->st, (size_t)kc * sizeof(TrajState), cudaMemcpyDeviceToHost, h->stream));
    QN_CUDA(cudaMemcpy2DAsync(fx.data(), sizeof(uint32_t), h->frame_x + n, (size_t)(G + 1) * sizeof(uint32_t),
                              sizeof(uint32_t), kc, cudaMemcpyDeviceToHost, h->stream));
    QN_CUDA(cudaMemcpyAsync(hf.data(), h->hfac, hf.size() * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    QN_CUDA(cudaStreamSynchronize(h->stream));
    // key: the n outcome bytes (n <= 30) packed into four words; groups in order of first occurrence
    struct HKey {
        uint64_t w[4];
        bool operator==(const HKey &o) const {
            return w[0] == o.w[0] && w[1] == o.w[1] && w[2] == o.w[2] && w[3] == o.w[3];
        }
    };
    struct HKeyHash {
        size_t operator()(const HKey &k) const {
            uint64_t x = 0;
            for (int i = 0; i < 4; ++i) x = (x ^ k.w[i]) * 0x9E3779B97F4A7C15ull;
            return (size_t)(x ^ (x >> 29));
        }
    };
    static_assert(kMaxQubits <= 32, "the H-layer key holds 32 bytes");
    std::unordered_map<HKey, int, HKeyHash> key_slot;
    key_slot.reserve((size_t)std::min(kc, 1 << 16));
    std::vector<std::vector<int32_t>> groups;
    for (int t = 0; t < kc; ++t) {
        HKey key{{0, 0, 0, 0}};
        std::memcpy(key.w, &hbr[(size_t)t * n], (size_t)n);
        auto it = key_slot.find(key);
        if (it == key_slot.end()) {
            key_slot.emplace(key, (int)groups.size());
            groups.push_back({t});
        } else {
            groups[it->second].push_back(t);
        }
    }
    const int ns = (int)groups.size();
    std::vector<int32_t> members;
    std::vector<int2> range((size_t)ns);
    std::vector<TrajState> sst((size_t)ns);
    std::vector<float> shf((size_t)ns * n * 2);
    for (int sl = 0; sl < ns; ++sl) {
        range[sl] = make_int2((int)members.size(), (int)groups[sl].size());
        members.insert(members.end(), groups[sl].begin(), groups[sl].end());
        const int rep = groups[sl][0];
        TrajState st;
        st.J = fx[rep] ^ tst[rep].J;
        st.pend = 0;
        st.pq0 = st.pq1 = 0;
        st.f[0] = st.f[1] = st.f[2] = st.f[3] = 1.0f;
        sst[sl] = st;
        std::copy(hf.begin() + (size_t)rep * n * 2, hf.begin() + (size_t)(rep + 1) * n * 2,
                  shf.begin() + (size_t)sl * n * 2);
    }
    const int32_t ctr[4] = {ns, ns, 0, 0};  // slot_count, active, fork_count
    QN_CUDA(cudaMemcpyAsync(h->sh_members, members.data(), members.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                            h->stream));
    QN_CUDA(cudaMemcpyAsync(h->sh_range, range.data(), range.size() * sizeof(int2), cudaMemcpyHostToDevice,
                            h->stream));
    QN_CUDA(cudaMemcpyAsync(h->st, sst.data(), sst.size() * sizeof(TrajState), cudaMemcpyHostToDevice, h->stream));
    QN_CUDA(cudaMemcpyAsync(h->hfac, shf.data(), shf.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    QN_CUDA(cudaMemcpyAsync(h->sh_ctr, ctr, sizeof ctr, cudaMemcpyHostToDevice, h->stream));
    QN_CUDA(cudaMemsetAsync(h->frame_x, 0, (size_t)kc * (G + 1) * sizeof(uint32_t), h->stream));
    QN_CUDA(cudaMemsetAsync(h->counters, 0, (size_t)kc * sizeof(unsigned int), h->stream));
    QN_CUDA(cudaStreamSynchronize(h->stream));  // host vectors above go out of scope

    SlotView sv;
    sv.members = h->sh_members;
    sv.tmp = h->sh_tmp;
    sv.cls = h->sh_cls;
    sv.range = h->sh_range;
    sv.slot_count = h->sh_ctr;
    sv.active = h->sh_ctr + 1;
    sv.forks = h->sh_forks;
    sv.fork_count = h->sh_ctr + 2;
    sv.marg = h->sh_marg;
    sv.max_slots = kc;
    if (h->launch_mode != 0) return run_shared_dev(h, v, sv, t0, kc, ns);

    BatchView vs = v;
    vs.b = ns;
    EventPair ep;
    QN_TRY(prof_begin(h, &ep, 1, (double)ns * 8.0 * (double)((size_t)1 << n)));
    QN_CUDA(launch_init(vs, h->stream));
    QN_TRY(prof_end(h, &ep));
    h->launches += 1;
    // the live-slot count is read into the handle's page-locked word (from a pool that
    // is never freed: cudaFreeHost would synchronise the device), else a pageable one
    if (!h->pinned_tried) {
        h->pinned_tried = true;
        h->pinned_word = pinned_word_take();
    }
    int32_t active_word = ns;
    int32_t *active_host = h->pinned_word ? h->pinned_word : &active_word;
    *active_host = ns;
    int active = ns;
    bool final_norms = false;  // the last sweep formed 1 / ||psi||^2 of every state
    // the last sweep kept the states (a full mixer block off qubit 0): the sigma pass applies it
    bool keep = false;
    MixMap keep_mm;
    MixTail keep_tail{};
    ReadTail read_tail{};
    const double amp_count = (double)((size_t)1 << n);
    for (int g = n; g < G; ++g) {
        const int gi = grouped ? h->group_at[g] : -1;
        if (gi >= 0) {
            // a group: (joint pass,) decide + forks, one sweep that applies the
            // group and forms the next group's joint
            const GateGroup &z = h->groups[gi];
            const int ng = (int)h->groups.size();
            const GateGroup *nz = gi + 1 < ng && h->groups[gi + 1].g0 == z.g0 + z.m ? &h->groups[gi + 1] : nullptr;
            // a phase group needs its own joint pass unless the sweep before it
            // (a phase group or the previous layer's last mixer block) formed it
            const bool first = z.kind == 0 && (gi == 0 || h->groups[gi - 1].g0 + h->groups[gi - 1].m != z.g0);
            // a phase group before the layer's first mixer block (qubits 0-7) also rotates qubits
            // 0-3 and forms that block's joint (k_group_mix)
            const bool wide_next = z.kind == 0 && nz && nz->kind == 1 && nz->s == kWideBlock && nz->sp[0] == 0;
            GroupView gv = group_view(h, gi, nz, sv, kc);
            cudaError_t e = cudaSuccess;
            if (first) {
                QN_TRY(prof_begin(h, &ep, 3, (double)active * 8.0 * amp_count));
                e = launch_group_hist(v, sv, gv, active, h->stream);
                if (e == cudaSuccess) QN_TRY(prof_end(h, &ep));
                h->sweep_bytes += (double)active * 8.0 * amp_count;
                h->launches += 1;
            }
            const MixMap mm = group_mix_map(h, z, nz, wide_next);
            // the circuit's last mixer block, a full block off qubit 0: its states are read once
            // more by the sigma pass anyway, so no sweep applies it -- that pass does, on the fly,
            // and the decide forms the final norms from the joint the block was drawn from
            const bool last_block = z.kind == 1 && mm.keep;
            gv.final_norm = last_block ? 1 : 0;
            if (e == cudaSuccess) e = launch_group_decide(v, sv, gv, z.s, active, h->nz.gamma, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(active_host, sv.active, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                                      h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return fail(QN_ECUDA, "shared-prefix group at gate %d: %s", g, cudaGetErrorString(e));
            const int old_active = active;
            active = *active_host;
            if (z.kind == 1) final_norms = final_norms || mm.final_norm;
            if (last_block) {
                keep = true;
                keep_mm = mm;
                keep_tail.grp = gv.grp;
                keep_tail.T = gv.T;
                keep_tail.parent = gv.parent;
                keep_tail.first_new = old_active;
                read_tail = keep_read_tail(z, gv, old_active);
                h->launches += 2;  // decide, finish
                g += z.m - 1;
                continue;
            }
            // the slots forked here first, reading their parents' states; then
            // the older slots in place (the launch order keeps parents unread-over)
            const double sweep_b = (double)active * 16.0 * amp_count;
            QN_TRY(prof_begin(h, &ep, z.kind == 0 ? 3 : 4, sweep_b));
            for (int part = 0; part < 2 && e == cudaSuccess; ++part) {
                const int first = part == 0 ? old_active : 0;
                const int count = part == 0 ? active - old_active : old_active;
                if (count <= 0) continue;
                gv.src = part == 0 ? gv.parent : nullptr;
                gv.slot_base = first;
                e = z.kind == 1 ? launch_mix_sweep(v, gv, mm, count, h->stream)
                    : wide_next ? launch_group_mix(v, gv, mm, count, h->stream)
                                : launch_group_apply(v, sv, gv, count, h->stream);
                h->launches += 1;
            }
            if (e != cudaSuccess) return fail(QN_ECUDA, "shared-prefix group at gate %d: %s", g, cudaGetErrorString(e));
            QN_TRY(prof_end(h, &ep));
            h->sweep_bytes += sweep_b;
            h->launches += 2;  // decide, finish
            g += z.m - 1;
            continue;
        }
        QN_TRY(prof_begin(h, &ep, 0, (double)active * 16.0 * (double)((size_t)1 << n)));
        cudaError_t e = launch_slot_sweep(v, sv, active, g, h->dgates_host[g], h->damping_on, h->stream);
        if (e == cudaSuccess) {
            QN_TRY(prof_end(h, &ep));
            e = launch_slot_fork(v, sv, active, g, h->dgates_host[g], h->nz, h->damping_on, h->stream);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(active_host, sv.active, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                                  h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return fail(QN_ECUDA, "shared-prefix gate %d: %s", g, cudaGetErrorString(e));
        h->sweep_bytes += (double)active * 16.0 * (double)((size_t)1 << n);
        active = *active_host;
        h->launches += 4;
    }
    // deterministic accumulation order: slots by their first member
    int32_t nslots = 0;
    QN_CUDA(cudaMemcpyAsync(&nslots, h->sh_ctr, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    QN_TRY(check_status(h));  // synchronises
    if (nslots > kc) return fail(QN_ESTATE, "shared-prefix run created %d slots for %d trajectories", nslots, kc);
    std::vector<int2> fr((size_t)nslots);
    std::vector<int32_t> fm((size_t)kc);
    QN_CUDA(cudaMemcpyAsync(fr.data(), h->sh_range, fr.size() * sizeof(int2), cudaMemcpyDeviceToHost, h->stream));
    QN_CUDA(cudaMemcpyAsync(fm.data(), h->sh_members, fm.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    QN_CUDA(cudaStreamSynchronize(h->stream));
    std::vector<int32_t> order((size_t)nslots);
    std::vector<double> weights((size_t)nslots);
    for (int sl = 0; sl < nslots; ++sl) {
        order[sl] = sl;
        weights[sl] = (double)fr[sl].y;
    }
    std::sort(order.begin(), order.end(), [&](int a, int b) { return fm[fr[a].x] < fm[fr[b].x]; });
    QN_CUDA(cudaMemcpyAsync(h->sh_order, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                            h->stream));
    QN_CUDA(cudaMemcpyAsync(h->sh_weights, weights.data(), weights.size() * sizeof(double), cudaMemcpyHostToDevice,
                            h->stream));
    BatchView vo = v;
    vo.b = nslots;
    AccumView a = shared_accum(h, final_norms);  // the last sweep left no pending op
    QN_TRY(probs_rows(h, nslots, &a, keep ? 2 : (final_norms ? 1 : 0)));
    QN_TRY(prof_begin(h, &ep, 2, (double)nslots * (final_norms ? 8.0 : 16.0) * (double)((size_t)1 << n)));
    if (!final_norms) QN_CUDA(launch_observe(vo, a, h->stream));
    if (keep) QN_CUDA(launch_probs_mix(vo, a, keep_mm, keep_tail, h->stream));
    else QN_CUDA(launch_probs(vo, a, h->stream));
    QN_TRY(prof_end(h, &ep));
    h->launches += (final_norms ? 1 : 2) + (a.parts > 1 ? 1 : 0);
    h->sh_slots += nslots;
    QN_CUDA(cudaStreamSynchronize(h->stream));  // order / weights host vectors
    h->sh_valid = true;
    h->sh_last_t0 = t0;
    h->sh_last_kc = kc;
    h->sh_range_host = std::move(fr);
    h->sh_members_host = std::move(fm);
    h->sh_order_host = std::move(order);
    h->sh_tail = read_tail;
    return QN_OK;
}

qn_status check_status(const qn_batch *h) {
    int st = 0;
    QN_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    QN_CUDA(cudaStreamSynchronize(h->stream));
    if (st != 0) return fail(QN_ESTATE, "a kernel flagged a zero or non-finite norm (status %d)", st);
    return QN_OK;
}

}  // namespace

namespace qn {

qn_status set_error(qn_status st, const char *msg) { return fail(st, "%s", msg); }

qn_status plan_qaoa(int32_t n, const qn_graph *graph, int32_t p, const double *gammas, const double *betas,
                    const qn_noise *noise, QaoaPlan *out) {
    if (n < 1 || n > kMaxQubits) return fail(QN_EINVAL, "n = %d outside [1, %d]", n, kMaxQubits);
    qn_batch tmp;  // host-only description; owns no device memory
    tmp.n = n;
    QN_TRY(validate_graph(&tmp, graph));
    QN_TRY(validate_noise(noise));
    if (p < 0) return fail(QN_EINVAL, "p = %d < 0", p);
    if (p > 0 && (!gammas || !betas)) return fail(QN_EINVAL, "gammas/betas is NULL");
    for (int l = 0; l < p; ++l)
        if (!std::isfinite(gammas[l]) || !std::isfinite(betas[l])) return fail(QN_EINVAL, "angle %d not finite", l);
    const int64_t G = (int64_t)n + (int64_t)p * (graph->num_edges + n);
    if (G > kMaxGates) return fail(QN_EINVAL, "circuit has %lld gates (max %lld)", (long long)G, (long long)kMaxGates);
    tmp.edges.assign(graph->edges, graph->edges + 2 * graph->num_edges);
    tmp.p = p;
    tmp.gammas.assign(gammas, gammas + p);
    tmp.betas.assign(betas, betas + p);
    build_gates(&tmp);
    double pr1[4], pr2[16];
    probs_1q(*noise, pr1);
    probs_2q(*noise, pr2);
    thresholds(pr1, 4, out->nz.thr1);
    thresholds(pr2, 16, out->nz.thr2);
    out->nz.gamma = noise->damping;
    out->damping_on = noise->damping > 0.0;
    out->gates = tmp.dgates_host;
    out->edges = tmp.edges_host;
    return QN_OK;
}

}  // namespace qn

extern "C" {

qn_status qn_batch_create(int32_t n, int64_t trajectories, uint64_t seed, qn_batch **out) {
    if (!out) return fail(QN_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kMaxQubits) return fail(QN_EINVAL, "n = %d outside [1, %d]", n, kMaxQubits);
    if (trajectories < 1) return fail(QN_EINVAL, "trajectories = %lld < 1", (long long)trajectories);
    qn_batch *h = new (std::nothrow) qn_batch();
    if (!h) return fail(QN_ENOMEM, "host allocation failed");
    h->n = n;
    h->K = trajectories;
    h->seed = seed;
    *out = h;
    return ok();
}

qn_status qn_batch_set_stream(qn_batch *h, void *cuda_stream) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    return ok();
}

qn_status qn_batch_set_allocator(qn_batch *h, void *(*alloc)(size_t, void *), void (*free_fn)(void *, void *),
                                 void *ctx) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (!h->blocks.empty()) return fail(QN_ESTATE, "allocator must be set before the first run");
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(QN_EINVAL, "alloc and free must both be set");
    h->alloc_fn = alloc;
    h->free_fn = free_fn;
    h->alloc_ctx = ctx;
    return ok();
}

qn_status qn_batch_set_launch_batch(qn_batch *h, int64_t B) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (B < 0 || B > 65535) return fail(QN_EINVAL, "launch batch %lld outside [0, 65535]", (long long)B);
    h->B_req = B;
    return ok();
}

qn_status qn_batch_set_fusion(qn_batch *h, int32_t on) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (on != 0 && on != 1) return fail(QN_EINVAL, "fusion must be 0 or 1");
    h->fusion = on;
    h->has_run = false;
    return ok();
}

qn_status qn_batch_set_precision(qn_batch *h, int32_t mode) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (mode != kPrecFP32 && mode != kPrecTF32 && mode != kPrecBF16x3)
        return fail(QN_EINVAL, "precision must be 0 (FP32), 1 (TF32 tensor cores) or 2 (BF16x3 tensor cores)");
    h->precision = mode;
    h->has_run = false;
    return ok();
}

qn_status qn_batch_set_sharing(qn_batch *h, int32_t on) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (on != 0 && on != 1) return fail(QN_EINVAL, "sharing must be 0 or 1");
    h->sharing = on;
    h->has_run = false;
    return ok();
}

qn_status qn_batch_set_launch_mode(qn_batch *h, int32_t mode) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (mode < 0 || mode > 2) return fail(QN_EINVAL, "launch mode must be 0, 1 or 2");
    h->launch_mode = mode;
    h->has_run = false;
    return ok();
}

qn_status qn_graph_info(const qn_batch *h, int64_t *captures, int64_t *replays, int64_t *updates) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (captures) *captures = h->graph_captures;
    if (replays) *replays = h->graph_replays;
    if (updates) *updates = h->graph_updates;
    return ok();
}

qn_status qn_batch_set_offset(qn_batch *h, int64_t first_trajectory) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (first_trajectory < 0) return fail(QN_EINVAL, "first trajectory id < 0");
    h->offset = first_trajectory;
    h->has_run = false;
    return ok();
}

qn_status qn_run_qaoa(qn_batch *h, const qn_graph *graph, int32_t p, const double *gammas, const double *betas,
                      const qn_noise *noise) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    QN_TRY(validate_graph(h, graph));
    QN_TRY(validate_noise(noise));
    if (p < 0) return fail(QN_EINVAL, "p = %d < 0", p);
    if (p > 0 && (!gammas || !betas)) return fail(QN_EINVAL, "gammas/betas is NULL");
    for (int l = 0; l < p; ++l)
        if (!std::isfinite(gammas[l]) || !std::isfinite(betas[l])) return fail(QN_EINVAL, "angle %d not finite", l);
    const int64_t G = (int64_t)h->n + (int64_t)p * (graph->num_edges + h->n);
    if (G > kMaxGates) return fail(QN_EINVAL, "circuit has %lld gates (max %lld)", (long long)G, (long long)kMaxGates);

    h->edges.assign(graph->edges, graph->edges + 2 * graph->num_edges);
    h->p = p;
    h->gammas.assign(gammas, gammas + p);
    h->betas.assign(betas, betas + p);
    h->noise = *noise;
    build_gates(h);
    build_groups(h);
    double pr1[4], pr2[16];
    probs_1q(*noise, pr1);
    probs_2q(*noise, pr2);
    thresholds(pr1, 4, h->nz.thr1);
    thresholds(pr2, 16, h->nz.thr2);
    h->nz.gamma = noise->damping;
    h->damping_on = noise->damping > 0.0;

    int64_t B = h->B_req;
    if (B == 0) {
        // shared-prefix mode keeps one slot per distinct prefix alive: give it
        // up to a quarter of the free memory for statevectors
        size_t budget = kDefaultBatchBytes;
        if (h->sharing) {
            size_t fb = 0, tb = 0;
            QN_CUDA(cudaMemGetInfo(&fb, &tb));
            budget = std::max(budget, fb / 4);
        }
        B = std::max<int64_t>(1, (int64_t)(budget / state_bytes(h->n)));
    }
    B = std::min<int64_t>(std::min<int64_t>(B, h->K), 65535);
    h->B = B;
    h->has_run = false;
    h->final_states = false;
    QN_TRY(ensure_buffers(h, B, (int32_t)G, graph->num_edges));
    QN_CUDA(cudaMemcpyAsync(h->dgates, h->dgates_host.data(), h->dgates_host.size() * sizeof(DevGate),
                            cudaMemcpyHostToDevice, h->stream));
    if (!h->edges_host.empty())
        QN_CUDA(cudaMemcpyAsync(h->dedges, h->edges_host.data(), h->edges_host.size() * sizeof(int2),
                                cudaMemcpyHostToDevice, h->stream));
    QN_CUDA(cudaMemsetAsync(h->probs, 0, sizeof(double) << h->n, h->stream));
    QN_CUDA(cudaMemsetAsync(h->sums, 0, 2 * sizeof(double), h->stream));
    QN_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    if (use_fusion(h)) QN_TRY(prepare_fusion(h));
    h->launches = 0;
    h->sweep_bytes = 0.0;
    h->sh_slots = 0;
    h->sh_valid = false;
    for (int64_t t0 = 0; t0 < h->K; t0 += B) {
        const int b = (int)std::min<int64_t>(B, h->K - t0);
        if (h->sharing && !use_fusion(h)) QN_TRY(run_shared(h, t0, b));
        else QN_TRY(run_batch(h, t0, b, true));
    }
    h->has_run = true;
    h->final_states = !(h->sharing && !use_fusion(h)) && B >= h->K;
    return ok();
}

qn_status qn_expectation(const qn_batch *h, double *mean, double *std_err) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (!mean || !std_err) return fail(QN_EINVAL, "output pointer is NULL");
    if (!h->has_run) return fail(QN_ESTATE, "no completed qn_run_qaoa on this handle");
    double s[2];
    QN_CUDA(cudaMemcpyAsync(s, h->sums, sizeof s, cudaMemcpyDeviceToHost, h->stream));
    QN_TRY(check_status(h));
    const double K = (double)h->K;
    const double m = s[0] / K;
    const double var = std::max(0.0, s[1] / K - m * m);
    *mean = m;
    *std_err = std::sqrt(var / K);
    return ok();
}

qn_status qn_probs(const qn_batch *h, double *out, int64_t len) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (!out) return fail(QN_EINVAL, "out is NULL");
    if (len != ((int64_t)1 << h->n)) return fail(QN_EINVAL, "len = %lld, expected 2^n = %lld", (long long)len,
                                                 (long long)((int64_t)1 << h->n));
    if (!h->has_run) return fail(QN_ESTATE, "no completed qn_run_qaoa on this handle");
    QN_CUDA(cudaMemcpyAsync(out, h->probs, sizeof(double) * (size_t)len, cudaMemcpyDeviceToHost, h->stream));
    QN_TRY(check_status(h));
    // sigma_approx = the ensemble's sum over trajectories of phi_t / ||phi_t||^2, scaled to unit
    // mass: the norms are exact to FP32 rounding (a shared-prefix run that ends on a mixer block
    // takes them from the block's joint), so the mass is K to that accuracy.  Eight partial sums
    // in fixed order (independent chains: the loop runs at the memory rate)
    double part[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t x0 = 0;
    for (; x0 + 8 <= len; x0 += 8)
        for (int k = 0; k < 8; ++k) part[k] += out[x0 + k];
    for (; x0 < len; ++x0) part[0] += out[x0];
    const double sum = ((part[0] + part[1]) + (part[2] + part[3])) + ((part[4] + part[5]) + (part[6] + part[7]));
    if (!(sum > 0.0) || !std::isfinite(sum)) return fail(QN_ESTATE, "sigma has mass %g", sum);
    const double inv = 1.0 / sum;
    for (int64_t x = 0; x < len; ++x) out[x] *= inv;
    return ok();
}

qn_status qn_traj_debug(qn_batch *h, int64_t t0, int64_t count, float *amps, uint8_t *branches,
                        double *c_per_traj) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (!h->has_run) return fail(QN_ESTATE, "no completed qn_run_qaoa on this handle");
    if (t0 < 0 || count < 0 || t0 + count > h->K)
        return fail(QN_EINVAL, "trajectories [%lld, %lld) outside [0, %lld)", (long long)t0,
                    (long long)(t0 + count), (long long)h->K);
    const int n = h->n;
    const int G = (int)h->gates.size();
    if (amps && !h->readout) {
        QN_TRY(alloc_t(h, &h->readout, (size_t)h->cap_B << n));
    }
    h->sh_valid = false;  // the re-simulation reuses the buffers a shared-prefix run left
    h->final_states = false;
    const int64_t saved_launches = h->launches;
    for (int64_t c0 = 0; c0 < count; c0 += h->cap_B) {
        const int b = (int)std::min<int64_t>(h->cap_B, count - c0);
        QN_TRY(run_batch(h, t0 + c0, b, false));
        if (amps) {
            BatchView v = view_for(h, h->offset + t0 + c0, b);
            QN_CUDA(launch_readout(v, h->readout, h->stream));
            QN_CUDA(cudaMemcpyAsync(amps + ((size_t)c0 << n) * 2, h->readout, ((size_t)b << n) * sizeof(float2),
                                    cudaMemcpyDeviceToHost, h->stream));
        }
        if (branches)
            QN_CUDA(cudaMemcpyAsync(branches + (size_t)c0 * G, h->branch, (size_t)b * G, cudaMemcpyDeviceToHost,
                                    h->stream));
        if (c_per_traj)
            QN_CUDA(cudaMemcpyAsync(c_per_traj + c0, h->c_dbg, (size_t)b * sizeof(double), cudaMemcpyDeviceToHost,
                                    h->stream));
        QN_CUDA(cudaStreamSynchronize(h->stream));
    }
    h->launches = saved_launches;
    QN_TRY(check_status(h));
    return ok();
}

qn_status qn_shared_readout(qn_batch *h, int64_t t0, int64_t count, float *amps, uint8_t *branches,
                            double *c_per_traj) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (!h->has_run) return fail(QN_ESTATE, "no completed qn_run_qaoa on this handle");
    if (!h->sh_valid) return fail(QN_ESTATE, "the last run did not evolve shared prefixes (sharing off, or Pauli-only "
                                             "noise with fusion on)");
    const int64_t lo = h->sh_last_t0, hi = h->sh_last_t0 + h->sh_last_kc;
    if (count < 0 || t0 < lo || t0 + count > hi)
        return fail(QN_EINVAL, "trajectories [%lld, %lld) outside the last prefix tree [%lld, %lld)", (long long)t0,
                    (long long)(t0 + count), (long long)lo, (long long)hi);
    const int n = h->n;
    const int G = (int)h->gates.size();
    const int kc = h->sh_last_kc;
    const int nslots = (int)h->sh_range_host.size();
    // final slot of every trajectory of the tree, and each slot's place in the sigma pass
    std::vector<int32_t> slot_of((size_t)kc, -1), pos((size_t)nslots, -1);
    for (int sl = 0; sl < nslots; ++sl) {
        const int2 r = h->sh_range_host[sl];
        for (int i = 0; i < r.y; ++i) slot_of[h->sh_members_host[(size_t)r.x + i]] = sl;
    }
    for (int i = 0; i < nslots; ++i) pos[h->sh_order_host[i]] = i;
    const int64_t b0 = t0 - lo;  // batch-local id of the first output
    for (int64_t i = 0; i < count; ++i)
        if (slot_of[b0 + i] < 0) return fail(QN_ESTATE, "trajectory %lld has no final slot", (long long)(t0 + i));
    if (branches && count > 0)
        QN_CUDA(cudaMemcpyAsync(branches, h->branch + (size_t)b0 * G, (size_t)count * G, cudaMemcpyDeviceToHost,
                                h->stream));
    if (c_per_traj && count > 0) {
        std::vector<double> cs((size_t)nslots);
        QN_CUDA(cudaMemcpyAsync(cs.data(), h->c_dbg, (size_t)nslots * sizeof(double), cudaMemcpyDeviceToHost,
                                h->stream));
        QN_CUDA(cudaStreamSynchronize(h->stream));
        for (int64_t i = 0; i < count; ++i) c_per_traj[i] = cs[pos[slot_of[b0 + i]]];
    }
    if (amps && count > 0) {
        const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(count, 64),
                                                                     (int64_t)(kDefaultBatchBytes / state_bytes(n))));
        if (h->sh_readcap < chunk) {
            QN_TRY(alloc_t(h, &h->sh_readbuf, (size_t)chunk << n));
            QN_TRY(alloc_t(h, &h->sh_readidx, (size_t)2 * chunk));
            h->sh_readcap = chunk;
        }
        BatchView v = view_for(h, h->offset + lo, kc);
        std::vector<int32_t> idx((size_t)2 * chunk);
        for (int64_t c0 = 0; c0 < count; c0 += chunk) {
            const int m = (int)std::min<int64_t>(chunk, count - c0);
            for (int i = 0; i < m; ++i) {
                idx[i] = slot_of[b0 + c0 + i];
                idx[chunk + i] = (int32_t)(b0 + c0 + i);
            }
            QN_CUDA(cudaMemcpyAsync(h->sh_readidx, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                    h->stream));
            QN_CUDA(launch_slot_readout(v, h->sh_readidx, h->sh_readidx + chunk, m, h->sh_tail, h->sh_readbuf,
                                        h->stream));
            QN_CUDA(cudaMemcpyAsync(amps + ((size_t)c0 << n) * 2, h->sh_readbuf, ((size_t)m << n) * sizeof(float2),
                                    cudaMemcpyDeviceToHost, h->stream));
            QN_CUDA(cudaStreamSynchronize(h->stream));  // idx is reused
        }
    }
    QN_TRY(check_status(h));
    return ok();
}

}  // extern "C"

namespace {

// Parameter index of gate g (>= n): 2l for the phase gates of layer l, 2l+1 for
// its mixer gates.
// Windows (first qubit, qubits) of the fused adjoint's mixer sweeps: qubits 0-3 (qubit 0
// in the float4, three on the register index), then the others in windows of two or
// three (a single one only when one qubit is left after the first window).
std::vector<std::pair<int, int>> adj_windows(int n) {
    std::vector<std::pair<int, int>> w;
    const int first = std::min(4, n);
    w.emplace_back(0, first);
    const int rest = n - first;
    if (rest <= 0) return w;
    const int count = (rest + 2) / 3;
    int q_lo = first;
    for (int i = 0; i < count; ++i) {
        const int m = rest / count + (i < rest % count ? 1 : 0);
        w.emplace_back(q_lo, m);
        q_lo += m;
    }
    return w;
}

// The tiled reverse windows of one layer for n >= 12 (launch_adj_win): qubits 0-9, then
// ceil((n - 10) / 6) windows of balanced sizes (at most 6, the larger ones first); the
// last window also undoes the cost diagonal.
std::vector<std::pair<int, int>> adj_tile_windows(int n) {
    std::vector<std::pair<int, int>> w;
    w.emplace_back(0, 10);
    const int rest = n - 10;
    const int count = (rest + 5) / 6;
    int q_lo = 10;
    for (int i = 0; i < count; ++i) {
        const int m = rest / count + (i < rest % count ? 1 : 0);
        w.emplace_back(q_lo, m);
        q_lo += m;
    }
    return w;
}

int param_of(const qn_batch *h, int g) {
    const int E = (int)h->edges.size() / 2;
    const int r = g - h->n;
    const int l = r / (E + h->n);
    return (r % (E + h->n)) < E ? 2 * l : 2 * l + 1;
}

// Per-trajectory adjoint gradients of trajectories [t0, t0 + count) (handle-local
// ids) into h->grad[(t0 + i) * 2p + param].
qn_status run_grad(qn_batch *h, int64_t t0, int64_t count) {
    if (!h->has_run) return fail(QN_ESTATE, "no completed qn_run_qaoa on this handle");
    if (h->noise.damping > 0.0)
        return fail(QN_EINVAL, "the adjoint gradient needs Pauli-only noise (damping = 0): damping makes "
                               "trajectories non-unitary");
    const int n = h->n;
    const int G = (int)h->gates.size();
    const int np = 2 * h->p;
    if (np == 0) return QN_OK;
    if (!h->lambda) QN_TRY(alloc_t(h, &h->lambda, (size_t)h->cap_B << n));
    if (!h->grad || h->grad_cap != np) {
        QN_TRY(alloc_t(h, &h->grad, (size_t)h->K * np));
        h->grad_cap = np;
    }
    QN_CUDA(cudaMemsetAsync(h->grad + (size_t)t0 * np, 0, (size_t)count * np * sizeof(double), h->stream));
    h->sh_valid = false;  // the re-simulation reuses the buffers a shared-prefix run left
    const int64_t saved_launches = h->launches;
    // the whole ensemble in one launch batch whose final states the run left: no re-simulation
    const bool reuse = h->final_states && t0 == 0 && count == h->K;
    h->final_states = false;  // the reverse sweeps take the states back to the start
    for (int64_t c0 = 0; c0 < count; c0 += h->cap_B) {
        const int b = (int)std::min<int64_t>(h->cap_B, count - c0);
        if (!reuse) QN_TRY(run_batch(h, t0 + c0, b, false));
        BatchView v = view_for(h, h->offset + t0 + c0, b);
        AccumView a = {};
        a.num_edges = (int32_t)h->edges_host.size();
        a.edges = h->dedges;
        QN_CUDA(launch_adj_init(v, h->lambda, a, h->stream));
        double *gr = h->grad + (size_t)(t0 + c0) * np;
        if (use_fusion(h)) {
            // the fused forward left every layer's parameters: the reverse takes a layer's
            // mixer in windows of a few qubits and its cost diagonal in one sweep
            for (int l = h->p - 1; l >= 0; --l) {
                const LayerView L = layer_view(h, l);
                if (n >= 12) {  // tiles through shared memory, the cost diagonal in the last window's sweep
                    const std::vector<std::pair<int, int>> ws = adj_tile_windows(n);
                    for (size_t i = 0; i < ws.size(); ++i)
                        QN_CUDA(launch_adj_win(v, h->lambda, L, ws[i].first, ws[i].second, i + 1 == ws.size(), gr,
                                               2 * l + 1, 2 * l, np, h->stream));
                    continue;
                }
                for (const auto &wd : adj_windows(n))
                    QN_CUDA(launch_adj_mixer(v, h->lambda, L, wd.first, wd.second, gr, 2 * l + 1, np, h->stream));
                QN_CUDA(launch_adj_phase(v, h->lambda, L, gr, 2 * l, np, h->stream));
            }
        } else {
            for (int g = G - 1; g >= n; --g)
                QN_CUDA(launch_adj_sweep(v, h->lambda, g, h->dgates_host[g], gr, param_of(h, g), np, h->stream));
        }
    }
    h->launches = saved_launches;
    QN_TRY(check_status(h));
    return QN_OK;
}

}  // namespace

extern "C" {

qn_status qn_grad(qn_batch *h, double *dgamma, double *dbeta) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (h->p > 0 && (!dgamma || !dbeta)) return fail(QN_EINVAL, "output pointer is NULL");
    QN_TRY(run_grad(h, 0, h->K));
    const int np = 2 * h->p;
    if (np == 0) return ok();
    std::vector<double> all((size_t)h->K * np);
    QN_CUDA(cudaMemcpyAsync(all.data(), h->grad, all.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    QN_CUDA(cudaStreamSynchronize(h->stream));
    for (int l = 0; l < h->p; ++l) {
        double sg = 0.0, sb = 0.0;
        for (int64_t t = 0; t < h->K; ++t) {
            sg += all[(size_t)t * np + 2 * l];
            sb += all[(size_t)t * np + 2 * l + 1];
        }
        dgamma[l] = sg / (double)h->K;
        dbeta[l] = sb / (double)h->K;
    }
    return ok();
}

qn_status qn_grad_traj(qn_batch *h, int64_t t0, int64_t count, double *dgamma, double *dbeta) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (t0 < 0 || count < 0 || t0 + count > h->K)
        return fail(QN_EINVAL, "trajectories [%lld, %lld) outside [0, %lld)", (long long)t0, (long long)(t0 + count),
                    (long long)h->K);
    if (h->p > 0 && count > 0 && (!dgamma || !dbeta)) return fail(QN_EINVAL, "output pointer is NULL");
    QN_TRY(run_grad(h, t0, count));
    const int np = 2 * h->p;
    if (np == 0 || count == 0) return ok();
    std::vector<double> all((size_t)count * np);
    QN_CUDA(cudaMemcpyAsync(all.data(), h->grad + (size_t)t0 * np, all.size() * sizeof(double),
                            cudaMemcpyDeviceToHost, h->stream));
    QN_CUDA(cudaStreamSynchronize(h->stream));
    for (int64_t i = 0; i < count; ++i)
        for (int l = 0; l < h->p; ++l) {
            dgamma[i * h->p + l] = all[(size_t)i * np + 2 * l];
            dbeta[i * h->p + l] = all[(size_t)i * np + 2 * l + 1];
        }
    return ok();
}

qn_status qn_fidelity_error(const double *sa, const double *se, int64_t len, double *out) {
    if (!sa || !se || !out) return fail(QN_EINVAL, "NULL argument");
    if (len < 0) return fail(QN_EINVAL, "len < 0");
    double s = 0.0;
    for (int64_t x = 0; x < len; ++x) {
        if (!(sa[x] >= 0.0) || !(se[x] >= 0.0)) return fail(QN_EINVAL, "negative or NaN entry at %lld", (long long)x);
        s += std::sqrt(sa[x] * se[x]);
    }
    *out = 1.0 - s * s;
    return ok();
}

qn_status qn_run_info(const qn_batch *h, int64_t *gates, int64_t *launches, double *sweep_bytes, int64_t *states) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (states) *states = (h->sharing && !use_fusion(h)) ? h->sh_slots : h->K;
    if (gates) *gates = (int64_t)h->gates.size();
    if (launches) *launches = h->launches;
    if (sweep_bytes) *sweep_bytes = h->sweep_bytes;
    return ok();
}

qn_status qn_group_plan(int32_t n, const qn_graph *graph, int32_t p, int32_t capacity, int32_t *kind,
                        int32_t *first_gate, int32_t *gates, uint32_t *qubit_mask, int32_t *count) {
    if (!count) return fail(QN_EINVAL, "count is NULL");
    if (n < 1 || n > kMaxQubits) return fail(QN_EINVAL, "n = %d outside [1, %d]", n, kMaxQubits);
    if (p < 0) return fail(QN_EINVAL, "p = %d < 0", p);
    if (capacity < 0 || (capacity > 0 && (!kind || !first_gate || !gates || !qubit_mask)))
        return fail(QN_EINVAL, "capacity < 0 or an output array is NULL");
    qn_batch tmp;  // host-only description; owns no device memory
    tmp.n = n;
    QN_TRY(validate_graph(&tmp, graph));
    tmp.edges.assign(graph->edges, graph->edges + 2 * graph->num_edges);
    tmp.p = p;
    tmp.gammas.assign((size_t)p, 0.0);
    tmp.betas.assign((size_t)p, 0.0);
    build_gates(&tmp);
    build_groups(&tmp);
    *count = (int32_t)tmp.groups.size();
    for (int i = 0; i < (int)tmp.groups.size() && i < capacity; ++i) {
        const GateGroup &z = tmp.groups[i];
        kind[i] = z.kind;
        first_gate[i] = z.g0;
        gates[i] = z.m;
        uint32_t mask = 0;
        for (int k = 0; k < z.s; ++k) mask |= 1u << z.sp[k];
        qubit_mask[i] = mask;
    }
    return ok();
}

qn_status qn_fused_windows(int32_t n, int32_t reverse, int32_t capacity, int32_t *q_lo, int32_t *qubits,
                           int32_t *count) {
    if (!count) return fail(QN_EINVAL, "count is NULL");
    if (n < 2 || n > kMaxQubits) return fail(QN_EINVAL, "n = %d outside [2, %d]", n, kMaxQubits);
    if (reverse != 0 && reverse != 1) return fail(QN_EINVAL, "reverse must be 0 or 1");
    if (capacity < 0 || (capacity > 0 && (!q_lo || !qubits))) return fail(QN_EINVAL, "bad output arrays");
    const std::vector<std::pair<int, int>> w = reverse ? (n >= 12 ? adj_tile_windows(n) : adj_windows(n))
                                                       : fused_windows(n);
    for (size_t i = 0; i < w.size() && (int32_t)i < capacity; ++i) {
        q_lo[i] = w[i].first;
        qubits[i] = w[i].second;
    }
    *count = (int32_t)w.size();
    return ok();
}

qn_status qn_mix_tile_map(int32_t n, int32_t q_lo, int32_t m, int32_t m_next, int8_t *lane_bits, int8_t *a_bits,
                          int8_t *b_bits, int8_t *tile_bits, int32_t *ntile) {
    if (!lane_bits || !a_bits || !b_bits || !tile_bits || !ntile) return fail(QN_EINVAL, "an output is NULL");
    if (n < 12 || n > kMaxQubits || m < 1 || m > kMixQ || m_next < 0 || m_next > kMixQ || q_lo < 0 ||
        q_lo + m + m_next > n)
        return fail(QN_EINVAL, "no mixer block of %d qubits at %d (next %d) for n = %d", m, q_lo, m_next, n);
    std::vector<int> next;
    for (int k = 0; k < m_next; ++k) next.push_back(q_lo + m + k);
    const MixMap mm = mix_map(n, q_lo, m, next);
    for (int i = 0; i < kMixL; ++i) lane_bits[i] = mm.fL[i];
    for (int i = 0; i < kMixQ; ++i) {
        a_bits[i] = mm.fA[i];
        b_bits[i] = mm.fB[i];
    }
    for (int i = 0; i < 32; ++i) tile_bits[i] = i < mm.ntile ? mm.ftile[i] : (int8_t)-1;
    *ntile = mm.ntile;
    return ok();
}

qn_status qn_batch_set_profiling(qn_batch *h, int32_t period) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (period < 0) return fail(QN_EINVAL, "profiling period < 0");
    h->prof_period = period;
    h->prof_counter = 0;
    return ok();
}

qn_status qn_profile_read(qn_batch *h, int32_t kind, int64_t *launches, double *ms, double *bytes) {
    if (!h) return fail(QN_EINVAL, "handle is NULL");
    if (kind < 0 || kind > 4) return fail(QN_EINVAL, "kind must be 0 .. 4");
    QN_TRY(prof_collect(h));
    if (launches) *launches = h->prof_launches[kind];
    if (ms) *ms = h->prof_ms[kind];
    if (bytes) *bytes = h->prof_bytes[kind];
    h->prof_launches[kind] = 0;
    h->prof_ms[kind] = 0.0;
    h->prof_bytes[kind] = 0.0;
    return ok();
}

const char *qn_last_error(void) { return g_last_error.c_str(); }

void qn_batch_destroy(qn_batch *h) {
    if (!h) return;
    release_all(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    pinned_word_give(h->pinned_word);
    for (EventPair &ep : h->events) {
        cudaEventDestroy(ep.a);
        cudaEventDestroy(ep.b);
    }
    for (EventPair &ep : h->spare) {
        cudaEventDestroy(ep.a);
        cudaEventDestroy(ep.b);
    }
    delete h;
}

}  // extern "C"
