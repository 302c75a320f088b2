// qn_noalloc.cu -- qn_run_qaoa_noalloc: one batch of noisy-QAOA trajectories
// without any device allocation by the library.
//
// Who needs this: callers that are not allowed to allocate device memory
// themselves or through libraries they call -- code whose device memory is
// owned by another runtime or pool allocator that must account for every
// byte, services that carve a fixed memory budget at start-up, and loops that
// cannot take the device-wide synchronisation cudaMalloc and cudaFree may
// imply.  They pass in the statevector workspace and the output buffers; every
// other buffer the pipeline needs (branch tables, X-frames, damping draws,
// per-trajectory state, reduction partials and counters, the gate list) is
// carved out of one fixed-size array in device global memory that this file
// declares statically.
//
// The array is kScratchBytes (8 MiB) per device, reserved on every GPU that
// loads libqnoise.so until the process exits.  Its device address is looked up
// with cudaGetSymbolAddress once per device, by the first call made with that
// device current; that first call should come before any stream capture (the
// lookup may load the module).  All calls share the one array and find the
// previous call's contents in it: the counters and flags that must start at
// zero are cleared on the stream at the start of every call, and calls whose
// work overlaps on the GPU (different streams without ordering, or several
// host threads) race on it.  The call returns after its work has finished.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "qn.h"
#include "qn_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)8 << 20;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
qn_status scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "cudaGetDevice failed: %s", cudaGetErrorString(e));
        return qn::set_error(QN_ECUDA, msg);
    }
    if (dev < 0 || dev >= kMaxDevices) return qn::set_error(QN_EINVAL, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
            return qn::set_error(QN_ECUDA, msg);
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return QN_OK;
}

// Bump allocator over the scratch array (256-byte aligned slices).
struct Carve {
    unsigned char *base;
    size_t used;
    template <typename T>
    T *take(size_t count) {
        used = (used + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + used);
        used += count * sizeof(T);
        return p;
    }
};

size_t scratch_needed(int n, int count, int G, int E) {
    Carve c{nullptr, 0};
    const size_t tiles = (size_t)qn::tiles_for(n);
    c.take<uint8_t>((size_t)count * G);
    c.take<uint32_t>((size_t)count * G * 2);
    c.take<uint32_t>((size_t)count * (G + 1));
    c.take<uint8_t>((size_t)count);
    c.take<float>((size_t)count * n * 2);
    c.take<qn::TrajState>((size_t)count);
    c.take<double>((size_t)count * tiles * 4);
    c.take<double>((size_t)count);
    c.take<double>((size_t)count * qn::accumulate_xblocks(n));
    c.take<unsigned int>((size_t)count);
    c.take<unsigned int>(1);
    c.take<int>(1);
    c.take<qn::DevGate>((size_t)(G > 0 ? G : 1));
    c.take<int2>((size_t)(E > 0 ? E : 1));
    return c.used;
}

#define NA_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            char msg_[256];                                                            \
            snprintf(msg_, sizeof msg_, "%s failed: %s", #call, cudaGetErrorString(e_)); \
            return qn::set_error(QN_ECUDA, msg_);                                      \
        }                                                                              \
    } while (0)

}  // namespace

extern "C" qn_status qn_run_qaoa_noalloc(int32_t n, const qn_graph *graph, int32_t p, const double *gammas,
                                         const double *betas, const qn_noise *noise, uint64_t seed,
                                         int64_t first_trajectory, int32_t count, void *psi, double *c_out,
                                         double *probs_out, void *cuda_stream) {
    using namespace qn;
    if (count < 1 || count > 65535) return set_error(QN_EINVAL, "count outside [1, 65535]");
    if (first_trajectory < 0) return set_error(QN_EINVAL, "first_trajectory < 0");
    if (!psi || !c_out || !probs_out) return set_error(QN_EINVAL, "psi, c_out and probs_out must be device pointers");
    if ((reinterpret_cast<uintptr_t>(psi) & 15u) != 0) return set_error(QN_EINVAL, "psi must be 16-byte aligned");
    QaoaPlan plan;
    qn_status st = plan_qaoa(n, graph, p, gammas, betas, noise, &plan);
    if (st != QN_OK) return st;
    const int G = (int)plan.gates.size();
    const int E = (int)plan.edges.size();
    const size_t need = scratch_needed(n, count, G, E);
    if (need > kScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "needs %zu bytes of scratch but the allocation-free path has %zu; lower count or n", need,
                 kScratchBytes);
        return set_error(QN_EINVAL, msg);
    }
    void *base = nullptr;
    st = scratch_address(&base);
    if (st != QN_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    Carve c{static_cast<unsigned char *>(base), 0};
    BatchView v;
    v.psi = static_cast<float2 *>(psi);
    v.n = n;
    v.b = count;
    v.t0 = first_trajectory;
    v.G = G;
    v.tiles = (int32_t)tiles_for(n);
    v.stiles = (int32_t)sweep_tiles_for(n);
    v.branch = c.take<uint8_t>((size_t)count * G);
    v.dwords = c.take<uint32_t>((size_t)count * G * 2);
    v.frame_x = c.take<uint32_t>((size_t)count * (G + 1));
    v.yphase = c.take<uint8_t>((size_t)count);
    v.hfac = c.take<float>((size_t)count * n * 2);
    v.st = c.take<TrajState>((size_t)count);
    v.partials = c.take<double>((size_t)count * v.tiles * 4);
    v.inv_norm = c.take<double>((size_t)count);
    double *cpart = c.take<double>((size_t)count * accumulate_xblocks(n));
    v.counters = c.take<unsigned int>((size_t)count);
    unsigned int *acc_counter = c.take<unsigned int>(1);
    v.status = c.take<int>(1);
    DevGate *dgates = c.take<DevGate>((size_t)(G > 0 ? G : 1));
    int2 *dedges = c.take<int2>((size_t)(E > 0 ? E : 1));

    // zero what the kernels expect zeroed; the array holds the previous call's data
    NA_CUDA(cudaMemsetAsync(v.counters, 0, (size_t)count * sizeof(unsigned int), s));
    NA_CUDA(cudaMemsetAsync(acc_counter, 0, sizeof(unsigned int), s));
    NA_CUDA(cudaMemsetAsync(v.status, 0, sizeof(int), s));
    NA_CUDA(cudaMemsetAsync(probs_out, 0, sizeof(double) << n, s));
    NA_CUDA(cudaMemcpyAsync(dgates, plan.gates.data(), (size_t)G * sizeof(DevGate), cudaMemcpyHostToDevice, s));
    if (E > 0)
        NA_CUDA(cudaMemcpyAsync(dedges, plan.edges.data(), (size_t)E * sizeof(int2), cudaMemcpyHostToDevice, s));

    NA_CUDA(launch_prepare(v, dgates, seed, plan.nz, plan.damping_on, s));
    NA_CUDA(launch_init(v, s));
    for (int g = n; g < G; ++g) NA_CUDA(launch_sweep(v, g, plan.gates[g], plan.nz, plan.damping_on, s));
    AccumView a;
    a.num_edges = E;
    a.edges = dedges;
    a.order = nullptr;
    a.weights = nullptr;
    a.cpart = cpart;
    a.acc_counter = acc_counter;
    a.c_out = c_out;
    a.probs = probs_out;
    a.sums = nullptr;
    NA_CUDA(launch_observe(v, a, s));
    NA_CUDA(launch_probs(v, a, s));
    // the host copies of the gate list and edges must outlive the async copies above
    NA_CUDA(cudaStreamSynchronize(s));
    int flag = 0;
    NA_CUDA(cudaMemcpy(&flag, v.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag != 0) return set_error(QN_ESTATE, "a kernel flagged a zero or non-finite norm");
    return set_error(QN_OK, "");
}
