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
// with cudaGetSymbolAddress once per device (again if the device's context was
// destroyed and recreated since), by the first call made with that device
// current; that first call should come before any stream capture (the lookup
// may load the module).  Every call checks that psi, c_out, probs_out and the
// stream belong to the current device before it queues anything, and returns
// QN_EINVAL for host memory or another GPU's buffers.  All calls share the one
// array and find the
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
// Per device: the scratch address and the id of the CUDA context it belongs to.
// A context torn down and created again (cudaDeviceReset, or a driver-level
// reset by another library) loads the module anew, so the address is looked up
// again whenever the current context's id differs from the cached one.
void *g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Driver entry points for the current context's unique id, fetched through the
// runtime so the library need not link libcuda.  Null when the driver lacks
// them; the cache then keys on the device alone.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);
struct CtxFns {
    CtxGetCurrentFn get_current = nullptr;
    CtxGetIdFn get_id = nullptr;
};
const CtxFns &ctx_fns() {
    static const CtxFns fns = [] {
        CtxFns f;
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa = cudaDriverEntryPointSymbolNotFound, qb = qa;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess && qb == cudaDriverEntryPointSuccess && a && b) {
            f.get_current = reinterpret_cast<CtxGetCurrentFn>(a);
            f.get_id = reinterpret_cast<CtxGetIdFn>(b);
        }
        cudaGetLastError();
        return f;
    }();
    return fns;
}

// Id of the current context (0 when it cannot be read).
unsigned long long current_ctx_id() {
    const CtxFns &f = ctx_fns();
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (f.get_current && f.get_current(&ctx) == 0 && ctx && f.get_id(ctx, &id) == 0) return id;
    return 0;
}

// Device address of g_scratch in the current device's context (looked up once per
// device and context; when the context id cannot be read, on every call).
// *dev_out receives the current device.
qn_status scratch_address(void **out, int *dev_out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "cudaGetDevice failed: %s", cudaGetErrorString(e));
        return qn::set_error(QN_ECUDA, msg);
    }
    if (dev < 0 || dev >= kMaxDevices) return qn::set_error(QN_EINVAL, "device ordinal beyond 63");
    // a context that does not exist yet (or no longer exists) reads as id 0 and
    // never matches a cached id; the lookup below creates it
    const unsigned long long ctx = current_ctx_id();
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
            return qn::set_error(QN_ECUDA, msg);
        }
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = current_ctx_id();
    }
    *out = g_scratch_ptr[dev];
    *dev_out = dev;
    return QN_OK;
}

// Bump allocator over the scratch array (256-byte aligned slices).  With a null
// base it only measures: the same carve() call both sizes and lays out the
// scratch, so the size check cannot drift from the real layout.
struct Carve {
    unsigned char *base;
    size_t used;
    template <typename T>
    T *take(size_t count) {
        used = (used + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + used) : nullptr;
        used += count * sizeof(T);
        return p;
    }
};

// Every scratch buffer of one batch of `count` trajectories.
struct Scratch {
    uint8_t *branch;
    uint32_t *dwords, *frame_x;
    uint8_t *yphase;
    float *hfac;
    qn::TrajState *st;
    double *partials, *inv_norm, *cpart;
    unsigned int *counters, *acc_counter;
    int *status;
    qn::DevGate *dgates;
    int2 *dedges;
};

Scratch carve(Carve &c, int n, int count, int G, int E) {
    Scratch s;
    const size_t tiles = (size_t)qn::tiles_for(n);
    s.branch = c.take<uint8_t>((size_t)count * G);
    s.dwords = c.take<uint32_t>((size_t)count * G * 2);
    s.frame_x = c.take<uint32_t>((size_t)count * (G + 1));
    s.yphase = c.take<uint8_t>((size_t)count);
    s.hfac = c.take<float>((size_t)count * n * 2);
    s.st = c.take<qn::TrajState>((size_t)count);
    s.partials = c.take<double>((size_t)count * tiles * 4);
    s.inv_norm = c.take<double>((size_t)count);
    s.cpart = c.take<double>((size_t)count * qn::accumulate_xblocks(n));
    s.counters = c.take<unsigned int>((size_t)count);
    s.acc_counter = c.take<unsigned int>(1);
    s.status = c.take<int>(1);
    s.dgates = c.take<qn::DevGate>((size_t)(G > 0 ? G : 1));
    s.dedges = c.take<int2>((size_t)(E > 0 ? E : 1));
    return s;
}

size_t scratch_needed(int n, int count, int G, int E) {
    Carve c{nullptr, 0};
    carve(c, n, count, G, E);
    return c.used;
}

// A caller buffer must be device memory (or managed memory) of device `dev`:
// a host pointer or another GPU's buffer would fault inside the kernels.
qn_status check_device_buffer(const void *ptr, int dev, const char *name) {
    cudaPointerAttributes at;
    const cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char msg[256];
        snprintf(msg, sizeof msg, "%s: cudaPointerGetAttributes failed: %s", name, cudaGetErrorString(e));
        return qn::set_error(QN_EINVAL, msg);
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) {
        char msg[256];
        snprintf(msg, sizeof msg, "%s is not device memory (pointer type %d)", name, (int)at.type);
        return qn::set_error(QN_EINVAL, msg);
    }
    if (at.device != dev) {
        char msg[256];
        snprintf(msg, sizeof msg, "%s belongs to device %d but device %d is current", name, at.device, dev);
        return qn::set_error(QN_EINVAL, msg);
    }
    return QN_OK;
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
    int dev = -1;
    st = scratch_address(&base, &dev);
    if (st != QN_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // every buffer and the stream must belong to the current device, checked before anything is queued
    if ((st = check_device_buffer(psi, dev, "psi")) != QN_OK) return st;
    if ((st = check_device_buffer(c_out, dev, "c_out")) != QN_OK) return st;
    if ((st = check_device_buffer(probs_out, dev, "probs_out")) != QN_OK) return st;
    {
        int sdev = -1;
        const cudaError_t e = cudaStreamGetDevice(s, &sdev);
        if (e != cudaSuccess) {
            cudaGetLastError();
            char msg[256];
            snprintf(msg, sizeof msg, "cudaStreamGetDevice failed: %s", cudaGetErrorString(e));
            return set_error(QN_EINVAL, msg);
        }
        if (sdev != dev) {
            char msg[256];
            snprintf(msg, sizeof msg, "the stream belongs to device %d but device %d is current", sdev, dev);
            return set_error(QN_EINVAL, msg);
        }
    }

    Carve c{static_cast<unsigned char *>(base), 0};
    const Scratch sc = carve(c, n, count, G, E);
    BatchView v;
    v.psi = static_cast<float2 *>(psi);
    v.n = n;
    v.b = count;
    v.t0 = first_trajectory;
    v.G = G;
    v.tiles = (int32_t)tiles_for(n);
    v.stiles = (int32_t)sweep_tiles_for(n);
    v.branch = sc.branch;
    v.dwords = sc.dwords;
    v.frame_x = sc.frame_x;
    v.yphase = sc.yphase;
    v.hfac = sc.hfac;
    v.st = sc.st;
    v.partials = sc.partials;
    v.inv_norm = sc.inv_norm;
    double *cpart = sc.cpart;
    v.counters = sc.counters;
    unsigned int *acc_counter = sc.acc_counter;
    v.status = sc.status;
    DevGate *dgates = sc.dgates;
    int2 *dedges = sc.dedges;

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
