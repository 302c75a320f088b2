// qn_kernels.cu -- sm_103a kernels of the stochastic noisy-QAOA ensemble.
//
// Stored state.  Each trajectory keeps a complex64 vector phi and an X-frame F
// (an n-bit mask) with psi_x = i^k phi_{x xor F}.  A Pauli X on qubit q only
// flips bit q of F; a Z (and the Z half of Y = iXZ) multiplies the amplitudes
// whose *true* bit (y_q xor F_q) is 1 by -1; Y adds a factor i (k += 1).  The
// amplitude-damping jump K1 = sqrt(gamma) X P1 becomes the projector onto true
// bit 1 plus a frame flip, and K0 is diagonal.  exp(-i beta X) commutes with
// every X-frame, and the ZZ phase is diagonal.  So a gate sweep applies
//
//     phi <- Z-part(P_g) * U_g * D_{g-1} * phi
//
// where D_{g-1} is the damping operator (with renormalisation) chosen for the
// previous gate, U_g the gate, and the X-part of P_g goes into the frame.  The
// same sweep reduces |phi|^2 into the marginal of gate g's qubits (true bits,
// after its Pauli); the last block of each trajectory then draws the damping
// branch of gate g in FP64 (Sec. "Stochastic Noise Implementation": one
// uniform number per channel picks the Kraus operator).
//
// Layout: phi is float2[b][2^n]; one float4 holds the amplitude pair (2f, 2f+1).
// A sweep tile is 256 threads x 4 float4 (2048 amplitudes) of one trajectory;
// grid = (tiles per trajectory, trajectories).  Every load and store is a
// coalesced 16-byte access; each amplitude is read once and written once.
#include "qn_internal.h"

#include <array>
#include <mutex>
#include <unordered_map>

namespace qn {
namespace {

constexpr double kTwoM32 = 2.3283064365386962890625e-10;  // 2^-32

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplications of counter words 0 and 2, high halves XORed into the other
// words and the key, key advanced by the Weyl increments after each round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t lo0 = m0 * c.x, hi0 = __umulhi(m0, c.x);
        uint32_t lo1 = m1 * c.z, hi1 = __umulhi(m1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ int pick_code(uint32_t w, const uint64_t *thr, int count) {
    for (int k = 0; k < count - 1; ++k)
        if ((uint64_t)w < thr[k]) return k;
    return count - 1;
}

__device__ __forceinline__ uint32_t xpart_1q(int code) { return (uint32_t)((code ^ (code >> 1)) & 1); }
__device__ __forceinline__ uint32_t zpart_1q(int code) { return (uint32_t)((code >> 1) & 1); }

// Work items of a sweep launch: one tile of one slot each.  A launch sized on the host
// (v.dyn_hi == nullptr) gives each block one item, tile blockIdx.x of slot base +
// blockIdx.y.  A device-driven launch has a persistent grid: its items k = 0, 1, ...
// cover the v.dyn_tiles tiles of each slot in [*v.dyn_lo, *v.dyn_hi) (read on the
// device, after grid_dependency_wait: the kernel before wrote them), tile k % dyn_tiles
// of slot lo + k / dyn_tiles, and are handed out in order from the launch's counter
// v.dyn_queue (zero at launch).  So the blocks at work at any moment hold consecutive
// items -- the order in which the hardware starts the blocks of a host-sized grid,
// which keeps the tiles of a slot in flight together -- and the host never reads the
// live-slot count: a whole run can be captured in a CUDA graph.  Thread 0 claims each
// item one item ahead (nxt, its register), so the counter's round trip overlaps the
// work on the item before; an item claimed beyond the end is dropped.  q_* are the
// block's shared words; `it` counts the block's items.  Called by every thread.
template <bool DYN>
__device__ __forceinline__ bool sweep_item(const BatchView &v, int base, int it, int &q_item, int &q_lo, int &q_n,
                                           int &nxt, int &tile, int &slot) {
    if (!DYN) {
        tile = (int)blockIdx.x;
        slot = base + (int)blockIdx.y;
        return it == 0;
    }
    __syncthreads();  // the previous item's shared memory is free
    if (threadIdx.x == 0) {
        if (it == 0) {
            q_lo = v.dyn_lo ? *v.dyn_lo : 0;
            q_n = v.dyn_tiles * max(*v.dyn_hi - q_lo, 0);
            nxt = atomicAdd(v.dyn_queue, 1);
        }
        q_item = nxt;
        if (nxt < q_n) nxt = atomicAdd(v.dyn_queue, 1);
    }
    __syncthreads();
    const int k = q_item;
    if (k >= q_n) return false;
    tile = k % v.dyn_tiles;
    slot = q_lo + k / v.dyn_tiles;
    return true;
}
// FP32 arithmetic of the sweeps in one fixed rounding sequence (no contraction left to
// the compiler), so that every variant of a kernel -- host-sized or device-driven, whose
// code the compiler schedules differently -- gives bit-identical values.
__device__ __forceinline__ float norm2_rn(float re, float im) { return __fmaf_rn(re, re, __fmul_rn(im, im)); }
__device__ __forceinline__ void cmul_rn(float ar, float ai, float br, float bi, float &re, float &im) {
    re = __fmaf_rn(ar, br, -__fmul_rn(ai, bi));
    im = __fmaf_rn(ar, bi, __fmul_rn(ai, br));
}

// The same, DYN decided at run time (the small sweeps: init, observables).
__device__ __forceinline__ bool sweep_item_rt(const BatchView &v, int base, int it, int &q_item, int &q_lo, int &q_n,
                                              int &nxt, int &tile, int &slot) {
    return v.dyn_hi ? sweep_item<true>(v, base, it, q_item, q_lo, q_n, nxt, tile, slot)
                    : sweep_item<false>(v, base, it, q_item, q_lo, q_n, nxt, tile, slot);
}
// Tiles per slot of a sweep launch (the host-sized grid's x extent).
template <bool DYN>
__device__ __forceinline__ int sweep_tiles(const BatchView &v) { return DYN ? v.dyn_tiles : (int)gridDim.x; }

// ---------------------------------------------------------------------------
// Per-trajectory preparation: Philox draws for every gate, Pauli codes, X-frame
// prefix, Y count, and the analytic noisy Hadamard layer.  One thread per
// trajectory.  The H layer acts on a product state, so every qubit's marginal
// is exactly 1/2 when its damping branch is drawn and each qubit's factor
// (Z sign, damping weight, normalisation) is independent of the others.
// ---------------------------------------------------------------------------
__global__ void k_prepare(BatchView v, const DevGate *__restrict__ gates, uint64_t seed, NoiseDev nz,
                          int damp) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= v.b) return;
    const uint64_t tg = (uint64_t)(v.t0 + t);
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const double gamma = nz.gamma;
    const double r2 = 0.70710678118654752440;
    uint32_t F = 0, J = 0, ycnt = 0;
    for (int g = 0; g < v.G; ++g) {
        const DevGate gt = gates[g];
        const uint4 w = philox4x32_10(make_uint4((uint32_t)g, 0u, (uint32_t)tg, (uint32_t)(tg >> 32)), key);
        const bool twoq = gt.kind == kGateZZ;
        const int code = twoq ? pick_code(w.x, nz.thr2, 16) : pick_code(w.x, nz.thr1, 4);
        uint8_t rec = (uint8_t)code;
        v.frame_x[(size_t)t * (v.G + 1) + g] = F;
        if (damp) {
            v.dwords[((size_t)t * v.G + g) * 2 + 0] = w.y;
            v.dwords[((size_t)t * v.G + g) * 2 + 1] = w.z;
        }
        if (gt.kind == kGateH) {
            // |+> ; Z part: sign on stored bit 1 (frame bit 0 before the flip);
            // X part: frame bit fb; damping acts on the true bit y ^ fb.
            const uint32_t fb = xpart_1q(code);
            const double s1 = zpart_1q(code) ? -r2 : r2;
            double d0 = 1.0, d1 = 1.0;
            if (damp) {
                const double u = ((double)w.y + 0.5) * kTwoM32;
                const bool jump = u < gamma * 0.5;
                if (jump) {
                    d0 = 0.0;
                    d1 = sqrt(2.0);  // sqrt(gamma) / sqrt(gamma / 2)
                    J ^= 1u << gt.q0;
                    rec |= 0x10;
                } else {
                    const double nn = sqrt(1.0 - 0.5 * gamma);
                    d0 = 1.0 / nn;
                    d1 = sqrt(1.0 - gamma) / nn;
                }
            }
            float *hf = v.hfac + ((size_t)t * v.n + gt.q0) * 2;
            hf[0] = (float)(r2 * (fb ? d1 : d0));
            hf[1] = (float)(s1 * (fb ? d0 : d1));
        }
        if (twoq) {
            const int a = code >> 2, b = code & 3;
            F ^= (xpart_1q(a) << gt.q0) ^ (xpart_1q(b) << gt.q1);
            ycnt += (a == 2) + (b == 2);
        } else {
            F ^= xpart_1q(code) << gt.q0;
            ycnt += (code == 2);
        }
        v.branch[(size_t)t * v.G + g] = rec;
    }
    v.frame_x[(size_t)t * (v.G + 1) + v.G] = F;
    v.yphase[t] = (uint8_t)(ycnt & 3u);
    TrajState s;
    s.J = J;
    s.pend = 0;
    s.pq0 = 0;
    s.pq1 = 0;
    s.f[0] = s.f[1] = s.f[2] = s.f[3] = 1.0f;
    v.st[t] = s;
    v.counters[t] = 0;
}

// ---------------------------------------------------------------------------
// State init: phi_y = prod_q hfac[q][y_q] (write-only sweep).  Factors of bits
// 0..5 and 6..10 come from two shared tables, the tile's high bits from one
// per-block scalar.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_init(BatchView v) {
    __shared__ int q_item, q_lo, q_n;
    int nxt = 0;  // thread 0: the next item claimed
    int tile, t;
    for (int it = 0; sweep_item_rt(v, 0, it, q_item, q_lo, q_n, nxt, tile, t); ++it) {
    __shared__ float lo[64], mid[32];
    __shared__ float hi_s;
    const float *hf = v.hfac + (size_t)t * v.n * 2;
    const int n = v.n;
    if (threadIdx.x < 64) {
        float p = 1.0f;
        for (int q = 0; q < 6 && q < n; ++q) p *= hf[2 * q + ((threadIdx.x >> q) & 1)];
        lo[threadIdx.x] = p;
    } else if (threadIdx.x < 96) {
        const int m = threadIdx.x - 64;
        float p = 1.0f;
        for (int q = 6; q < 11 && q < n; ++q) p *= hf[2 * q + ((m >> (q - 6)) & 1)];
        mid[m] = p;
    } else if (threadIdx.x == 96) {
        // tile covers bits 0..10 of y (2048 amplitudes); higher bits are fixed
        const uint32_t ybase = (uint32_t)tile << 11;
        float p = 1.0f;
        for (int q = 11; q < n; ++q) p *= hf[2 * q + ((ybase >> q) & 1)];
        hi_s = p;
    }
    __syncthreads();
    const int64_t nf = (int64_t)1 << (n - 1 > 0 ? n - 1 : 0);
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)t << n));
    const float h = hi_s;
#pragma unroll
    for (int k = 0; k < kF4PerThread; ++k) {
        const int64_t f = (int64_t)tile * kTileF4 + threadIdx.x + k * kThreads;
        if (f >= nf) break;
        const uint32_t y = (uint32_t)(2 * f);
        float a0, a1;
        if (n == 1) {
            a0 = hf[0];
            a1 = hf[1];
        } else {
            const float m = h * mid[(y >> 6) & 31];
            a0 = m * lo[y & 63];
            a1 = m * lo[(y & 63) | 1];
        }
        p4[f] = make_float4(a0, 0.0f, a1, 0.0f);
    }
    }
}

// ---------------------------------------------------------------------------
// Gate sweep.
// ---------------------------------------------------------------------------
struct SweepCtx {
    uint32_t Fa, Fb, Fc;  // frames: pending-op, gate/Z-part, bins
    int pq0, pq1;
    float f[4];
    int code;
};

__device__ __forceinline__ float pend_factor(const SweepCtx &c, uint32_t y) {
    const uint32_t ta = y ^ c.Fa;
    const uint32_t b0 = (ta >> c.pq0) & 1u, b1 = (ta >> c.pq1) & 1u;
    const float lo = b0 ? c.f[1] : c.f[0];
    const float hi = b0 ? c.f[3] : c.f[2];
    return b1 ? hi : lo;
}

// One branch class of gate g: Pauli `code` (its X part flips frame bits, its Z
// part signs true bits), then amplitude damping on the gate's qubits with
// outcomes ji, jj.  m[b0 | b1 << 1] is the weight of the state after the gate
// by true bits (b0, b1) of its qubits *before* the class's Pauli (a 1q gate uses
// m[0], m[3]).  Fills the pending op the next sweep applies: f indexed the same
// way (Z sign x damping Kraus factor x renormalisation), the frame flips of the
// Pauli X part (xmask) and of the jumps (jmask).
struct ClassOp {
    double f[4];
    uint32_t xmask, jmask;
    bool bad;
};

__device__ __forceinline__ void class_marginal(const DevGate &gt, const double m[4], int code, double mc[4]) {
    if (gt.kind == kGateZZ) {
        const int x = (int)(xpart_1q(code >> 2) | (xpart_1q(code & 3) << 1));
        for (int k = 0; k < 4; ++k) mc[k] = m[k ^ x];
    } else {
        const bool x = xpart_1q(code) != 0;
        mc[0] = x ? m[3] : m[0];
        mc[3] = x ? m[0] : m[3];
        mc[1] = mc[2] = 0.0;
    }
}

// Damping draws of one trajectory in class `code` (the second conditioned on the
// first), from the post-Pauli marginal mc.
__device__ __forceinline__ void damping_draws(const DevGate &gt, const double mc[4], double u0, double u1,
                                              double gamma, bool &ji, bool &jj) {
    const double sg = sqrt(gamma), sg1 = sqrt(1.0 - gamma);
    if (gt.kind == kGateZZ) {
        const double N = mc[0] + mc[1] + mc[2] + mc[3];
        ji = u0 < gamma * (mc[1] + mc[3]) / N;
        const double ki0 = ji ? 0.0 : 1.0, ki1 = ji ? sg : sg1;
        const double Ni = (mc[0] + mc[2]) * ki0 * ki0 + (mc[1] + mc[3]) * ki1 * ki1;
        jj = u1 < gamma * (mc[2] * ki0 * ki0 + mc[3] * ki1 * ki1) / Ni;
    } else {
        ji = u0 < gamma * mc[3] / (mc[0] + mc[3]);
        jj = false;
    }
}

__device__ __noinline__ ClassOp class_op(const DevGate &gt, const double m[4], int code, bool ji, bool jj, double gamma,
                                     bool damp) {
    ClassOp op;
    double mc[4];
    class_marginal(gt, m, code, mc);
    const double sg = sqrt(gamma), sg1 = sqrt(1.0 - gamma);
    const double ki0 = !damp ? 1.0 : (ji ? 0.0 : 1.0), ki1 = !damp ? 1.0 : (ji ? sg : sg1);
    const double kj0 = !damp ? 1.0 : (jj ? 0.0 : 1.0), kj1 = !damp ? 1.0 : (jj ? sg : sg1);
    if (gt.kind == kGateZZ) {
        const int a = code >> 2, b = code & 3;
        const uint32_t xa = xpart_1q(a), xb = xpart_1q(b), za = zpart_1q(a), zb = zpart_1q(b);
        // norm after the ops, from post-Pauli bins
        const double Nf = mc[0] * ki0 * ki0 * kj0 * kj0 + mc[1] * ki1 * ki1 * kj0 * kj0 +
                          mc[2] * ki0 * ki0 * kj1 * kj1 + mc[3] * ki1 * ki1 * kj1 * kj1;
        const double sc = damp ? 1.0 / sqrt(Nf) : 1.0;
        for (int idx = 0; idx < 4; ++idx) {
            const uint32_t b0 = idx & 1, b1 = (idx >> 1) & 1;
            const double zs = ((za & b0) ^ (zb & b1)) ? -1.0 : 1.0;
            const double k0 = (b0 ^ xa) ? ki1 : ki0, k1 = (b1 ^ xb) ? kj1 : kj0;
            op.f[idx] = zs * k0 * k1 * sc;
        }
        op.xmask = (xa << gt.q0) | (xb << gt.q1);
        op.jmask = ((uint32_t)(damp && ji) << gt.q0) | ((uint32_t)(damp && jj) << gt.q1);
        op.bad = damp && (!(Nf > 0.0) || !isfinite(sc));
    } else {
        const uint32_t x = xpart_1q(code), z = zpart_1q(code);
        const double Nf = mc[0] * ki0 * ki0 + mc[3] * ki1 * ki1;
        const double sc = damp ? 1.0 / sqrt(Nf) : 1.0;
        op.f[0] = (x ? ki1 : ki0) * sc;
        op.f[3] = (z ? -1.0 : 1.0) * (x ? ki0 : ki1) * sc;
        op.f[1] = op.f[2] = 0.0;
        op.xmask = x << gt.q0;
        op.jmask = (uint32_t)(damp && ji) << gt.q0;
        op.bad = damp && (!(Nf > 0.0) || !isfinite(sc));
    }
    return op;
}

__device__ __forceinline__ void set_pending(TrajState &s, const DevGate &gt, const ClassOp &op) {
    s.J ^= s.pend;
    s.pend = op.xmask ^ op.jmask;
    s.pq0 = gt.q0;
    s.pq1 = gt.kind == kGateZZ ? gt.q1 : gt.q0;
    for (int k = 0; k < 4; ++k) s.f[k] = (float)op.f[k];
}

// Damping branch of gate g for one trajectory of a launch batch.  m[4] is the
// marginal after the gate's Pauli (already applied by the sweep: Z part on the
// data, X part in the frame), so the branch class here is the identity Pauli.
__device__ void decide_damping(const BatchView &v, int t, int g, const DevGate &gt, const double m[4],
                               double gamma) {
    TrajState s = v.st[t];
    const uint32_t *dw = v.dwords + ((size_t)t * v.G + g) * 2;
    const double u0 = ((double)dw[0] + 0.5) * kTwoM32;
    const double u1 = ((double)dw[1] + 0.5) * kTwoM32;
    bool ji, jj;
    damping_draws(gt, m, u0, u1, gamma, ji, jj);
    const ClassOp op = class_op(gt, m, 0, ji, jj, gamma, true);
    if (op.bad || !((m[0] + m[1] + m[2] + m[3]) > 0.0)) atomicOr(v.status, 1);
    set_pending(s, gt, op);
    v.st[t] = s;
    v.branch[(size_t)t * v.G + g] |= (uint8_t)(((uint32_t)ji << 4) | ((uint32_t)(jj && gt.kind == kGateZZ) << 5));
}

// Programmatic dependent launch: a sweep may be scheduled while the previous
// kernel drains; it waits here before touching anything that kernel wrote.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependent_launch() { asm volatile("griddepcontrol.launch_dependents;"); }


// Block reduction of the damping marginal of one unit -> partials[t][tile];
// returns true in the last block to finish trajectory (or slot) t, with the
// trajectory's marginal (FP64, fixed summation order) in m_out (shared).
__device__ __forceinline__ bool reduce_marginal(const BatchView &v, int t, int tile, float acc0, float acc1, float acc2,
                                                float acc3, double *m_out) {
    __shared__ float red[kThreads / 32][4];
    __shared__ double redd[kThreads / 32][4];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[4] = {acc0, acc1, acc2, acc3};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float a = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) red[warp][k] = a;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += (double)red[w][threadIdx.x];
        v.partials[((size_t)t * v.stiles + tile) * 4 + threadIdx.x] = s;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&v.counters[t], 1u);
        last = prev == (unsigned)(v.stiles - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < v.stiles; i += kThreads) {
        const double *pp = v.partials + ((size_t)t * v.stiles + i) * 4;
#pragma unroll
        for (int k = 0; k < 4; ++k) s[k] += __ldcg(pp + k);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double a = s[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) redd[warp][k] = a;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double a = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) a += redd[w][threadIdx.x];
        m_out[threadIdx.x] = a;
    }
    if (threadIdx.x == 0) v.counters[t] = 0;
    __syncthreads();
    return true;
}

// Context of trajectory t for gate g, read by every thread (uniform addresses,
// served from L1 after the first warp).
__device__ __forceinline__ SweepCtx load_ctx(const BatchView &v, int t, int g, bool damp) {
    SweepCtx c;
    const uint32_t fxg = v.frame_x[(size_t)t * (v.G + 1) + g];
    const uint32_t fxg1 = v.frame_x[(size_t)t * (v.G + 1) + g + 1];
    c.code = v.branch[(size_t)t * v.G + g] & 15;
    if (damp) {
        const TrajState s = v.st[t];
        c.Fa = fxg ^ s.J;
        c.Fb = c.Fa ^ s.pend;
        c.Fc = fxg1 ^ s.J ^ s.pend;
        c.pq0 = s.pq0;
        c.pq1 = s.pq1;
        for (int k = 0; k < 4; ++k) c.f[k] = s.f[k];
    } else {
        c.Fa = c.Fb = fxg;
        c.Fc = fxg1;
        c.pq0 = c.pq1 = 0;
        c.f[0] = c.f[1] = c.f[2] = c.f[3] = 1.0f;
    }
    return c;
}

// Context of a shared-prefix slot: its whole frame lives in J ^ pend and the
// slot itself always takes the identity Pauli (other classes fork off).
__device__ __forceinline__ SweepCtx load_slot_ctx(const BatchView &v, int slot) {
    SweepCtx c;
    const TrajState s = v.st[slot];
    c.code = 0;
    c.Fa = s.J;
    c.Fb = c.Fc = s.J ^ s.pend;
    c.pq0 = s.pq0;
    c.pq1 = s.pq1;
    for (int k = 0; k < 4; ++k) c.f[k] = s.f[k];
    return c;
}

__device__ __forceinline__ void load_tile(float4 (&dst)[kF4PerThread], const float4 *p4, int64_t f0, int64_t nf) {
#pragma unroll
    for (int k = 0; k < kF4PerThread; ++k)
        if (f0 + k * kThreads < nf) dst[k] = p4[f0 + k * kThreads];
}

// ZZ phase on one unit (kSub tiles) of trajectory or slot t: phi_y *=
// D_{g-1}(y) * (true bits of q0, q1 differ ? e^{-i gamma} : 1) * (Z part of the
// Pauli), then bins of |phi|^2 by the true bits after the Pauli.  The next
// tile is prefetched into registers while the current one is computed.
template <bool DAMP, bool SLOT>
__device__ __forceinline__ void zz_unit(const BatchView &v, int t, int tile, int g, const DevGate &gt, float &acc0,
                                        float &acc1, float &acc2, float &acc3) {
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1);
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)t << n));
    const int64_t fbase = (int64_t)tile * kTileF4 * kSub + threadIdx.x;
    float4 cur[kF4PerThread], nxt[kF4PerThread];
    load_tile(cur, p4, fbase, nf);
    const SweepCtx c = SLOT ? load_slot_ctx(v, t) : load_ctx(v, t, g, DAMP);
    constexpr bool PEND = DAMP || SLOT;  // pending factors to apply
    const int q0 = gt.q0, q1 = gt.q1;
    const uint32_t za = (uint32_t)(c.code >> 3) & 1u, zb = (uint32_t)(c.code >> 1) & 1u;
    const uint32_t fb0 = (c.Fb >> q0) & 1u, fb1 = (c.Fb >> q1) & 1u;
    const uint32_t fc0 = (c.Fc >> q0) & 1u, fc1 = (c.Fc >> q1) & 1u;
    const uint32_t fa0 = (c.Fa >> c.pq0) & 1u, fa1 = (c.Fa >> c.pq1) & 1u;
    // bit 0 (the two halves of a float4) touches no qubit of this op: one
    // coefficient per float4
    const bool pair_uniform = q0 != 0 && q1 != 0 && (!PEND || (c.pq0 != 0 && c.pq1 != 0));
#pragma unroll
    for (int sub = 0; sub < kSub; ++sub) {
        const int64_t f0 = fbase + (int64_t)sub * kTileF4;
        if (sub + 1 < kSub) load_tile(nxt, p4, f0 + kTileF4, nf);
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k) {
            const int64_t f = f0 + k * kThreads;
            if (f >= nf) continue;
            const uint32_t y = (uint32_t)(2 * f);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (e == 1 && pair_uniform) break;
                const uint32_t ye = y | (uint32_t)e;
                const uint32_t y0 = (ye >> q0) & 1u, y1 = (ye >> q1) & 1u;
                float fa = 1.0f;
                if (PEND) {
                    const uint32_t a0 = ((ye >> c.pq0) & 1u) ^ fa0, a1 = ((ye >> c.pq1) & 1u) ^ fa1;
                    fa = a1 ? (a0 ? c.f[3] : c.f[2]) : (a0 ? c.f[1] : c.f[0]);
                }
                const uint32_t b0 = y0 ^ fb0, b1 = y1 ^ fb1;
                const float sgn = ((za & b0) ^ (zb & b1)) ? -fa : fa;
                const bool diff = (b0 ^ b1) != 0u;
                const float pc = diff ? gt.c * sgn : sgn;
                const float ps = diff ? gt.s * sgn : 0.0f;
                float p;
                if (pair_uniform) {
                    const float r0 = cur[k].x, i0 = cur[k].y, r1 = cur[k].z, i1 = cur[k].w;
                    cur[k].x = r0 * pc + i0 * ps;
                    cur[k].y = i0 * pc - r0 * ps;
                    cur[k].z = r1 * pc + i1 * ps;
                    cur[k].w = i1 * pc - r1 * ps;
                    p = cur[k].x * cur[k].x + cur[k].y * cur[k].y + cur[k].z * cur[k].z + cur[k].w * cur[k].w;
                } else {
                    float &re = e ? cur[k].z : cur[k].x;
                    float &im = e ? cur[k].w : cur[k].y;
                    const float nr = re * pc + im * ps, ni = im * pc - re * ps;
                    re = nr;
                    im = ni;
                    p = nr * nr + ni * ni;
                }
                if (DAMP) {
                    const uint32_t idx = (y0 ^ fc0) | ((y1 ^ fc1) << 1);
                    acc0 += idx == 0u ? p : 0.0f;
                    acc1 += idx == 1u ? p : 0.0f;
                    acc2 += idx == 2u ? p : 0.0f;
                    acc3 += idx == 3u ? p : 0.0f;
                }
            }
            p4[f] = cur[k];
        }
        if (sub + 1 < kSub) {
#pragma unroll
            for (int k = 0; k < kF4PerThread; ++k) cur[k] = nxt[k];
        }
    }
}

// exp(-i beta X) on qubit q for one unit: pairs (y0, y0 | 2^q) after D_{g-1};
// the Z part of the Pauli negates the element whose true bit is 1; bins by the
// true bit of q after the Pauli (acc0: true bit 0, acc3: true bit 1).
template <bool DAMP, bool SLOT>
__device__ __forceinline__ void rx_unit(const BatchView &v, int t, int tile, int g, const DevGate &gt, float &acc0,
                                        float &acc3) {
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1);
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)t << n));
    const int q = gt.q0;
    constexpr bool PEND = DAMP || SLOT;
    float acc_lo = 0.0f, acc_hi = 0.0f;  // weight of rows 0 (stored bit 0) and 1
    uint32_t fcq = 0;
    if (q == 0) {
        const int64_t fbase = (int64_t)tile * kTileF4 * kSub + threadIdx.x;
        float4 cur[kF4PerThread], nxt[kF4PerThread];
        load_tile(cur, p4, fbase, nf);
        const SweepCtx c = SLOT ? load_slot_ctx(v, t) : load_ctx(v, t, g, DAMP);
        const uint32_t fbq = c.Fb & 1u;
        fcq = c.Fc & 1u;
        const float s0 = ((c.code >> 1) & 1) && fbq ? -1.0f : 1.0f;   // row of stored bit 0
        const float s1 = ((c.code >> 1) & 1) && !fbq ? -1.0f : 1.0f;  // row of stored bit 1
        const float c0 = gt.c * s0, sn0 = gt.s * s0, c1 = gt.c * s1, sn1 = gt.s * s1;
#pragma unroll
        for (int sub = 0; sub < kSub; ++sub) {
            const int64_t f0 = fbase + (int64_t)sub * kTileF4;
            if (sub + 1 < kSub) load_tile(nxt, p4, f0 + kTileF4, nf);
#pragma unroll
            for (int k = 0; k < kF4PerThread; ++k) {
                const int64_t f = f0 + k * kThreads;
                if (f >= nf) continue;
                const uint32_t y = (uint32_t)(2 * f);
                const float fa0 = PEND ? pend_factor(c, y) : 1.0f, fa1 = PEND ? pend_factor(c, y | 1u) : 1.0f;
                const float r0 = cur[k].x * fa0, i0 = cur[k].y * fa0, r1 = cur[k].z * fa1, i1 = cur[k].w * fa1;
                cur[k].x = c0 * r0 + sn0 * i1;
                cur[k].y = c0 * i0 - sn0 * r1;
                cur[k].z = c1 * r1 + sn1 * i0;
                cur[k].w = c1 * i1 - sn1 * r0;
                acc_lo += cur[k].x * cur[k].x + cur[k].y * cur[k].y;
                acc_hi += cur[k].z * cur[k].z + cur[k].w * cur[k].w;
                p4[f] = cur[k];
            }
            if (sub + 1 < kSub) {
#pragma unroll
                for (int k = 0; k < kF4PerThread; ++k) cur[k] = nxt[k];
            }
        }
    } else {
        const int sh = q - 1;
        const int64_t npairs = nf >> 1;
        constexpr int kPairs = kF4PerThread / 2;
        const int64_t rbase = (int64_t)tile * (kTileF4 / 2) * kSub + threadIdx.x;
        const int64_t hib = (int64_t)1 << sh;
        float4 lo[kPairs], hi[kPairs], nlo[kPairs], nhi[kPairs];
        auto load_pairs = [&](float4 (&dl)[kPairs], float4 (&dh)[kPairs], int64_t r0) {
#pragma unroll
            for (int k = 0; k < kPairs; ++k) {
                const int64_t r = r0 + k * kThreads;
                const int64_t fl = ((r >> sh) << (sh + 1)) | (r & (hib - 1));
                if (r < npairs) {
                    dl[k] = p4[fl];
                    dh[k] = p4[fl | hib];
                }
            }
        };
        load_pairs(lo, hi, rbase);
        const SweepCtx c = SLOT ? load_slot_ctx(v, t) : load_ctx(v, t, g, DAMP);
        const uint32_t fbq = (c.Fb >> q) & 1u;
        fcq = (c.Fc >> q) & 1u;
        const float s0 = ((c.code >> 1) & 1) && fbq ? -1.0f : 1.0f;
        const float s1 = ((c.code >> 1) & 1) && !fbq ? -1.0f : 1.0f;
        const float c0 = gt.c * s0, sn0 = gt.s * s0, c1 = gt.c * s1, sn1 = gt.s * s1;
        const bool quad_uniform = !PEND || (c.pq0 != 0 && c.pq0 != q && c.pq1 != 0 && c.pq1 != q);
#pragma unroll
        for (int sub = 0; sub < kSub; ++sub) {
            const int64_t r0 = rbase + (int64_t)sub * (kTileF4 / 2);
            if (sub + 1 < kSub) load_pairs(nlo, nhi, r0 + kTileF4 / 2);
#pragma unroll
            for (int k = 0; k < kPairs; ++k) {
                const int64_t r = r0 + k * kThreads;
                if (r >= npairs) continue;
                const int64_t fl = ((r >> sh) << (sh + 1)) | (r & (hib - 1));
                const uint32_t y0 = (uint32_t)(2 * fl);
                const uint32_t qb = 1u << q;
                float fl0, fl1, fh0, fh1;  // pending factors of lo.xy, lo.zw, hi.xy, hi.zw
                if (!PEND) {
                    fl0 = fl1 = fh0 = fh1 = 1.0f;
                } else if (quad_uniform) {
                    fl0 = fl1 = fh0 = fh1 = pend_factor(c, y0);
                } else {
                    fl0 = pend_factor(c, y0);
                    fl1 = pend_factor(c, y0 | 1u);
                    fh0 = pend_factor(c, y0 | qb);
                    fh1 = pend_factor(c, y0 | 1u | qb);
                }
                const float a0r = lo[k].x * fl0, a0i = lo[k].y * fl0, b0r = hi[k].x * fh0, b0i = hi[k].y * fh0;
                const float a1r = lo[k].z * fl1, a1i = lo[k].w * fl1, b1r = hi[k].z * fh1, b1i = hi[k].w * fh1;
                lo[k].x = c0 * a0r + sn0 * b0i;
                lo[k].y = c0 * a0i - sn0 * b0r;
                hi[k].x = c1 * b0r + sn1 * a0i;
                hi[k].y = c1 * b0i - sn1 * a0r;
                lo[k].z = c0 * a1r + sn0 * b1i;
                lo[k].w = c0 * a1i - sn0 * b1r;
                hi[k].z = c1 * b1r + sn1 * a1i;
                hi[k].w = c1 * b1i - sn1 * a1r;
                acc_lo += lo[k].x * lo[k].x + lo[k].y * lo[k].y + lo[k].z * lo[k].z + lo[k].w * lo[k].w;
                acc_hi += hi[k].x * hi[k].x + hi[k].y * hi[k].y + hi[k].z * hi[k].z + hi[k].w * hi[k].w;
                p4[fl] = lo[k];
                p4[fl | hib] = hi[k];
            }
            if (sub + 1 < kSub) {
#pragma unroll
                for (int k = 0; k < kPairs; ++k) {
                    lo[k] = nlo[k];
                    hi[k] = nhi[k];
                }
            }
        }
    }
    acc0 = fcq ? acc_hi : acc_lo;
    acc3 = fcq ? acc_lo : acc_hi;
}

// Gate sweeps of a launch batch: grid (sweep tiles, trajectories).
template <bool DAMP>
__global__ void __launch_bounds__(kThreads, 4) k_sweep_zz(BatchView v, int g, DevGate gt, double gamma) {
    grid_dependency_wait();
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    zz_unit<DAMP, false>(v, blockIdx.y, blockIdx.x, g, gt, a0, a1, a2, a3);
    allow_dependent_launch();
    if (DAMP) {
        __shared__ double m[4];
        if (reduce_marginal(v, blockIdx.y, blockIdx.x, a0, a1, a2, a3, m) && threadIdx.x == 0)
            decide_damping(v, blockIdx.y, g, gt, m, gamma);
    }
}

template <bool DAMP>
__global__ void __launch_bounds__(kThreads, 4) k_sweep_rx(BatchView v, int g, DevGate gt, double gamma) {
    grid_dependency_wait();
    float a0 = 0.0f, a3 = 0.0f;
    rx_unit<DAMP, false>(v, blockIdx.y, blockIdx.x, g, gt, a0, a3);
    allow_dependent_launch();
    if (DAMP) {
        __shared__ double m[4];
        if (reduce_marginal(v, blockIdx.y, blockIdx.x, a0, 0.0f, 0.0f, a3, m) && threadIdx.x == 0)
            decide_damping(v, blockIdx.y, g, gt, m, gamma);
    }
}

// ---------------------------------------------------------------------------
// Shared-prefix mode.  Trajectories whose Kraus strings agree so far share one
// statevector ("slot").  A slot always takes the identity Pauli and, with
// damping, the no-jump branch; after every gate the last block of each slot
// draws, for every member trajectory, its own Pauli (from the member's Philox
// word) and damping outcomes (from the slot's marginal, permuted by that
// Pauli's X part), groups the members by outcome, keeps the identity / no-jump
// group and forks every other group into a new slot that copies the state and
// carries its class's Z sign, damping factors and renormalisation as the
// pending op.  Every trajectory therefore sees exactly the state and branch
// draws it would see alone; only the work on common prefixes is shared.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void decide_slot(const BatchView &v, const SlotView &sv, int s, int g, const DevGate &gt,
                            const double *m_sh, double gamma, bool damp) {
    __shared__ int ccount[64], cstart[64], order[64];
    __shared__ int norder, child_base, run;
    __shared__ int wcnt[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int2 rg = sv.range[s];
    const int off = rg.x, cnt = rg.y;
    if (threadIdx.x < 64) ccount[threadIdx.x] = 0;
    __syncthreads();
    double m[4];
    for (int k = 0; k < 4; ++k) m[k] = damp ? m_sh[k] : 0.0;
    for (int i = threadIdx.x; i < cnt; i += kThreads) {
        const int t = sv.members[off + i];
        const int code = v.branch[(size_t)t * v.G + g] & 15;
        int cls = code;
        if (damp) {
            const uint32_t *dw = v.dwords + ((size_t)t * v.G + g) * 2;
            double mc[4];
            class_marginal(gt, m, code, mc);
            bool ji, jj;
            damping_draws(gt, mc, ((double)dw[0] + 0.5) * kTwoM32, ((double)dw[1] + 0.5) * kTwoM32, gamma, ji, jj);
            cls |= ((int)ji << 4) | ((int)jj << 5);
            v.branch[(size_t)t * v.G + g] = (uint8_t)cls;
        }
        sv.cls[off + i] = (uint8_t)cls;
        atomicAdd(&ccount[cls], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int first = ccount[0] > 0 ? 0 : -1;
        for (int c = 1; c < 64 && first < 0; ++c)
            if (ccount[c] > 0) first = c;
        int no = 0;
        order[no++] = first;
        for (int c = 0; c < 64; ++c)
            if (c != first && ccount[c] > 0) order[no++] = c;
        int pos = 0;
        for (int k = 0; k < no; ++k) {
            cstart[order[k]] = pos;
            pos += ccount[order[k]];
        }
        norder = no;
        child_base = no > 1 ? atomicAdd(sv.slot_count, no - 1) : 0;
    }
    __syncthreads();
    const int no = norder;
    if (no > 1) {
        // stable partition of the members by class, into tmp[off ..]
        for (int k = 0; k < no; ++k) {
            const int c = order[k];
            if (threadIdx.x == 0) run = 0;
            __syncthreads();
            for (int i0 = 0; i0 < cnt; i0 += kThreads) {
                const int i = i0 + threadIdx.x;
                const bool flag = i < cnt && sv.cls[off + i] == c;
                const unsigned bal = __ballot_sync(0xffffffffu, flag);
                if (lane == 0) wcnt[warp] = __popc(bal);
                __syncthreads();
                int before = run;
                for (int w = 0; w < warp; ++w) before += wcnt[w];
                if (flag) sv.tmp[off + cstart[c] + before + __popc(bal & ((1u << lane) - 1u))] = sv.members[off + i];
                __syncthreads();
                if (threadIdx.x == 0)
                    for (int w = 0; w < kThreads / 32; ++w) run += wcnt[w];
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < cnt; i += kThreads) sv.members[off + i] = sv.tmp[off + i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const TrajState parent = v.st[s];
        for (int k = 0; k < no; ++k) {
            const int c = order[k];
            const ClassOp op = class_op(gt, m, c & 15, (c >> 4) & 1, (c >> 5) & 1, gamma, damp);
            if (op.bad) atomicOr(v.status, 1);
            TrajState ns = parent;
            set_pending(ns, gt, op);
            const int2 r = make_int2(off + cstart[c], ccount[c]);
            if (k == 0) {
                v.st[s] = ns;
                sv.range[s] = r;
            } else {
                const int child = child_base + k - 1;
                if (child >= sv.max_slots) {
                    atomicOr(v.status, 4);
                    continue;
                }
                v.st[child] = ns;
                sv.range[child] = r;
                const int f = atomicAdd(sv.fork_count, 1);
                sv.forks[f] = make_int2(s, child);
            }
        }
    }
    __syncthreads();
}

// Slot sweeps: grid (sweep tiles, slots alive before this gate), one unit per
// block, the same body as the batch sweeps; the last block of a slot stores the
// slot's marginal for k_slot_decide.
template <bool DAMP, int KIND, bool DYN = false>
__global__ void __launch_bounds__(kThreads, 4) k_slot_sweep(BatchView v, SlotView sv, int g, DevGate gt) {
    grid_dependency_wait();
    __shared__ int q_item, q_lo, q_n;
    int nxt = 0;  // thread 0: the next item claimed
    int tile, slot;
    for (int it = 0; sweep_item<DYN>(v, 0, it, q_item, q_lo, q_n, nxt, tile, slot); ++it) {
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
        if (KIND == kGateZZ) zz_unit<DAMP, true>(v, slot, tile, g, gt, a0, a1, a2, a3);
        else rx_unit<DAMP, true>(v, slot, tile, g, gt, a0, a3);
        allow_dependent_launch();
        if (DAMP) {
            __shared__ double m[4];
            if (reduce_marginal(v, slot, tile, a0, a1, a2, a3, m) && threadIdx.x < 4)
                sv.marg[(size_t)slot * 4 + threadIdx.x] = m[threadIdx.x];
        }
    }
}

// Branch classes of every live slot at gate g: one block per slot.
template <bool DAMP>
__global__ void __launch_bounds__(kThreads) k_slot_decide(BatchView v, SlotView sv, int g, DevGate gt, double gamma) {
    grid_dependency_wait();
    // a block per live slot (device-driven runs: blocks stride over the live count)
    const int active = sv.dyn ? *sv.active : (int)gridDim.x;
    for (int slot = blockIdx.x; slot < active; slot += gridDim.x) {
        decide_slot(v, sv, slot, g, gt, sv.marg + (size_t)slot * 4, gamma, DAMP);
        if (slot + (int)gridDim.x < active) __syncthreads();
    }
    allow_dependent_launch();
}

// |fac * a|^2 with fixed rounding (no contraction), so that the norm pass and
// the probability pass see bit-identical FP32 values and sum(sigma) = 1 to FP64
// rounding.
__device__ __forceinline__ float prob_of(float fac, float re, float im) {
    return __fmul_rn(__fmul_rn(fac, fac), __fadd_rn(__fmul_rn(re, re), __fmul_rn(im, im)));
}

// Compensated FP32 sums (double-float): FP64 is slow on this part, so the
// per-amplitude accumulations run as FP32 pairs (hi, lo) with the exact error
// of every step kept in lo (Knuth's TwoSum; the product error from one FMA),
// and only short sums are carried this way before they are added in FP64.
// The _rn intrinsics keep the compiler from contracting or reordering them.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__device__ __forceinline__ void df_add(float &hi, float &lo, float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
}

// (hi, lo) += x * (mh + ml), with x * mh split exactly into product and error.
__device__ __forceinline__ void df_add_prod(float &hi, float &lo, float x, float mh, float ml) {
    const float p = __fmul_rn(x, mh);
    const float pe = __fmaf_rn(x, ml, __fmaf_rn(x, mh, -p));
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

// Warp sum of double-float pairs (fixed butterfly order), returned as FP64.
__device__ __forceinline__ double df_warp_sum(float hi, float lo) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, off), ol = __shfl_xor_sync(0xffffffffu, lo, off);
        float s, e;
        two_sum(hi, oh, s, e);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(ol, e));
    }
    return (double)hi + (double)lo;
}

// ---------------------------------------------------------------------------
// Phase-gate groups in shared-prefix mode.  A group is a run of consecutive
// phase gates of one layer on a qubit set S of at most 10 qubits.  Every op of
// the group -- phase, Z part of a Pauli, K0 -- is diagonal in the stored basis,
// and every X part or K1 jump only relabels true bits, so the branch of every
// damping site in the group follows from the joint distribution of the true
// bits of S when the group starts.  The group decide (k_gd_*) draws all
// members' branches from that joint in FP32 (the same draws, conditioned the
// same way, as one gate at a time), forks every outcome string other than the
// shared one and writes per slot a table T of 2^|S| amplitude factors;
// k_group_apply multiplies the state by T in one sweep and accumulates the
// next group's joint on the way.  Joints are summed in warp-private shared
// histograms in a fixed order (or, in the last mixer block of a layer, in one
// block histogram of integers) and added across blocks as 2^-60 fixed-point
// integers, so they do not depend on the order in which blocks or warps run.
// ---------------------------------------------------------------------------
constexpr double kHistScale = 1152921504606846976.0;  // 2^60
constexpr double kHistUnit = 1.0 / kHistScale;
// Phase-group sweeps stream kGSub sub-tiles per block (twice the gate sweeps'
// kSub), so the per-block histogram work is spread over more amplitudes.
constexpr int kGSub = 8;
constexpr int kGLow = 14;  // amplitude bits a group-sweep block covers
static_assert(kThreads == 256 && kTileF4 == 1024 && kF4PerThread == 4 && kGSub == 8,
              "group bins assume y = e | tid << 1 | k << 9 | sub << 11 | tile << 14");

__device__ __forceinline__ int group_bin(const GateGroup *gp, uint32_t y) {
    return gp->tab[0][y & 255u] | gp->tab[1][(y >> 8) & 255u] | gp->tab[2][(y >> 16) & 255u] | gp->tab[3][y >> 24];
}

// Bins of one group-sweep block split into a per-thread part (tid bits), a
// block part (tile bits) and a part that depends only on the unrolled loop
// indices (e, k, sub), kept in the shared table vtab[e | k << 1 | sub << 3].
// A group-sweep block covers amplitude bits 0 .. kGLow-1 and fixes the higher
// ones, so it touches only the bins of S's qubits below kGLow -- the low `nlow`
// bin bits (S is numbered in ascending qubit order) -- above a block-constant
// part `hi`.  The block's histogram is indexed by the low bits alone.
struct GroupBins {
    int base;        // low bins of this thread's tid bits
    unsigned lmask;  // lane bits that are no qubit of S
    int hi;          // the block's high bins (its tile bits)
    int nlow;        // S's qubits below kGLow
};

__device__ __forceinline__ GroupBins group_bins(const GateGroup *gp, int tile, uint16_t *vtab) {
    GroupBins gb;
    int nlow = 0;
    while (nlow < gp->s && gp->sp[nlow] < kGLow) ++nlow;
    gb.nlow = nlow;
    gb.base = group_bin(gp, (uint32_t)threadIdx.x << 1);
    gb.hi = group_bin(gp, (uint32_t)tile << kGLow);
    unsigned lm = 0;
    for (int i = 0; i < 5; ++i)
        if (group_bin(gp, 2u << i) == 0) lm |= 1u << i;
    gb.lmask = lm;
    if (threadIdx.x < 2 * 4 * kGSub) {  // j = e | k << 1 | sub << 3
        const uint32_t j = threadIdx.x;
        vtab[j] = (uint16_t)group_bin(gp, (j & 1u) | (((j >> 1) & 3u) << 9) | ((j >> 3) << 11));
    }
    return gb;
}

// Add x, summed over the lanes that differ only outside S, to the warp's
// histogram (lanes left after the butterfly hold distinct bins).
__device__ __forceinline__ void hist_flush(float *hw, float x, int bin, unsigned lmask) {
#pragma unroll
    for (int i = 0; i < 5; ++i)
        if ((lmask >> i) & 1u) x += __shfl_xor_sync(0xffffffffu, x, 1 << i);
    if (((threadIdx.x & 31u) & lmask) == 0u) hw[bin] += x;
    __syncwarp();
}

// The same into a block-wide histogram of 2^-60 fixed-point integers: each
// flushed value is quantised once and integer adds commute, so the block's
// sums do not depend on the order in which its warps arrive.
constexpr float kHistScaleF = 1152921504606846976.0f;  // 2^60
__device__ __forceinline__ void hist_flush(unsigned long long *h, float x, int bin, unsigned lmask) {
#pragma unroll
    for (int i = 0; i < 5; ++i)
        if ((lmask >> i) & 1u) x += __shfl_xor_sync(0xffffffffu, x, 1 << i);
    if (((threadIdx.x & 31u) & lmask) == 0u && x > 0.0f) atomicAdd(h + bin, (unsigned long long)__float2ull_rn(x * kHistScaleF));
}

// Run of consecutive (e = 0, e = 1) probabilities with the same loop-index bin
// `ks`; flushed when ks changes (ks is warp-uniform).  e1 = bin bits of y bit 0.
struct HistRun {
    float r0 = 0.0f, r1 = 0.0f;
    int ks = -1;
};

template <class Sink>
__device__ __forceinline__ void hist_close(Sink *hw, const GroupBins &gb, int e1, const HistRun &run) {
    if (run.ks < 0) return;
    if (e1) {
        hist_flush(hw, run.r0, gb.base | run.ks, gb.lmask);
        hist_flush(hw, run.r1, gb.base | run.ks | e1, gb.lmask);
    } else {
        hist_flush(hw, run.r0 + run.r1, gb.base | run.ks, gb.lmask);
    }
}

template <class Sink>
__device__ __forceinline__ void hist_push(Sink *hw, const GroupBins &gb, int e1, int ks, float p0, float p1,
                                          HistRun &run) {
    if (ks != run.ks) {
        hist_close(hw, gb, e1, run);
        run.ks = ks;
        run.r0 = p0;
        run.r1 = p1;
    } else {
        run.r0 += p0;
        run.r1 += p1;
    }
}

// Block histogram -> the slot's global joint (fixed-point integer adds).
__device__ __forceinline__ void hist_commit(const float *hw, const GroupBins &gb, unsigned long long *H) {
    for (int b = threadIdx.x; b < (1 << gb.nlow); b += kThreads) {
        double acc = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) acc += (double)hw[w * kGroupBins + b];
        if (acc > 0.0) atomicAdd(H + (gb.hi | b), __double2ull_rn(acc * kHistScale));
    }
}

// Zero the block's histogram rows (the low bins only).
__device__ __forceinline__ void hist_zero(float *hw, int nlow) {
    const int nb = 1 << nlow;
    for (int i = threadIdx.x; i < (kThreads / 32) * nb; i += kThreads) hw[(i / nb) * kGroupBins + (i % nb)] = 0.0f;
}

__device__ __forceinline__ SweepCtx pending_ctx(const TrajState &s) {
    SweepCtx c;
    c.code = 0;
    c.Fa = s.J;
    c.Fb = c.Fc = s.J ^ s.pend;
    c.pq0 = s.pq0;
    c.pq1 = s.pq1;
    for (int k = 0; k < 4; ++k) c.f[k] = s.f[k];
    return c;
}

// Joint of the first group of a layer: a read-only pass that applies the
// pending op of the gate before on the fly.  Grid (sweep tiles, live slots).
template <bool PEND, bool DYN = false>
__global__ void __launch_bounds__(kThreads, 4) k_group_hist(BatchView v, GroupView gv) {
    grid_dependency_wait();
    __shared__ int q_item, q_lo, q_n;
    int nxt = 0;  // thread 0: the next item claimed
    int tile, slot;
    for (int it = 0; sweep_item<DYN>(v, 0, it, q_item, q_lo, q_n, nxt, tile, slot); ++it) {
    const GateGroup *gp = gv.grp;
    __shared__ float hw[kThreads / 32][kGroupBins];
    __shared__ uint16_t vtab[2 * 4 * kGSub];
    const GroupBins gb = group_bins(gp, tile, vtab);
    hist_zero(&hw[0][0], gb.nlow);
    __syncthreads();
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1);
    const float4 *p4 = reinterpret_cast<const float4 *>(v.psi + ((size_t)slot << n));
    const int64_t fbase = (int64_t)tile * kTileF4 * kGSub + threadIdx.x;
    const SweepCtx c = pending_ctx(v.st[slot]);
    float *my = hw[threadIdx.x >> 5];
    const int e1 = vtab[1];
    HistRun run;
    float4 cur[kF4PerThread], nxt[kF4PerThread];
    load_tile(cur, p4, fbase, nf);
#pragma unroll
    for (int sub = 0; sub < kGSub; ++sub) {
        const int64_t f0 = fbase + (int64_t)sub * kTileF4;
        if (sub + 1 < kGSub) load_tile(nxt, p4, f0 + kTileF4, nf);
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k) {
            const int64_t f = f0 + k * kThreads;
            float p0 = 0.0f, p1 = 0.0f;
            if (f < nf) {
                const uint32_t y = (uint32_t)(2 * f);
                const float fa0 = PEND ? pend_factor(c, y) : 1.0f, fa1 = PEND ? pend_factor(c, y | 1u) : 1.0f;
                p0 = __fmul_rn(__fmul_rn(fa0, fa0), norm2_rn(cur[k].x, cur[k].y));
                p1 = __fmul_rn(__fmul_rn(fa1, fa1), norm2_rn(cur[k].z, cur[k].w));
            }
            hist_push(my, gb, e1, vtab[(k << 1) | (sub << 3)], p0, p1, run);
        }
        if (sub + 1 < kGSub) {
#pragma unroll
            for (int k = 0; k < kF4PerThread; ++k) cur[k] = nxt[k];
        }
    }
    hist_close(my, gb, e1, run);
    __syncthreads();
    allow_dependent_launch();
    hist_commit(&hw[0][0], gb, gv.Hcur + (size_t)slot * kGroupBins);
    }
}

// Per-block joint of a mixer block (at most 4 qubits): the per-warp rows
// hw[warps][kJointBins] are summed in fixed order (after a block barrier) and the
// block's 2^nb bins added to H as 2^-60 fixed-point integers.
constexpr int kJointBins = 16;  // bins of a mixer block's joint (at most 4 qubits)

__device__ __forceinline__ void lane_joint_commit(int nb, int warps, const float *hw, unsigned long long *H) {
    if ((int)threadIdx.x < nb) {
        double sum = 0.0;
        for (int w = 0; w < warps; ++w) sum += (double)hw[w * kJointBins + threadIdx.x];
        if (sum > 0.0) atomicAdd(H + threadIdx.x, __double2ull_rn(sum * kHistScale));
    }
}

// Apply a phase group: phi_y *= D(y) * T[slot][stored bits of S], D the pending
// op of the gate before the group, and accumulate the next phase group's joint
// (NEXT = 1, gv.next) on the way.  PEND: the gate before left a pending op
// (else it is the identity and skipped).  The last phase group of a layer is
// applied by k_group_mix instead, which also starts the mixer layer.
template <bool PEND, int NEXT, bool DYN = false>
__global__ void __launch_bounds__(kThreads, 4) k_group_apply(BatchView v, GroupView gv) {
    grid_dependency_wait();
    __shared__ int q_item, q_lo, q_n;
    int nxt = 0;  // thread 0: the next item claimed
    int tile, slot;
    for (int it = 0; sweep_item<DYN>(v, gv.slot_base, it, q_item, q_lo, q_n, nxt, tile, slot); ++it) {
    const int from = gv.src ? gv.src[slot] : slot;  // a new slot's first sweep reads its parent
    const GateGroup *gp = gv.grp;
    const GateGroup *nx = NEXT == 1 ? gv.next : nullptr;
    __shared__ float2 Ts[kGroupBins];
    __shared__ float hw[kThreads / 32][kGroupBins];
    __shared__ uint16_t vT[2 * 4 * kGSub], vN[2 * 4 * kGSub];
    for (int i = threadIdx.x; i < (1 << gp->s); i += kThreads) Ts[i] = gv.T[(size_t)slot * kGroupBins + i];
    const GroupBins gt = group_bins(gp, tile, vT);
    GroupBins gn{0, 0u, 0, 0};
    if (NEXT == 1) {
        gn = group_bins(nx, tile, vN);
        hist_zero(&hw[0][0], gn.nlow);
    }
    __syncthreads();
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1);
    const float4 *q4 = reinterpret_cast<const float4 *>(v.psi + ((size_t)from << n));
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)slot << n));
    const int64_t fbase = (int64_t)tile * kTileF4 * kGSub + threadIdx.x;
    const SweepCtx c = pending_ctx(gv.st_prev[slot]);
    float *my = hw[threadIdx.x >> 5];
    const int tE1 = vT[1];
    const int nE1 = NEXT == 1 ? vN[1] : 0;
    HistRun run;
    float4 cur[kF4PerThread], nxt[kF4PerThread];
    load_tile(cur, q4, fbase, nf);
#pragma unroll
    for (int sub = 0; sub < kGSub; ++sub) {
        const int64_t f0 = fbase + (int64_t)sub * kTileF4;
        if (sub + 1 < kGSub) load_tile(nxt, q4, f0 + kTileF4, nf);
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k) {
            const int64_t f = f0 + k * kThreads;
            float4 o = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (f < nf) {
                const uint32_t y = (uint32_t)(2 * f);
                const int tb = gt.hi | gt.base | vT[(k << 1) | (sub << 3)];
                const float fa0 = PEND ? pend_factor(c, y) : 1.0f, fa1 = PEND ? pend_factor(c, y | 1u) : 1.0f;
                const float2 w0 = Ts[tb], w1 = Ts[tb | tE1];
                const float wr0 = __fmul_rn(w0.x, fa0), wi0 = __fmul_rn(w0.y, fa0);
                const float wr1 = __fmul_rn(w1.x, fa1), wi1 = __fmul_rn(w1.y, fa1);
                const float4 a = cur[k];
                cmul_rn(a.x, a.y, wr0, wi0, o.x, o.y);
                cmul_rn(a.z, a.w, wr1, wi1, o.z, o.w);
                p4[f] = o;
            }
            if (NEXT == 1) hist_push(my, gn, nE1, vN[(k << 1) | (sub << 3)], norm2_rn(o.x, o.y), norm2_rn(o.z, o.w), run);
        }
        if (sub + 1 < kGSub) {
#pragma unroll
            for (int k = 0; k < kF4PerThread; ++k) cur[k] = nxt[k];
        }
    }
    if (NEXT == 1) hist_close(my, gn, nE1, run);
    __syncthreads();
    allow_dependent_launch();
    if (NEXT == 1) hist_commit(&hw[0][0], gn, gv.Hnext + (size_t)slot * kGroupBins);
    }
}

// 16-byte asynchronous global -> shared copies (the copy engine of the SM
// streams the next tile while the current one is computed).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int kMixTile = 2048;  // float4 per tile
constexpr size_t kMixSmem = 2 * kMixTile * sizeof(float4);
constexpr int kMixE = 1 << kMixQ;  // float4 per thread and phase

// exp(-i beta X) on a pair up to the common factor sc (cos beta when TANF,
// sin beta otherwise): (I - i t X) with t = tan beta, or (t I - i X) with
// t = cot beta -- four FMAs per pair, and |t| <= 1 either way.
template <bool TANF>
__device__ __forceinline__ void rx_pair_t(float &ar, float &ai, float &br, float &bi, float t) {
    float nar, nai, nbr, nbi;
    if (TANF) {
        nar = __fmaf_rn(t, bi, ar);
        nai = __fmaf_rn(-t, br, ai);
        nbr = __fmaf_rn(t, ai, br);
        nbi = __fmaf_rn(-t, ar, bi);
    } else {
        nar = __fmaf_rn(t, ar, bi);
        nai = __fmaf_rn(t, ai, -br);
        nbr = __fmaf_rn(t, br, ai);
        nbi = __fmaf_rn(t, bi, -ar);
    }
    ar = nar;
    ai = nai;
    br = nbr;
    bi = nbi;
}

template <bool TANF>
__device__ __forceinline__ void rx_pair4_t(float4 &a, float4 &b, float t) {
    rx_pair_t<TANF>(a.x, a.y, b.x, b.y, t);
    rx_pair_t<TANF>(a.z, a.w, b.z, b.w, t);
}

// Mixer block sweep (shared-prefix mode): exp(-i beta X) on the block's (up
// to kMixQ consecutive) qubits, then the block's drawn Pauli and damping ops
// as the real factor T[slot][stored bits of the block] (drawn beforehand from
// the joint after the rotations, so the state is final when written).  Tiles
// of 2048 float4 stream through two shared buffers (cp.async, one tile
// ahead), each copied by the threads that take it in phase 1: (1) per thread
// the float4 along the block's qubits (A bits) are rotated, scaled and stored
// to HBM (and back to the tile); (2) per thread the float4 along the next
// block's qubits (B bits) are read from the tile and rotated without being
// kept, and their squared magnitudes give that block's joint after its
// rotations.  Register pairs only, no shuffles; the tile is read in lane order
// (tile index = L | A << kMixL | B << (kMixL + kMixQ)).
// Variants with every bound a constant (all for full blocks of kMixQ qubits):
//   kMixMid   not qubit 0, a full next block
//   kMixHist  not qubit 0, no next block, the next layer's first phase-group joint
//   kMixKeep  not qubit 0, the circuit's last block: forms the final norms and
//             stores nothing (the states stay as they were; the sigma pass,
//             k_probs_mix, applies the block again on the fly)
// and kMixAny, which reads everything from the map (and stores the final states
// of a last block it sweeps); and
//   kMixWide  the qubits 4-7 of a block that covers qubits 0-7 (the sweep before
//             rotated qubits 0-3, k_group_mix): a full next block, and the factor
//             table of all eight qubits (qubit 0 = the float4 half, qubits 1-3 =
//             the lane bits L, qubits 4-7 = the element index j)
//   kMixW1    (MixMap::wide 2) the factors of the block over qubits 0-7, all eight
//             rotated by the sweep before (k_group_mix FULL); A = the first half of
//             the next, 8-qubit block, B its second half; that block's joint has
//             256 bins, A | B << 4
//   kMixW2    (MixMap::wide 3) the second half A of an 8-qubit block whose first
//             half (tile f bits wsh .. wsh+3) kMixW1 rotated: the block's factors
//             by A << 4 | first half, and a full next block
enum { kMixAny = 0, kMixMid = 1, kMixHist = 2, kMixWide = 8, kMixW1 = 16, kMixW2 = 32 };

template <bool TANF, int VAR, bool DYN = false>
__global__ void __launch_bounds__(kMixThreads, 3) k_mix_sweep(BatchView v, GroupView gv, MixMap mm) {
    extern __shared__ float4 mix_buf[];  // [2][kMixTile]
    constexpr int kWarps = kMixThreads / 32;
    grid_dependency_wait();
    __shared__ int q_item, q_lo, q_n;
    int nxt = 0;  // thread 0: the next item claimed
    int bx, slot;  // the block of tiles (kMixSubs per block) and the slot this item sweeps
    for (int it = 0; sweep_item<DYN>(v, gv.slot_base, it, q_item, q_lo, q_n, nxt, bx, slot); ++it) {
    const int from = gv.src ? gv.src[slot] : slot;  // a new slot's first sweep reads its parent
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tL = threadIdx.x & ((1 << kMixL) - 1), tH = threadIdx.x >> kMixL;  // L part, A or B part
    constexpr bool kFix = VAR != kMixAny;
    // next layer's first phase group: its joint is formed here
    const GateGroup *nx = kFix ? (VAR == kMixHist ? gv.next : nullptr) : gv.next;
    const bool has0 = kFix ? false : mm.has0 != 0;
    const int M = kFix ? kMixQ : mm.M;
    constexpr bool kW8 = VAR == kMixWide || VAR == kMixW1 || VAR == kMixW2;  // 256-entry factor table
    const int nN = kFix ? ((VAR == kMixMid || kW8) ? kMixQ : 0) : mm.nN;
    const bool final_norm = kFix ? false : mm.final_norm != 0;
    const float c = gv.grp->c, sn = gv.grp->sn;
    const float rt = TANF ? sn / c : c / sn, rsc = TANF ? c : sn;  // rotation = rsc * (tangent form)
    float scM = 1.0f;  // rsc^M: the block's rotations, folded into its factors
    for (int i = 0; i < M; ++i) scM *= rsc;
    constexpr int kDf = kW8 ? 256 : 16;
    __shared__ float Df[kDf];
    // the block's histogram of the next phase group's joint (variants that form one; 2^-60
    // fixed point, one row for all warps), and the per-warp rows of the next mixer block's joint
    constexpr bool kHist = VAR == kMixAny || VAR == kMixHist;
    __shared__ unsigned long long hist[kHist ? kGroupBins : 1];
    __shared__ float red[kWarps * kJointBins];
    if (kW8) {
        for (int i = threadIdx.x; i < kDf; i += kMixThreads) Df[i] = gv.T[(size_t)slot * kGroupBins + i].x * scM;
    } else if (threadIdx.x < 16u) {
        Df[threadIdx.x] = threadIdx.x < (1u << M) ? gv.T[(size_t)slot * kGroupBins + threadIdx.x].x * scM : 0.0f;
    }
    if (nx)
        for (int i = threadIdx.x; i < kGroupBins; i += kMixThreads) hist[i] = 0ull;
    // float4 indices fit 32 bits (n <= 30)
    uint32_t offL = 0, offW = 0, ao[kMixQ];
#pragma unroll
    for (int i = 0; i < kMixL; ++i) offL |= (uint32_t)((tL >> i) & 1) << mm.fL[i];
#pragma unroll
    for (int i = 0; i < kMixQ; ++i) {
        offW |= (uint32_t)((tH >> i) & 1) << mm.fB[i];
        ao[i] = 1u << mm.fA[i];
    }
    auto aoff = [&](int j) {
        uint32_t o = 0;
#pragma unroll
        for (int i = 0; i < kMixQ; ++i) o |= (j & (1 << i)) ? ao[i] : 0u;
        return o;
    };
    const float4 *q4 = reinterpret_cast<const float4 *>(v.psi + ((size_t)from << v.n));
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)slot << v.n));
    const int nqa = has0 ? M - 1 : M;  // block qubits on A bits
    const int dmask = (1 << nqa) - 1;
    const int nsubs = mm.ntile >= 2 ? kMixSubs : (1 << mm.ntile);
    // tile offsets: the block's first tile, plus sub-tile steps (tile bits 0, 1)
    uint32_t tbits = 0;  // tile bits of the block's first tile
    {
        const uint32_t t0 = (uint32_t)bx * nsubs;
#pragma unroll
        for (int i = 0; i < 32; ++i)  // constant indices: the map stays in parameter space
            if (i < mm.ntile) tbits |= ((t0 >> i) & 1u) << mm.ftile[i];
    }
    const uint32_t tbase = tbits | offL | offW;
    const uint32_t ts1 = mm.ntile > 0 ? 1u << mm.ftile[0] : 0u;
    const uint32_t ts2 = mm.ntile > 1 ? 1u << mm.ftile[1] : 0u;
    auto tile_base = [&](int sub) { return tbase | ((sub & 1) ? ts1 : 0u) | ((sub & 2) ? ts2 : 0u); };
    // shared tile slot of tile index i: the low A bits are XOR-ed into the L bits, so
    // that eight lanes apart by A (the copy order of the qubit-0 block) hit distinct banks
    auto sw = [](int i) { return i ^ ((i >> kMixL) & ((1 << kMixL) - 1)); };
    auto idx1 = [&](int j) { return sw(tL | (j << kMixL) | (tH << (kMixL + kMixQ))); };  // phase 1: j along A
    auto idx2 = [&](int j) { return sw(tL | (tH << kMixL) | (j << (kMixL + kMixQ))); };  // phase 2: j along B
    // The block holding qubit 0 has its own qubits on the lowest f bits, where
    // the phase-1 order would give every lane its own 128-byte line: it copies
    // in an order with A bits 0-2 on lane bits 0-2 instead, and takes a block
    // barrier before phase 1 (threads then read what others copied).
    uint32_t cbase = 0;
    int cidx = 0;
    uint32_t bo[kMixQ];
#pragma unroll
    for (int i = 0; i < kMixQ; ++i) bo[i] = 1u << mm.fB[i];
    if (has0) {
        const int la = lane & 7, ll = ((lane >> 3) & 3) | ((warp & 1) << 2), ah = warp >> 1;
        cidx = ll | (la << kMixL) | (ah << (kMixL + 3));
#pragma unroll
        for (int i = 0; i < kMixL; ++i) cbase |= (uint32_t)((ll >> i) & 1) << mm.fL[i];
#pragma unroll
        for (int i = 0; i < 3; ++i) cbase |= (uint32_t)((la >> i) & 1) << mm.fA[i];
        cbase |= (uint32_t)ah << mm.fA[3];
    }
    auto fetch = [&](int sub) {  // tile `sub` into its buffer
        const uint32_t ts = ((sub & 1) ? ts1 : 0u) | ((sub & 2) ? ts2 : 0u);
        float4 *buf = mix_buf + (sub & 1) * kMixTile;
        if (has0) {
#pragma unroll
            for (int j = 0; j < kMixE; ++j) {
                uint32_t bofs = 0;
#pragma unroll
                for (int i = 0; i < kMixQ; ++i) bofs |= (j & (1 << i)) ? bo[i] : 0u;
                cp_async16(buf + sw(cidx | (j << (kMixL + kMixQ))), q4 + (tbits | ts | cbase | bofs));
            }
        } else {
            const uint32_t fb = tbase | ts;
#pragma unroll
            for (int j = 0; j < kMixE; ++j) cp_async16(buf + idx1(j), q4 + (fb | aoff(j)));
        }
        cp_async_commit();
    };
    // next phase group's bins: this thread's part, the A part of element j, the float4 half
    GroupBins gn{0, 0u};
    int nab[kMixQ], ne1 = 0;
    int nb0 = 0, nb1 = 0, nb2 = 0;  // bins of the first tile's thread offset and of the sub-tile steps
#pragma unroll
    for (int i = 0; i < kMixQ; ++i) nab[i] = 0;
    if (nx) {
#pragma unroll
        for (int i = 0; i < kMixQ; ++i) nab[i] = group_bin(nx, (uint32_t)(2 * ao[i]));
        ne1 = group_bin(nx, 1u);
        // a bin is the OR of its bits' bins, so a tile's is the first's with the steps' ORed in
        nb0 = group_bin(nx, 2u * tbase);
        nb1 = group_bin(nx, 2u * ts1);
        nb2 = group_bin(nx, 2u * ts2);
        // lane bits: kMixL bits of L, then the low B bits
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const int fbit = i < kMixL ? mm.fL[i] : mm.fB[i - kMixL];
            if (group_bin(nx, 2u << fbit) == 0) gn.lmask |= 1u << i;
        }
    }
    HistRun run;
    float acc[kMixE];  // phase 2: sum of |.|^2 by B index j (folded into the next block's bins at the end)
#pragma unroll
    for (int j = 0; j < kMixE; ++j) acc[j] = 0.0f;
    float nh = 0.0f, nl = 0.0f;  // final norm (double-float), same FP32 terms as k_probs forms
    fetch(0);
    __syncthreads();  // Df, hw
    for (int sub = 0; sub < nsubs; ++sub) {
        if (sub + 1 < nsubs) {
            fetch(sub + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        if (has0) __syncthreads();  // copies by other threads
        float4 *buf = mix_buf + (sub & 1) * kMixTile;
        const uint32_t fb = tile_base(sub);
        float4 x[kMixE];
#pragma unroll
        for (int j = 0; j < kMixE; ++j) x[j] = buf[idx1(j)];  // this thread's own copies unless has0
        // phase 1: the block's rotations, then its factors
        if (has0) {
#pragma unroll
            for (int j = 0; j < kMixE; ++j) rx_pair_t<TANF>(x[j].x, x[j].y, x[j].z, x[j].w, rt);
        }
#pragma unroll
        for (int i = 0; i < kMixQ; ++i) {
            if (i >= nqa) break;
#pragma unroll
            for (int j = 0; j < kMixE; ++j)
                if (!(j & (1 << i))) rx_pair4_t<TANF>(x[j], x[j | (1 << i)], rt);
        }
#pragma unroll
        for (int j = 0; j < kMixE; ++j) {
            const int d = j & dmask;
            float f0 = has0 ? Df[d << 1] : Df[d], f1 = has0 ? Df[(d << 1) | 1] : Df[d];
            if (VAR == kMixWide) {  // qubit 0 the half, qubits 1-3 the lane bits L, qubits 4-7 j
                f0 = Df[(j << 4) | (tL << 1)];
                f1 = Df[(j << 4) | (tL << 1) | 1];
            }
            if (VAR == kMixW1) {  // qubit 0 the half, qubits 1-3 L, qubits 4-7 the tile's f bits
                const int t47 = (int)((fb >> mm.wsh) & 15u) << 4;
                f0 = Df[t47 | (tL << 1)];
                f1 = Df[t47 | (tL << 1) | 1];
            }
            if (VAR == kMixW2) {  // the block's first half on the tile's f bits, its second j
                f0 = f1 = Df[(j << 4) | (int)((fb >> mm.wsh) & 15u)];
            }
            x[j].x *= f0;
            x[j].y *= f0;
            x[j].z *= f1;
            x[j].w *= f1;
            if (has0) buf[idx1(j)] = x[j];  // stored from the tile in copy order below
            else p4[fb | aoff(j)] = x[j];
            if (nN > 0 && !has0) buf[idx1(j)] = x[j];
            if (nx) {
                if (j == 0) gn.base = nb0 | ((sub & 1) ? nb1 : 0) | ((sub & 2) ? nb2 : 0);
                int ks = 0;
#pragma unroll
                for (int i = 0; i < kMixQ; ++i) ks |= (j & (1 << i)) ? nab[i] : 0;
                hist_push(hist, gn, ne1, ks, norm2_rn(x[j].x, x[j].y), norm2_rn(x[j].z, x[j].w), run);
            }
            if (final_norm) {
                df_add(nh, nl, prob_of(1.0f, x[j].x, x[j].y));
                df_add(nh, nl, prob_of(1.0f, x[j].z, x[j].w));
            }
        }
        if (nx) {  // the per-thread bin part changes with the tile
            hist_close(hist, gn, ne1, run);
            run = HistRun();
        }
        if (nN > 0 || has0) __syncthreads();
        if (has0) {
            const uint32_t ts = ((sub & 1) ? ts1 : 0u) | ((sub & 2) ? ts2 : 0u);
#pragma unroll
            for (int j = 0; j < kMixE; ++j) {
                uint32_t bofs = 0;
#pragma unroll
                for (int i = 0; i < kMixQ; ++i) bofs |= (j & (1 << i)) ? bo[i] : 0u;
                p4[tbits | ts | cbase | bofs] = buf[sw(cidx | (j << (kMixL + kMixQ)))];
            }
        }
        if (nN > 0) {
            // phase 2: the next block's rotations on the tile, kept only as squared magnitudes
#pragma unroll
            for (int j = 0; j < kMixE; ++j) x[j] = buf[idx2(j)];
#pragma unroll
            for (int i = 0; i < kMixQ; ++i) {
                if (i >= nN) break;
#pragma unroll
                for (int j = 0; j < kMixE; ++j)
                    if (!(j & (1 << i))) rx_pair4_t<TANF>(x[j], x[j | (1 << i)], rt);
            }
#pragma unroll
            for (int j = 0; j < kMixE; ++j)
                acc[j] = __fadd_rn(acc[j], __fadd_rn(norm2_rn(x[j].x, x[j].y), norm2_rn(x[j].z, x[j].w)));
        }
        if (nN > 0 || has0) __syncthreads();  // the buffer is refilled two tiles on
    }
    allow_dependent_launch();
    if (VAR == kMixW1) {
        // 256 bins A | B << 4: this thread's A is tH and its B is j; sum over the L lanes
        float sc2 = 1.0f;  // B was rotated up to rsc per qubit: restore |.|^2
        for (int i = 0; i < kMixQ; ++i) sc2 *= rsc * rsc;
        __syncthreads();  // the tile buffers now hold the bins
        float *bins = reinterpret_cast<float *>(mix_buf);
#pragma unroll
        for (int j = 0; j < kMixE; ++j) {
            float x = __fmul_rn(acc[j], sc2);
#pragma unroll
            for (int off = 1; off < (1 << kMixL); off <<= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (tL == 0) bins[tH | (j << 4)] = x;
        }
        __syncthreads();
        unsigned long long *H = gv.Hnext + (size_t)slot * kGroupBins;
        for (int b = threadIdx.x; b < 256; b += kMixThreads)
            if (bins[b] > 0.0f) atomicAdd(H + b, __double2ull_rn((double)bins[b] * kHistScale));
    } else if (nN > 0) {
        // bins of the next block are the low nN bits of j: fold, then lanes and warps
        const int nb = 1 << nN;
#pragma unroll
        for (int half = kMixE / 2; half >= 1; half >>= 1) {
            if (nb <= half) {
#pragma unroll
                for (int j = 0; j < half; ++j) acc[j] += acc[j + half];
            }
        }
        float sc2 = 1.0f;  // the next block's rotations were taken up to rsc each: restore |.|^2
        for (int i = 0; i < nN; ++i) sc2 *= rsc * rsc;
#pragma unroll
        for (int b = 0; b < kMixE; ++b) {
            float x = __fmul_rn(acc[b], sc2);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0) red[warp * kJointBins + b] = x;
        }
        __syncthreads();
        lane_joint_commit(nb, kWarps, red, gv.Hnext + (size_t)slot * kGroupBins);
    }
    if (nx) {
        __syncthreads();
        for (int b = threadIdx.x; b < (1 << nx->s); b += kMixThreads)
            if (hist[b]) atomicAdd(gv.Hnext + (size_t)slot * kGroupBins + b, hist[b]);
    }
    if (final_norm) {
        // block partial -> partials[slot][block]; the slot's last block forms 1/N
        __shared__ double redd[kWarps];
        __shared__ int last;
        const double ws = df_warp_sum(nh, nl);
        if (lane == 0) redd[warp] = ws;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (int w = 0; w < kWarps; ++w) sum += redd[w];
            v.partials[((size_t)slot * v.tiles + bx) * 4] = sum;
            __threadfence();
            const unsigned prev = atomicAdd(&v.counters[slot], 1u);
            last = prev == (unsigned)sweep_tiles<DYN>(v) - 1;
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            __threadfence();
            double N = 0.0;
            for (int i = 0; i < sweep_tiles<DYN>(v); ++i) N += __ldcg(v.partials + ((size_t)slot * v.tiles + i) * 4);
            if (!(N > 0.0) || !isfinite(N)) atomicOr(v.status, 2);
            v.inv_norm[slot] = 1.0 / N;
            v.counters[slot] = 0;
        }
    }
    }
}

// exp(-i beta X) up to the common factor (see rx_pair_t) on a qubit whose two
// values sit in lanes that differ in `lanebit`.  The rotation treats both
// values alike, so each lane forms its own from its value and its partner's,
// with the same operations rx_pair_t takes for that value.
template <bool TANF>
__device__ __forceinline__ void rx_lanes_t(float4 &o, int lanebit, float t) {
    const float px = __shfl_xor_sync(0xffffffffu, o.x, lanebit), py = __shfl_xor_sync(0xffffffffu, o.y, lanebit);
    const float pz = __shfl_xor_sync(0xffffffffu, o.z, lanebit), pw = __shfl_xor_sync(0xffffffffu, o.w, lanebit);
    if (TANF) {
        o.x = __fmaf_rn(t, py, o.x);
        o.y = __fmaf_rn(-t, px, o.y);
        o.z = __fmaf_rn(t, pw, o.z);
        o.w = __fmaf_rn(-t, pz, o.w);
    } else {
        o.x = __fmaf_rn(t, o.x, py);
        o.y = __fmaf_rn(t, o.y, -px);
        o.z = __fmaf_rn(t, o.z, pw);
        o.w = __fmaf_rn(t, o.w, -pz);
    }
}

// The last phase group of a layer, applied together with the rotations of
// qubits 0-3 of the layer's first mixer block, whose other four qubits (4-7)
// the next sweep rotates: that block covers qubits 0-7 and its Kraus draws
// come from the joint of all eight after their rotations (the same draws as
// gate by gate: an op on one qubit commutes with rotations of the others), which
// this sweep forms by rotating qubits 4-7 in registers without keeping them.
// Tile: the contiguous f bits 0-10 -- qubit 0 inside the float4, qubits 1-3 lane
// bits 0-2, qubits 4-7 the register index j, f7-f10 lane bits 3-4 and the warp.
// Per element: the phase group's factor T[stored bits of S] (and rsc^4 of the
// tangent-form rotations), the rotations of qubits 0-3, the store; then the
// rotations of qubits 4-7, binned by the stored bits of qubits 0-7 (256 bins:
// e | lane bits 0-2 << 1 | j << 4).  No pending op (the gate before is a group).
// FULL: the rotations of qubits 4-7 are kept too (stored after them), so the
// block's joint is binned from the stored state and its own sweep only applies
// its factors (MixMap::wide 2).
template <bool TANF, bool FULL, bool DYN = false>
__global__ void __launch_bounds__(kMixThreads, 3) k_group_mix(BatchView v, GroupView gv, MixMap mm) {
    extern __shared__ float4 mix_buf[];  // [2][kMixE][kMixThreads]
    constexpr int kWarps = kMixThreads / 32;
    static_assert(kMixThreads == 128 && kMixE == 16 && kMixQ == 4, "the tile is f0-f10: 16 float4 x 128 threads");
    grid_dependency_wait();
    __shared__ int q_item, q_lo, q_n;
    int nxt = 0;  // thread 0: the next item claimed
    int bx, slot;  // the block of tiles (kMixSubs per block) and the slot this item sweeps
    for (int it = 0; sweep_item<DYN>(v, gv.slot_base, it, q_item, q_lo, q_n, nxt, bx, slot); ++it) {
    const int from = gv.src ? gv.src[slot] : slot;  // a new slot's first sweep reads its parent
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const GateGroup *gp = gv.grp;
    const float c = gv.vc, sn = gv.vs;  // the mixer layer's angle
    const float rt = TANF ? sn / c : c / sn, rsc = TANF ? c : sn;
    float scM = 1.0f;  // rsc^4 (FULL: rsc^8): the tangent-form rotations kept, folded into T
    for (int i = 0; i < (FULL ? 2 : 1) * kMixQ; ++i) scM *= rsc;
    __shared__ float2 Ts[kGroupBins];
    __shared__ uint16_t binj[kMixE];
    float *red = reinterpret_cast<float *>(mix_buf);  // [kWarps][256], after the tile loop
    for (int i = threadIdx.x; i < (1 << gp->s); i += kMixThreads) {
        const float2 t = gv.T[(size_t)slot * kGroupBins + i];
        Ts[i] = make_float2(t.x * scM, t.y * scM);
    }
    if (threadIdx.x < (unsigned)kMixE) binj[threadIdx.x] = (uint16_t)group_bin(gp, 2u * (threadIdx.x << 3));
    const int bin1 = group_bin(gp, 1u);
    const float4 *q4 = reinterpret_cast<const float4 *>(v.psi + ((size_t)from << v.n));
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)slot << v.n));
    const int nsubs = mm.ntile >= 2 ? kMixSubs : (1 << mm.ntile);
    uint32_t tbits = 0;  // tile bits of the block's first tile
    {
        const uint32_t t0 = (uint32_t)bx * nsubs;
#pragma unroll
        for (int i = 0; i < 32; ++i)  // constant indices: the map stays in parameter space
            if (i < mm.ntile) tbits |= ((t0 >> i) & 1u) << mm.ftile[i];
    }
    const uint32_t ts1 = mm.ntile > 0 ? 1u << mm.ftile[0] : 0u;
    const uint32_t ts2 = mm.ntile > 1 ? 1u << mm.ftile[1] : 0u;
    const uint32_t fth = (uint32_t)(lane & 7) | ((uint32_t)(lane >> 3) << 7) | ((uint32_t)warp << 9);
    auto tile_f = [&](int sub) { return tbits | ((sub & 1) ? ts1 : 0u) | ((sub & 2) ? ts2 : 0u) | fth; };
    auto fetch = [&](int sub) {
        const uint32_t fb = tile_f(sub);
        float4 *buf = mix_buf + (sub & 1) * kMixTile + threadIdx.x;
#pragma unroll
        for (int j = 0; j < kMixE; ++j) cp_async16(buf + j * kMixThreads, q4 + (fb | ((uint32_t)j << 3)));
        cp_async_commit();
    };
    float acc0[kMixE], acc1[kMixE];  // |.|^2 after the rotations of qubits 4-7 by j, for qubit 0 = 0 / 1
#pragma unroll
    for (int j = 0; j < kMixE; ++j) acc0[j] = acc1[j] = 0.0f;
    fetch(0);
    __syncthreads();  // Ts, binj
    for (int sub = 0; sub < nsubs; ++sub) {
        if (sub + 1 < nsubs) {
            fetch(sub + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        const float4 *buf = mix_buf + (sub & 1) * kMixTile + threadIdx.x;
        const uint32_t fb = tile_f(sub);
        const int binb = group_bin(gp, 2u * fb);  // the bits of S outside j and qubit 0
        float4 x[kMixE];
#pragma unroll
        for (int j = 0; j < kMixE; ++j) {
            const float4 a = buf[j * kMixThreads];
            const int bj = binb | binj[j];
            const float2 w0 = Ts[bj], w1 = Ts[bj | bin1];
            cmul_rn(a.x, a.y, w0.x, w0.y, x[j].x, x[j].y);
            cmul_rn(a.z, a.w, w1.x, w1.y, x[j].z, x[j].w);
        }
#pragma unroll
        for (int j = 0; j < kMixE; ++j) rx_pair_t<TANF>(x[j].x, x[j].y, x[j].z, x[j].w, rt);  // qubit 0
#pragma unroll
        for (int i = 0; i < 3; ++i) {  // qubits 1-3
#pragma unroll
            for (int j = 0; j < kMixE; ++j) rx_lanes_t<TANF>(x[j], 1 << i, rt);
        }
        if (!FULL) {
#pragma unroll
            for (int j = 0; j < kMixE; ++j) p4[fb | ((uint32_t)j << 3)] = x[j];
        }
        // the rotations of qubits 4-7, kept only as squared magnitudes unless FULL
#pragma unroll
        for (int i = 0; i < kMixQ; ++i) {
#pragma unroll
            for (int j = 0; j < kMixE; ++j)
                if (!(j & (1 << i))) rx_pair4_t<TANF>(x[j], x[j | (1 << i)], rt);
        }
        if (FULL) {
#pragma unroll
            for (int j = 0; j < kMixE; ++j) p4[fb | ((uint32_t)j << 3)] = x[j];
        }
#pragma unroll
        for (int j = 0; j < kMixE; ++j) {
            acc0[j] = __fadd_rn(acc0[j], norm2_rn(x[j].x, x[j].y));
            acc1[j] = __fadd_rn(acc1[j], norm2_rn(x[j].z, x[j].w));
        }
    }
    allow_dependent_launch();
    float sc2 = 1.0f;  // qubits 4-7 were rotated up to rsc each: restore |.|^2 (FULL: in T)
    for (int i = 0; i < (FULL ? 0 : kMixQ); ++i) sc2 *= rsc * rsc;
    __syncthreads();  // every thread is done with the tile buffers, which now hold the per-warp bins
    // sum over lane bits 3-4 (f7-f8); lanes 0-7 then hold the bins of their qubits 1-3
#pragma unroll
    for (int j = 0; j < kMixE; ++j) {
        float a = __fmul_rn(acc0[j], sc2), b = __fmul_rn(acc1[j], sc2);
        a += __shfl_xor_sync(0xffffffffu, a, 8);
        a += __shfl_xor_sync(0xffffffffu, a, 16);
        b += __shfl_xor_sync(0xffffffffu, b, 8);
        b += __shfl_xor_sync(0xffffffffu, b, 16);
        if (lane < 8) {
            red[warp * 256 + ((j << 4) | (lane << 1))] = a;
            red[warp * 256 + ((j << 4) | (lane << 1) | 1)] = b;
        }
    }
    __syncthreads();
    unsigned long long *H = gv.Hnext + (size_t)slot * kGroupBins;
    for (int b = threadIdx.x; b < 256; b += kMixThreads) {
        double sum = 0.0;
        for (int w = 0; w < kWarps; ++w) sum += (double)red[w * 256 + b];
        if (sum > 0.0) atomicAdd(H + b, __double2ull_rn(sum * kHistScale));
    }
    }
}

__device__ __forceinline__ float warp_sumf(float x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = __fadd_rn(x, __shfl_xor_sync(0xffffffffu, x, off));
    return x;
}

// Stable block-wide selection over [0, cnt): out(rank, i) for every i with
// pred(i), ranks in increasing i; returns how many.  Called by the whole block.
template <class Pred, class Out>
__device__ int block_select(int cnt, Pred pred, Out out) {
    __shared__ int wcnt[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int run = 0;
    for (int i0 = 0; i0 < cnt; i0 += kThreads) {
        const int i = i0 + (int)threadIdx.x;
        const bool flag = i < cnt && pred(i);
        const unsigned bal = __ballot_sync(0xffffffffu, flag);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        int before = run, total = run;
        for (int w = 0; w < kThreads / 32; ++w) {
            if (w < warp) before += wcnt[w];
            total += wcnt[w];
        }
        if (flag) out(before + __popc(bal & ((1u << lane) - 1u)), i);
        __syncthreads();
        run = total;
    }
    return run;
}

// X and Z parts of a gate's Pauli on its (one or two) qubits.
struct GateCode {
    uint32_t xa, za, xb, zb;
    int sites;  // damping sites of the gate
};

__device__ __forceinline__ GateCode gate_code(int kind, int code) {
    GateCode g;
    if (kind == 0) {
        g.xa = xpart_1q(code >> 2);
        g.za = zpart_1q(code >> 2);
        g.xb = xpart_1q(code & 3);
        g.zb = zpart_1q(code & 3);
        g.sites = 2;
    } else {
        g.xa = xpart_1q(code);
        g.za = zpart_1q(code);
        g.xb = g.zb = 0;
        g.sites = 1;
    }
    return g;
}

// Warp sum of the weights w[r] of patterns b = lane + 32 r whose current bit qi
// (b ^ flip) is set, or of all of them for qi < 0: a pairwise tree per lane, then
// the butterfly -- a fixed order, so equal inputs give equal sums everywhere.
template <int R>
__device__ __forceinline__ float site_weight(const float (&w)[R], int lane, uint32_t flip, int qi) {
    float t[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool bit = qi < 0 || ((((uint32_t)(lane + 32 * r) ^ flip) >> qi) & 1u) != 0;
        t[r] = bit ? w[r] : 0.0f;
    }
#pragma unroll
    for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int r = 0; r < h; ++r) t[r] = __fadd_rn(t[r], t[r + h]);
    }
    return warp_sumf(t[0]);
}

// The draws of a group, in four steps.  FP32 throughout (FP64 is slow on this
// part and the joint comes from FP32 amplitudes); the shared path and every
// member's own path run the same operations in the same order (site_weight,
// the closed-form total), so a member that never leaves the shared path draws
// exactly what the shared path drew.  A warp holds the patterns b = lane + 32 r
// (true bits of S, r < kPatR) of the joint: at the start of a phase group,
// after the rotations of a mixer block.
//   1 k_gd_joint    warp per slot: joint by true bits, the shared path's
//                   gamma P(q=1) per site, the slot of each member position
//   2 k_gd_members  thread per member: leaves the shared path? a warp per
//                   such member draws its outcome string (key)
//   3 k_gd_classes  block per slot: classes by first occurrence, the stable
//                   member partition, forks
//   4 k_gd_tables   warp per class: factor table and the state after the group

__device__ __forceinline__ void key_put(GroupKey &k, int e, uint64_t bits) {
    if (e < 10) k.x |= bits << (6 * e);
    else k.y |= bits << (6 * (e - 10));
}
__device__ __forceinline__ int key_gate(const GroupKey &k, int e) {  // the gate's 6 bits
    return (int)((e < 10 ? k.x >> (6 * e) : k.y >> (6 * (e - 10))) & 63u);
}
__device__ __forceinline__ bool key_eq(const GroupKey &a, const GroupKey &b) { return a.x == b.x && a.y == b.y; }
__device__ __forceinline__ bool key_zero(const GroupKey &a) { return (a.x | a.y) == 0; }

// The outcome string of one member from the slot's joint h0: its Pauli codes
// and damping words, staged in shared memory (codes[e], dws[2e + site]).
// Writes the jump bits into the member's branch bytes (lane 0).
template <int kPatR>
__device__ GroupKey member_key(const BatchView &v, const GateGroup *gp, const float (&h0)[kPatR], float tot0,
                               const uint8_t *codes, const uint32_t *dws, size_t gbase, float gf, float omg, int lane) {
    const int m = gp->m, kind = gp->kind, nsite = kind == 0 ? 2 : 1;
    float w[kPatR];
#pragma unroll
    for (int r = 0; r < kPatR; ++r) w[r] = h0[r];
    float tot = tot0;
    uint32_t flip = 0;
    GroupKey key = make_ulonglong2(0ull, 0ull);
    for (int e = 0; e < m; ++e) {
        const int code = codes[e];
        const GateCode gc = gate_code(kind, code);
        flip ^= (gc.xa << gp->ei[e]) ^ (gc.xb << gp->ej[e]);
        int jumps = 0;
        for (int k2 = 0; k2 < nsite; ++k2) {
            const int qi = k2 ? gp->ej[e] : gp->ei[e];
            const float one = site_weight<kPatR>(w, lane, flip, qi);
            const bool j = ((double)dws[2 * e + k2] + 0.5) * kTwoM32 < (double)__fdiv_rn(__fmul_rn(gf, one), tot);
            tot = j ? __fmul_rn(gf, one) : __fsub_rn(tot, __fmul_rn(gf, one));
#pragma unroll
            for (int r = 0; r < kPatR; ++r) {
                const bool bit = ((((uint32_t)(lane + 32 * r) ^ flip) >> qi) & 1u) != 0;
                w[r] = j ? (bit ? __fmul_rn(w[r], gf) : 0.0f) : (bit ? __fmul_rn(w[r], omg) : w[r]);
            }
            if (j) {
                flip ^= 1u << qi;
                jumps |= 1 << k2;
            }
        }
        key_put(key, e, (uint64_t)(code | (jumps << 4)));
        if (lane == 0) v.branch[gbase + e] = (uint8_t)(code | (jumps << 4));
    }
    return key;
}

template <int kPatR>
__global__ void __launch_bounds__(kThreads) k_gd_joint(BatchView v, SlotView sv, GroupView gv, double gamma, int active) {
    grid_dependency_wait();
    const int lane = threadIdx.x & 31;
    const int slot = blockIdx.x * (kThreads / 32) + (int)(threadIdx.x >> 5);  // warp per slot
    if (sv.dyn) active = *sv.active;  // device-driven runs: the grid covers every slot there can be
    if (slot >= active) return;
    const GateGroup *gp = gv.grp;
    const int m = gp->m, ns = gp->s, nbins = 1 << ns, nsite = gp->kind == 0 ? 2 : 1;
    const TrajState st = v.st[slot];
    const uint32_t Fb = st.J ^ st.pend;  // frame once the pending op is applied
    uint32_t fS = 0;
    for (int k = 0; k < ns; ++k) fS |= ((Fb >> gp->sp[k]) & 1u) << k;
    // the joint by true bits b = stored bits ^ fS, pattern b = lane + 32 r
    unsigned long long *Hs = gv.Hcur + (size_t)slot * kGroupBins;
    float w[kPatR];
#pragma unroll
    for (int r = 0; r < kPatR; ++r) {
        const int b = lane + 32 * r;
        w[r] = b < nbins ? (float)((double)Hs[b ^ fS] * kHistUnit) : 0.0f;
    }
    __syncwarp();  // every lane has read before any zeroes
    float *ht = gv.Htrue + (size_t)slot * kGroupBins;
#pragma unroll
    for (int r = 0; r < kPatR; ++r) {
        const int b = lane + 32 * r;
        if (b < nbins) Hs[b] = 0ull;  // zero again for the next group that accumulates here
        ht[b] = w[r];
    }
    // the identity / no-jump path: gamma P(q = 1) at every damping site
    const float gf = (float)gamma, omg = (float)(1.0 - gamma);
    float tot = site_weight<kPatR>(w, lane, 0u, -1);
    float *p1m = gv.p1m + (size_t)slot * 2 * kMaxGroupEdges;
    for (int e = 0; e < m; ++e)
        for (int k2 = 0; k2 < nsite; ++k2) {
            const int qi = k2 ? gp->ej[e] : gp->ei[e];
            const float one = site_weight<kPatR>(w, lane, 0u, qi);
            if (lane == 0) p1m[2 * e + k2] = __fdiv_rn(__fmul_rn(gf, one), tot);
            tot = __fsub_rn(tot, __fmul_rn(gf, one));  // no jump: the weight on bit 1 shrinks by 1 - gamma
#pragma unroll
            for (int r = 0; r < kPatR; ++r) {
                const bool bit = (((uint32_t)(lane + 32 * r) >> qi) & 1u) != 0;
                w[r] = bit ? __fmul_rn(w[r], omg) : w[r];
            }
        }
    if (lane == 0) gv.st_prev[slot] = st;
    const int2 rg = sv.range[slot];
    for (int i = lane; i < rg.y; i += 32) gv.pos_slot[rg.x + i] = slot;
    allow_dependent_launch();
}

// Members per k_gd_members block: a member that leaves the shared path costs its
// warp a serial walk over the group's sites (longer for more patterns per lane),
// so large groups spread their members thinly and give each event a warp of its own.
__host__ __device__ constexpr int gd_members_per_block(int pat_r) { return pat_r >= 32 ? 32 : pat_r >= 4 ? 64 : kThreads; }

template <int kPatR>
__global__ void __launch_bounds__(kThreads) k_gd_members(BatchView v, SlotView sv, GroupView gv, double gamma) {
    grid_dependency_wait();
    constexpr int kPer = gd_members_per_block(kPatR);
    const GateGroup *gp = gv.grp;
    const int m = gp->m, nsite = gp->kind == 0 ? 2 : 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pos = blockIdx.x * kPer + threadIdx.x;
    bool ev = false;
    if ((int)threadIdx.x < kPer && pos < gv.members) {
        // all of the member's codes and words first (independent loads), then the tests
        const int slot = gv.pos_slot[pos];
        const size_t g0 = (size_t)sv.members[pos] * v.G + gp->g0;
        const float *p1m = gv.p1m + (size_t)slot * 2 * kMaxGroupEdges;
        uint32_t codes = 0, dwv[2 * kMaxGroupEdges];
#pragma unroll
        for (int e = 0; e < kMaxGroupEdges; ++e)
            if (e < m) {
                codes |= (uint32_t)(v.branch[g0 + e] & 15);
                dwv[2 * e] = v.dwords[(g0 + e) * 2];
                dwv[2 * e + 1] = nsite == 2 ? v.dwords[(g0 + e) * 2 + 1] : 0xffffffffu;
            }
        ev = codes != 0;
#pragma unroll
        for (int e = 0; e < kMaxGroupEdges; ++e)
            if (e < m) {
                ev = ev || ((double)dwv[2 * e] + 0.5) * kTwoM32 < (double)p1m[2 * e];
                if (nsite == 2) ev = ev || ((double)dwv[2 * e + 1] + 0.5) * kTwoM32 < (double)p1m[2 * e + 1];
            }
        if (!ev) gv.ekey[pos] = make_ulonglong2(0ull, 0ull);
    }
    __shared__ int evl[kThreads];
    const int ne = block_select(kThreads, [&](int) { return ev; }, [&](int r, int i) { evl[r] = i; });
    __shared__ uint8_t s_code[kThreads / 32][kMaxGroupEdges];
    __shared__ uint32_t s_dw[kThreads / 32][2 * kMaxGroupEdges];
    const float gf = (float)gamma, omg = (float)(1.0 - gamma);
    for (int a = warp; a < ne; a += kThreads / 32) {  // their own draws: one warp each
        const int p = blockIdx.x * kPer + evl[a];
        const int slot = gv.pos_slot[p];
        const size_t gbase = (size_t)sv.members[p] * v.G + gp->g0;
        if (lane < m) s_code[warp][lane] = v.branch[gbase + lane] & 15;
        if (lane < 2 * m) s_dw[warp][lane] = v.dwords[gbase * 2 + lane];
        float h0[kPatR];
        const float *ht = gv.Htrue + (size_t)slot * kGroupBins;
#pragma unroll
        for (int r = 0; r < kPatR; ++r) h0[r] = ht[lane + 32 * r];
        const float tot0 = site_weight<kPatR>(h0, lane, 0u, -1);
        __syncwarp();
        const GroupKey key = member_key<kPatR>(v, gp, h0, tot0, s_code[warp], s_dw[warp], gbase, gf, omg, lane);
        if (lane == 0) gv.ekey[p] = key;
        __syncwarp();  // the staged codes are refilled for the warp's next member
    }
    allow_dependent_launch();
}

// Exclusive prefix sums of in[0 .. cnt) plus base into out[0 .. cnt), in place
// allowed; called by the whole block.
__device__ void block_scan_excl(int cnt, const int *in, int *out, int base) {
    __shared__ int wsum[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int run = base;
    for (int i0 = 0; i0 < cnt; i0 += kThreads) {
        const int i = i0 + (int)threadIdx.x;
        const int x = i < cnt ? in[i] : 0;
        int inc = x;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        int before = run, total = run;
        for (int w = 0; w < kThreads / 32; ++w) {
            if (w < warp) before += wsum[w];
            total += wsum[w];
        }
        if (i < cnt) out[i] = before + inc - x;
        __syncthreads();
        run = total;
    }
}

__global__ void __launch_bounds__(kThreads) k_gd_classes(BatchView v, SlotView sv, GroupView gv) {
    grid_dependency_wait();
    // a block per live slot (device-driven runs: blocks stride over the live count)
    const int active = sv.dyn ? *sv.active : (int)gridDim.x;
    for (int slot = blockIdx.x; slot < active; slot += gridDim.x) {
    if (slot != (int)blockIdx.x) __syncthreads();  // the previous slot's shared memory
    __shared__ int child_base;
    const int2 rg = sv.range[slot];
    const int off = rg.x, cnt = rg.y;
    const int32_t *mem = sv.members + off;
    const GroupKey *key = gv.ekey + off;
    int32_t *evt = gv.evt + off, *rep = gv.rep + off, *lead = gv.lead + off;
    int32_t *lcount = gv.lcount + off, *lstart = gv.lstart + off, *run = gv.pos_slot + off;  // run: scratch
    // members that left the shared path, in member order
    const int ne = block_select(cnt, [&](int i) { return !key_zero(key[i]); }, [&](int r, int i) { evt[r] = i; });
    // rep[a] = the first event b <= a with a's outcome string, over keys staged in
    // shared memory a chunk at a time (a thread keeps the same events a throughout)
    constexpr int kKeyChunk = 2 * kThreads;
    __shared__ GroupKey skey[kKeyChunk];
    for (int a = threadIdx.x; a < ne; a += kThreads) rep[a] = -1;
    for (int c0 = 0; c0 < ne; c0 += kKeyChunk) {
        const int cn = min(kKeyChunk, ne - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < cn; i += kThreads) skey[i] = key[evt[c0 + i]];
        __syncthreads();
        for (int a = c0 + (int)threadIdx.x; a < ne; a += kThreads) {
            if (rep[a] >= 0) continue;
            const GroupKey ka = key[evt[a]];
            const int bend = min(a + 1 - c0, cn);  // b <= a
            for (int b = 0; b < bend; ++b)
                if (key_eq(skey[b], ka)) {
                    rep[a] = c0 + b;
                    break;
                }
        }
    }
    __syncthreads();
    // classes: the shared path (if any member kept it), then one per distinct
    // outcome string in order of its first event; the rank of each leader goes to
    // lstart[leader] for the moment, and rep[a] becomes the class rank of event a
    const int nlead = block_select(ne, [&](int a) { return rep[a] == a; }, [&](int r, int a) {
        lead[r] = a;
        lstart[a] = r;
    });
    for (int a = threadIdx.x; a < ne; a += kThreads) rep[a] = lstart[rep[a]];
    const int mainc = cnt - ne;
    const int hasmain = mainc > 0 ? 1 : 0;
    const int nc = hasmain + nlead;
    __syncthreads();
    // members per class (integer counts, in any order), then the classes' starts
    for (int r = threadIdx.x; r < nlead; r += kThreads) {
        lcount[r] = 0;
        run[r] = 0;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < ne; a += kThreads) atomicAdd(&lcount[rep[a]], 1);
    __syncthreads();
    block_scan_excl(nlead, lcount, lstart, mainc);
    if (threadIdx.x == 0) child_base = nc > 1 ? atomicAdd(sv.slot_count, nc - 1) : 0;
    __syncthreads();
    if (nc > 1) {  // stable partition of the members by class into tmp[off ..]
        // the shared path's members, in member order, at the front
        block_select(cnt, [&](int i) { return key_zero(key[i]); }, [&](int r, int i) { sv.tmp[off + r] = mem[i]; });
        // events in order, a chunk of kThreads at a time: an event's place in its class is
        // the class's events in earlier chunks (run) plus those before it in its chunk
        __shared__ int srep[kThreads];
        for (int a0 = 0; a0 < ne; a0 += kThreads) {
            const int a = a0 + (int)threadIdx.x;
            const int r = a < ne ? rep[a] : -1;
            srep[threadIdx.x] = r;
            __syncthreads();
            if (a < ne) {
                int pos = 0;
                for (int b = 0; b < (int)threadIdx.x; ++b) pos += srep[b] == r;
                sv.tmp[off + lstart[r] + run[r] + pos] = mem[evt[a]];
            }
            __syncthreads();
            if (a < ne) atomicAdd(&run[r], 1);
            __syncthreads();
        }
        for (int i = threadIdx.x; i < cnt; i += kThreads) sv.members[off + i] = sv.tmp[off + i];
    }
    for (int c = threadIdx.x; c < nc; c += kThreads) {
        GroupClass gc;
        gc.key = make_ulonglong2(0ull, 0ull);
        gc.slot = slot;
        gc.start = off;
        gc.count = mainc;
        if (c >= hasmain) {
            const int r = c - hasmain;
            gc.key = key[evt[lead[r]]];
            gc.start = off + lstart[r];
            gc.count = lcount[r];
        }
        gc.target = c == 0 ? slot : child_base + c - 1;
        if (gc.target >= sv.max_slots) {
            atomicOr(v.status, 4);
            continue;
        }
        gv.cls[atomicAdd(gv.ncls, 1)] = gc;
    }
    }
    allow_dependent_launch();
}

template <int kPatR>
__device__ __forceinline__ void gd_table(const BatchView &v, const SlotView &sv, const GroupView &gv, double gamma,
                                         int c, int lane) {
    const GroupClass gc = gv.cls[c];
    const GateGroup *gp = gv.grp;
    const int m = gp->m, ns = gp->s, nbins = 1 << ns, kind = gp->kind, nsite = kind == 0 ? 2 : 1;
    const TrajState st = gv.st_prev[gc.slot];
    const uint32_t Fb = st.J ^ st.pend;
    uint32_t fS = 0;
    for (int k = 0; k < ns; ++k) fS |= ((Fb >> gp->sp[k]) & 1u) << k;
    const float sg = (float)sqrt(gamma), sg1 = (float)sqrt(1.0 - gamma);
    const float *ht = gv.Htrue + (size_t)gc.slot * kGroupBins;
    float ar[kPatR], ai[kPatR], w[kPatR];
    uint32_t flip = 0;
#pragma unroll
    for (int r = 0; r < kPatR; ++r) {
        ar[r] = 1.0f;
        ai[r] = 0.0f;
        w[r] = ht[lane + 32 * r];
    }
    const float gcos = gp->c, gsin = gp->sn;
    for (int e = 0; e < m; ++e) {
        const int code = key_gate(gc.key, e) & 15;
        const int qi = gp->ei[e], qj = gp->ej[e];
        const GateCode pc = gate_code(kind, code);
#pragma unroll
        for (int r = 0; r < kPatR; ++r) {  // phase, then the Pauli's Z part, on the bits before its X part
            const uint32_t cb = (uint32_t)(lane + 32 * r) ^ flip;
            const uint32_t ci = (cb >> qi) & 1u, cj = (cb >> qj) & 1u;
            if (kind == 0 && ci != cj) {
                const float nr = ar[r] * gcos + ai[r] * gsin, ni = ai[r] * gcos - ar[r] * gsin;
                ar[r] = nr;
                ai[r] = ni;
            }
            if ((pc.za & ci) ^ (pc.zb & cj)) {
                ar[r] = -ar[r];
                ai[r] = -ai[r];
            }
        }
        flip ^= (pc.xa << qi) ^ (pc.xb << qj);
        for (int k2 = 0; k2 < nsite; ++k2) {
            const int q = k2 ? qj : qi;
            const bool j = ((key_gate(gc.key, e) >> (4 + k2)) & 1) != 0;
#pragma unroll
            for (int r = 0; r < kPatR; ++r) {
                const bool bit = ((((uint32_t)(lane + 32 * r) ^ flip) >> q) & 1u) != 0;
                const float kf = j ? (bit ? sg : 0.0f) : (bit ? sg1 : 1.0f);
                ar[r] *= kf;
                ai[r] *= kf;
                w[r] *= kf * kf;
            }
            if (j) flip ^= 1u << q;
        }
    }
    float N = 0.0f;
#pragma unroll
    for (int r = 0; r < kPatR; ++r) N += w[r];
    N = warp_sumf(N);
    const float sc = 1.0f / sqrtf(N);
    if (lane == 0 && !(N > 0.0f && isfinite(sc))) atomicOr(v.status, 1);
    if (gv.final_norm) {
        // the class's final state T_b phi_b has norm sc^2 sum_b w_b (w_b = J_b |a_b|^2)
        double nd = 0.0;
#pragma unroll
        for (int r = 0; r < kPatR; ++r) nd += (double)w[r];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nd += __shfl_xor_sync(0xffffffffu, nd, off);
        if (lane == 0) v.inv_norm[gc.target] = 1.0 / (nd * (double)sc * (double)sc);
    }
#pragma unroll
    for (int r = 0; r < kPatR; ++r) {
        const int b = lane + 32 * r;
        if (b < nbins) gv.T[(size_t)gc.target * kGroupBins + (b ^ fS)] = make_float2(ar[r] * sc, ai[r] * sc);
    }
    if (lane == 0) {
        uint32_t qflip = 0;
        for (int k = 0; k < ns; ++k) qflip |= ((flip >> k) & 1u) << gp->sp[k];
        TrajState nst;
        nst.J = Fb ^ qflip;
        nst.pend = 0;
        nst.pq0 = nst.pq1 = 0;
        nst.f[0] = nst.f[1] = nst.f[2] = nst.f[3] = 1.0f;
        v.st[gc.target] = nst;
        sv.range[gc.target] = make_int2(gc.start, gc.count);
        if (gc.target != gc.slot) {
            gv.st_prev[gc.target] = st;      // the pending op of the gate before, applied with T
            gv.parent[gc.target] = gc.slot;  // its first sweep reads the parent's state
        }
    }
}

// Warp per class, over a grid sized to what is resident at once (the class
// count is known on the device only).
template <int kPatR>
__global__ void __launch_bounds__(kThreads) k_gd_tables(BatchView v, SlotView sv, GroupView gv, double gamma) {
    grid_dependency_wait();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ncls = *gv.ncls;
    for (int c = blockIdx.x * (kThreads / 32) + warp; c < ncls; c += gridDim.x * (kThreads / 32))
        gd_table<kPatR>(v, sv, gv, gamma, c, lane);
}

// Copy the parent's statevector into every slot forked at this gate.
__global__ void __launch_bounds__(kThreads) k_fork_copy(BatchView v, SlotView sv) {
    grid_dependency_wait();
    const int nforks = *sv.fork_count;
    const int64_t nf = (int64_t)1 << (v.n - 1 > 0 ? v.n - 1 : 0);
    const int64_t chunks = (nf + kTileF4 - 1) / kTileF4;
    const int64_t units = (int64_t)nforks * chunks;
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int2 fk = sv.forks[u / chunks];
        const int64_t f0 = (u % chunks) * kTileF4 + threadIdx.x;
        const float4 *src = reinterpret_cast<const float4 *>(v.psi + ((size_t)fk.x << v.n));
        float4 *dst = reinterpret_cast<float4 *>(v.psi + ((size_t)fk.y << v.n));
        float4 tmp[kF4PerThread];
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k)
            if (f0 + k * kThreads < nf) tmp[k] = src[f0 + k * kThreads];
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k)
            if (f0 + k * kThreads < nf) dst[f0 + k * kThreads] = tmp[k];
    }
    allow_dependent_launch();
}

// After the copies: the new slots join the next sweep.
__global__ void k_fork_finish(SlotView sv) {
    grid_dependency_wait();
    const int sc = *sv.slot_count;
    const int live = sc < sv.max_slots ? sc : sv.max_slots;
    if (sv.prev_active) *sv.prev_active = *sv.active;
    if (sv.live_log) sv.live_log[1 + sv.live_log[0]++] = live;
    *sv.active = live;
    *sv.fork_count = 0;
}

// The sigma pass takes the slots of a shared-prefix run in the order of their first
// members, so that its sums do not depend on how the forks numbered the slots.  A
// device-driven run forms that order on the device.  First each slot marks its first
// member's place among the K trajectories (pos[t] = slot; pos starts at -1) and records
// its member count as its weight; a slot without members, or a member index out of
// range, sets status bit 16.
__global__ void k_order_mark(SlotView sv, int32_t *pos, double *weights, int K, int *status) {
    const int ns = min(*sv.slot_count, sv.max_slots);
    for (int sl = blockIdx.x * blockDim.x + threadIdx.x; sl < ns; sl += gridDim.x * blockDim.x) {
        const int2 r = sv.range[sl];
        const int t = r.y > 0 && r.x >= 0 && r.x < K ? sv.members[r.x] : -1;
        if (t >= 0 && t < K) pos[t] = sl;
        else atomicOr(status, 16);
        weights[sl] = (double)r.y;
    }
}

// ... then one block lists the marked slots in trajectory order: chunks of kThreads
// trajectories, a ballot and a block scan per chunk.
__global__ void __launch_bounds__(kThreads) k_order_compact(const int32_t *pos, int K, int32_t *order) {
    __shared__ int wsum[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int carry = 0;  // slots listed by earlier chunks (the same in every thread)
    for (int c0 = 0; c0 < K; c0 += kThreads) {
        const int t = c0 + (int)threadIdx.x;
        const int sl = t < K ? pos[t] : -1;
        const unsigned m = __ballot_sync(0xffffffffu, sl >= 0);
        if (lane == 0) wsum[warp] = __popc(m);
        __syncthreads();
        int base = carry, total = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            if (w < warp) base += wsum[w];
            total += wsum[w];
        }
        if (sl >= 0) order[base + __popc(m & ((1u << lane) - 1u))] = sl;
        carry += total;
        __syncthreads();  // wsum is rewritten by the next chunk
    }
}

// ---------------------------------------------------------------------------
// Observables of the final state.  The last pending damping op is applied on
// the fly.  k_observe reduces N_t = ||psi_t||^2 per trajectory (FP64 above the
// float4 level) and stores 1/N_t: the final state is normalised exactly before
// phi = |psi|^2 is formed (the paper takes psi normalised).  k_probs owns a
// block of 2048 basis states x (true index), computes C(x) once for them and
// loops over the batch: sigma's FP64 sums get |psi_t,x|^2 / N_t in fixed
// order, and sum_x |psi_t,x|^2 C(x) is reduced per (t, block); its last block
// forms <C>_t and adds S1, S2 in trajectory order.
// ---------------------------------------------------------------------------

// The end of a norm pass over state t, blocks tile = 0 .. ntiles-1 (WARPS warps
// each, every thread holding its double-float sum (sh, sl)): the block
// sum goes to partials, and the last block to finish stores 1/N_t.
template <int WARPS = kThreads / 32>
__device__ void norm_finish(const BatchView &v, int t, int tile, int ntiles, float sh, float sl) {
    __shared__ double redd[WARPS];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double sn = df_warp_sum(sh, sl);
    if (lane == 0) redd[warp] = sn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < WARPS; ++w) sum += redd[w];
        v.partials[((size_t)t * v.tiles + tile) * 4] = sum;
        __threadfence();
        const unsigned prev = atomicAdd(&v.counters[t], 1u);
        last = prev == (unsigned)(ntiles - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s0 = 0.0;
    for (int i = threadIdx.x; i < ntiles; i += WARPS * 32) s0 += __ldcg(v.partials + ((size_t)t * v.tiles + i) * 4);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    __syncthreads();
    if (lane == 0) redd[warp] = s0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double N = 0.0;
        for (int w = 0; w < WARPS; ++w) N += redd[w];
        if (!(N > 0.0) || !isfinite(N)) atomicOr(v.status, 2);
        v.inv_norm[t] = 1.0 / N;
        v.counters[t] = 0;
    }
}

__global__ void __launch_bounds__(kThreads) k_observe(BatchView v) {
    __shared__ int q_item, q_lo, q_n;
    int nxt = 0;  // thread 0: the next item claimed
    int tile, t;
    for (int it = 0; sweep_item_rt(v, 0, it, q_item, q_lo, q_n, nxt, tile, t); ++it) {
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1 > 0 ? n - 1 : 0);
    const TrajState st = v.st[t];
    SweepCtx c;
    c.Fa = v.frame_x[(size_t)t * (v.G + 1) + v.G] ^ st.J;
    c.pq0 = st.pq0;
    c.pq1 = st.pq1;
    for (int k = 0; k < 4; ++k) c.f[k] = st.f[k];
    const float4 *p4 = reinterpret_cast<const float4 *>(v.psi + ((size_t)t << n));
    float sh = 0.0f, sl = 0.0f;
#pragma unroll
    for (int k = 0; k < kF4PerThread; ++k) {
        const int64_t f = (int64_t)tile * kTileF4 + threadIdx.x + k * kThreads;
        if (f < nf) {
            const float4 val = p4[f];
            const uint32_t y = (uint32_t)(2 * f);
            const float f0 = pend_factor(c, y), f1 = pend_factor(c, y | 1u);
            df_add(sh, sl, prob_of(f0, val.x, val.y));
            df_add(sh, sl, prob_of(f1, val.z, val.w));
        }
    }
    norm_finish(v, t, tile, v.tiles, sh, sl);
    }
}

constexpr int kAccChunk = 32;

// The end of a sigma pass, after a block's sigma terms are out: the last block
// to finish forms <C>_t of every state from the per-block partial sums and adds
// S1, S2 in state order.
__device__ void probs_finish(const BatchView &v, const AccumView &a, int64_t xblocks, int nb, int rows) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(a.acc_counter, 1u);
        last = prev == (unsigned)(xblocks * rows - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int tt = threadIdx.x; tt < nb; tt += blockDim.x) {
        double sum = 0.0;
        for (int64_t i = 0; i < xblocks; ++i) sum += __ldcg(a.cpart + (size_t)tt * xblocks + i);
        a.c_out[tt] = sum * v.inv_norm[a.order ? a.order[tt] : tt];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (a.sums) {
            double s1 = a.sums[0], s2 = a.sums[1];
            for (int tt = 0; tt < nb; ++tt) {
                const double cv = a.c_out[tt];
                const double w = a.weights ? a.weights[a.order ? a.order[tt] : tt] : 1.0;
                s1 += w * cv;
                s2 += w * cv * cv;
            }
            a.sums[0] = s1;
            a.sums[1] = s2;
        }
        *a.acc_counter = 0;
    }
}


// Row block blockIdx.y takes states [y b / P, (y + 1) b / P) of the b states, in chunks of
// kAccChunk; row 0 adds its sigma terms to probs, the others store theirs in spart (summed on in
// row order afterwards).
template <bool TRIVIAL>
__global__ void __launch_bounds__(kThreads) k_probs(BatchView v, AccumView a, int64_t xblocks) {
    // the states (device-driven runs: counted on the device) and the row blocks taken
    const int nb = v.dyn_hi ? *v.dyn_hi : v.b;
    const int rows = a.rows.used ? row_parts(a.rows, nb) : (int)gridDim.y;
    if ((int)blockIdx.y >= rows) return;
    const int xb = blockIdx.x;
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1 > 0 ? n - 1 : 0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kX = 2 * kF4PerThread;  // basis states per thread
    __shared__ float cw[kAccChunk][kThreads / 32];
    __shared__ int c_sl[kAccChunk], c_pq0[kAccChunk], c_pq1[kAccChunk];
    __shared__ uint32_t c_Ff[kAccChunk], c_pend[kAccChunk];
    __shared__ float4 c_f[kAccChunk];
    __shared__ float c_ih[kAccChunk], c_il[kAccChunk];
    __shared__ float s_cut[kX][kThreads];
    __shared__ double s_acc[kX][kThreads];
    const int64_t f0 = (int64_t)xb * kTileF4 + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kF4PerThread; ++k)
        for (int e = 0; e < 2; ++e) {
            const uint32_t x = (uint32_t)(2 * (f0 + k * kThreads) + e);
            int cnt = 0;
            for (int j = 0; j < a.num_edges; ++j) {
                const int2 ed = a.edges[j];
                cnt += (int)(((x >> ed.x) ^ (x >> ed.y)) & 1u);
            }
            s_cut[2 * k + e][threadIdx.x] = (float)cnt;
            s_acc[2 * k + e][threadIdx.x] = 0.0;
        }
    auto load_state = [&](int ci, float4 (&val)[kF4PerThread]) {
        const uint32_t Ff = c_Ff[ci];
        const float4 *p4 = reinterpret_cast<const float4 *>(v.psi + ((size_t)c_sl[ci] << n));
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k)
            if (f0 + k * kThreads < nf) val[k] = p4[(f0 + k * kThreads) ^ (int64_t)(Ff >> 1)];
    };
    // sigma terms of state ci into (ah, al); returns this thread's sum of p * C(x)
    auto take_state = [&](int ci, float4 (&val)[kF4PerThread], float (&ah)[kX], float (&al)[kX]) {
        const uint32_t Ff = c_Ff[ci], pend = c_pend[ci];
        const int pq0 = c_pq0[ci], pq1 = c_pq1[ci];
        const float4 fs = c_f[ci];
        const float ih = c_ih[ci], il = c_il[ci];
        float cp = 0.0f;
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k) {
            if (f0 + k * kThreads >= nf) continue;
            float4 vv = val[k];
            if (Ff & 1u) vv = make_float4(vv.z, vv.w, vv.x, vv.y);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const uint32_t x = (uint32_t)(2 * (f0 + k * kThreads) + e);
                float fac = 1.0f;
                if (!TRIVIAL) {
                    const uint32_t tb = x ^ pend;
                    const uint32_t b0 = (tb >> pq0) & 1u, b1 = (tb >> pq1) & 1u;
                    fac = b1 ? (b0 ? fs.w : fs.z) : (b0 ? fs.y : fs.x);
                }
                const float re = e ? vv.z : vv.x, im = e ? vv.w : vv.y;
                const float pr = prob_of(fac, re, im);
                if (a.probs) df_add_prod(ah[2 * k + e], al[2 * k + e], pr, ih, il);
                cp += pr * s_cut[2 * k + e][threadIdx.x];
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) cp += __shfl_xor_sync(0xffffffffu, cp, off);
        if (lane == 0) cw[ci][warp] = cp;
    };
    const int tbeg = (int)((int64_t)blockIdx.y * nb / rows);
    const int tlim = (int)((int64_t)(blockIdx.y + 1) * nb / rows);
    for (int t0c = tbeg; t0c < tlim; t0c += kAccChunk) {
        const int tend = min(tlim, t0c + kAccChunk);
        // the chunk's per-state parameters, once per block
        if ((int)threadIdx.x < tend - t0c) {
            const int tt = t0c + threadIdx.x;
            const int sl = a.order ? a.order[tt] : tt;
            const TrajState st = v.st[sl];
            c_sl[threadIdx.x] = sl;
            c_Ff[threadIdx.x] = v.frame_x[(size_t)sl * (v.G + 1) + v.G] ^ st.J ^ st.pend;
            c_pend[threadIdx.x] = st.pend;
            c_pq0[threadIdx.x] = st.pq0;
            c_pq1[threadIdx.x] = st.pq1;
            c_f[threadIdx.x] = make_float4(st.f[0], st.f[1], st.f[2], st.f[3]);
            const double inv = v.inv_norm[sl] * (a.weights ? a.weights[sl] : 1.0);
            const float ih = (float)inv;
            c_ih[threadIdx.x] = ih;
            c_il[threadIdx.x] = (float)(inv - (double)ih);
        }
        __syncthreads();
        float ah[kX], al[kX];  // sigma terms of this chunk (double-float)
#pragma unroll
        for (int i = 0; i < kX; ++i) ah[i] = al[i] = 0.0f;
        const int cn = tend - t0c;
        for (int ci = 0; ci < cn; ci += 2) {  // two states per step: eight loads in flight
            float4 va[kF4PerThread], vb[kF4PerThread];
            load_state(ci, va);
            if (ci + 1 < cn) load_state(ci + 1, vb);
            take_state(ci, va, ah, al);
            if (ci + 1 < cn) take_state(ci + 1, vb, ah, al);
        }
#pragma unroll
        for (int i = 0; i < kX; ++i) s_acc[i][threadIdx.x] += (double)ah[i] + (double)al[i];
        __syncthreads();
        if ((int)threadIdx.x < cn) {
            double sum = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) sum += (double)cw[threadIdx.x][w];
            a.cpart[(size_t)(t0c + threadIdx.x) * xblocks + xb] = sum;
        }
        __syncthreads();
    }
    if (a.probs) {
        double *dst = blockIdx.y == 0 ? nullptr : a.spart + (size_t)(blockIdx.y - 1) * (2 * (size_t)nf);
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k)
            if (f0 + k * kThreads < nf) {
                const int64_t x = 2 * (f0 + k * kThreads);
                if (dst) {
                    dst[x] = s_acc[2 * k][threadIdx.x];
                    dst[x + 1] = s_acc[2 * k + 1][threadIdx.x];
                } else {
                    a.probs[x] += s_acc[2 * k][threadIdx.x];
                    a.probs[x + 1] += s_acc[2 * k + 1][threadIdx.x];
                }
            }
    }
    probs_finish(v, a, xblocks, nb, rows);
}

// sigma += the other row blocks' terms, in row order.
__global__ void k_probs_combine(double *probs, const double *spart, int parts, int64_t dim, RowPlan rp,
                                const int32_t *nbp) {
    if (rp.used) parts = row_parts(rp, *nbp);
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < dim; x += (int64_t)gridDim.x * blockDim.x) {
        double acc = probs[x];
        for (int p = 0; p + 1 < parts; ++p) acc += spart[(size_t)p * dim + x];
        probs[x] = acc;
    }
}

// The sigma pass when the circuit ends on a full mixer block off qubit 0, which
// no sweep applies: every state is as it was before the block, and the group
// decide formed each final state's norm from the joint the block was drawn
// from.  The pass applies the block to each state on the fly -- the rotations of
// k_mix_sweep, then |f x|^2 with the drawn factor f -- so the final states are
// never written.  A slot forked at the block reads its parent's state.  Grid (half tiles of the block's map, row blocks) x
// kMixThreads: two lanes (lane bit 4 = the block's fourth qubit) share a fiber
// of 16 float4 along the block's qubits, 8 each (the first three qubits on the
// register index), at true bits fixed over the states.  Each float4 is read from
// its true position XOR the state's frame; since a rotation treats a pair's two
// values alike, rotating in true order gives the stored-order values moved.
template <bool TANF>
__global__ void __launch_bounds__(kMixThreads, 4) k_probs_mix(BatchView v, AccumView a, MixMap mm, MixTail tl,
                                                           int64_t xblocks) {
    constexpr int kR = kMixE / 2;  // float4 per thread
    constexpr int kE = 2 * kR;     // basis states per thread
    constexpr int kWarps = kMixThreads / 32;
    static_assert(kMixQ == 4 && kMixL == 3 && kMixThreads == 128, "lanes: 3 L bits, 1 B bit, the fourth qubit");
    // the states (device-driven runs: counted on the device) and the row blocks taken
    const int nb = v.dyn_hi ? *v.dyn_hi : v.b;
    const int rows = a.rows.used ? row_parts(a.rows, nb) : (int)gridDim.y;
    if ((int)blockIdx.y >= rows) return;
    const int first_new = tl.first_new_dev ? *tl.first_new_dev : tl.first_new;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ float cw[kAccChunk][kWarps];
    __shared__ int c_src[kAccChunk];
    __shared__ uint32_t c_Ff[kAccChunk];
    __shared__ float c_w[kAccChunk];
    __shared__ float c_df[kAccChunk][kMixE];
    __shared__ float s_cut[kE][kMixThreads];
    __shared__ double s_acc[kE][kMixThreads];
    const float c = tl.grp->c, sn = tl.grp->sn;
    const float rt = TANF ? sn / c : c / sn, rsc = TANF ? c : sn;
    float scM = 1.0f;  // rsc^4, folded into the factors as k_mix_sweep does
    for (int i = 0; i < kMixQ; ++i) scM *= rsc;
    // this thread's float4: true index base | aoff(j), j along the block's first three qubits;
    // lane bits 0-2 the L bits, lane bit 3 and the warp the B bits 0-2, lane bit 4 the fourth
    // qubit, blockIdx.x B bit 3 then the tile bits
    const int hi = lane >> 4;  // this lane's fourth-qubit bit
    uint32_t base = 0, ao[kMixQ - 1];
#pragma unroll
    for (int i = 0; i < kMixL; ++i) base |= (uint32_t)((lane >> i) & 1) << mm.fL[i];
    base |= (uint32_t)((lane >> 3) & 1) << mm.fB[0];
    base |= (uint32_t)(warp & 1) << mm.fB[1];
    base |= (uint32_t)((warp >> 1) & 1) << mm.fB[2];
    base |= (uint32_t)hi << mm.fA[3];
    base |= (uint32_t)(blockIdx.x & 1u) << mm.fB[3];
#pragma unroll
    for (int i = 0; i < 32; ++i)  // constant indices: the map stays in parameter space
        if (i < mm.ntile) base |= ((blockIdx.x >> (i + 1)) & 1u) << mm.ftile[i];
#pragma unroll
    for (int i = 0; i < kMixQ - 1; ++i) ao[i] = 1u << mm.fA[i];
    const uint32_t ao3 = 1u << mm.fA[3];
    auto aoff = [&](int j) {
        uint32_t o = 0;
#pragma unroll
        for (int i = 0; i < kMixQ - 1; ++i) o |= (j & (1 << i)) ? ao[i] : 0u;
        return o;
    };
#pragma unroll
    for (int j = 0; j < kR; ++j)
        for (int e = 0; e < 2; ++e) {
            const uint32_t x = 2u * (base | aoff(j)) + (uint32_t)e;
            int cnt = 0;
            for (int k = 0; k < a.num_edges; ++k) {
                const int2 ed = a.edges[k];
                cnt += (int)(((x >> ed.x) ^ (x >> ed.y)) & 1u);
            }
            s_cut[2 * j + e][threadIdx.x] = (float)cnt;
            s_acc[2 * j + e][threadIdx.x] = 0.0;
        }
    float cut[kE];  // C(x) of this thread's basis states, constant over the states
#pragma unroll
    for (int i = 0; i < kE; ++i) cut[i] = s_cut[i][threadIdx.x];
    const int tbeg = (int)((int64_t)blockIdx.y * nb / rows);
    const int tlim = (int)((int64_t)(blockIdx.y + 1) * nb / rows);
    for (int t0c = tbeg; t0c < tlim; t0c += kAccChunk) {
        const int cn = min(tlim, t0c + kAccChunk) - t0c;
        // the chunk's per-state parameters, once per block
        if ((int)threadIdx.x < cn) {
            const int tt = t0c + threadIdx.x;
            const int sl = a.order ? a.order[tt] : tt;
            const TrajState st = v.st[sl];
            c_src[threadIdx.x] = sl >= first_new ? tl.parent[sl] : sl;
            c_Ff[threadIdx.x] = v.frame_x[(size_t)sl * (v.G + 1) + v.G] ^ st.J ^ st.pend;
            c_w[threadIdx.x] = (float)(v.inv_norm[sl] * (a.weights ? a.weights[sl] : 1.0));
        }
        for (int i = threadIdx.x; i < cn * kMixE; i += kMixThreads) {
            const int tt = t0c + i / kMixE;
            const int sl = a.order ? a.order[tt] : tt;
            c_df[i / kMixE][i % kMixE] = tl.T[(size_t)sl * kGroupBins + i % kMixE].x * scM;
        }
        __syncthreads();
        // sigma terms of this chunk: FP32 sums of at most kAccChunk weighted probabilities,
        // added to the FP64 sums once per chunk (relative error below 2^-24 kAccChunk)
        float ah[kE];
#pragma unroll
        for (int i = 0; i < kE; ++i) ah[i] = 0.0f;
        // element j's stored index: (base | aoff(j)) ^ Fq = (base ^ Fq) ^ aoff(j); the next
        // state's float4 are loaded while the current one is computed
        auto load_state = [&](int ci, float4 (&dst)[kR]) {
            const uint32_t sb = base ^ (c_Ff[ci] >> 1);
            const float4 *q4 = reinterpret_cast<const float4 *>(v.psi + ((size_t)c_src[ci] << v.n));
#pragma unroll
            for (int j = 0; j < kR; ++j) dst[j] = q4[sb ^ aoff(j)];
        };
        float4 xn[kR];
        if (cn > 0) load_state(0, xn);
        for (int ci = 0; ci < cn; ++ci) {
            const uint32_t Ff = c_Ff[ci], Fq = Ff >> 1;  // Fq: the frame on float4 indices
            // this lane's pattern on the block's qubits is (j | hi << 3); stored: that ^ fa
            int fa = (Fq & ao3) ? 8 : 0;
#pragma unroll
            for (int i = 0; i < kMixQ - 1; ++i) fa |= (Fq & ao[i]) ? 1 << i : 0;
            float4 x[kR];
#pragma unroll
            for (int j = 0; j < kR; ++j) x[j] = xn[j];
            if (ci + 1 < cn) load_state(ci + 1, xn);
#pragma unroll
            for (int i = 0; i < kMixQ - 1; ++i) {
#pragma unroll
                for (int j = 0; j < kR; ++j)
                    if (!(j & (1 << i))) rx_pair4_t<TANF>(x[j], x[j | (1 << i)], rt);
            }
#pragma unroll
            for (int j = 0; j < kR; ++j) rx_lanes_t<TANF>(x[j], 16, rt);  // the fourth qubit
            const float wc = c_w[ci];  // the state's weight / ||psi||^2
            const int fd = fa ^ (hi << 3);
            float cp = 0.0f;
#pragma unroll
            for (int j = 0; j < kR; ++j) {
                const float f = c_df[ci][j ^ fd];  // |f x|^2 with the drawn factor f
                const float pa = prob_of(f, x[j].x, x[j].y), pb = prob_of(f, x[j].z, x[j].w);
                const float p0 = (Ff & 1u) ? pb : pa, p1 = (Ff & 1u) ? pa : pb;  // true qubit 0
                ah[2 * j] = __fmaf_rn(p0, wc, ah[2 * j]);
                ah[2 * j + 1] = __fmaf_rn(p1, wc, ah[2 * j + 1]);
                cp += p0 * cut[2 * j];
                cp += p1 * cut[2 * j + 1];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) cp += __shfl_xor_sync(0xffffffffu, cp, off);
            if (lane == 0) cw[ci][warp] = cp;
        }
#pragma unroll
        for (int i = 0; i < kE; ++i) s_acc[i][threadIdx.x] += (double)ah[i];
        __syncthreads();
        if ((int)threadIdx.x < cn) {
            double sum = 0.0;
            for (int w = 0; w < kWarps; ++w) sum += (double)cw[threadIdx.x][w];
            a.cpart[(size_t)(t0c + threadIdx.x) * xblocks + blockIdx.x] = sum;
        }
        __syncthreads();
    }
    if (a.probs) {
        double *dst = blockIdx.y == 0 ? a.probs : a.spart + (size_t)(blockIdx.y - 1) * ((size_t)1 << v.n);
#pragma unroll
        for (int j = 0; j < kR; ++j) {
            const size_t x = 2 * (size_t)(base | aoff(j));
            if (blockIdx.y == 0) {
                dst[x] += s_acc[2 * j][threadIdx.x];
                dst[x + 1] += s_acc[2 * j + 1][threadIdx.x];
            } else {
                dst[x] = s_acc[2 * j][threadIdx.x];
                dst[x + 1] = s_acc[2 * j + 1][threadIdx.x];
            }
        }
    }
    probs_finish(v, a, xblocks, nb, rows);
}

// ---------------------------------------------------------------------------
// Adjoint gradient (Pauli-only noise: every trajectory is a unitary circuit).
// With U_g = P_g G_g(theta), <C>_t = <psi_T|C|psi_T> and
//   d<C>_t/d theta = sum over gates g with parameter theta of
//                    2 Im <lambda_g'| H_g |chi_g>,
// where chi_g = G_g psi_{g-1} (after the gate, before its Pauli), H_g the
// gate's generator (G = exp(-i theta H)): the differing-bit indicator for the
// ZZ phase gate, X_q for exp(-i beta X_q), and lambda_g' = P_g^dagger U_{g+1}^dagger
// ... U_G^dagger C psi_T.  Both vectors stay in the trajectory's X-frame (the
// frame is a unitary shared by psi and lambda, so inner products and the
// diagonal C are evaluated on true bits).  The reverse sweep for gate g undoes
// the Pauli's Z part on phi and lambda, accumulates the term, then applies
// G_g^dagger to both.  One 2048-amplitude tile per block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_adj_init(BatchView v, float2 *lam, AccumView a) {
    const int t = blockIdx.y;
    const int tile = blockIdx.x;
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1 > 0 ? n - 1 : 0);
    const uint32_t F = v.frame_x[(size_t)t * (v.G + 1) + v.G];
    const float4 *p4 = reinterpret_cast<const float4 *>(v.psi + ((size_t)t << n));
    float4 *l4 = reinterpret_cast<float4 *>(lam + ((size_t)t << n));
#pragma unroll
    for (int k = 0; k < kF4PerThread; ++k) {
        const int64_t f = (int64_t)tile * kTileF4 + threadIdx.x + k * kThreads;
        if (f >= nf) continue;
        const float4 val = p4[f];
        float cw[2];
        for (int e = 0; e < 2; ++e) {
            const uint32_t x = (uint32_t)(2 * f + e) ^ F;
            int cnt = 0;
            for (int j = 0; j < a.num_edges; ++j) {
                const int2 ed = a.edges[j];
                cnt += (int)(((x >> ed.x) ^ (x >> ed.y)) & 1u);
            }
            cw[e] = (float)cnt;
        }
        l4[f] = make_float4(cw[0] * val.x, cw[0] * val.y, cw[1] * val.z, cw[1] * val.w);
    }
}

// The end of an adjoint sweep over trajectory t, in block blk of its nblk blocks
// (kThreads threads, every thread with its FP32 part of the inner product): the
// block's sum goes to partials[t][blk] in FP64, and the trajectory's last block
// to finish adds 2 x their sum / ||psi||^2 to grad[t][param], in block order.
__device__ void adj_finish(const BatchView &v, int t, int blk, int nblk, float acc, double *grad, int param,
                           int nparam) {
    __shared__ double redd[kThreads / 32];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double d = (double)acc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    if (lane == 0) redd[warp] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) sum += redd[w];
        v.partials[((size_t)t * v.tiles + blk) * 4] = sum;
        __threadfence();
        const unsigned prev = atomicAdd(&v.counters[t], 1u);
        last = prev == (unsigned)(nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s0 = 0.0;
    for (int i = threadIdx.x; i < nblk; i += kThreads) s0 += __ldcg(v.partials + ((size_t)t * v.tiles + i) * 4);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    __syncthreads();
    if (lane == 0) redd[warp] = s0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) sum += redd[w];
        grad[(size_t)t * nparam + param] += 2.0 * sum * v.inv_norm[t];
        v.counters[t] = 0;
    }
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_adj_sweep(BatchView v, float2 *lam, int g, DevGate gt, double *grad,
                                                         int param, int nparam) {
    const int t = blockIdx.y;
    const int tile = blockIdx.x;
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1 > 0 ? n - 1 : 0);
    const uint32_t Fb = v.frame_x[(size_t)t * (v.G + 1) + g];
    const int code = v.branch[(size_t)t * v.G + g] & 15;
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)t << n));
    float4 *l4 = reinterpret_cast<float4 *>(lam + ((size_t)t << n));
    float acc = 0.0f;
    if (KIND == kGateZZ) {
        const int q0 = gt.q0, q1 = gt.q1;
        const uint32_t za = (uint32_t)(code >> 3) & 1u, zb = (uint32_t)(code >> 1) & 1u;
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k) {
            const int64_t f = (int64_t)tile * kTileF4 + threadIdx.x + k * kThreads;
            if (f >= nf) continue;
            float4 ph = p4[f], la = l4[f];
            float pv[4] = {ph.x, ph.y, ph.z, ph.w}, lv[4] = {la.x, la.y, la.z, la.w};
            for (int e = 0; e < 2; ++e) {
                const uint32_t tb = (uint32_t)(2 * f + e) ^ Fb;
                const uint32_t b0 = (tb >> q0) & 1u, b1 = (tb >> q1) & 1u;
                const float sgn = ((za & b0) ^ (zb & b1)) ? -1.0f : 1.0f;
                float pr = pv[2 * e] * sgn, pi = pv[2 * e + 1] * sgn;
                float lr = lv[2 * e] * sgn, li = lv[2 * e + 1] * sgn;
                if (b0 ^ b1) {
                    // H = indicator: Im(conj(l) * p)
                    acc += lr * pi - li * pr;
                    // undo e^{-i gamma}: multiply by e^{+i gamma} = c + i s
                    const float npr = pr * gt.c - pi * gt.s, npi = pi * gt.c + pr * gt.s;
                    const float nlr = lr * gt.c - li * gt.s, nli = li * gt.c + lr * gt.s;
                    pr = npr; pi = npi; lr = nlr; li = nli;
                }
                pv[2 * e] = pr; pv[2 * e + 1] = pi; lv[2 * e] = lr; lv[2 * e + 1] = li;
            }
            p4[f] = make_float4(pv[0], pv[1], pv[2], pv[3]);
            l4[f] = make_float4(lv[0], lv[1], lv[2], lv[3]);
        }
    } else {
        const int q = gt.q0;
        const uint32_t z = (uint32_t)(code >> 1) & 1u;
        const uint32_t fbq = (Fb >> q) & 1u;
        // element with stored bit 0 has true bit fbq
        const float s0 = (z && fbq) ? -1.0f : 1.0f, s1 = (z && !fbq) ? -1.0f : 1.0f;
        const float cb = gt.c, sb = gt.s;
        auto pair = [&](float &a0r, float &a0i, float &a1r, float &a1i, float &m0r, float &m0i, float &m1r,
                        float &m1i) {
            a0r *= s0; a0i *= s0; a1r *= s1; a1i *= s1;
            m0r *= s0; m0i *= s0; m1r *= s1; m1i *= s1;
            // H = X: Im(conj(l0) p1 + conj(l1) p0)
            acc += (m0r * a1i - m0i * a1r) + (m1r * a0i - m1i * a0r);
            // exp(-i beta X)^dagger = [[c, i s], [i s, c]]
            float n0r = cb * a0r - sb * a1i, n0i = cb * a0i + sb * a1r;
            float n1r = cb * a1r - sb * a0i, n1i = cb * a1i + sb * a0r;
            a0r = n0r; a0i = n0i; a1r = n1r; a1i = n1i;
            n0r = cb * m0r - sb * m1i; n0i = cb * m0i + sb * m1r;
            n1r = cb * m1r - sb * m0i; n1i = cb * m1i + sb * m0r;
            m0r = n0r; m0i = n0i; m1r = n1r; m1i = n1i;
        };
        if (q == 0) {
#pragma unroll
            for (int k = 0; k < kF4PerThread; ++k) {
                const int64_t f = (int64_t)tile * kTileF4 + threadIdx.x + k * kThreads;
                if (f >= nf) continue;
                float4 ph = p4[f], la = l4[f];
                pair(ph.x, ph.y, ph.z, ph.w, la.x, la.y, la.z, la.w);
                p4[f] = ph;
                l4[f] = la;
            }
        } else {
            const int sh = q - 1;
            const int64_t npairs = nf >> 1, hib = (int64_t)1 << sh;
#pragma unroll
            for (int k = 0; k < kF4PerThread / 2; ++k) {
                const int64_t r = (int64_t)tile * (kTileF4 / 2) + threadIdx.x + k * kThreads;
                if (r >= npairs) continue;
                const int64_t fl = ((r >> sh) << (sh + 1)) | (r & (hib - 1));
                float4 plo = p4[fl], phi = p4[fl | hib], llo = l4[fl], lhi = l4[fl | hib];
                pair(plo.x, plo.y, phi.x, phi.y, llo.x, llo.y, lhi.x, lhi.y);
                pair(plo.z, plo.w, phi.z, phi.w, llo.z, llo.w, lhi.z, lhi.w);
                p4[fl] = plo; p4[fl | hib] = phi; l4[fl] = llo; l4[fl | hib] = lhi;
            }
        }
    }
    adj_finish(v, t, tile, v.tiles, acc, grad, param, nparam);
}

// ---------------------------------------------------------------------------
// Fused layers (Pauli-only noise).  Without damping no branch depends on the
// state, so a whole QAOA layer can be applied in few sweeps:
//  * the cost layer -- every edge's phase gate and every Pauli's Z part -- is
//    diagonal in the stored basis: phi_y *= (-1)^{popc(y & zm) + zc} *
//    e^{-i gamma k(y)}, k(y) = popc(EV(y) xor s), where EV(y) has bit e set when
//    the stored bits of edge e's endpoints differ (XOR of four byte tables) and
//    s_e flips edge e when the frame differs on its endpoints at that gate;
//  * the mixer layer is a tensor product of one 2x2 matrix per qubit (the
//    rotation with the row signs of its Pauli's Z part), applied in fibres over
//    windows of consecutive qubits: up to kFuse0 with qubit 0, kFuse without
//    (four qubits in registers, the others on lane bits).
// A sweep applies [phase of layer l] (first sweep) and the rotations of one
// qubit group; the last group of a layer also applies the next layer's phase.
// ---------------------------------------------------------------------------
__global__ void k_layer_params(BatchView v, LayerView L, int g0, int E) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= v.b) return;
    uint64_t sv = 0;
    uint32_t zm = 0, zc = 0, mz = 0, mf = 0;
    for (int e = 0; e < E; ++e) {
        const int g = g0 + e;
        const uint32_t F = v.frame_x[(size_t)t * (v.G + 1) + g];
        const int2 ed = L.edges[e];
        sv |= (uint64_t)(((F >> ed.x) ^ (F >> ed.y)) & 1u) << e;
        const int code = v.branch[(size_t)t * v.G + g] & 15;
        const uint32_t za = zpart_1q(code >> 2), zb = zpart_1q(code & 3);
        zm ^= (za << ed.x) ^ (zb << ed.y);
        zc ^= (za & (F >> ed.x)) ^ (zb & (F >> ed.y));
    }
    for (int q = 0; q < v.n; ++q) {
        const int g = g0 + E + q;
        const uint32_t F = v.frame_x[(size_t)t * (v.G + 1) + g];
        mz |= zpart_1q(v.branch[(size_t)t * v.G + g] & 15) << q;
        mf |= ((F >> q) & 1u) << q;
    }
    L.s[t] = sv;
    L.zm[t] = zm;
    L.zc[t] = zc & 1u;
    L.mz[t] = mz;
    L.mf[t] = mf;
}


__device__ __forceinline__ void cmul_inplace(float &re, float &im, float2 w) {
    const float r = re * w.x - im * w.y, i = re * w.y + im * w.x;
    re = r;
    im = i;
}

__device__ __forceinline__ uint64_t ev_of(const LayerView &L, uint32_t y) {
    return __ldg(L.ev + (y & 255u)) ^ __ldg(L.ev + 256 + ((y >> 8) & 255u)) ^ __ldg(L.ev + 512 + ((y >> 16) & 255u)) ^
           __ldg(L.ev + 768 + (y >> 24));
}

// The cost layer's phase table in shared memory with the Z sign folded in:
// ph2[2k + s] = (-1)^s e^{-i gamma k} (CONJ: its conjugate), k = 0 .. E, so that an
// amplitude's factor is one shared load at (popc(EV(y) ^ s) << 1) | (Z parity of y).
constexpr int kPh2 = 2 * 65;
template <bool CONJ = false>
__device__ __forceinline__ void load_phase2(const LayerView &L, float2 *ph2, int nthreads) {
    for (int i = threadIdx.x; i < 2 * (L.num_edges + 1); i += nthreads) {
        const float2 f = __ldg(L.phase + (i >> 1));
        const float sg = (i & 1) ? -1.0f : 1.0f;
        ph2[i] = make_float2(f.x * sg, CONJ ? -f.y * sg : f.y * sg);
    }
}
// e: EV of the thread's part of y xor the frame's edge flips; evk: EV of the element's part;
// par: the Z parity of y (bit 0)
__device__ __forceinline__ float2 phase2(const float2 *ph2, uint64_t e, uint64_t evk, uint32_t par) {
    return ph2[(__popcll(e ^ evk) << 1) | (par & 1u)];
}

// One fused sweep over a window of M = HAS0 + LQ + RQ qubits.  A fibre is the
// 2^(M - HAS0) float4 of one value of the float4-index bits outside the window:
//  * with HAS0 (q_lo == 0) qubit 0 is the float4 half, qubits 1 .. LQ are lane
//    bits 0 .. LQ-1 (float4-index bits 0 .. LQ-1) and the next RQ qubits the
//    register index; the upper lane bits index fibres, so runs of 2^LQ
//    consecutive float4 fill a warp's accesses;
//  * otherwise qubits q_lo .. q_lo+LQ-1 are lane bits 5-LQ .. 4 and the next RQ
//    the register index; lane bits 0 .. 4-LQ are the float4-index bits 0 .. 4-LQ
//    below the window.
// The rotation of a lane qubit takes the partner half from lane ^ (1 << b) by
// shuffle.  PRE: phase of layer `lp` before the rotations; POST: phase of layer
// `lq` after them.  The phase of register element k, half e, is that of
// y0 | 2 (k << rs) | e (rs the float4-index bit of register bit 0), split into
// the thread's y0 and the block-wide tables of the patterns 2 (k << rs) and e.
// A block takes kFuseChunks consecutive chunks of kThreads fibre-threads; each
// thread copies its next chunk's float4 into its own shared slots (cp.async)
// while it rotates the current one, so the loads stay in flight through the
// arithmetic.  NORM (the circuit's last sweep): the block also sums |psi|^2 of
// what it stores, and the last block of the state stores 1/N_t, as the norm
// pass does.
template <int LQ, int RQ, bool HAS0, bool PRE, bool POST, bool NORM>
__global__ void __launch_bounds__(kThreads, 2) k_fused_sweep(BatchView v, LayerView Lp, LayerView Lr, LayerView Lq,
                                                             int q_lo) {
    constexpr int NE = 1 << RQ;
    constexpr int DB = LQ + RQ;  // window bits in the float4 index
    constexpr int LO = 5 - LQ;   // lane bits that index fibres
    static_assert(NE <= 16 && LQ <= 3, "at most 16 float4 per thread and 3 lane qubits");
    extern __shared__ float4 fslot[];  // [NE][kThreads]: each thread's landing slots
    const int t = blockIdx.y;
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1);
    const int wlo = HAS0 ? 0 : q_lo - 1;  // lowest float4-index bit of the window
    const int rs = wlo + LQ;
    const int64_t nfib = nf >> DB;
    __shared__ uint64_t evk[NE + 1];  // EV of each register element's offset; [NE]: EV of bit 0
    __shared__ float2 ph2p[PRE ? kPh2 : 1], ph2q[POST ? kPh2 : 1];  // the layers' phase tables
    uint32_t pkp = 0, pkq = 0;  // bit k: the Z parity of register element k's offset (layers Lp, Lq)
    if (PRE || POST) {
        const LayerView &L = PRE ? Lp : Lq;  // the edge tables are the graph's, the same in every layer
        if ((int)threadIdx.x < NE) evk[threadIdx.x] = ev_of(L, 2u * ((uint32_t)threadIdx.x << rs));
        if ((int)threadIdx.x == NE) evk[NE] = ev_of(L, 1u);
        if (PRE) load_phase2(Lp, ph2p, kThreads);
        if (POST) load_phase2(Lq, ph2q, kThreads);
        const uint32_t zmp = PRE ? Lp.zm[blockIdx.y] : 0u, zmq = POST ? Lq.zm[blockIdx.y] : 0u;
#pragma unroll
        for (int k = 0; k < NE; ++k) {
            const uint32_t yk = 2u * ((uint32_t)k << rs);
            pkp |= ((uint32_t)__popc(yk & zmp) & 1u) << k;
            pkq |= ((uint32_t)__popc(yk & zmq) & 1u) << k;
        }
        __syncthreads();
    }
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)t << n));
    const uint32_t lane = threadIdx.x & 31u;
    // wb: the window's lane bits; the fibre r of chunk c.  With LQ > 0 a warp's
    // fibres are 2^LO consecutive ones, so a warp is in or out as a whole.
    const uint32_t wb = LQ == 0 ? 0u : HAS0 ? lane & ((1u << LQ) - 1u) : lane >> LO;
    auto fibre_of = [&](int64_t c, int64_t &fbase) -> bool {
        const int64_t tg = c * kThreads + threadIdx.x;
        const int64_t r = LQ == 0 ? tg
                          : HAS0  ? (int64_t)(lane >> LQ) | ((tg >> 5) << LO)
                                  : (int64_t)(lane & ((1u << LO) - 1u)) | ((tg >> 5) << LO);
        fbase = ((r >> wlo) << (wlo + DB)) | (r & (((int64_t)1 << wlo) - 1)) | ((int64_t)wb << wlo);
        return r < nfib;
    };
    const uint32_t mz = Lr.mz[t], mf = Lr.mf[t];
    const float cb = Lr.cb, sb = Lr.sb;
    // the 2x2 rotation of qubit q with the row signs of its Pauli's Z part:
    // row 0 (stored bit 0) c0, sn0; row 1 c1, sn1
    auto coeffs = [&](int q, float &c0, float &sn0, float &c1, float &sn1) {
        const uint32_t z = (mz >> q) & 1u, fb = (mf >> q) & 1u;
        const float s0 = (z && fb) ? -1.0f : 1.0f, s1 = (z && !fb) ? -1.0f : 1.0f;
        c0 = cb * s0;
        sn0 = sb * s0;
        c1 = cb * s1;
        sn1 = sb * s1;
    };
    const int ql = q_lo + (HAS0 ? 1 : 0);  // first lane qubit
    const int64_t c_begin = (int64_t)blockIdx.x * kFuseChunks;
    int64_t fnext;
    bool ok_next = fibre_of(c_begin, fnext);
    if (ok_next) {
#pragma unroll
        for (int k = 0; k < NE; ++k) cp_async16(&fslot[k * kThreads + threadIdx.x], p4 + fnext + ((int64_t)k << rs));
    }
    cp_async_commit();
    float sh = 0.0f, sl = 0.0f;  // NORM: this thread's sum of |psi|^2 (double-float)
    for (int j = 0; j < kFuseChunks; ++j) {
        const int64_t fbase = fnext;
        const bool ok = ok_next;
        float4 val[NE];
        cp_async_wait<0>();
        if (ok) {
#pragma unroll
            for (int k = 0; k < NE; ++k) val[k] = fslot[k * kThreads + threadIdx.x];
        }
        __syncwarp();  // the slots' reads are performed before the next chunk's copies land in them
        ok_next = j + 1 < kFuseChunks && fibre_of(c_begin + j + 1, fnext);
        if (ok_next) {
#pragma unroll
            for (int k = 0; k < NE; ++k) cp_async16(&fslot[k * kThreads + threadIdx.x], p4 + fnext + ((int64_t)k << rs));
        }
        cp_async_commit();
        if (!ok) continue;
        const uint32_t y0 = (uint32_t)(2 * fbase);
        if (PRE) {
            const uint32_t zm = Lp.zm[t];
            const uint64_t e0 = ev_of(Lp, y0) ^ Lp.s[t], e1 = e0 ^ evk[NE];
            const uint32_t zp0 = (uint32_t)__popc(y0 & zm) ^ Lp.zc[t], zp1 = zp0 ^ (zm & 1u);
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                cmul_inplace(val[k].x, val[k].y, phase2(ph2p, e0, evk[k], zp0 ^ (pkp >> k)));
                cmul_inplace(val[k].z, val[k].w, phase2(ph2p, e1, evk[k], zp1 ^ (pkp >> k)));
            }
        }
        if (HAS0) {
            float c0, sn0, c1, sn1;
            coeffs(0, c0, sn0, c1, sn1);
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                const float r0 = val[k].x, i0 = val[k].y, r1 = val[k].z, i1 = val[k].w;
                val[k].x = c0 * r0 + sn0 * i1;
                val[k].y = c0 * i0 - sn0 * r1;
                val[k].z = c1 * r1 + sn1 * i0;
                val[k].w = c1 * i1 - sn1 * r0;
            }
        }
#pragma unroll
        for (int jq = 0; jq < LQ; ++jq) {
            // own' = c own - i s partner with the row of the lane's own bit
            const int b = HAS0 ? jq : LO + jq;
            const uint32_t hb = (lane >> b) & 1u;
            float c0, sn0, c1, sn1;
            coeffs(ql + jq, c0, sn0, c1, sn1);
            const float co = hb ? c1 : c0, so = hb ? sn1 : sn0;
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                const float px = __shfl_xor_sync(0xffffffffu, val[k].x, 1 << b);
                const float py = __shfl_xor_sync(0xffffffffu, val[k].y, 1 << b);
                const float pz = __shfl_xor_sync(0xffffffffu, val[k].z, 1 << b);
                const float pw = __shfl_xor_sync(0xffffffffu, val[k].w, 1 << b);
                val[k] = make_float4(co * val[k].x + so * py, co * val[k].y - so * px, co * val[k].z + so * pw,
                                     co * val[k].w - so * pz);
            }
        }
#pragma unroll
        for (int jq = 0; jq < RQ; ++jq) {
            float c0, sn0, c1, sn1;
            coeffs(ql + LQ + jq, c0, sn0, c1, sn1);
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                if (k & (1 << jq)) continue;
                float4 &a = val[k];
                float4 &b = val[k | (1 << jq)];
                const float nx = c0 * a.x + sn0 * b.y, ny = c0 * a.y - sn0 * b.x;
                const float mx = c1 * b.x + sn1 * a.y, my = c1 * b.y - sn1 * a.x;
                const float nz = c0 * a.z + sn0 * b.w, nw = c0 * a.w - sn0 * b.z;
                const float mzv = c1 * b.z + sn1 * a.w, mw = c1 * b.w - sn1 * a.z;
                a = make_float4(nx, ny, nz, nw);
                b = make_float4(mx, my, mzv, mw);
            }
        }
        if (POST) {
            const uint32_t zm = Lq.zm[t];
            const uint64_t e0 = ev_of(Lq, y0) ^ Lq.s[t], e1 = e0 ^ evk[NE];
            const uint32_t zp0 = (uint32_t)__popc(y0 & zm) ^ Lq.zc[t], zp1 = zp0 ^ (zm & 1u);
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                cmul_inplace(val[k].x, val[k].y, phase2(ph2q, e0, evk[k], zp0 ^ (pkq >> k)));
                cmul_inplace(val[k].z, val[k].w, phase2(ph2q, e1, evk[k], zp1 ^ (pkq >> k)));
            }
        }
#pragma unroll
        for (int k = 0; k < NE; ++k) p4[fbase + ((int64_t)k << rs)] = val[k];
        if (NORM) {
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                df_add(sh, sl, prob_of(1.0f, val[k].x, val[k].y));
                df_add(sh, sl, prob_of(1.0f, val[k].z, val[k].w));
            }
        }
    }
    if (NORM) norm_finish(v, t, blockIdx.x, gridDim.x, sh, sl);
}

// The first window of a fused layer for n >= 13: the mixer rotations of qubits 0-11 (and,
// with PRE, layer Lp's phase before them), one 2048-float4 tile of consecutive float4 at a
// time -- qubit 0 the float4 half, qubits 1-11 the tile's float4-index bits 0-10.  Tiles
// stream through two shared buffers (cp.async, one tile ahead, 512 contiguous bytes per
// warp copy); each tile takes three register phases over the buffer, 16 float4 per thread:
//   A  register index j = bits 0-3 (the phase, qubits 0 and 1-4),
//   B  j = bits 4-7 (qubits 5-8),
//   C  j bit 0 = bit 7, bits 1-3 = bits 8-10 (qubits 9-11), stored to HBM from there.
// The rotations take the tangent form (rx_pair_t) with the common factor rsc^12 and the
// row signs of the drawn Paulis' Z parts applied once, after the window: qubit q's row r
// carries -1 when z_q and r != x_q (the frame's X bit), so an amplitude y of the window
// carries (-1)^popc(z & (x ^ y)).  Slot of float4 f in a buffer: f ^ ((f >> 4) & 7), so
// that each quarter warp of every phase hits eight distinct 16-byte bank groups.
// Grid (blocks of up to kT12Subs tiles, trajectories) x 128 threads.
constexpr int kT12Subs = 4;
constexpr size_t kT12Smem = 2 * 2048 * sizeof(float4);

template <bool TANF, bool PRE>
__global__ void __launch_bounds__(128, 3) k_fused_tile12(BatchView v, LayerView Lp, LayerView Lr) {
    extern __shared__ float4 t12_buf[];  // [2][2048]
    __shared__ uint64_t evk[17];         // PRE: EV of the phase-A register offsets 2j; [16]: EV of bit 0
    __shared__ float2 ph2[PRE ? kPh2 : 1];  // PRE: layer Lp's phase table
    const int t = blockIdx.y;
    const uint32_t tid = threadIdx.x;
    const float4 *q4 = reinterpret_cast<const float4 *>(v.psi + ((size_t)t << v.n));
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)t << v.n));
    const int ntiles = 1 << (v.n - 12);
    const int nsubs = ntiles < kT12Subs ? ntiles : kT12Subs;
    const uint32_t tile0 = (uint32_t)blockIdx.x * (uint32_t)nsubs;
    uint32_t pk = 0;  // PRE: bit j, the Z parity of the phase-A register offset 2j
    if (PRE) {
        if (tid < 16u) evk[tid] = ev_of(Lp, 2u * tid);
        if (tid == 16u) evk[16] = ev_of(Lp, 1u);
        load_phase2(Lp, ph2, 128);
        const uint32_t zm = Lp.zm[t];
#pragma unroll
        for (int j = 0; j < 16; ++j) pk |= ((uint32_t)__popc((2u * (uint32_t)j) & zm) & 1u) << j;
    }
    const float cb = Lr.cb, sb = Lr.sb;
    const float rt = TANF ? sb / cb : cb / sb, rsc = TANF ? cb : sb;
    float sc12 = 1.0f;
#pragma unroll
    for (int i = 0; i < 12; ++i) sc12 *= rsc;
    const uint32_t zw = Lr.mz[t] & 0xfffu;
    const uint32_t sgn0 = (uint32_t)__popc(zw & Lr.mf[t]);  // the parity's constant part
    auto sw = [](uint32_t f) { return f ^ ((f >> 4) & 7u); };
    auto fetch = [&](int sub) {
        float4 *buf = t12_buf + (sub & 1) * 2048;
        const float4 *src = q4 + ((size_t)(tile0 + (uint32_t)sub) << 11);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t f = tid | ((uint32_t)k << 7);
            cp_async16(buf + sw(f), src + f);
        }
        cp_async_commit();
    };
    fetch(0);
    for (int sub = 0; sub < nsubs; ++sub) {
        if (sub + 1 < nsubs) {
            fetch(sub + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();  // every thread's copies of this tile (and evk)
        float4 *buf = t12_buf + (sub & 1) * 2048;
        const uint32_t tb = (tile0 + (uint32_t)sub) << 11;  // the tile's first float4 (n <= 30)
        float4 x[16];
        // phase A: f = j | tid << 4
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = buf[sw((uint32_t)j | (tid << 4))];
        if (PRE) {
            const uint32_t zm = Lp.zm[t];
            const uint32_t y0 = 2u * (tb | (tid << 4));
            const uint64_t e0 = ev_of(Lp, y0) ^ Lp.s[t], e1 = e0 ^ evk[16];
            const uint32_t zp0 = (uint32_t)__popc(y0 & zm) ^ Lp.zc[t], zp1 = zp0 ^ (zm & 1u);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                cmul_inplace(x[j].x, x[j].y, phase2(ph2, e0, evk[j], zp0 ^ (pk >> j)));
                cmul_inplace(x[j].z, x[j].w, phase2(ph2, e1, evk[j], zp1 ^ (pk >> j)));
            }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) rx_pair_t<TANF>(x[j].x, x[j].y, x[j].z, x[j].w, rt);  // qubit 0
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (!(j & (1 << i))) rx_pair4_t<TANF>(x[j], x[j | (1 << i)], rt);
#pragma unroll
        for (int j = 0; j < 16; ++j) buf[sw((uint32_t)j | (tid << 4))] = x[j];
        __syncthreads();
        // phase B: f = (tid & 15) | j << 4 | (tid >> 4) << 8
        const uint32_t fB = (tid & 15u) | ((tid >> 4) << 8);
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = buf[sw(fB | ((uint32_t)j << 4))];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (!(j & (1 << i))) rx_pair4_t<TANF>(x[j], x[j | (1 << i)], rt);
#pragma unroll
        for (int j = 0; j < 16; ++j) buf[sw(fB | ((uint32_t)j << 4))] = x[j];
        __syncthreads();
        // phase C: f = tid | (j & 1) << 7 | (j >> 1) << 8
        auto fC = [&](int j) { return tid | ((uint32_t)(j & 1) << 7) | ((uint32_t)(j >> 1) << 8); };
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = buf[sw(fC(j))];
#pragma unroll
        for (int i = 1; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (!(j & (1 << i))) rx_pair4_t<TANF>(x[j], x[j | (1 << i)], rt);
        const uint32_t pt = sgn0 ^ (uint32_t)__popc(zw & (2u * tid));  // parity of the thread's part
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint32_t par = pt ^ (uint32_t)__popc(zw & (2u * (fC(j) & ~tid)));
            const float s0 = (par & 1u) ? -sc12 : sc12, s1 = ((par ^ zw) & 1u) ? -sc12 : sc12;
            p4[tb + fC(j)] = make_float4(x[j].x * s0, x[j].y * s0, x[j].z * s1, x[j].w * s1);
        }
        __syncthreads();  // the buffer's reads are done before the next copy into it
    }
}

// A fused window off qubit 0: the mixer rotations of M = 4..7 qubits q_lo .. q_lo+M-1,
// float4-index bits w .. w+M-1 (w = q_lo - 1 >= 11 - M), with the next layer's phase
// after them (MODE kWinPost) or the final norms (kWinNorm, the circuit's last sweep).
// A tile is 2^(11-M) consecutive float4 (the run, bits 0 .. 10-M of the float4 index,
// all below the window) times the 2^M values of the window's bits: tile index
// i = run | window << (11 - M).  Tiles stream through two shared buffers (cp.async, one
// tile ahead, copied in index order, so a warp copies runs of at least 256 contiguous
// bytes however far apart the window's bits place them); then 16 float4 per thread:
//   phase 1  register index j = window bits 0-3, the thread = the run and window bits 4..
//   phase 2  (M > 4) j = run bits 3 .. 10-M and window bits 4 .., the thread = run bits
//            0-2 and window bits 0-3,
// the row signs of the drawn Paulis (folded into the phase's sign with kWinPost) and the
// phase or the norm terms on the last phase's registers, back to the buffer, and stored
// in index order.  Buffer slot of i: i itself (in every access the eight threads of a
// quarter warp differ exactly in tile-index bits 0-2, eight distinct 16-byte bank groups).
// Grid (blocks of up to kT12Subs tiles, trajectories) x 128 threads.
enum { kWinPlain = 0, kWinPost = 1, kWinNorm = 2 };

template <int M, int MODE>
__global__ void __launch_bounds__(128, 3) k_fused_win(BatchView v, LayerView Lr, LayerView Lq, int q_lo) {
    constexpr int RL = 11 - M;  // run bits
    constexpr int LJ = 8 - M;   // phase 2: run bits in the register index (bits 3 .. RL-1)
    static_assert(M >= 4 && M <= 7, "windows of 4 to 7 qubits");
    extern __shared__ float4 win_buf[];  // [2][2048]
    __shared__ uint64_t evk[17];         // kWinPost: EV of the last phase's register offsets; [16]: EV of bit 0
    __shared__ float2 ph2[MODE == kWinPost ? kPh2 : 1];  // kWinPost: layer Lq's phase table
    const int t = blockIdx.y;
    const uint32_t tid = threadIdx.x;
    const int w = q_lo - 1;
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)t << v.n));
    const int ntiles = 1 << (v.n - 12);
    const int nsubs = ntiles < kT12Subs ? ntiles : kT12Subs;
    const uint32_t tile0 = (uint32_t)blockIdx.x * (uint32_t)nsubs;
    // float4 offset of tile index i, and the first float4 of tile u (its n-12 bits: the
    // bits between the run and the window, then those above the window)
    auto off = [&](uint32_t i) { return (i & ((1u << RL) - 1u)) | ((i >> RL) << w); };
    auto tile_base = [&](uint32_t u) {
        const uint32_t mid = (uint32_t)(w - RL);
        return ((u & ((1u << mid) - 1u)) << RL) | ((u >> mid) << (w + M));
    };
    // the last phase's tile index: the thread's part and register j's part
    const uint32_t it_last = M == 4 ? (tid & ((1u << RL) - 1u)) | ((tid >> RL) << (RL + 4)) : (tid & 7u) | ((tid >> 3) << RL);
    auto ij_last = [](int j) -> uint32_t {
        if (M == 4) return (uint32_t)j << RL;
        return ((uint32_t)(j & ((1 << LJ) - 1)) << 3) | ((uint32_t)(j >> LJ) << (RL + 4));
    };
    // Rotations without the row signs; those are a diagonal after the window's rotations:
    // -1 on qubit q's row r when z_q and r != x_q, so a tile index i carries
    // (-1)^popc(zw & (xw ^ (i >> RL))) (zw, xw: the window's Z and frame bits).
    const uint32_t zw = (Lr.mz[t] >> q_lo) & ((1u << M) - 1u), xw = (Lr.mf[t] >> q_lo) & ((1u << M) - 1u);
    const float cb = Lr.cb, sb = Lr.sb;
    uint32_t pj = 0;  // bit j: the parity of register j's part (and, with kWinPost, of its phase sign)
    const uint32_t zmq = MODE == kWinPost ? Lq.zm[t] : 0u;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const uint32_t ij = ij_last(j);
        uint32_t par = (uint32_t)__popc(zw & (ij >> RL));
        if (MODE == kWinPost) par ^= (uint32_t)__popc(2u * off(ij) & zmq);
        pj |= (par & 1u) << j;
    }
    const uint32_t pt = (uint32_t)__popc(zw & xw) ^ (uint32_t)__popc(zw & (it_last >> RL));  // the thread's part
    if (MODE == kWinPost) {
        if (tid < 16u) evk[tid] = ev_of(Lq, 2u * off(ij_last((int)tid)));
        if (tid == 16u) evk[16] = ev_of(Lq, 1u);
        load_phase2(Lq, ph2, 128);
    }
    auto rot = [&](float4 *x, int bit) {  // exp(-i beta X) on register bit `bit`
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j & (1 << bit)) continue;
            float4 &a = x[j];
            float4 &b = x[j | (1 << bit)];
            const float nx = cb * a.x + sb * b.y, ny = cb * a.y - sb * b.x;
            const float mx = cb * b.x + sb * a.y, my = cb * b.y - sb * a.x;
            const float nz = cb * a.z + sb * b.w, nw = cb * a.w - sb * b.z;
            const float mzv = cb * b.z + sb * a.w, mw = cb * b.w - sb * a.z;
            a = make_float4(nx, ny, nz, nw);
            b = make_float4(mx, my, mzv, mw);
        }
    };
    // index order: thread tid takes i = tid | k << 7, k = 0..15; tile-index bit 7 is a
    // window bit (RL <= 7), float4 offset 2^kst
    const uint32_t off_t = off(tid);
    const int kst = w + 7 - RL;
    auto fetch = [&](int sub) {
        float4 *buf = win_buf + (sub & 1) * 2048 + tid;
        const float4 *src = p4 + tile_base(tile0 + (uint32_t)sub) + off_t;
#pragma unroll
        for (int k = 0; k < 16; ++k) cp_async16(buf + (k << 7), src + ((size_t)k << kst));
        cp_async_commit();
    };
    float sh = 0.0f, sl = 0.0f;  // kWinNorm: this thread's sum of |psi|^2 (double-float)
    fetch(0);
    for (int sub = 0; sub < nsubs; ++sub) {
        if (sub + 1 < nsubs) {
            fetch(sub + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();  // every thread's copies of this tile (and evk)
        float4 *buf = win_buf + (sub & 1) * 2048;
        float4 x[16];
        // phase 1: j = window bits 0-3
        const uint32_t i1 = (tid & ((1u << RL) - 1u)) | ((tid >> RL) << (RL + 4));
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = buf[i1 | ((uint32_t)j << RL)];
#pragma unroll
        for (int b = 0; b < 4; ++b) rot(x, b);
        if (M > 4) {
#pragma unroll
            for (int j = 0; j < 16; ++j) buf[i1 | ((uint32_t)j << RL)] = x[j];
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 16; ++j) x[j] = buf[it_last | ij_last(j)];
#pragma unroll
            for (int b = LJ; b < 4; ++b) rot(x, b);
        }
        if (MODE == kWinPost) {  // the next layer's phase, with the row signs folded into its sign
            const uint32_t y0 = 2u * (tile_base(tile0 + (uint32_t)sub) | off(it_last));
            const uint64_t e0 = ev_of(Lq, y0) ^ Lq.s[t], e1 = e0 ^ evk[16];
            const uint32_t p0 = (uint32_t)__popc(y0 & zmq) ^ Lq.zc[t] ^ pt;
            const uint32_t p1 = p0 ^ (zmq & 1u);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                cmul_inplace(x[j].x, x[j].y, phase2(ph2, e0, evk[j], p0 ^ (pj >> j)));
                cmul_inplace(x[j].z, x[j].w, phase2(ph2, e1, evk[j], p1 ^ (pj >> j)));
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if ((pt ^ (pj >> j)) & 1u) x[j] = make_float4(-x[j].x, -x[j].y, -x[j].z, -x[j].w);
        }
        if (MODE == kWinNorm) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                df_add(sh, sl, prob_of(1.0f, x[j].x, x[j].y));
                df_add(sh, sl, prob_of(1.0f, x[j].z, x[j].w));
            }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) buf[it_last | ij_last(j)] = x[j];  // the slots this thread read
        __syncthreads();
        float4 *dst = p4 + tile_base(tile0 + (uint32_t)sub) + off_t;
#pragma unroll
        for (int k = 0; k < 16; ++k) dst[(size_t)k << kst] = buf[tid + (k << 7)];
        __syncthreads();  // the buffer's reads are done before the next copy into it
    }
    if (MODE == kWinNorm) norm_finish<4>(v, t, blockIdx.x, gridDim.x, sh, sl);
}

// Phase only (a circuit whose layers have no mixer qubits left to fuse with).
__global__ void __launch_bounds__(kThreads) k_phase_sweep(BatchView v, LayerView L) {
    const int t = blockIdx.y;
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1 > 0 ? n - 1 : 0);
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)t << n));
    const uint64_t sv = L.s[t];
    const uint32_t zm = L.zm[t], zc = L.zc[t];
    for (int64_t f = (int64_t)blockIdx.x * kThreads + threadIdx.x; f < nf; f += (int64_t)gridDim.x * kThreads) {
        float4 val = p4[f];
        const uint32_t y = (uint32_t)(2 * f);
        cmul_inplace(val.x, val.y, layer_phase(L, y, sv, zm, zc));
        cmul_inplace(val.z, val.w, layer_phase(L, y | 1u, sv, zm, zc));
        p4[f] = val;
    }
}

// ---------------------------------------------------------------------------
// Fused adjoint (Pauli-only noise), the reverse of the fused layers on psi and
// lambda together.  In the stored basis a layer is the cost diagonal D(y) =
// (-1)^{popc(y & zm) + zc} e^{-i gamma k(y)} followed by the mixer, a tensor
// product of M_q = S_q exp(-i beta X_q) over the qubits (S_q the row signs of the
// qubit's Pauli's Z part on its true bit).  So, at the point after the layer,
//   d<C>_t/d beta  += sum_q 2 sigma_q Im <lambda|X_q|psi>   (S X S = sigma X,
//                     sigma_q = -1 when the Pauli has a Z part),
// and, at the point after the cost layer (the mixer undone),
//   d<C>_t/d gamma += 2 Im <lambda|k|psi>                   (dD/dgamma = -i k D).
// The qubits' terms may be taken window by window: the rotations of the other
// windows commute with X_q.  A window sweep takes the terms of its qubits and then
// applies M_q^dagger = exp(+i beta X_q) S_q to both vectors; the phase sweep takes
// the k term and applies D^dagger.  32 B per amplitude per sweep.
// ---------------------------------------------------------------------------

// One qubit of a window: the pair (a0, a1) of psi and (m0, m1) of lambda at stored
// bits 0 and 1 of the qubit.  Adds sigma Im(conj(m0) a1 + conj(m1) a0) to acc, then
// applies S (s0, s1) and exp(+i beta X) = [[c, i s], [i s, c]] to both pairs.
__device__ __forceinline__ void adj_pair(float &a0r, float &a0i, float &a1r, float &a1i, float &m0r, float &m0i,
                                         float &m1r, float &m1i, float sg, float s0, float s1, float cb, float sb,
                                         float &acc) {
    acc += sg * ((m0r * a1i - m0i * a1r) + (m1r * a0i - m1i * a0r));
    a0r *= s0;
    a0i *= s0;
    a1r *= s1;
    a1i *= s1;
    m0r *= s0;
    m0i *= s0;
    m1r *= s1;
    m1i *= s1;
    float n0r = cb * a0r - sb * a1i, n0i = cb * a0i + sb * a1r;
    float n1r = cb * a1r - sb * a0i, n1i = cb * a1i + sb * a0r;
    a0r = n0r;
    a0i = n0i;
    a1r = n1r;
    a1i = n1i;
    n0r = cb * m0r - sb * m1i;
    n0i = cb * m0i + sb * m1r;
    n1r = cb * m1r - sb * m0i;
    n1i = cb * m1i + sb * m0r;
    m0r = n0r;
    m0i = n0i;
    m1r = n1r;
    m1i = n1i;
}

// Reverse of one mixer window of layer L: qubits q_lo .. q_lo + HAS0 + R - 1.  With
// HAS0 (q_lo == 0) qubit 0 is the float4 half and qubits 1 .. R the float4-index bits
// 0 .. R-1; otherwise qubits q_lo .. q_lo + R - 1 are the float4-index bits q_lo - 1 ..
// A thread holds one fibre of 2^R float4 of each vector (the window's bits varied,
// the others fixed); consecutive threads take consecutive values of the bits below
// the window.  Grid (fibres / kThreads, trajectories).
template <int R, bool HAS0>
__global__ void __launch_bounds__(kThreads) k_adj_mixer(BatchView v, float2 *lam, LayerView L, int q_lo, double *grad,
                                                         int param, int nparam) {
    constexpr int E = 1 << R;
    const int t = blockIdx.y;
    const int64_t nf = (int64_t)1 << (v.n - 1 > 0 ? v.n - 1 : 0);
    const int wlo = HAS0 ? 0 : q_lo - 1;  // float4-index bit of the window's first register qubit
    const int q1 = HAS0 ? 1 : q_lo;       // qubit on register bit 0
    const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    float acc = 0.0f;
    if (r < (nf >> R)) {
        const int64_t lowm = ((int64_t)1 << wlo) - 1;
        const int64_t base = ((r & ~lowm) << R) | (r & lowm);
        float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)t << v.n));
        float4 *l4 = reinterpret_cast<float4 *>(lam + ((size_t)t << v.n));
        float4 a[E], m[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            a[j] = p4[base | ((int64_t)j << wlo)];
            m[j] = l4[base | ((int64_t)j << wlo)];
        }
        const uint32_t mz = L.mz[t], mf = L.mf[t];
        const float cb = L.cb, sb = L.sb;
        if (HAS0) {
            const uint32_t z = mz & 1u, fq = mf & 1u;
            const float sg = z ? -1.0f : 1.0f, s0 = (z && fq) ? -1.0f : 1.0f, s1 = (z && !fq) ? -1.0f : 1.0f;
#pragma unroll
            for (int j = 0; j < E; ++j)
                adj_pair(a[j].x, a[j].y, a[j].z, a[j].w, m[j].x, m[j].y, m[j].z, m[j].w, sg, s0, s1, cb, sb, acc);
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int q = q1 + i;
            const uint32_t z = (mz >> q) & 1u, fq = (mf >> q) & 1u;
            const float sg = z ? -1.0f : 1.0f, s0 = (z && fq) ? -1.0f : 1.0f, s1 = (z && !fq) ? -1.0f : 1.0f;
#pragma unroll
            for (int j = 0; j < E; ++j) {
                if (j & (1 << i)) continue;
                const int k = j | (1 << i);
                adj_pair(a[j].x, a[j].y, a[k].x, a[k].y, m[j].x, m[j].y, m[k].x, m[k].y, sg, s0, s1, cb, sb, acc);
                adj_pair(a[j].z, a[j].w, a[k].z, a[k].w, m[j].z, m[j].w, m[k].z, m[k].w, sg, s0, s1, cb, sb, acc);
            }
        }
#pragma unroll
        for (int j = 0; j < E; ++j) {
            p4[base | ((int64_t)j << wlo)] = a[j];
            l4[base | ((int64_t)j << wlo)] = m[j];
        }
    }
    adj_finish(v, t, blockIdx.x, gridDim.x, acc, grad, param, nparam);
}

// Reverse of the cost layer L: adds 2 Im <lambda|k|psi> to d<C>_t/d gamma (via
// adj_finish), then applies D^dagger = (-1)^{popc(y & zm) + zc} e^{+i gamma k(y)} to
// both vectors.  One tile of kTileF4 float4 per block, grid (tiles, trajectories).
__global__ void __launch_bounds__(kThreads) k_adj_phase(BatchView v, float2 *lam, LayerView L, double *grad, int param,
                                                         int nparam) {
    const int t = blockIdx.y, tile = blockIdx.x;
    const int64_t nf = (int64_t)1 << (v.n - 1 > 0 ? v.n - 1 : 0);
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)t << v.n));
    float4 *l4 = reinterpret_cast<float4 *>(lam + ((size_t)t << v.n));
    const uint64_t sv = L.s[t];
    const uint32_t zm = L.zm[t], zc = L.zc[t];
    const uint64_t ev1 = ev_of(L, 1u);
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < kF4PerThread; ++k) {
        const int64_t f = (int64_t)tile * kTileF4 + threadIdx.x + k * kThreads;
        if (f >= nf) continue;
        float4 a = p4[f], m = l4[f];
        const uint32_t y = (uint32_t)(2 * f);
        const uint64_t e0 = ev_of(L, y);
        float av[4] = {a.x, a.y, a.z, a.w}, mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int kk = __popcll((e ? e0 ^ ev1 : e0) ^ sv);
            const float2 ph = __ldg(L.phase + kk);  // e^{-i gamma k}
            const float sg = ((__popc((y | (uint32_t)e) & zm) ^ zc) & 1u) ? -1.0f : 1.0f;
            float &ar = av[2 * e], &ai = av[2 * e + 1], &mr = mv[2 * e], &mi = mv[2 * e + 1];
            acc += (float)kk * (mr * ai - mi * ar);
            const float cr = ph.x * sg, ci = -ph.y * sg;  // conj(D(y))
            const float nar = ar * cr - ai * ci, nai = ar * ci + ai * cr;
            const float nmr = mr * cr - mi * ci, nmi = mr * ci + mi * cr;
            ar = nar;
            ai = nai;
            mr = nmr;
            mi = nmi;
        }
        p4[f] = make_float4(av[0], av[1], av[2], av[3]);
        l4[f] = make_float4(mv[0], mv[1], mv[2], mv[3]);
    }
    adj_finish(v, t, tile, v.tiles, acc, grad, param, nparam);
}

// The end of a tiled adjoint sweep: as adj_finish for NV inner products at once (WARPS
// warps per block), each into partials slot v of the block and grad[t][param[v]].
template <int WARPS, int NV>
__device__ void adj_finish_n(const BatchView &v, int t, int blk, int nblk, const float *acc, double *grad,
                             const int *param, int nparam) {
    __shared__ double redd[NV][WARPS];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double d = (double)acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
        if (lane == 0) redd[k][warp] = d;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < NV; ++k) {
            double sum = 0.0;
            for (int w = 0; w < WARPS; ++w) sum += redd[k][w];
            v.partials[((size_t)t * v.tiles + blk) * 4 + k] = sum;
        }
        __threadfence();
        const unsigned prev = atomicAdd(&v.counters[t], 1u);
        last = prev == (unsigned)(nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s0 = 0.0;
        for (int i = threadIdx.x; i < nblk; i += WARPS * 32) s0 += __ldcg(v.partials + ((size_t)t * v.tiles + i) * 4 + k);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        __syncthreads();
        if (lane == 0) redd[k][warp] = s0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < NV; ++k) {
            double sum = 0.0;
            for (int w = 0; w < WARPS; ++w) sum += redd[k][w];
            grad[(size_t)t * nparam + param[k]] += 2.0 * sum * v.inv_norm[t];
        }
        v.counters[t] = 0;
    }
}

// The layout of a tiled adjoint window.  A tile is 1024 float4 of psi and the same 1024
// of lambda, tile index i (10 bits).  HAS0: the tile is float4 bits 0-9 and the window
// qubits 0-9 (qubit 0 the float4 half, qubits 1-9 tile bits 0-8); otherwise tile bits
// 0 .. L-1 are the run (float4 bits 0 .. L-1, below the window) and bits L .. 9 the
// window's NB qubits q_lo .. (float4 bits q_lo-1 ..).  A thread holds 8 float4 of each
// vector per phase: in phase p register bit b is tile bit rb(p, b) -- window bits
// 3p .. 3p+2, or, past the window's last, the run's top bits -- and the thread's 7 bits
// are the other tile bits in increasing order (so its bits 0-2 are tile bits 3-5 in
// phase 0 with HAS0, tile bits 0-2 otherwise).  Buffer slot of i: i + (i >> 3), which
// puts the eight threads of a quarter warp on distinct 16-byte bank groups in every
// phase and adds over disjoint bit fields (base + constant addressing).
template <bool HAS0, int NB>
struct AdjWin {
    static constexpr int L = HAS0 ? 10 : 10 - NB;
    static constexpr int NP = HAS0 ? 3 : (NB > 3 ? 2 : 1);
    __host__ __device__ static constexpr int wp(int p) { return HAS0 ? 3 : (NB - 3 * p < 3 ? NB - 3 * p : 3); }
    __host__ __device__ static constexpr int rb(int p, int b) {
        return HAS0 ? 3 * p + b : (b < wp(p) ? L + 3 * p + b : L - 1 - (b - wp(p)));
    }
    __host__ __device__ static constexpr bool in_rb(int p, int bit) {
        return rb(p, 0) == bit || rb(p, 1) == bit || rb(p, 2) == bit;
    }
    __host__ __device__ static constexpr int tb(int p, int k) {  // tile bit of thread bit k
        int c = 0;
        for (int bit = 0; bit < 10; ++bit)
            if (!in_rb(p, bit)) {
                if (c == k) return bit;
                ++c;
            }
        return -1;
    }
    __host__ __device__ static constexpr uint32_t ij(int p, int j) {  // register j's tile bits
        return ((uint32_t)(j & 1) << rb(p, 0)) | ((uint32_t)((j >> 1) & 1) << rb(p, 1)) |
               ((uint32_t)((j >> 2) & 1) << rb(p, 2));
    }
    __host__ __device__ static constexpr uint32_t slot(uint32_t i) { return i + (i >> 3); }
};
constexpr int kAdjTile = 1024;                       // float4 per vector and tile
constexpr int kAdjSlots = kAdjTile + kAdjTile / 8;   // with one pad slot per eight
constexpr int kAdjSubs = 4;                          // tiles per block
constexpr size_t kAdjSmem = 2 * 2 * kAdjSlots * sizeof(float4);  // [buffer][psi, lambda][slot]

// The reverse of one mixer window of layer L over tiles of psi and lambda (layout
// AdjWin), and with PHASE also of the layer's cost diagonal (the window is the layer's
// last to be undone).  Per tile: phase 0 applies the window's Pauli row signs S_q to both
// vectors (a diagonal: (-1)^popc(z & (x ^ y)) over the window); then per phase, for each
// register qubit, the term Im(conj(m0) a1 + conj(m1) a0) of d<C>_t/d beta (the row signs
// are in: S_q's two signs multiply to sigma_q) and exp(+i beta X_q) on both vectors in
// the tangent form of k_fused_tile12 with beta -> -beta (the common factor rsc^N taken
// in phase 0).
// With PHASE the last phase adds k(y) Im(conj(m) a) to d<C>_t/d gamma and applies
// D(y)^dagger.  The terms of the other windows' qubits are unaffected (their rotations
// commute with X_q).  Tiles stream through two buffers (cp.async, one tile ahead); the last
// phase stores its registers to HBM.
// Grid (blocks of kAdjSubs tiles, trajectories) x 128 threads.
template <bool HAS0, int NB, bool PHASE, bool TANF>
__global__ void __launch_bounds__(128, 3) k_adj_win(BatchView v, float2 *lam, LayerView L, int q_lo, double *grad,
                                                     int pbeta, int pgamma, int nparam) {
    using A = AdjWin<HAS0, NB>;
    constexpr int RL = A::L;
    extern __shared__ float4 adj_buf[];  // [2][2][kAdjSlots]
    __shared__ uint64_t evk[9];          // PHASE: EV of the last phase's register offsets; [8]: EV of bit 0
    __shared__ float2 ph2[PHASE ? kPh2 : 1];  // PHASE: the conjugate phase table of layer L
    const int t = blockIdx.y;
    const uint32_t tid = threadIdx.x;
    const int w = HAS0 ? 0 : q_lo - 1;
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)t << v.n));
    float4 *l4 = reinterpret_cast<float4 *>(lam + ((size_t)t << v.n));
    const int ntiles = 1 << (v.n - 11);
    const int nsubs = ntiles < kAdjSubs ? ntiles : kAdjSubs;
    const uint32_t tile0 = (uint32_t)blockIdx.x * (uint32_t)nsubs;
    // float4 offset of tile index i, and the first float4 of tile u
    auto off = [&](uint32_t i) -> uint32_t {
        if constexpr (HAS0) return i;
        else return (i & ((1u << RL) - 1u)) | ((i >> RL) << w);
    };
    auto tile_base = [&](uint32_t u) -> uint32_t {
        if constexpr (HAS0) {
            return u << 10;
        } else {
            const uint32_t mid = (uint32_t)(w - RL);
            return ((u & ((1u << mid) - 1u)) << RL) | ((u >> mid) << (w + NB));
        }
    };
    auto it_of = [&](int p) {  // the thread's tile bits in phase p
        uint32_t i = 0;
#pragma unroll
        for (int k = 0; k < 7; ++k) i |= ((tid >> k) & 1u) << A::tb(p, k);
        return i;
    };
    // the window's amplitude bits of tile index i (float4 half 0): the Z and frame bits
    // of its qubits line up with them
    auto wbits = [&](uint32_t i) -> uint32_t {
        return HAS0 ? (2u * i) & 0x3ffu : (i >> RL) & ((1u << NB) - 1u);
    };
    const uint32_t wmask = HAS0 ? 0x3ffu : (1u << NB) - 1u;
    const uint32_t zw = (HAS0 ? L.mz[t] : L.mz[t] >> q_lo) & wmask, xw = (HAS0 ? L.mf[t] : L.mf[t] >> q_lo) & wmask;
    uint32_t pj0 = 0;  // bit j: the row-sign parity of phase-0 register j's bits
#pragma unroll
    for (int j = 0; j < 8; ++j) pj0 |= ((uint32_t)__popc(zw & wbits(A::ij(0, j))) & 1u) << j;
    const uint32_t pt0 = (uint32_t)__popc(zw & xw) ^ (uint32_t)__popc(zw & wbits(it_of(0)));
    // exp(+i beta X) = exp(-i (-beta) X): the forward's tangent form with sin beta negated
    const float cb = L.cb, sb = -L.sb;
    const float rt = TANF ? sb / cb : cb / sb, rsc = TANF ? cb : sb;
    constexpr int PL = A::NP - 1;  // the last phase
    uint32_t pjD = 0;
    const uint32_t zmD = PHASE ? L.zm[t] : 0u;
    if (PHASE) {
#pragma unroll
        for (int j = 0; j < 8; ++j) pjD |= ((uint32_t)__popc(2u * off(A::ij(PL, j)) & zmD) & 1u) << j;
        if (tid < 8u) evk[tid] = ev_of(L, 2u * off(A::ij(PL, (int)tid)));
        if (tid == 8u) evk[8] = ev_of(L, 1u);
        load_phase2<true>(L, ph2, 128);
    }
    const uint32_t off_t = off(tid);  // index order: i = tid | k << 7
    auto fetch = [&](int sub) {
        float4 *bp = adj_buf + (sub & 1) * 2 * kAdjSlots;
        const uint32_t tbs = tile_base(tile0 + (uint32_t)sub);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t i = tid | ((uint32_t)k << 7);
            const uint32_t o = tbs + off_t + off((uint32_t)k << 7);
            cp_async16(bp + A::slot(i), p4 + o);
            cp_async16(bp + kAdjSlots + A::slot(i), l4 + o);
        }
        cp_async_commit();
    };
    float accb = 0.0f, accg = 0.0f;
    // Phase 0 scales both vectors by rsc^N (N: the window's qubits) with the row signs, so
    // that after the window's N tangent-form rotations they carry their true scale; the
    // terms of phase p, taken on values still short of the rotations before it, are scaled
    // by rsc^(2 (N - nprev)) and corrected once per phase.
    constexpr int NQ = HAS0 ? 10 : NB;
    float rscN = 1.0f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) rscN *= rsc;
    float corr[A::NP];  // 1 / rsc^(2 (N - qubits rotated before phase p))
    {
        int prev = 0;
#pragma unroll
        for (int p = 0; p < A::NP; ++p) {
            float c = 1.0f;
            for (int q = prev; q < NQ; ++q) c *= rsc * rsc;
            corr[p] = 1.0f / c;
            prev += A::wp(p) + ((HAS0 && p == 0) ? 1 : 0);
        }
    }
    float accp = 0.0f;  // the current phase's terms
    auto term = [&](float a0r, float a0i, float a1r, float a1i, float m0r, float m0i, float m1r, float m1i) {
        accp += (m0r * a1i - m0i * a1r) + (m1r * a0i - m1i * a0r);
    };
    fetch(0);
    for (int sub = 0; sub < nsubs; ++sub) {
        if (sub + 1 < nsubs) {
            fetch(sub + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();  // every thread's copies of this tile (and evk)
        float4 *bp = adj_buf + (sub & 1) * 2 * kAdjSlots;
        float4 a[8], m[8];
#pragma unroll
        for (int p = 0; p < A::NP; ++p) {
            const uint32_t st = A::slot(it_of(p));
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                a[j] = bp[st + A::slot(A::ij(p, j))];
                m[j] = bp[kAdjSlots + st + A::slot(A::ij(p, j))];
            }
            if (p == 0) {  // the row signs of the window's qubits, and rsc^N
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t par = pt0 ^ (pj0 >> j);
                    const float s0 = (par & 1u) ? -rscN : rscN;
                    const float s1 = HAS0 ? (((par ^ zw) & 1u) ? -rscN : rscN) : s0;
                    a[j] = make_float4(a[j].x * s0, a[j].y * s0, a[j].z * s1, a[j].w * s1);
                    m[j] = make_float4(m[j].x * s0, m[j].y * s0, m[j].z * s1, m[j].w * s1);
                }
            }
            // the terms of the phase's qubits, all on the values as the phase read them (the
            // tangent-form rotations are unitary only up to rsc, applied at the phase's end)
            if (HAS0 && p == 0) {  // qubit 0: the float4 halves
#pragma unroll
                for (int j = 0; j < 8; ++j) term(a[j].x, a[j].y, a[j].z, a[j].w, m[j].x, m[j].y, m[j].z, m[j].w);
            }
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (b >= A::wp(p)) break;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (j & (1 << b)) continue;
                    const int k = j | (1 << b);
                    term(a[j].x, a[j].y, a[k].x, a[k].y, m[j].x, m[j].y, m[k].x, m[k].y);
                    term(a[j].z, a[j].w, a[k].z, a[k].w, m[j].z, m[j].w, m[k].z, m[k].w);
                }
            }
            accb = __fmaf_rn(accp, corr[p], accb);
            accp = 0.0f;
            if (HAS0 && p == 0) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    rx_pair_t<TANF>(a[j].x, a[j].y, a[j].z, a[j].w, rt);
                    rx_pair_t<TANF>(m[j].x, m[j].y, m[j].z, m[j].w, rt);
                }
            }
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (b >= A::wp(p)) break;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (j & (1 << b)) continue;
                    rx_pair4_t<TANF>(a[j], a[j | (1 << b)], rt);
                    rx_pair4_t<TANF>(m[j], m[j | (1 << b)], rt);
                }
            }
            if (PHASE && p == PL) {  // the cost diagonal: its gamma term, then D^dagger
                const uint32_t y0 = 2u * (tile_base(tile0 + (uint32_t)sub) | off(it_of(p)));
                const uint64_t e0 = ev_of(L, y0) ^ L.s[t], e1 = e0 ^ evk[8];
                const uint32_t p0 = (uint32_t)__popc(y0 & zmD) ^ L.zc[t];
                const uint32_t p1 = p0 ^ (zmD & 1u);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t k0 = (uint32_t)__popcll(e0 ^ evk[j]), k1 = (uint32_t)__popcll(e1 ^ evk[j]);
                    accg += (float)k0 * (m[j].x * a[j].y - m[j].y * a[j].x);
                    accg += (float)k1 * (m[j].z * a[j].w - m[j].w * a[j].z);
                    const float2 d0 = ph2[(k0 << 1) | ((p0 ^ (pjD >> j)) & 1u)];
                    const float2 d1 = ph2[(k1 << 1) | ((p1 ^ (pjD >> j)) & 1u)];
                    cmul_inplace(a[j].x, a[j].y, d0);
                    cmul_inplace(a[j].z, a[j].w, d1);
                    cmul_inplace(m[j].x, m[j].y, d0);
                    cmul_inplace(m[j].z, m[j].w, d1);
                }
            }
            if (p < PL) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {  // back to the slots this thread read
                    bp[st + A::slot(A::ij(p, j))] = a[j];
                    bp[kAdjSlots + st + A::slot(A::ij(p, j))] = m[j];
                }
                __syncthreads();
            } else {  // the last phase stores to HBM: a warp's lanes cover tile bits 0-4 (runs of >= 256 bytes)
                const uint32_t ob = tile_base(tile0 + (uint32_t)sub) + off(it_of(p));
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t o = ob + off(A::ij(p, j));
                    p4[o] = a[j];
                    l4[o] = m[j];
                }
            }
        }
        __syncthreads();  // the buffer's reads are done before the next copy into it
    }
    const float acc2[2] = {accb, accg};
    const int par2[2] = {pbeta, pgamma};
    adj_finish_n<4, PHASE ? 2 : 1>(v, t, blockIdx.x, gridDim.x, acc2, grad, par2, nparam);
}

// Readout of psi_x = i^k * D * phi_{x xor F} in the true basis (debug path).
__global__ void __launch_bounds__(kThreads) k_readout(BatchView v, float2 *out) {
    const int t = blockIdx.y;
    const int n = v.n;
    const int64_t dim = (int64_t)1 << n;
    const TrajState s = v.st[t];
    const uint32_t Ff = v.frame_x[(size_t)t * (v.G + 1) + v.G] ^ s.J ^ s.pend;
    const int k = v.yphase[t];
    for (int64_t x = (int64_t)blockIdx.x * kThreads + threadIdx.x; x < dim; x += (int64_t)gridDim.x * kThreads) {
        const uint32_t y = (uint32_t)x ^ Ff;
        const float2 a = v.psi[((size_t)t << n) + y];
        const uint32_t tb = (uint32_t)x ^ s.pend;
        const float fac = s.f[((tb >> s.pq0) & 1u) | (((tb >> s.pq1) & 1u) << 1)];
        const float sc = fac * (float)sqrt(v.inv_norm[t]);
        float re = a.x * sc, im = a.y * sc;
        float2 r;
        if (k == 0) r = make_float2(re, im);
        else if (k == 1) r = make_float2(-im, re);
        else if (k == 2) r = make_float2(-re, -im);
        else r = make_float2(im, -re);
        out[((size_t)t << n) + x] = r;
    }
}

// Readout of the states a shared-prefix run evolved (debug path, no
// re-simulation): output o is trajectory otraj[o] (batch-local) whose final
// state is slot oslot[o].  psi_x = i^k * sqrt(1/N_s) * phi'_{x xor F}, where phi'
// is the slot's stored state with its pending op applied, or -- when the
// circuit's last mixer block was kept pending (its sweep formed only the norms)
// -- that block applied here: phi'_y = f(y_S) * sum_a prod_i R(y_qi, a_i)
// phi_src(y with the block's bits set to a), R = exp(-i beta X) entry by entry,
// f the block's drawn factor by stored bits, src the parent of a slot forked at
// the block.  Written plainly (one output amplitude per thread, FP32 terms
// summed in FP64), independently of the sigma pass that applies the same block.
__global__ void __launch_bounds__(kThreads) k_slot_readout(BatchView v, const int32_t *oslot, const int32_t *otraj,
                                                           ReadTail rt, float2 *out) {
    const int o = blockIdx.y;
    const int sl = oslot[o], t = otraj[o];
    const int n = v.n;
    const int64_t dim = (int64_t)1 << n;
    const TrajState s = v.st[sl];
    const uint32_t Ff = v.frame_x[(size_t)sl * (v.G + 1) + v.G] ^ s.J ^ s.pend;
    const int k = v.yphase[t];
    const double sc = sqrt(v.inv_norm[sl]);
    const bool keep = rt.keep != 0;
    const int src = keep && sl >= rt.first_new ? rt.parent[sl] : sl;
    const float2 *phi = v.psi + ((size_t)src << n);
    for (int64_t x = (int64_t)blockIdx.x * kThreads + threadIdx.x; x < dim; x += (int64_t)gridDim.x * kThreads) {
        const uint32_t y = (uint32_t)x ^ Ff;
        double re = 0.0, im = 0.0;
        if (keep) {
            int yS = 0;
            uint32_t ybase = y;
            for (int i = 0; i < rt.M; ++i) {
                yS |= (int)((y >> rt.q[i]) & 1u) << i;
                ybase &= ~(1u << rt.q[i]);
            }
            for (int a = 0; a < (1 << rt.M); ++a) {
                // prod_i R(y_i, a_i): cos beta where the bits agree, -i sin beta where they differ
                double cr = 1.0, ci = 0.0;
                uint32_t ya = ybase;
                for (int i = 0; i < rt.M; ++i) {
                    const int ai = (a >> i) & 1;
                    ya |= (uint32_t)ai << rt.q[i];
                    const bool same = ai == ((yS >> i) & 1);
                    const double er = same ? (double)rt.c : 0.0, ei = same ? 0.0 : -(double)rt.s;
                    const double nr = cr * er - ci * ei, ni = cr * ei + ci * er;
                    cr = nr;
                    ci = ni;
                }
                const float2 p = phi[ya];
                re += cr * p.x - ci * p.y;
                im += cr * p.y + ci * p.x;
            }
            const double f = rt.T[(size_t)sl * kGroupBins + yS].x;
            re *= f;
            im *= f;
        } else {
            const float2 p = phi[y];
            const uint32_t tb = (uint32_t)x ^ s.pend;
            const double f = s.f[((tb >> s.pq0) & 1u) | (((tb >> s.pq1) & 1u) << 1)];
            re = f * p.x;
            im = f * p.y;
        }
        re *= sc;
        im *= sc;
        float2 r;
        if (k == 0) r = make_float2((float)re, (float)im);
        else if (k == 1) r = make_float2((float)-im, (float)re);
        else if (k == 2) r = make_float2((float)-re, (float)-im);
        else r = make_float2((float)im, (float)-re);
        out[((size_t)o << n) + x] = r;
    }
}

}  // namespace

cudaError_t launch_prepare(const BatchView &v, const DevGate *gates, uint64_t seed, const NoiseDev &nz,
                           int damping_on, cudaStream_t s) {
    const int threads = 128;
    k_prepare<<<(v.b + threads - 1) / threads, threads, 0, s>>>(v, gates, seed, nz, damping_on);
    return cudaGetLastError();
}

// Blocks of one kernel that fit on one SM at once (cached per kernel).
static int blocks_per_sm(const void *kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::unordered_map<const void *, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(kernel);
    if (it != cache.end()) return it->second;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess) per = 1;
    per = std::max(per, 1);
    cache.emplace(kernel, per);
    return per;
}

static int sm_count() {
    static const int sms = [] {  // initialised once, safely under concurrent first calls
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : 152;
    }();
    return sms;
}

// The grid of a sweep launch of gx blocks (tiles) per slot over `most` slots.  Sized on
// the host: (gx, most), one block per tile and slot.  Device-driven (v.dyn_hi set; `most` =
// the slots there can be): a persistent grid of as many blocks as the device holds of this
// kernel at once (at most gx * most), which take the items of v's counter (*lv: v with the
// tile count set).
static dim3 sweep_grid(const BatchView &v, const void *kernel, int threads, size_t smem, unsigned gx, int most,
                       BatchView *lv) {
    *lv = v;
    if (!v.dyn_hi) return dim3(gx, (unsigned)most);
    lv->dyn_tiles = (int32_t)gx;
    const int64_t resident = (int64_t)blocks_per_sm(kernel, threads, smem) * sm_count();
    return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(resident, (int64_t)gx * std::max(most, 1))));
}

// Blocks of a block-per-slot decide kernel: one per live slot, or (device-driven) enough to
// fill the device, each striding over the slots.
static unsigned slot_blocks(const SlotView &sv, const void *kernel, int active) {
    if (!sv.dyn) return (unsigned)active;
    return (unsigned)std::max(1, std::min(active, blocks_per_sm(kernel, kThreads, 0) * sm_count()));
}

cudaError_t launch_init(const BatchView &v, cudaStream_t s) {
    BatchView lv;
    const dim3 grid = sweep_grid(v, (const void *)k_init, kThreads, 0, (unsigned)v.tiles, v.b, &lv);
    k_init<<<grid, kThreads, 0, s>>>(lv);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const BatchView &v, int g, const DevGate &gate, const NoiseDev &nz, int damping_on,
                         cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)v.stiles, (unsigned)v.b);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (gate.kind == kGateZZ) {
        if (damping_on) return cudaLaunchKernelEx(&cfg, k_sweep_zz<true>, v, g, gate, nz.gamma);
        return cudaLaunchKernelEx(&cfg, k_sweep_zz<false>, v, g, gate, nz.gamma);
    }
    if (damping_on) return cudaLaunchKernelEx(&cfg, k_sweep_rx<true>, v, g, gate, nz.gamma);
    return cudaLaunchKernelEx(&cfg, k_sweep_rx<false>, v, g, gate, nz.gamma);
}

int64_t accumulate_xblocks(int n) { return tiles_for(n); }

static int persistent_blocks() {
    static const int blocks = [] {  // initialised once, safely under concurrent first calls
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fork_copy, kThreads, 0);
        return (sms > 0 ? sms : 152) * (per > 0 ? per : 4);
    }();
    return blocks;
}


template <typename K, typename... Args>
static cudaError_t launch_pdl_smem(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename K, typename... Args>
static cudaError_t launch_pdl(K kernel, dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    return launch_pdl_smem(kernel, grid, block, 0, s, args...);
}

cudaError_t launch_slot_sweep(const BatchView &v, const SlotView &sv, int active, int g, const DevGate &gate,
                              int damping_on, cudaStream_t s) {
    BatchView lv;
    const dim3 grid = sweep_grid(v, (const void *)k_slot_sweep<true, kGateZZ, true>, kThreads, 0, (unsigned)v.stiles,
                                 active, &lv),
               block(kThreads);
#define QN_SLOT(D, K)                                                                                    \
    (v.dyn_hi ? launch_pdl(k_slot_sweep<D, K, true>, grid, block, s, lv, sv, g, gate)                   \
              : launch_pdl(k_slot_sweep<D, K, false>, grid, block, s, lv, sv, g, gate))
    if (gate.kind == kGateZZ) return damping_on ? QN_SLOT(true, kGateZZ) : QN_SLOT(false, kGateZZ);
    return damping_on ? QN_SLOT(true, kGateRX) : QN_SLOT(false, kGateRX);
#undef QN_SLOT
}

cudaError_t launch_slot_fork(const BatchView &v, const SlotView &sv, int active, int g, const DevGate &gate,
                             const NoiseDev &nz, int damping_on, cudaStream_t s) {
    const int blocks = persistent_blocks();
    const dim3 block(kThreads);
    const dim3 slots(slot_blocks(sv, (const void *)k_slot_decide<true>, active));
    cudaError_t e = damping_on ? launch_pdl(k_slot_decide<true>, slots, block, s, v, sv, g, gate, nz.gamma)
                               : launch_pdl(k_slot_decide<false>, slots, block, s, v, sv, g, gate, nz.gamma);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_fork_copy, dim3(blocks), block, s, v, sv);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_fork_finish, dim3(1), dim3(1), s, sv);
}

cudaError_t launch_slot_order(const SlotView &sv, int32_t *pos, int32_t *order, double *weights, int K, int *status,
                              cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(pos, 0xff, (size_t)K * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(order, 0, (size_t)K * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)std::max(1, std::min((K + kThreads - 1) / kThreads, 4 * sm_count()));
    k_order_mark<<<blocks, kThreads, 0, s>>>(sv, pos, weights, K, status);
    k_order_compact<<<1, kThreads, 0, s>>>(pos, K, order);
    return cudaGetLastError();
}

cudaError_t launch_observe(const BatchView &v, const AccumView &, cudaStream_t s) {
    BatchView lv;
    const dim3 grid = sweep_grid(v, (const void *)k_observe, kThreads, 0, (unsigned)v.tiles, v.b, &lv);
    k_observe<<<grid, kThreads, 0, s>>>(lv);
    return cudaGetLastError();
}

RowPlan probs_row_plan(int n, int kind) {
    // blocks per state: k_probs covers 2048 amplitudes per block, k_probs_mix 2048 (half a mixer tile)
    const int64_t xb = kind == 2 ? std::max<int64_t>(2, (int64_t)1 << std::max(0, n - 11)) : accumulate_xblocks(n);
    // resident blocks of each pass, initialised once (safely under concurrent first calls)
    static const std::array<int, 3> resident = [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int occ[3] = {0, 0, 0};
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], k_probs<false>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], k_probs<true>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], k_probs_mix<true>, kMixThreads, 0);
        std::array<int, 3> r{};
        for (int k = 0; k < 3; ++k) r[k] = std::max(sms, 1) * std::max(occ[k], 1);
        return r;
    }();
    RowPlan r{};
    r.xb = xb;
    r.res = resident[kind < 0 ? 0 : kind > 2 ? 2 : kind];
    // rows past the first hold a sigma copy (8 B per basis state), 64 MiB at most
    const int64_t copies = std::max<int64_t>(0, ((int64_t)64 << 20) / ((int64_t)8 << n));
    r.pmax = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)kMaxProbParts, 1 + copies));
    r.used = 0;
    return r;
}

int probs_parts(int n, int b, int kind) { return row_parts(probs_row_plan(n, kind), b); }

cudaError_t launch_probs(const BatchView &v, const AccumView &a, cudaStream_t s) {
    const int64_t xb = accumulate_xblocks(v.n);
    const int parts = a.probs && a.spart ? a.parts : 1;
    const dim3 grid((unsigned)xb, (unsigned)parts);
    if (a.trivial_pending) k_probs<true><<<grid, kThreads, 0, s>>>(v, a, xb);
    else k_probs<false><<<grid, kThreads, 0, s>>>(v, a, xb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || parts == 1) return e;
    const int64_t dim = (int64_t)1 << v.n;
    k_probs_combine<<<(unsigned)std::min<int64_t>((dim + 255) / 256, 4096), 256, 0, s>>>(a.probs, a.spart, parts, dim,
                                                                                        a.rows, v.dyn_hi);
    return cudaGetLastError();
}

cudaError_t launch_probs_mix(const BatchView &v, const AccumView &a, const MixMap &mm, const MixTail &tl,
                             cudaStream_t s) {
    const int64_t xb = (int64_t)2 << mm.ntile;  // half tiles
    const int parts = a.probs && a.spart ? a.parts : 1;
    const dim3 grid((unsigned)xb, (unsigned)parts);
    if (mm.tanf) k_probs_mix<true><<<grid, kMixThreads, 0, s>>>(v, a, mm, tl, xb);
    else k_probs_mix<false><<<grid, kMixThreads, 0, s>>>(v, a, mm, tl, xb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || parts == 1) return e;
    const int64_t dim = (int64_t)1 << v.n;
    k_probs_combine<<<(unsigned)std::min<int64_t>((dim + 255) / 256, 4096), 256, 0, s>>>(a.probs, a.spart, parts, dim,
                                                                                        a.rows, v.dyn_hi);
    return cudaGetLastError();
}

cudaError_t launch_readout(const BatchView &v, float2 *out, cudaStream_t s) {
    const int64_t dim = (int64_t)1 << v.n;
    int64_t blocks = (dim + kThreads - 1) / kThreads;
    if (blocks > 4096) blocks = 4096;
    k_readout<<<dim3((unsigned)blocks, (unsigned)v.b), kThreads, 0, s>>>(v, out);
    return cudaGetLastError();
}

cudaError_t launch_slot_readout(const BatchView &v, const int32_t *oslot, const int32_t *otraj, int nout,
                                const ReadTail &rt, float2 *out, cudaStream_t s) {
    if (nout <= 0) return cudaSuccess;
    const int64_t dim = (int64_t)1 << v.n;
    int64_t blocks = (dim + kThreads - 1) / kThreads;
    if (blocks > 4096) blocks = 4096;
    k_slot_readout<<<dim3((unsigned)blocks, (unsigned)nout), kThreads, 0, s>>>(v, oslot, otraj, rt, out);
    return cudaGetLastError();
}

cudaError_t launch_adj_init(const BatchView &v, float2 *lam, const AccumView &a, cudaStream_t s) {
    k_adj_init<<<dim3((unsigned)v.tiles, (unsigned)v.b), kThreads, 0, s>>>(v, lam, a);
    return cudaGetLastError();
}

cudaError_t launch_adj_sweep(const BatchView &v, float2 *lam, int g, const DevGate &gate, double *grad, int param,
                             int nparam, cudaStream_t s) {
    const dim3 grid((unsigned)v.tiles, (unsigned)v.b);
    if (gate.kind == kGateZZ) k_adj_sweep<kGateZZ><<<grid, kThreads, 0, s>>>(v, lam, g, gate, grad, param, nparam);
    else k_adj_sweep<kGateRX><<<grid, kThreads, 0, s>>>(v, lam, g, gate, grad, param, nparam);
    return cudaGetLastError();
}

cudaError_t launch_adj_mixer(const BatchView &v, float2 *lam, const LayerView &L, int q_lo, int m, double *grad,
                             int param, int nparam, cudaStream_t s) {
    const bool has0 = q_lo == 0;
    const int R = has0 ? m - 1 : m;
    if (R < 0 || R > 3 || (!has0 && R == 0) || q_lo + m > v.n) return cudaErrorInvalidValue;
    const int64_t nf = (int64_t)1 << (v.n - 1 > 0 ? v.n - 1 : 0);
    const int64_t fibres = nf >> R;
    const dim3 grid((unsigned)((fibres + kThreads - 1) / kThreads), (unsigned)v.b);
    if ((int64_t)grid.x > v.tiles) return cudaErrorInvalidValue;  // partials hold v.tiles per trajectory
#define QN_ADJM(RR, H) k_adj_mixer<RR, H><<<grid, kThreads, 0, s>>>(v, lam, L, q_lo, grad, param, nparam)
    if (has0) {
        switch (R) {
        case 0: QN_ADJM(0, true); break;
        case 1: QN_ADJM(1, true); break;
        case 2: QN_ADJM(2, true); break;
        default: QN_ADJM(3, true); break;
        }
    } else {
        switch (R) {
        case 1: QN_ADJM(1, false); break;
        case 2: QN_ADJM(2, false); break;
        default: QN_ADJM(3, false); break;
        }
    }
#undef QN_ADJM
    return cudaGetLastError();
}

template <bool HAS0, int NB, bool PHASE>
static cudaError_t adj_win_launch(const BatchView &v, float2 *lam, const LayerView &L, int q_lo, double *grad,
                                  int pbeta, int pgamma, int nparam, cudaStream_t s) {
    static const cudaError_t attr = [] {
        cudaError_t e = cudaFuncSetAttribute(k_adj_win<HAS0, NB, PHASE, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_adj_win<HAS0, NB, PHASE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kAdjSmem);
        return e;
    }();
    if (attr != cudaSuccess) return attr;
    const int ntiles = 1 << (v.n - 11);
    const int blocks = ntiles < kAdjSubs ? 1 : ntiles / kAdjSubs;
    if (blocks > v.tiles) return cudaErrorInvalidValue;  // partials hold v.tiles per trajectory
    const dim3 grid((unsigned)blocks, (unsigned)v.b);
    if (std::fabs(L.cb) >= std::fabs(L.sb))
        k_adj_win<HAS0, NB, PHASE, true><<<grid, 128, kAdjSmem, s>>>(v, lam, L, q_lo, grad, pbeta, pgamma, nparam);
    else
        k_adj_win<HAS0, NB, PHASE, false><<<grid, 128, kAdjSmem, s>>>(v, lam, L, q_lo, grad, pbeta, pgamma, nparam);
    return cudaGetLastError();
}

cudaError_t launch_adj_win(const BatchView &v, float2 *lam, const LayerView &L, int q_lo, int m, bool phase,
                           double *grad, int pbeta, int pgamma, int nparam, cudaStream_t s) {
    if (v.n < 12 || v.n > 30) return cudaErrorInvalidValue;
    if (q_lo == 0) {
        if (m != 10 || phase) return cudaErrorInvalidValue;
        return adj_win_launch<true, 9, false>(v, lam, L, 0, grad, pbeta, pgamma, nparam, s);
    }
    if (q_lo < 10 || m < 2 || m > 6 || q_lo + m > v.n) return cudaErrorInvalidValue;
#define QN_ADJW(NB)                                                                                  \
    return phase ? adj_win_launch<false, NB, true>(v, lam, L, q_lo, grad, pbeta, pgamma, nparam, s) \
                 : adj_win_launch<false, NB, false>(v, lam, L, q_lo, grad, pbeta, pgamma, nparam, s)
    switch (m) {
    case 2: QN_ADJW(2);
    case 3: QN_ADJW(3);
    case 4: QN_ADJW(4);
    case 5: QN_ADJW(5);
    default: QN_ADJW(6);
    }
#undef QN_ADJW
}

cudaError_t launch_adj_phase(const BatchView &v, float2 *lam, const LayerView &L, double *grad, int param, int nparam,
                             cudaStream_t s) {
    k_adj_phase<<<dim3((unsigned)v.tiles, (unsigned)v.b), kThreads, 0, s>>>(v, lam, L, grad, param, nparam);
    return cudaGetLastError();
}

cudaError_t launch_layer_params(const BatchView &v, const LayerView &L, int g0, int E, cudaStream_t s) {
    k_layer_params<<<(v.b + 127) / 128, 128, 0, s>>>(v, L, g0, E);
    return cudaGetLastError();
}

template <int LQ, int RQ, bool HAS0, bool PRE, bool POST, bool NORM = false>
static cudaError_t fused_launch(const BatchView &v, const LayerView &Lp, const LayerView &Lr, const LayerView &Lq,
                                int q_lo, cudaStream_t s) {
    constexpr size_t smem = sizeof(float4) * (size_t)(1 << RQ) * kThreads;  // the threads' landing slots
    static const cudaError_t attr = cudaFuncSetAttribute(k_fused_sweep<LQ, RQ, HAS0, PRE, POST, NORM>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    const int64_t threads = ((int64_t)1 << (v.n - 1)) >> RQ;  // 2^LQ threads per fibre of LQ + RQ bits
    const int64_t per_block = (int64_t)kThreads * kFuseChunks;
    const int64_t blocks = (threads + per_block - 1) / per_block;
    if (NORM && blocks > v.tiles) return cudaErrorInvalidValue;  // the partial sums hold v.tiles per state
    const dim3 grid((unsigned)blocks, (unsigned)v.b);
    k_fused_sweep<LQ, RQ, HAS0, PRE, POST, NORM><<<grid, kThreads, smem, s>>>(v, Lp, Lr, Lq, q_lo);
    return cudaGetLastError();
}

template <int LQ, int RQ, bool HAS0>
static cudaError_t fused_dispatch(const BatchView &v, const LayerView &Lp, const LayerView &Lr, const LayerView &Lq,
                                  int q_lo, bool pre, bool post, bool norm, cudaStream_t s) {
    if (!HAS0 && pre) return cudaErrorInvalidValue;  // the first layer's phase rides on the qubit-0 window
    if (norm) {
        // the circuit's last window (off qubit 0, so n > 5): no later phase
        if constexpr (HAS0) return cudaErrorInvalidValue;
        else return post ? cudaErrorInvalidValue : fused_launch<LQ, RQ, false, false, false, true>(v, Lp, Lr, Lq, q_lo, s);
    }
    if constexpr (HAS0 && LQ > 0) {
        // the 8-qubit window needs n >= 10, so it is never a layer's last
        if (post) return cudaErrorInvalidValue;
        if (pre) return fused_launch<LQ, RQ, true, true, false>(v, Lp, Lr, Lq, q_lo, s);
        return fused_launch<LQ, RQ, true, false, false>(v, Lp, Lr, Lq, q_lo, s);
    } else {
        if (HAS0 && pre && post) return fused_launch<LQ, RQ, HAS0, HAS0, true>(v, Lp, Lr, Lq, q_lo, s);
        if (HAS0 && pre) return fused_launch<LQ, RQ, HAS0, HAS0, false>(v, Lp, Lr, Lq, q_lo, s);
        if (post) return fused_launch<LQ, RQ, HAS0, false, true>(v, Lp, Lr, Lq, q_lo, s);
        return fused_launch<LQ, RQ, HAS0, false, false>(v, Lp, Lr, Lq, q_lo, s);
    }
}

cudaError_t launch_fused_sweep(const BatchView &v, const LayerView &Lp, const LayerView &Lr, const LayerView &Lq,
                               int q_lo, int m, bool pre, bool post, bool norm, cudaStream_t s) {
    if (m < 1 || q_lo < 0 || q_lo + m > v.n) return cudaErrorInvalidValue;
    // lane qubits need whole warps of fibres (2^(RQ+5) float4 per state, RQ = 4) and,
    // off qubit 0, the 5 - LQ float4-index bits below the window free (q_lo - 1 >= 5 - LQ,
    // LQ = m - 4)
    const bool lanes_ok = v.n >= 10 && (q_lo == 0 || q_lo - 1 >= 9 - m);
    if (q_lo == 0) {
        switch (m) {
        case 1: return fused_dispatch<0, 0, true>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
        case 2: return fused_dispatch<0, 1, true>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
        case 3: return fused_dispatch<0, 2, true>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
        case 4: return fused_dispatch<0, 3, true>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
        case 5: return fused_dispatch<0, 4, true>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
        case 8:  // qubit 0 in the float4, 1-3 on lane bits, 4-7 in registers
            if (!lanes_ok) return cudaErrorInvalidValue;
            return fused_dispatch<3, 4, true>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (m) {
    case 1: return fused_dispatch<0, 1, false>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
    case 2: return fused_dispatch<0, 2, false>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
    case 3: return fused_dispatch<0, 3, false>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
    case 4: return fused_dispatch<0, 4, false>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
    case 5:
    case 6:
    case 7:  // m - 4 qubits on lane bits, 4 in registers
        if (!lanes_ok) return cudaErrorInvalidValue;
        if (m == 5) return fused_dispatch<1, 4, false>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
        if (m == 6) return fused_dispatch<2, 4, false>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
        return fused_dispatch<3, 4, false>(v, Lp, Lr, Lq, q_lo, pre, post, norm, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fused_tile12(const BatchView &v, const LayerView &Lp, const LayerView &Lr, bool pre,
                                cudaStream_t s) {
    if (v.n < 13 || v.n > 30) return cudaErrorInvalidValue;
    static const cudaError_t attr = [] {
        for (auto k : {k_fused_tile12<true, true>, k_fused_tile12<true, false>, k_fused_tile12<false, true>,
                       k_fused_tile12<false, false>}) {
            const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kT12Smem);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }();
    if (attr != cudaSuccess) return attr;
    const int ntiles = 1 << (v.n - 12);
    const dim3 grid((unsigned)(ntiles < kT12Subs ? 1 : ntiles / kT12Subs), (unsigned)v.b);
    const bool tanf = std::fabs(Lr.cb) >= std::fabs(Lr.sb);
    if (tanf) {
        if (pre) k_fused_tile12<true, true><<<grid, 128, kT12Smem, s>>>(v, Lp, Lr);
        else k_fused_tile12<true, false><<<grid, 128, kT12Smem, s>>>(v, Lp, Lr);
    } else {
        if (pre) k_fused_tile12<false, true><<<grid, 128, kT12Smem, s>>>(v, Lp, Lr);
        else k_fused_tile12<false, false><<<grid, 128, kT12Smem, s>>>(v, Lp, Lr);
    }
    return cudaGetLastError();
}

template <int M, int MODE>
static cudaError_t win_launch(const BatchView &v, const LayerView &Lr, const LayerView &Lq, int q_lo, cudaStream_t s) {
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_fused_win<M, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kT12Smem);
    if (attr != cudaSuccess) return attr;
    const int ntiles = 1 << (v.n - 12);
    const int blocks = ntiles < kT12Subs ? 1 : ntiles / kT12Subs;
    if (MODE == kWinNorm && blocks > v.tiles) return cudaErrorInvalidValue;  // partial sums: v.tiles per state
    k_fused_win<M, MODE><<<dim3((unsigned)blocks, (unsigned)v.b), 128, kT12Smem, s>>>(v, Lr, Lq, q_lo);
    return cudaGetLastError();
}

// Which windows take k_fused_win (measured on the fused layers at n = 16-26): the tiled form
// streams at the copy rate wherever the register sweep's lane runs are short (64 bytes for a
// 7-qubit window, far apart at the top qubits), and for the plain and norm sweeps; the
// register sweep (256 threads, more warps in flight) applies the next layer's phase faster
// in windows of up to six qubits.  Plain windows of four or five qubits off qubit 0 do not
// occur for n <= 30.
bool fused_win_ok(int n, int q_lo, int m, bool post, bool norm) {
    if (n < 12 || n > 30 || m < 4 || m > 7 || q_lo < 1 || q_lo - 1 < 11 - m || q_lo + m > n || (post && norm))
        return false;
    if (post) return m == 7;
    return norm || m >= 6;
}

cudaError_t launch_fused_win(const BatchView &v, const LayerView &Lr, const LayerView &Lq, int q_lo, int m, bool post,
                             bool norm, cudaStream_t s) {
    if (!fused_win_ok(v.n, q_lo, m, post, norm)) return cudaErrorInvalidValue;
    if (norm) {
        switch (m) {
        case 4: return win_launch<4, kWinNorm>(v, Lr, Lq, q_lo, s);
        case 5: return win_launch<5, kWinNorm>(v, Lr, Lq, q_lo, s);
        case 6: return win_launch<6, kWinNorm>(v, Lr, Lq, q_lo, s);
        default: return win_launch<7, kWinNorm>(v, Lr, Lq, q_lo, s);
        }
    }
    if (post) return win_launch<7, kWinPost>(v, Lr, Lq, q_lo, s);
    return m == 6 ? win_launch<6, kWinPlain>(v, Lr, Lq, q_lo, s) : win_launch<7, kWinPlain>(v, Lr, Lq, q_lo, s);
}

cudaError_t launch_phase_sweep(const BatchView &v, const LayerView &L, cudaStream_t s) {
    const int64_t nf = (int64_t)1 << (v.n - 1 > 0 ? v.n - 1 : 0);
    int64_t blocks = (nf + kThreads - 1) / kThreads;
    if (blocks > 65535) blocks = 65535;
    k_phase_sweep<<<dim3((unsigned)blocks, (unsigned)v.b), kThreads, 0, s>>>(v, L);
    return cudaGetLastError();
}

// Blocks of a group sweep per state (kGSub sub-tiles each).
static unsigned group_tiles(int n) {
    const int64_t nf = (int64_t)1 << (n - 1);
    return (unsigned)((nf + (int64_t)kTileF4 * kGSub - 1) / ((int64_t)kTileF4 * kGSub));
}

cudaError_t launch_group_hist(const BatchView &v, const SlotView &, const GroupView &gv, int active, cudaStream_t s) {
    BatchView lv;
    const dim3 grid = sweep_grid(v, (const void *)k_group_hist<true, true>, kThreads, 0, group_tiles(v.n), active, &lv);
    if (v.dyn_hi)
        return gv.pend ? launch_pdl(k_group_hist<true, true>, grid, dim3(kThreads), s, lv, gv)
                       : launch_pdl(k_group_hist<false, true>, grid, dim3(kThreads), s, lv, gv);
    return gv.pend ? launch_pdl(k_group_hist<true>, grid, dim3(kThreads), s, lv, gv)
                   : launch_pdl(k_group_hist<false>, grid, dim3(kThreads), s, lv, gv);
}

cudaError_t launch_group_decide(const BatchView &v, const SlotView &sv, const GroupView &gv, int ns, int active,
                                double gamma, cudaStream_t s) {
    const dim3 blk(kThreads);
    const dim3 slots(slot_blocks(sv, (const void *)k_gd_classes, active));
    const dim3 slot_warps((unsigned)((active + kThreads / 32 - 1) / (kThreads / 32)));
    const int class_blocks = (sv.max_slots + kThreads / 32 - 1) / (kThreads / 32);
    cudaError_t e;
#define QN_GD(R)                                                                                \
    const int resident = blocks_per_sm((const void *)k_gd_tables<R>, kThreads, 0) * sm_count();  \
    const dim3 classes((unsigned)std::min(class_blocks, resident));                             \
    const dim3 members((unsigned)((gv.members + gd_members_per_block(R) - 1) / gd_members_per_block(R))); \
    e = launch_pdl(k_gd_joint<R>, slot_warps, blk, s, v, sv, gv, gamma, active);                \
    if (e == cudaSuccess) e = launch_pdl(k_gd_members<R>, members, blk, s, v, sv, gv, gamma);   \
    if (e == cudaSuccess) e = launch_pdl(k_gd_classes, slots, blk, s, v, sv, gv);               \
    if (e == cudaSuccess) e = launch_pdl(k_gd_tables<R>, classes, blk, s, v, sv, gv, gamma);
    if (ns <= 5) {
        QN_GD(1)
    } else if (ns <= 7) {
        QN_GD(4)
    } else if (ns <= 8) {  // the 8-qubit first mixer block, and 8-qubit phase groups
        QN_GD(8)
    } else {
        QN_GD(kGroupBins / 32)
    }
#undef QN_GD
    if (e != cudaSuccess) return e;
    return launch_pdl(k_fork_finish, dim3(1), dim3(1), s, sv);
}

// The mixer sweeps' dynamic shared memory (two tiles), set once for every variant.
static cudaError_t launch_mix_sweep_attrs() {
    static const cudaError_t attr = [] {
#define QN_KS(D)                                                                                          \
    (const void *)k_mix_sweep<true, kMixAny, D>, (const void *)k_mix_sweep<true, kMixMid, D>,             \
        (const void *)k_mix_sweep<true, kMixHist, D>,                                                     \
        (const void *)k_mix_sweep<false, kMixAny, D>, (const void *)k_mix_sweep<false, kMixMid, D>,       \
        (const void *)k_mix_sweep<false, kMixHist, D>,                                                    \
        (const void *)k_mix_sweep<true, kMixWide, D>, (const void *)k_mix_sweep<false, kMixWide, D>,      \
        (const void *)k_mix_sweep<true, kMixW1, D>, (const void *)k_mix_sweep<false, kMixW1, D>,          \
        (const void *)k_mix_sweep<true, kMixW2, D>, (const void *)k_mix_sweep<false, kMixW2, D>,          \
        (const void *)k_group_mix<true, false, D>, (const void *)k_group_mix<false, false, D>,            \
        (const void *)k_group_mix<true, true, D>, (const void *)k_group_mix<false, true, D>
        const void *ks[] = {QN_KS(false), QN_KS(true)};
#undef QN_KS
        for (const void *k : ks) {
            const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMixSmem);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }();
    return attr;
}

cudaError_t launch_mix_sweep(const BatchView &vh, const GroupView &gv, const MixMap &mm, int active, cudaStream_t s) {
    const cudaError_t attr = launch_mix_sweep_attrs();
    if (attr != cudaSuccess) return attr;
    const unsigned blocks = mm.ntile >= 2 ? (1u << mm.ntile) / kMixSubs : 1u;
    BatchView v;
    const dim3 grid = sweep_grid(vh, (const void *)k_mix_sweep<true, kMixMid, true>, kMixThreads, kMixSmem, blocks,
                                 active, &v),
               block(kMixThreads);
#define QN_MIX(T, V)                                                                                     \
    (v.dyn_hi ? launch_pdl_smem(k_mix_sweep<T, V, true>, grid, block, kMixSmem, s, v, gv, mm)            \
              : launch_pdl_smem(k_mix_sweep<T, V, false>, grid, block, kMixSmem, s, v, gv, mm))
    int var = kMixAny;
    if (mm.wide == 2 || mm.wide == 3) {
        // full blocks off qubit 0 with a full next block; the other half's four f bits
        // (wsh ..) lie on tile bits; kMixW1 also needs qubits 1-3 on the L bits
        bool ok = mm.M == kMixQ && !mm.has0 && mm.nN == kMixQ && !gv.next && !mm.final_norm && mm.wsh >= 0 &&
                  mm.wsh + 4 <= v.n - 1;
        for (int i = 0; i < 5 && ok; ++i) {
            const int f = i < kMixL ? mm.fL[i] : -1;
            if (f >= mm.wsh && f < mm.wsh + 4) ok = false;
        }
        for (int i = 0; i < kMixQ && ok; ++i)
            if ((mm.fA[i] >= mm.wsh && mm.fA[i] < mm.wsh + 4) || (mm.fB[i] >= mm.wsh && mm.fB[i] < mm.wsh + 4))
                ok = false;
        if (mm.wide == 2) ok = ok && mm.fL[0] == 0 && mm.fL[1] == 1 && mm.fL[2] == 2 && mm.wsh == 3;
        if (!ok) return cudaErrorInvalidValue;
        if (mm.wide == 2)
            return mm.tanf ? QN_MIX(true, kMixW1)
                           : QN_MIX(false, kMixW1);
        return mm.tanf ? QN_MIX(true, kMixW2)
                       : QN_MIX(false, kMixW2);
    }
    if (mm.wide) {
        // qubits 4-7 with the factors of qubits 0-7: the lane bits must be qubits 1-3, the block
        // qubits 4-7 and a full next block
        const bool ok = mm.M == kMixQ && !mm.has0 && mm.nN == kMixQ && !gv.next && !mm.final_norm &&
                        mm.fL[0] == 0 && mm.fL[1] == 1 && mm.fL[2] == 2 && mm.fA[0] == 3 && mm.fA[1] == 4 &&
                        mm.fA[2] == 5 && mm.fA[3] == 6;
        if (!ok) return cudaErrorInvalidValue;
        return mm.tanf ? QN_MIX(true, kMixWide)
                       : QN_MIX(false, kMixWide);
    }
    if (mm.M == kMixQ) {
        const bool next_full = mm.nN == kMixQ && !gv.next && !mm.final_norm;
        if (next_full && !mm.has0) var = kMixMid;
        else if (!mm.has0 && mm.nN == 0 && gv.next && !mm.final_norm) var = kMixHist;
    }
    switch (var) {
    case kMixMid: return mm.tanf ? QN_MIX(true, kMixMid) : QN_MIX(false, kMixMid);
    case kMixHist: return mm.tanf ? QN_MIX(true, kMixHist) : QN_MIX(false, kMixHist);
    default: return mm.tanf ? QN_MIX(true, kMixAny) : QN_MIX(false, kMixAny);
    }
#undef QN_MIX
}

cudaError_t launch_group_mix(const BatchView &vh, const GroupView &gv, const MixMap &mm, int active, cudaStream_t s) {
    cudaError_t e = launch_mix_sweep_attrs();
    if (e != cudaSuccess) return e;
    const bool natural = mm.has0 && mm.M == kMixQ && mm.nN == kMixQ && mm.fA[0] == 0 && mm.fA[1] == 1 &&
                         mm.fA[2] == 2 && mm.fA[3] == 7 && mm.fB[0] == 3 && mm.fB[1] == 4 && mm.fB[2] == 5 &&
                         mm.fB[3] == 6 && mm.fL[0] == 8 && mm.fL[1] == 9 && mm.fL[2] == 10;
    if (!natural || gv.pend) return cudaErrorInvalidValue;
    const unsigned blocks = mm.ntile >= 2 ? (1u << mm.ntile) / kMixSubs : 1u;
    BatchView v;
    const dim3 grid = sweep_grid(vh, (const void *)k_group_mix<true, true, true>, kMixThreads, kMixSmem, blocks, active,
                                 &v),
               block(kMixThreads);
#define QN_GMIX(T, F)                                                                                    \
    (v.dyn_hi ? launch_pdl_smem(k_group_mix<T, F, true>, grid, block, kMixSmem, s, v, gv, mm)            \
              : launch_pdl_smem(k_group_mix<T, F, false>, grid, block, kMixSmem, s, v, gv, mm))
    if (mm.full8) return mm.tanf ? QN_GMIX(true, true) : QN_GMIX(false, true);
    return mm.tanf ? QN_GMIX(true, false) : QN_GMIX(false, false);
#undef QN_GMIX
}

cudaError_t prewarm_dev_launches() {
    const cudaError_t e = launch_mix_sweep_attrs();
    if (e != cudaSuccess) return e;
    (void)sm_count();
    const void *plain[] = {(const void *)k_init, (const void *)k_observe, (const void *)k_group_hist<true, true>,
                           (const void *)k_group_apply<true, 1, true>, (const void *)k_slot_sweep<true, kGateZZ, true>,
                           (const void *)k_slot_decide<true>, (const void *)k_gd_classes,
                           (const void *)k_gd_tables<1>, (const void *)k_gd_tables<4>, (const void *)k_gd_tables<8>,
                           (const void *)k_gd_tables<kGroupBins / 32>};
    for (const void *k : plain) (void)blocks_per_sm(k, kThreads, 0);
    (void)blocks_per_sm((const void *)k_mix_sweep<true, kMixMid, true>, kMixThreads, kMixSmem);
    (void)blocks_per_sm((const void *)k_group_mix<true, true, true>, kMixThreads, kMixSmem);
    (void)persistent_blocks();
    (void)probs_row_plan(1, 0);
    return cudaGetLastError();
}

cudaError_t launch_group_apply(const BatchView &vh, const SlotView &, const GroupView &gv, int active, cudaStream_t s) {
    BatchView v;
    const dim3 grid = sweep_grid(vh, (const void *)k_group_apply<true, 1, true>, kThreads, 0, group_tiles(vh.n), active,
                                 &v),
               blk(kThreads);
    const int next = gv.next ? 1 : 0;
#define QN_APPLY(P, N)                                                                                   \
    (v.dyn_hi ? launch_pdl(k_group_apply<P, N, true>, grid, blk, s, v, gv)                               \
              : launch_pdl(k_group_apply<P, N, false>, grid, blk, s, v, gv))
    if (gv.pend) return next == 1 ? QN_APPLY(true, 1) : QN_APPLY(true, 0);
    return next == 1 ? QN_APPLY(false, 1) : QN_APPLY(false, 0);
#undef QN_APPLY
}

}  // namespace qn


