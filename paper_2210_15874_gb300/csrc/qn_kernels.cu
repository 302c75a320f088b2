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
    const int t = blockIdx.y;
    const int tile = blockIdx.x;
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

__device__ __forceinline__ void add_bin(float acc[4], int idx, float p) {
    acc[0] += idx == 0 ? p : 0.0f;
    acc[1] += idx == 1 ? p : 0.0f;
    acc[2] += idx == 2 ? p : 0.0f;
    acc[3] += idx == 3 ? p : 0.0f;
}

// Damping branch of gate g from its marginal m[4] (FP64).  m[b0 | b1 << 1] is
// the weight of true bits (b0, b1) of the gate's qubits after its Pauli (for a
// 1q gate only m[0] and m[3]).  Draws in the order first qubit, second qubit,
// the second conditioned on the first.  Writes the pending op for the next sweep.
__device__ void decide_damping(const BatchView &v, int t, int g, const DevGate &gt, const double m[4],
                               double gamma) {
    TrajState s = v.st[t];
    const uint32_t *dw = v.dwords + ((size_t)t * v.G + g) * 2;
    const double u0 = ((double)dw[0] + 0.5) * kTwoM32;
    const double u1 = ((double)dw[1] + 0.5) * kTwoM32;
    const double sg = sqrt(gamma), sg1 = sqrt(1.0 - gamma);
    uint32_t newpend = 0;
    uint8_t jb = 0;
    double f[4];
    bool bad = false;
    if (gt.kind == kGateZZ) {
        const double N = m[0] + m[1] + m[2] + m[3];
        const bool ji = u0 < gamma * (m[1] + m[3]) / N;
        const double ki0 = ji ? 0.0 : 1.0, ki1 = ji ? sg : sg1;
        const double Ni = (m[0] + m[2]) * ki0 * ki0 + (m[1] + m[3]) * ki1 * ki1;
        const bool jj = u1 < gamma * (m[2] * ki0 * ki0 + m[3] * ki1 * ki1) / Ni;
        const double kj0 = jj ? 0.0 : 1.0, kj1 = jj ? sg : sg1;
        const double Nf = m[0] * ki0 * ki0 * kj0 * kj0 + m[1] * ki1 * ki1 * kj0 * kj0 +
                          m[2] * ki0 * ki0 * kj1 * kj1 + m[3] * ki1 * ki1 * kj1 * kj1;
        const double sc = 1.0 / sqrt(Nf);
        f[0] = ki0 * kj0 * sc;
        f[1] = ki1 * kj0 * sc;
        f[2] = ki0 * kj1 * sc;
        f[3] = ki1 * kj1 * sc;
        newpend = ((uint32_t)ji << gt.q0) | ((uint32_t)jj << gt.q1);
        jb = (uint8_t)(((uint32_t)ji << 4) | ((uint32_t)jj << 5));
        bad = !(N > 0.0) || !(Ni > 0.0) || !(Nf > 0.0) || !isfinite(sc);
    } else {
        const double N = m[0] + m[3];
        const bool j = u0 < gamma * m[3] / N;
        const double k0 = j ? 0.0 : 1.0, k1 = j ? sg : sg1;
        const double Nf = m[0] * k0 * k0 + m[3] * k1 * k1;
        const double sc = 1.0 / sqrt(Nf);
        f[0] = k0 * sc;
        f[3] = k1 * sc;
        f[1] = f[2] = 0.0;
        newpend = (uint32_t)j << gt.q0;
        jb = (uint8_t)((uint32_t)j << 4);
        bad = !(N > 0.0) || !(Nf > 0.0) || !isfinite(sc);
    }
    if (bad) atomicOr(v.status, 1);
    s.J ^= s.pend;
    s.pend = newpend;
    s.pq0 = gt.q0;
    s.pq1 = gt.kind == kGateZZ ? gt.q1 : gt.q0;
    for (int k = 0; k < 4; ++k) s.f[k] = (float)f[k];
    v.st[t] = s;
    v.branch[(size_t)t * v.G + g] |= jb;
}

template <int KIND, bool DAMP>
__global__ void __launch_bounds__(kThreads) k_sweep(BatchView v, int g, DevGate gt, double gamma) {
    const int t = blockIdx.y;
    const int tile = blockIdx.x;
    __shared__ SweepCtx sc;
    __shared__ float red[kThreads / 32][4];
    __shared__ double redd[kThreads / 32][4];
    __shared__ int last;
    if (threadIdx.x == 0) {
        const uint32_t fxg = v.frame_x[(size_t)t * (v.G + 1) + g];
        const uint32_t fxg1 = v.frame_x[(size_t)t * (v.G + 1) + g + 1];
        SweepCtx c;
        c.code = v.branch[(size_t)t * v.G + g] & 15;
        if (DAMP) {
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
        sc = c;
    }
    __syncthreads();
    const SweepCtx c = sc;
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1);
    float4 *p4 = reinterpret_cast<float4 *>(v.psi + ((size_t)t << n));
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};

    if (KIND == kGateZZ) {
        const int q0 = gt.q0, q1 = gt.q1;
        const uint32_t za = (uint32_t)(c.code >> 3) & 1u, zb = (uint32_t)(c.code >> 1) & 1u;
        auto proc = [&](float &re, float &im, uint32_t y) {
            if (DAMP) {
                const float fa = pend_factor(c, y);
                re *= fa;
                im *= fa;
            }
            const uint32_t tb = y ^ c.Fb;
            const uint32_t b0 = (tb >> q0) & 1u, b1 = (tb >> q1) & 1u;
            const float sgn = ((za & b0) ^ (zb & b1)) ? -1.0f : 1.0f;
            const bool diff = (b0 ^ b1) != 0u;
            const float pc = (diff ? gt.c : 1.0f) * sgn;
            const float ps = (diff ? gt.s : 0.0f) * sgn;
            const float nr = re * pc + im * ps;
            const float ni = im * pc - re * ps;
            re = nr;
            im = ni;
            if (DAMP) {
                const uint32_t tc = y ^ c.Fc;
                add_bin(acc, (int)(((tc >> q0) & 1u) | (((tc >> q1) & 1u) << 1)), nr * nr + ni * ni);
            }
        };
        float4 val[kF4PerThread];
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k) {
            const int64_t f = (int64_t)tile * kTileF4 + threadIdx.x + k * kThreads;
            if (f < nf) val[k] = p4[f];
        }
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k) {
            const int64_t f = (int64_t)tile * kTileF4 + threadIdx.x + k * kThreads;
            if (f < nf) {
                const uint32_t y = (uint32_t)(2 * f);
                proc(val[k].x, val[k].y, y);
                proc(val[k].z, val[k].w, y | 1u);
                p4[f] = val[k];
            }
        }
    } else {  // RX
        const int q = gt.q0;
        const float cb = gt.c, sb = gt.s;
        const uint32_t z = (uint32_t)(c.code >> 1) & 1u;
        const uint32_t fbq = (c.Fb >> q) & 1u;  // true bit of the element with stored bit 0
        const uint32_t fcq = (c.Fc >> q) & 1u;
        // (a0 at y0 with stored bit q = 0, a1 at y1 = y0 | 2^q)
        auto proc = [&](float &r0, float &i0, float &r1, float &i1, uint32_t y0, uint32_t y1) {
            if (DAMP) {
                const float f0 = pend_factor(c, y0), f1 = pend_factor(c, y1);
                r0 *= f0; i0 *= f0; r1 *= f1; i1 *= f1;
            }
            float w0r = cb * r0 + sb * i1, w0i = cb * i0 - sb * r1;
            float w1r = cb * r1 + sb * i0, w1i = cb * i1 - sb * r0;
            if (z) {  // negate the element whose true bit is 1
                if (fbq) { w0r = -w0r; w0i = -w0i; } else { w1r = -w1r; w1i = -w1i; }
            }
            r0 = w0r; i0 = w0i; r1 = w1r; i1 = w1i;
            if (DAMP) {
                const float p0 = w0r * w0r + w0i * w0i, p1 = w1r * w1r + w1i * w1i;
                acc[0] += fcq ? p1 : p0;
                acc[3] += fcq ? p0 : p1;
            }
        };
        if (q == 0) {
            float4 val[kF4PerThread];
#pragma unroll
            for (int k = 0; k < kF4PerThread; ++k) {
                const int64_t f = (int64_t)tile * kTileF4 + threadIdx.x + k * kThreads;
                if (f < nf) val[k] = p4[f];
            }
#pragma unroll
            for (int k = 0; k < kF4PerThread; ++k) {
                const int64_t f = (int64_t)tile * kTileF4 + threadIdx.x + k * kThreads;
                if (f < nf) {
                    const uint32_t y = (uint32_t)(2 * f);
                    proc(val[k].x, val[k].y, val[k].z, val[k].w, y, y | 1u);
                    p4[f] = val[k];
                }
            }
        } else {
            const int sh = q - 1;
            const int64_t npairs = nf >> 1;
            constexpr int kPairs = kF4PerThread / 2;
            float4 lo[kPairs], hi[kPairs];
            int64_t flo[kPairs];
#pragma unroll
            for (int k = 0; k < kPairs; ++k) {
                const int64_t r = (int64_t)tile * (kTileF4 / 2) + threadIdx.x + k * kThreads;
                flo[k] = ((r >> sh) << (sh + 1)) | (r & (((int64_t)1 << sh) - 1));
                if (r < npairs) {
                    lo[k] = p4[flo[k]];
                    hi[k] = p4[flo[k] | ((int64_t)1 << sh)];
                }
            }
#pragma unroll
            for (int k = 0; k < kPairs; ++k) {
                const int64_t r = (int64_t)tile * (kTileF4 / 2) + threadIdx.x + k * kThreads;
                if (r < npairs) {
                    const uint32_t y0 = (uint32_t)(2 * flo[k]);
                    const uint32_t qb = 1u << q;
                    proc(lo[k].x, lo[k].y, hi[k].x, hi[k].y, y0, y0 | qb);
                    proc(lo[k].z, lo[k].w, hi[k].z, hi[k].w, y0 | 1u, y0 | 1u | qb);
                    p4[flo[k]] = lo[k];
                    p4[flo[k] | ((int64_t)1 << sh)] = hi[k];
                }
            }
        }
    }

    if (!DAMP) return;

    // ---- epilogue: marginal of gate g's qubits, then the damping draw ----
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
        v.partials[((size_t)t * v.tiles + tile) * 4 + threadIdx.x] = s;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&v.counters[t], 1u);
        last = prev == (unsigned)(v.tiles - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < v.tiles; i += kThreads) {
        const double *pp = v.partials + ((size_t)t * v.tiles + i) * 4;
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
    if (threadIdx.x == 0) {
        double m[4];
        for (int k = 0; k < 4; ++k) {
            double a = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) a += redd[w][k];
            m[k] = a;
        }
        decide_damping(v, t, g, gt, m, gamma);
        v.counters[t] = 0;
    }
}

// ---------------------------------------------------------------------------
// Observables of the final state.  The last pending damping op is applied on
// the fly.  k_observe reduces, per trajectory, N_t = ||psi_t||^2 and
// sum_x |psi_t,x|^2 C(x) in FP64 (per-amplitude FP64 adds: this pass runs once
// per trajectory, so its FP64 cost is small next to the gate sweeps), then the
// last block of the trajectory stores 1/N_t and <C>_t = sum |psi|^2 C / N_t:
// the final state is normalised exactly (the paper takes psi normalised before
// phi = |psi|^2 is formed).  k_probs then adds |psi_t,x|^2 / N_t over the batch
// into sigma's FP64 sums, one fixed-order update per basis state x and batch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cut_of(uint32_t x, int num_edges, const int2 *__restrict__ edges) {
    int cnt = 0;
    for (int j = 0; j < num_edges; ++j) {
        const int2 ed = edges[j];
        cnt += (int)(((x >> ed.x) ^ (x >> ed.y)) & 1u);
    }
    return cnt;
}

__global__ void __launch_bounds__(kThreads) k_observe(BatchView v, AccumView a) {
    const int t = blockIdx.y;
    const int tile = blockIdx.x;
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1 > 0 ? n - 1 : 0);
    __shared__ SweepCtx sc;
    __shared__ double redd[kThreads / 32][2];
    __shared__ int last;
    if (threadIdx.x == 0) {
        const TrajState s = v.st[t];
        SweepCtx c;
        c.Fa = v.frame_x[(size_t)t * (v.G + 1) + v.G] ^ s.J;
        c.Fb = c.Fa ^ s.pend;  // final frame
        c.Fc = 0;
        c.pq0 = s.pq0;
        c.pq1 = s.pq1;
        for (int k = 0; k < 4; ++k) c.f[k] = s.f[k];
        c.code = 0;
        sc = c;
    }
    __syncthreads();
    const SweepCtx c = sc;
    const float4 *p4 = reinterpret_cast<const float4 *>(v.psi + ((size_t)t << n));
    double sn = 0.0, scut = 0.0;
#pragma unroll
    for (int k = 0; k < kF4PerThread; ++k) {
        const int64_t f = (int64_t)tile * kTileF4 + threadIdx.x + k * kThreads;
        if (f < nf) {
            const float4 val = p4[f];
            const uint32_t y = (uint32_t)(2 * f);
            const float f0 = pend_factor(c, y), f1 = pend_factor(c, y | 1u);
            const float p0 = f0 * f0 * (val.x * val.x + val.y * val.y);
            const float p1 = f1 * f1 * (val.z * val.z + val.w * val.w);
            const int c0 = cut_of(y ^ c.Fb, a.num_edges, a.edges);
            const int c1 = cut_of((y | 1u) ^ c.Fb, a.num_edges, a.edges);
            sn += (double)p0 + (double)p1;
            scut += (double)p0 * c0 + (double)p1 * c1;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sn += __shfl_xor_sync(0xffffffffu, sn, off);
        scut += __shfl_xor_sync(0xffffffffu, scut, off);
    }
    if (lane == 0) {
        redd[warp][0] = sn;
        redd[warp][1] = scut;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double sum = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) sum += redd[w][threadIdx.x];
        v.partials[((size_t)t * v.tiles + tile) * 4 + threadIdx.x] = sum;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&v.counters[t], 1u);
        last = prev == (unsigned)(v.tiles - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < v.tiles; i += kThreads) {
        const double *pp = v.partials + ((size_t)t * v.tiles + i) * 4;
        s0 += __ldcg(pp);
        s1 += __ldcg(pp + 1);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    }
    __syncthreads();
    if (lane == 0) {
        redd[warp][0] = s0;
        redd[warp][1] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double N = 0.0, C = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            N += redd[w][0];
            C += redd[w][1];
        }
        if (!(N > 0.0) || !isfinite(N)) atomicOr(v.status, 2);
        v.inv_norm[t] = 1.0 / N;
        a.c_out[t] = C / N;
        v.counters[t] = 0;
    }
}

__global__ void __launch_bounds__(kThreads) k_probs(BatchView v, AccumView a) {
    const int xb = blockIdx.x;
    const int n = v.n;
    const int64_t nf = (int64_t)1 << (n - 1 > 0 ? n - 1 : 0);
    __shared__ int last;
    int64_t fp[kF4PerThread];
    double acc[2 * kF4PerThread];
#pragma unroll
    for (int k = 0; k < kF4PerThread; ++k) {
        fp[k] = (int64_t)xb * kTileF4 + threadIdx.x + k * kThreads;
        acc[2 * k] = acc[2 * k + 1] = 0.0;
    }
    for (int tt = 0; tt < v.b; ++tt) {
        const TrajState s = v.st[tt];
        const uint32_t Ff = v.frame_x[(size_t)tt * (v.G + 1) + v.G] ^ s.J ^ s.pend;
        const double inv = v.inv_norm[tt];
        const float4 *p4 = reinterpret_cast<const float4 *>(v.psi + ((size_t)tt << n));
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k) {
            if (fp[k] < nf) {
                const int64_t f = fp[k] ^ (int64_t)(Ff >> 1);
                float4 val = p4[f];
                if (Ff & 1u) val = make_float4(val.z, val.w, val.x, val.y);
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const uint32_t x = (uint32_t)(2 * fp[k] + e);
                    const uint32_t tb = x ^ s.pend;
                    const uint32_t b0 = (tb >> s.pq0) & 1u, b1 = (tb >> s.pq1) & 1u;
                    const float fac = b1 ? (b0 ? s.f[3] : s.f[2]) : (b0 ? s.f[1] : s.f[0]);
                    const float re = e ? val.z : val.x, im = e ? val.w : val.y;
                    acc[2 * k + e] = fma((double)(fac * fac * (re * re + im * im)), inv, acc[2 * k + e]);
                }
            }
        }
    }
    if (a.probs) {
#pragma unroll
        for (int k = 0; k < kF4PerThread; ++k)
            if (fp[k] < nf) {
                a.probs[2 * fp[k]] += acc[2 * k];
                a.probs[2 * fp[k] + 1] += acc[2 * k + 1];
            }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(a.acc_counter, 1u);
        last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    if (a.sums) {
        double s1 = a.sums[0], s2 = a.sums[1];
        for (int tt = 0; tt < v.b; ++tt) {
            const double cv = __ldcg(a.c_out + tt);
            s1 += cv;
            s2 += cv * cv;
        }
        a.sums[0] = s1;
        a.sums[1] = s2;
    }
    *a.acc_counter = 0;
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

}  // namespace

cudaError_t launch_prepare(const BatchView &v, const DevGate *gates, uint64_t seed, const NoiseDev &nz,
                           int damping_on, cudaStream_t s) {
    const int threads = 128;
    k_prepare<<<(v.b + threads - 1) / threads, threads, 0, s>>>(v, gates, seed, nz, damping_on);
    return cudaGetLastError();
}

cudaError_t launch_init(const BatchView &v, cudaStream_t s) {
    k_init<<<dim3((unsigned)v.tiles, (unsigned)v.b), kThreads, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const BatchView &v, int g, const DevGate &gate, const NoiseDev &nz, int damping_on,
                         cudaStream_t s) {
    const dim3 grid((unsigned)v.tiles, (unsigned)v.b);
    if (gate.kind == kGateZZ) {
        if (damping_on) k_sweep<kGateZZ, true><<<grid, kThreads, 0, s>>>(v, g, gate, nz.gamma);
        else k_sweep<kGateZZ, false><<<grid, kThreads, 0, s>>>(v, g, gate, nz.gamma);
    } else {
        if (damping_on) k_sweep<kGateRX, true><<<grid, kThreads, 0, s>>>(v, g, gate, nz.gamma);
        else k_sweep<kGateRX, false><<<grid, kThreads, 0, s>>>(v, g, gate, nz.gamma);
    }
    return cudaGetLastError();
}

int64_t accumulate_xblocks(int n) { return tiles_for(n); }

cudaError_t launch_observe(const BatchView &v, const AccumView &a, cudaStream_t s) {
    k_observe<<<dim3((unsigned)v.tiles, (unsigned)v.b), kThreads, 0, s>>>(v, a);
    return cudaGetLastError();
}

cudaError_t launch_probs(const BatchView &v, const AccumView &a, cudaStream_t s) {
    k_probs<<<(unsigned)accumulate_xblocks(v.n), kThreads, 0, s>>>(v, a);
    return cudaGetLastError();
}

cudaError_t launch_readout(const BatchView &v, float2 *out, cudaStream_t s) {
    const int64_t dim = (int64_t)1 << v.n;
    int64_t blocks = (dim + kThreads - 1) / kThreads;
    if (blocks > 4096) blocks = 4096;
    k_readout<<<dim3((unsigned)blocks, (unsigned)v.b), kThreads, 0, s>>>(v, out);
    return cudaGetLastError();
}

}  // namespace qn
