// qn_tc.cu -- the fused layers of Pauli-only noise on the tensor cores
// (tcgen05.mma, accumulators in TMEM).
//
// A QAOA mixer layer is exp(-i beta X) on every qubit, and the Z parts of the
// layer's Paulis are signs on true bits; the cost layer is diagonal.  A sweep
// here applies the mixer rotations of up to five consecutive qubits -- a
// window W of five qubits, of which the bits in `act` are rotated -- as one
// dense 32 x 32 operator per window pattern, with the cost-layer phases before
// (PRE) and after (POST) and the Z signs folded in elementwise.  The dense
// operator is written through the Hadamard factorisation
//
//     exp(-i beta X) = H diag(e^{-i beta}, e^{+i beta}) H,   H = [[1,1],[1,-1]]/sqrt(2)
//     =>  RX^(x5) = H5 D H5 / 32,   H5[j][k] = (-1)^popc(j & k),
//                                   D(j) = e^{-i beta (a - 2 popc(j & act))}, a = popc(act)
//
// (a window bit outside `act` has D independent of it, so H.H / 2 = I there).
// H5 is real with entries +-1, exact in TF32 and BF16, so each sweep is two
// real GEMMs on the tensor cores with an elementwise complex diagonal between
// them: T = H5 Psi, T' = D T / 32, Psi' = H5 T'.  Real and imaginary parts are
// separate GEMM rows.
//
// Tile: 2048 amplitudes of one state -- the 32 window patterns (GEMM K / N)
// times 64 positions r of the six lowest amplitude bits outside W.  The 128
// GEMM rows (M) are (r, re/im), one per thread.  Per tile:
//   1. the tile is staged in shared memory (cp.async, one tile ahead), rows of
//      32 amplitudes padded to 68 floats;
//   2. thread m gathers its row x[b] (b = window pattern), applies PRE, and
//      writes it as the K-major A operand (128-byte swizzle): TF32 as FP32
//      words; BF16x3 as the exact split x = hi + mid + lo into three bf16
//      terms (the operand [hi | mid] and [lo]), whose products with the +-1
//      matrix are exact, so the only rounding is the FP32 accumulation;
//   3. one thread issues the MMAs (M = 128, N = 32; TF32: 4 x K=8, BF16: 6 x
//      K=16) into TMEM columns 0..31 and commits them to an mbarrier;
//   4. every thread loads its row of T (tcgen05.ld 32x32b), applies D / 32
//      (re/im partner: the neighbouring lane), writes the second A operand;
//   5. the second GEMM into TMEM columns 32..63; its row gets the Z signs and
//      POST, goes back to the staged tile, and the tile is stored (coalesced
//      16-byte stores).
// Every mbarrier wait is bounded (about two seconds of SM clock); on timeout
// the kernel flags status bit 8, drains its copies, frees its TMEM and exits.
#include <cuda_bf16.h>

#include "qn_internal.h"

namespace qn {
namespace {

constexpr int kTcThreads = 128;                    // GEMM rows (r, re/im)
constexpr int kTcPitch = 68;                       // floats per staged row of 32 amplitudes
constexpr int kTcRawBytes = 64 * kTcPitch * 4;     // one staged tile: 17408 B
constexpr int kTcOpBytes = 128 * 128;              // one K-major operand: 128 rows x 128 B
constexpr int kTcBBytes = 32 * 128;                // H5 (BF16: [H5 | H5]): 32 rows x 128 B
constexpr uint32_t kTcCols = 64;                   // TMEM columns: D1 0..31, D2 32..63
constexpr int kTcChunk = 8;                        // consecutive tiles per block (one staged ahead)

template <int KIND>
__host__ __device__ constexpr int tc_ops() { return KIND == kPrecTF32 ? 1 : 2; }
// Resident blocks per SM the register budget is compiled for (shared memory admits as many).
template <int KIND>
__host__ __device__ constexpr int kTcMinBlocks() { return KIND == kPrecTF32 ? 4 : 3; }
template <int KIND>
__host__ __device__ constexpr int tc_smem_bytes() { return 1024 + tc_ops<KIND>() * kTcOpBytes + kTcBBytes + 2 * kTcRawBytes; }

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand with the 128-byte swizzle:
// 8-row atoms of 1024 B (SBO), start address in 16-byte units, descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Byte offset of the 16-byte chunk `chunk` of row r in a K-major SW128 operand.
__device__ __forceinline__ uint32_t sw128_chunk(int r, int chunk) {
    const int rr = r & 7;
    return (uint32_t)((r >> 3) * 1024 + rr * 128 + ((chunk ^ rr) << 4));
}

// Instruction descriptor: D in FP32, A and B of format fmt (TF32 = 2, BF16 = 1), both
// K-major, N = 32, M = 128.
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(int kind, uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    if (kind == kPrecTF32)
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                     "l"(a), "l"(b), "r"(tc_idesc(2)), "r"(acc));
    else
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                     "l"(a), "l"(b), "r"(tc_idesc(1)), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// Wait for phase `parity` of the mbarrier, for at most ~2 s of SM clock.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > 4000000000ll) return false;
    }
}

// This thread's row (its TMEM lane) of 32 FP32 columns starting at `col`.
__device__ __forceinline__ void tc_load32(uint32_t taddr, float (&x)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Row m of the A operand from the 32 values x[b]: TF32 as FP32 words; BF16x3 as
// x = hi + mid + lo (each step exact in FP32), [hi | mid] into op0, [lo] into op1.
template <int KIND>
__device__ __forceinline__ void tc_put_row(unsigned char *op0, unsigned char *op1, int m, const float (&x)[32]) {
    if (KIND == kPrecTF32) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
            *reinterpret_cast<float4 *>(op0 + sw128_chunk(m, c)) =
                make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
    } else {
        uint32_t hi[16], mid[16], lo[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            __nv_bfloat16 h[2], md[2], l[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float v = x[2 * j + e];
                h[e] = __float2bfloat16_rn(v);
                const float r1 = __fsub_rn(v, __bfloat162float(h[e]));
                md[e] = __float2bfloat16_rn(r1);
                l[e] = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(md[e])));
            }
            hi[j] = pack_bf16(h[0], h[1]);
            mid[j] = pack_bf16(md[0], md[1]);
            lo[j] = pack_bf16(l[0], l[1]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            *reinterpret_cast<uint4 *>(op0 + sw128_chunk(m, c)) = make_uint4(hi[4 * c], hi[4 * c + 1], hi[4 * c + 2], hi[4 * c + 3]);
            *reinterpret_cast<uint4 *>(op0 + sw128_chunk(m, c + 4)) =
                make_uint4(mid[4 * c], mid[4 * c + 1], mid[4 * c + 2], mid[4 * c + 3]);
            *reinterpret_cast<uint4 *>(op1 + sw128_chunk(m, c)) = make_uint4(lo[4 * c], lo[4 * c + 1], lo[4 * c + 2], lo[4 * c + 3]);
        }
    }
}

// D[128 x 32] (TMEM column `col`) = A[128 x K] H5^T.
template <int KIND>
__device__ __forceinline__ void tc_gemm(uint32_t tmem, uint32_t col, uint32_t sop0, uint32_t sop1, uint32_t sb) {
    if (KIND == kPrecTF32) {
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)  // K = 8 per instruction: 32 B steps inside the 128-byte rows
            tc_mma(KIND, tmem + col, sw128_desc(sop0 + 32 * ks), sw128_desc(sb + 32 * ks), ks > 0);
    } else {
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)  // [hi | mid] against [H5 | H5]: K = 16 per instruction
            tc_mma(KIND, tmem + col, sw128_desc(sop0 + 32 * ks), sw128_desc(sb + 32 * ks), ks > 0);
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)  // [lo] against H5
            tc_mma(KIND, tmem + col, sw128_desc(sop1 + 32 * ks), sw128_desc(sb + 32 * ks), 1u);
    }
}

// The cost layer's factor at y = y0 | (b << wl) (layer_phase, split over the disjoint bits of
// y0 and of the window pattern b: the edge-difference vector and the Z parity are both
// linear in y).  ev0 = EV(y0), evb = EV(b << wl), zp0 = popc(y0 & zm) ^ zc.
__device__ __forceinline__ float2 tc_phase(const LayerView &L, uint64_t ev0, uint64_t evb, uint64_t sv, uint32_t zp0,
                                           uint32_t yb, uint32_t zm) {
    const int k = __popcll(ev0 ^ evb ^ sv);
    const float2 ph = __ldg(L.phase + k);
    const float sg = ((zp0 ^ __popc(yb & zm)) & 1u) ? -1.0f : 1.0f;
    return make_float2(ph.x * sg, ph.y * sg);
}

__device__ __forceinline__ uint64_t tc_ev(const LayerView &L, uint32_t y) {
    return __ldg(L.ev + (y & 255u)) ^ __ldg(L.ev + 256 + ((y >> 8) & 255u)) ^ __ldg(L.ev + 512 + ((y >> 16) & 255u)) ^
           __ldg(L.ev + 768 + (y >> 24));
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gmem) : "memory");
}

template <int KIND, bool PRE, bool POST>
__global__ void __launch_bounds__(kTcThreads, kTcMinBlocks<KIND>()) k_tc_sweep(BatchView v, LayerView Lp, LayerView Lr, LayerView Lq,
                                                         TcSweep sw) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char *smem = tc_smem_raw + ((1024u - (su32(tc_smem_raw) & 1023u)) & 1023u);
    unsigned char *op0 = smem;
    unsigned char *op1 = smem + (tc_ops<KIND>() - 1) * kTcOpBytes;  // BF16x3 only
    unsigned char *sB = smem + tc_ops<KIND>() * kTcOpBytes;
    float *raw0 = reinterpret_cast<float *>(sB + kTcBBytes);
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    __shared__ float2 dph[6];
    __shared__ uint64_t evw[32];  // edge-difference vector of each window pattern (the cost layer is linear in y)
    const int tid = threadIdx.x, warp = tid >> 5;
    const int n = v.n;
    const int wl = sw.wl;
    const uint32_t act = sw.act;
    const int ws = wl < 6 ? wl : 6;  // position of the window bits in the tile-local index
    const int tiles = 1 << (n - 11);
    const int units = v.b * tiles;

    // H5 as the B operand ([N = 32 patterns][K]), once per block
    {
        const int row = tid >> 2, part = tid & 3;  // 4 threads per row, 2 chunks each
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = part * 2 + cc;
            if (KIND == kPrecTF32) {
                float w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) w[e] = (__popc(row & (4 * c + e)) & 1) ? -1.0f : 1.0f;
                *reinterpret_cast<float4 *>(sB + sw128_chunk(row, c)) = make_float4(w[0], w[1], w[2], w[3]);
            } else {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k0 = (8 * c + 2 * e) & 31, k1 = (8 * c + 2 * e + 1) & 31;
                    w[e] = pack_bf16(__float2bfloat16_rn((__popc(row & k0) & 1) ? -1.0f : 1.0f),
                                     __float2bfloat16_rn((__popc(row & k1) & 1) ? -1.0f : 1.0f));
                }
                *reinterpret_cast<uint4 *>(sB + sw128_chunk(row, c)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
    if (tid < 6) dph[tid] = sw.dph[tid];
    if ((PRE || POST) && tid < 32) {
        const uint32_t y = (uint32_t)tid << wl;
        const LayerView &L = PRE ? Lp : Lq;
        evw[tid] = __ldg(L.ev + (y & 255u)) ^ __ldg(L.ev + 256 + ((y >> 8) & 255u)) ^
                   __ldg(L.ev + 512 + ((y >> 16) & 255u)) ^ __ldg(L.ev + 768 + (y >> 24));
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tbase)),
                     "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    const uint32_t sbar = su32(&bar);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;

    // tile-local index u (11 bits; the window at bits ws .. ws+4) -> amplitude offset in the state
    auto spread = [&](uint32_t u) -> uint32_t { return wl < 6 ? u : ((u & 63u) | ((u >> 6) << wl)); };
    auto tile_base = [&](int tile) -> uint32_t {
        if (wl < 6) return (uint32_t)tile << 11;
        const uint32_t t = (uint32_t)tile;
        return ((t & ((1u << (wl - 6)) - 1u)) << 6) | ((t >> (wl - 6)) << (wl + 5));
    };
    auto raw_of = [&](int slot) { return raw0 + slot * (kTcRawBytes / 4); };
    auto fetch = [&](int unit, int slot) {
        const int t = unit / tiles, tile = unit - t * tiles;
        const float2 *src = v.psi + ((size_t)t << n);
        const uint32_t base = tile_base(tile);
        const uint32_t dst = su32(raw_of(slot));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t u = 2u * (uint32_t)(tid + kTcThreads * j);
            cp_async16(dst + ((u >> 5) * kTcPitch + (u & 31u) * 2u) * 4u, src + (base | spread(u)));
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    // this thread's GEMM row: position r (deposited into the tile-local bits outside the window), re/im
    const int r = tid >> 1, ri = tid & 1;
    const uint32_t ur = wl < 6 ? (((uint32_t)r & ((1u << wl) - 1u)) | (((uint32_t)r >> wl) << (wl + 5))) : (uint32_t)r;
    const int apop = __popc(act);
    uint32_t phase = 0;
    bool aborted = false;
    int slot = 0;
    const int ubeg = (int)blockIdx.x * kTcChunk;
    const int uend = ubeg + kTcChunk < units ? ubeg + kTcChunk : units;
    if (ubeg < uend) fetch(ubeg, 0);
    for (int unit = ubeg; unit < uend; ++unit) {
        const int next = unit + 1;
        __syncthreads();  // the other buffer's last tile has been stored
        if (next < uend) {
            fetch(next, slot ^ 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();  // this tile is staged
        float *raw = raw_of(slot);
        const int t = unit / tiles, tile = unit - t * tiles;
        const uint32_t base = tile_base(tile);
        float x[32];
        const uint32_t y0 = base | spread(ur);  // this thread's amplitude at window pattern 0
        const uint64_t ev0 = (PRE || POST) ? tc_ev(PRE ? Lp : Lq, y0) : 0ull;
        {  // 1-2: gather, PRE, operand A
            uint64_t sv = 0;
            uint32_t zm = 0, zp0 = 0;
            if (PRE) {
                sv = Lp.s[t];
                zm = Lp.zm[t];
                zp0 = (uint32_t)__popc(y0 & zm) ^ Lp.zc[t];
            }
#pragma unroll
            for (int b = 0; b < 32; ++b) {
                const uint32_t u = ur | ((uint32_t)b << ws);
                const float2 a = *reinterpret_cast<const float2 *>(raw + (u >> 5) * kTcPitch + (u & 31u) * 2u);
                float re = a.x, im = a.y;
                if (PRE) {
                    const float2 w = tc_phase(Lp, ev0, evw[b], sv, zp0, (uint32_t)b << wl, zm);
                    const float nr = re * w.x - im * w.y, ni = re * w.y + im * w.x;
                    re = nr;
                    im = ni;
                }
                x[b] = ri ? im : re;
            }
            tc_put_row<KIND>(op0, op1, tid, x);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tc_gemm<KIND>(tmem, 0, su32(op0), su32(op1), su32(sB));
            tc_commit(sbar);
        }
        if (__syncthreads_or(!tc_wait(sbar, phase))) {
            aborted = true;
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        {  // 4: T' = D T / 32 -> operand A of the second GEMM
            tc_load32(tmem + lane_base, x);
#pragma unroll
            for (int b = 0; b < 32; ++b) {
                const float other = __shfl_xor_sync(0xffffffffu, x[b], 1);
                const float tr = ri ? other : x[b], ti = ri ? x[b] : other;
                const float2 w = dph[__popc((uint32_t)b & act)];
                x[b] = ri ? (tr * w.y + ti * w.x) : (tr * w.x - ti * w.y);
            }
            tc_put_row<KIND>(op0, op1, tid, x);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tc_gemm<KIND>(tmem, 32, su32(op0), su32(op1), su32(sB));
            tc_commit(sbar);
        }
        if (__syncthreads_or(!tc_wait(sbar, phase))) {
            aborted = true;
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        {  // 5: Z signs, POST, back to the staged tile
            tc_load32(tmem + lane_base + 32u, x);
            const uint32_t mz = Lr.mz[t], mf = Lr.mf[t];
            const uint32_t zW = (mz >> wl) & act, fW = (mf >> wl) & act;
            uint64_t sv = 0;
            uint32_t zm = 0, zp0 = 0;
            if (POST) {
                sv = Lq.s[t];
                zm = Lq.zm[t];
                zp0 = (uint32_t)__popc(y0 & zm) ^ Lq.zc[t];
            }
#pragma unroll
            for (int b = 0; b < 32; ++b) {
                float y = (__popc(((uint32_t)b ^ fW) & zW) & 1) ? -x[b] : x[b];
                const uint32_t u = ur | ((uint32_t)b << ws);
                if (POST) {
                    const float other = __shfl_xor_sync(0xffffffffu, y, 1);
                    const float re = ri ? other : y, im = ri ? y : other;
                    const float2 w = tc_phase(Lq, ev0, evw[b], sv, zp0, (uint32_t)b << wl, zm);
                    y = ri ? (re * w.y + im * w.x) : (re * w.x - im * w.y);
                }
                raw[(u >> 5) * kTcPitch + (u & 31u) * 2u + (uint32_t)ri] = y;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        {  // the tile back to the state, 16-byte stores in address order
            float4 *dst = reinterpret_cast<float4 *>(v.psi + ((size_t)t << n));
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t u = 2u * (uint32_t)(tid + kTcThreads * j);
                const float4 val = *reinterpret_cast<const float4 *>(raw + (u >> 5) * kTcPitch + (u & 31u) * 2u);
                dst[(base | spread(u)) >> 1] = val;
            }
        }
        slot ^= 1;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (aborted && tid == 0) atomicOr(v.status, 8);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

template <int KIND, bool PRE, bool POST>
cudaError_t tc_launch(const BatchView &v, const LayerView &Lp, const LayerView &Lr, const LayerView &Lq,
                      const TcSweep &sw, cudaStream_t s) {
    auto kern = k_tc_sweep<KIND, PRE, POST>;
    constexpr int smem = tc_smem_bytes<KIND>();
    static const cudaError_t attr = [&] {  // once per instantiation, on first use
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        return e;
    }();
    if (attr != cudaSuccess) return attr;
    // kTcChunk consecutive tiles per block; the hardware keeps as many blocks resident as
    // registers, shared memory and TMEM (64 of 512 columns each) admit
    const int64_t units = (int64_t)v.b << (v.n - 11);
    const int64_t blocks = (units + kTcChunk - 1) / kTcChunk;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    kern<<<(unsigned)blocks, kTcThreads, smem, s>>>(v, Lp, Lr, Lq, sw);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_sweep(const BatchView &v, const LayerView &Lp, const LayerView &Lr, const LayerView &Lq,
                            const TcSweep &sw, bool pre, bool post, int kind, cudaStream_t s) {
    if (v.n < 11 || sw.wl < 0 || sw.wl + 5 > v.n) return cudaErrorInvalidValue;
    if (kind == kPrecTF32) {
        if (pre && post) return tc_launch<kPrecTF32, true, true>(v, Lp, Lr, Lq, sw, s);
        if (pre) return tc_launch<kPrecTF32, true, false>(v, Lp, Lr, Lq, sw, s);
        if (post) return tc_launch<kPrecTF32, false, true>(v, Lp, Lr, Lq, sw, s);
        return tc_launch<kPrecTF32, false, false>(v, Lp, Lr, Lq, sw, s);
    }
    if (kind == kPrecBF16x3) {
        if (pre && post) return tc_launch<kPrecBF16x3, true, true>(v, Lp, Lr, Lq, sw, s);
        if (pre) return tc_launch<kPrecBF16x3, true, false>(v, Lp, Lr, Lq, sw, s);
        if (post) return tc_launch<kPrecBF16x3, false, true>(v, Lp, Lr, Lq, sw, s);
        return tc_launch<kPrecBF16x3, false, false>(v, Lp, Lr, Lq, sw, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace qn
