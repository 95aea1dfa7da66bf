// The surrogate network on the fifth-generation tensor cores: a warpgroup
// (128 threads, one photon per thread) evaluates 3 -> 64 -> 64 -> 64 -> 3.
// Layer 1 (3 inputs) runs on the CUDA cores; layers 2-4 are single-CTA
// tcgen05 MMAs (M = 128, K = 64 as four K = 16 steps, BF16 operands in shared
// memory in the no-swizzle K-major core-matrix layout, FP32 accumulators in
// tensor memory).  The accumulators come back with tcgen05.ld for the bias
// and tanh epilogue, which writes the next layer's operand -- the activation
// as a BF16 hi + lo pair, two MMAs per step -- back to shared memory.
#pragma once

#include "mlp_common.cuh"

namespace cs {

constexpr int kTcRows = 128;                         // rows per warpgroup tile
constexpr int kTcATile = kTcRows * kHid * 2;         // one BF16 A tile: 16 KB
constexpr int kTcW2 = 0, kTcW3 = kHid * kHid * 2, kTcW4 = 2 * kHid * kHid * 2;
constexpr int kTcN4 = 16;                            // output layer padded to the smallest MMA width
constexpr int kTcWBytes = kTcW4 + kTcN4 * kHid * 2;  // W2 | W3 | W4: 18 KB
constexpr int kTcSpin = 1 << 20;                     // polls of an MMA completion before giving up

// Shared memory of the tensor-core network, per CTA of NWG warpgroups; the
// CTA holds NWG x 64 tensor-memory columns (64 FP32 accumulators per row).
template <int NWG>
struct TcSmem {
    static_assert(NWG == 2 || NWG == 4, "tensor-memory allocations are powers of two >= 32 columns");
    static constexpr unsigned int kCols = 64 * NWG;
    __align__(128) unsigned char a[NWG][2][kTcATile];  // [warpgroup][hi, lo] activations
    __align__(128) unsigned char w[kTcWBytes];         // BF16 weights, core-matrix layout
    float4 w1p[kHid / 2][2];                           // layer 1, units 2i and 2i + 1 side by side:
                                                       // {W1[.][0], W1[.][1]}, {W1[.][2], b1[.]}
    float4 b23[2][kHid / 4];                           // biases of layers 2 and 3
    float b4[4];
    unsigned long long mbar[NWG];                      // MMA completion, per warpgroup
    unsigned int tmem_base;
    int abort[NWG];                                    // a wait ran out (per warpgroup)
    unsigned int phase[NWG];                           // parity of the next completion
};

// Set when a tensor-core wait ran out (one flag per translation unit); read
// and cleared by that unit's host calls through tc_take_timeout().
static __device__ unsigned int g_tc_timeout = 0;

static inline bool tc_take_timeout() {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof v) != cudaSuccess) return false;
    if (v) {
        const unsigned int z = 0;
        cudaMemcpyToSymbol(g_tc_timeout, &z, sizeof z);
    }
    return v != 0;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N)
// byte offsets, the fixed 0b001 field, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M = 128.
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

// Byte offset of element (r, k) in a K-major no-swizzle tile of `rows` rows:
// 8 x 16-byte core matrices, consecutive rows 16 bytes apart, K groups of 8
// elements rows * 16 bytes apart.
__host__ __device__ constexpr int tc_off(int r, int k, int rows) { return (k >> 3) * rows * 16 + r * 16 + (k & 7) * 2; }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void wg_barrier(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_polls(uint32_t a, uint32_t parity, int polls) {
    for (int it = 0; it < polls; ++it)
        if (mbar_try_wait(a, parity)) return true;
    return false;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t a, uint32_t parity) { return mbar_wait_polls(a, parity, kTcSpin); }

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    // the registers are defined once the load has completed: make the wait their producer
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])::"memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tc_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3])::"memory");
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}

// tanh of two pre-activations, rounded to BF16 first, by the hardware's packed
// BF16 approximation: the single-BF16 inference path (the network's part of
// the fields is a small correction to the first-order baseline, so a BF16
// activation's resolution suffices there).
__device__ __forceinline__ uint32_t tanh_bf16x2(float lo, float hi) {
    uint32_t r, v = pack_bf16x2(lo, hi);
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(r) : "r"(v));
    return r;
}

// Eight pre-activations of one row (K group g) through the packed tanh into the A tile.
__device__ __forceinline__ void tc_tanh_store8(unsigned char* a, int row, int g, const float (&z)[8]) {
    const int off = tc_off(row, 8 * g, kTcRows);
    *reinterpret_cast<uint4*>(a + off) =
        make_uint4(tanh_bf16x2(z[0], z[1]), tanh_bf16x2(z[2], z[3]), tanh_bf16x2(z[4], z[5]), tanh_bf16x2(z[6], z[7]));
}

// Eight activations of one row (K group g) as BF16 hi (+ lo) into the A tiles.
template <bool SPLIT>
__device__ __forceinline__ void tc_store8(unsigned char* a_hi, unsigned char* a_lo, int row, int g, const float (&h)[8]) {
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        hi[j] = pack_bf16x2(h[2 * j], h[2 * j + 1]);
        if (SPLIT) {
            const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&hi[j]);
            lo[j] = pack_bf16x2(h[2 * j] - __low2float(b), h[2 * j + 1] - __high2float(b));
        }
    }
    const int off = tc_off(row, 8 * g, kTcRows);
    *reinterpret_cast<uint4*>(a_hi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    if (SPLIT) *reinterpret_cast<uint4*>(a_lo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

// Per-CTA set-up (all threads): tensor memory, completion barriers, weights.
template <int NWG>
__device__ __forceinline__ void tc_setup(TcSmem<NWG>& T, const SurrogateView& sv) {
    const int t = threadIdx.x;
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&T.tmem_base)),
                     "r"(TcSmem<NWG>::kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        for (int wg = 0; wg < NWG; ++wg) {
            mbar_init(smem_u32(&T.mbar[wg]), 1);
            T.abort[wg] = 0;
            T.phase[wg] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // weights: global [n][k] rows of 64 BF16 -> core-matrix layout, 16 bytes at a time
    const uint4* src = reinterpret_cast<const uint4*>(sv.wb);
    for (int i = t; i < (2 * kHid + kTcN4) * (kHid / 8); i += blockDim.x) {
        const int n = i / (kHid / 8), g = i % (kHid / 8);   // row n of W2 | W3 | W4, K group g
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        int dst;
        if (n < kHid) {
            v = __ldg(src + (size_t)(kBOffW2 / 8) + n * (kHid / 8) + g);
            dst = kTcW2 + tc_off(n, 8 * g, kHid);
        } else if (n < 2 * kHid) {
            v = __ldg(src + (size_t)(kBOffW3 / 8) + (n - kHid) * (kHid / 8) + g);
            dst = kTcW3 + tc_off(n - kHid, 8 * g, kHid);
        } else {
            const int r = n - 2 * kHid;
            if (r < kNOutP) v = __ldg(src + (size_t)(kBOffW4 / 8) + r * (kHid / 8) + g);
            dst = kTcW4 + tc_off(r, 8 * g, kTcN4);
        }
        *reinterpret_cast<uint4*>(T.w + dst) = v;
    }
    const float* p = sv.p;
    for (int i = t; i < kHid / 2; i += blockDim.x) {
        const int u = 2 * i, v = u + 1;
        T.w1p[i][0] = make_float4(p[kOffW1 + 3 * u], p[kOffW1 + 3 * v], p[kOffW1 + 3 * u + 1], p[kOffW1 + 3 * v + 1]);
        T.w1p[i][1] = make_float4(p[kOffW1 + 3 * u + 2], p[kOffW1 + 3 * v + 2], p[kOffB1 + u], p[kOffB1 + v]);
    }
    for (int i = t; i < 2 * kHid; i += blockDim.x)
        reinterpret_cast<float*>(T.b23)[i] = p[(i < kHid ? kOffB2 : kOffB3 - kHid) + i];
    if (t < 4) T.b4[t] = t < kNOut ? p[kOffB4 + t] : 0.0f;
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Per-CTA tear-down (all threads): after a wait that ran out, give the
// outstanding MMAs a bounded chance to finish; then free the tensor memory.
template <int NWG>
__device__ __forceinline__ void tc_teardown(TcSmem<NWG>& T) {
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int wg = 0; wg < NWG; ++wg)
            if (T.abort[wg]) {
                mbar_wait_bounded(smem_u32(&T.mbar[wg]), T.phase[wg]);
                atomicOr(&g_tc_timeout, 1u);
            }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(T.tmem_base),
                     "r"(TcSmem<NWG>::kCols)
                     : "memory");
    }
}

// The network on the 128 rows of warpgroup wg (row = thread index within the
// warpgroup): normalised inputs x in, normalised outputs y out.  All 128
// threads of the warpgroup call it together.  Returns false (outputs zero)
// once a wait of this warpgroup has run out.
template <bool SPLIT, int NWG>
__device__ __forceinline__ bool net128_tc(const SurrogateView& sv, TcSmem<NWG>& T, const float (&x)[3], float (&y)[3]) {
    const int wg = threadIdx.x >> 7, row = threadIdx.x & 127;
    y[0] = y[1] = y[2] = 0.0f;
    if (T.abort[wg]) return false;   // uniform: set before one of this warpgroup's barriers
    unsigned char* a_hi = T.a[wg][0];
    unsigned char* a_lo = T.a[wg][1];
    // layer 1 (3 inputs): FP32 on the CUDA cores
#pragma unroll 1
    for (int g = 0; g < 8; ++g) {
        float h[8];
        // two units per packed FP32 instruction (the same fused operations in the same order)
        const float2 x0 = make_float2(x[0], x[0]), x1 = make_float2(x[1], x[1]), x2 = make_float2(x[2], x[2]);
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            const float4 wa = T.w1p[(8 * g + j) >> 1][0], wb = T.w1p[(8 * g + j) >> 1][1];
            float2 z = __ffma2_rn(make_float2(wa.x, wa.y), x0, make_float2(wb.z, wb.w));
            z = __ffma2_rn(make_float2(wa.z, wa.w), x1, z);
            z = __ffma2_rn(make_float2(wb.x, wb.y), x2, z);
            h[j] = z.x;
            h[j + 1] = z.y;
        }
        if (SPLIT) {
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = tanh_act(h[j]);
        }
        if (SPLIT) tc_store8<true>(a_hi, a_lo, row, g, h);
        else tc_tanh_store8(a_hi, row, g, h);
    }
    const uint32_t d_tmem = T.tmem_base + (uint32_t)(wg * kHid);
    const uint32_t t_lane = d_tmem + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16);
    const uint32_t mbar = smem_u32(&T.mbar[wg]);
#pragma unroll 1
    for (int L = 0; L < 3; ++L) {
        // the operand tile is complete and earlier reads of the accumulators are done
        fence_async_smem();
        tc_fence_before();
        wg_barrier(1 + wg);
        if (row == 0) {
            tc_fence_after();
            const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo);
            const int rows_b = L == 2 ? kTcN4 : kHid;
            const uint32_t wb = smem_u32(T.w) + (uint32_t)(L == 0 ? kTcW2 : L == 1 ? kTcW3 : kTcW4);
            const uint32_t lbo_b = (uint32_t)rows_b * 16, idesc = tc_idesc(rows_b);
#pragma unroll
            for (int s = 0; s < kHid / 16; ++s) {   // K = 16 per MMA: two K groups
                const uint64_t bd = tc_desc(wb + (uint32_t)s * 2 * lbo_b, lbo_b, 128);
                tc_mma(d_tmem, tc_desc(ah + (uint32_t)s * 2 * kTcRows * 16, kTcRows * 16, 128), bd, idesc, s > 0);
                if (SPLIT) tc_mma(d_tmem, tc_desc(al + (uint32_t)s * 2 * kTcRows * 16, kTcRows * 16, 128), bd, idesc, 1);
            }
            tc_commit(mbar);
        }
        const bool done = mbar_wait_polls(mbar, T.phase[wg], sv.polls);
        if (!done) T.abort[wg] = 1;
        wg_barrier(1 + wg);   // every thread has seen the completion, or the give-up
        if (row == 0 && done) T.phase[wg] ^= 1u;
        if (T.abort[wg]) return false;
        tc_fence_after();
        if (L < 2) {
            const float4* bias = T.b23[L];
#pragma unroll 1
            for (int c = 0; c < kHid / 16; ++c) {
                float v[16];
                tc_ld16(t_lane + (uint32_t)(16 * c), v);
                float h0[8], h1[8];
#pragma unroll
                for (int q = 0; q < 2; ++q) {   // bias adds two per packed FP32 instruction
                    const float4 b0 = bias[4 * c + q], b1 = bias[4 * c + 2 + q];
                    float2 z;
                    z = __fadd2_rn(make_float2(v[4 * q + 0], v[4 * q + 1]), make_float2(b0.x, b0.y));
                    h0[4 * q + 0] = z.x;
                    h0[4 * q + 1] = z.y;
                    z = __fadd2_rn(make_float2(v[4 * q + 2], v[4 * q + 3]), make_float2(b0.z, b0.w));
                    h0[4 * q + 2] = z.x;
                    h0[4 * q + 3] = z.y;
                    z = __fadd2_rn(make_float2(v[8 + 4 * q + 0], v[8 + 4 * q + 1]), make_float2(b1.x, b1.y));
                    h1[4 * q + 0] = z.x;
                    h1[4 * q + 1] = z.y;
                    z = __fadd2_rn(make_float2(v[8 + 4 * q + 2], v[8 + 4 * q + 3]), make_float2(b1.z, b1.w));
                    h1[4 * q + 2] = z.x;
                    h1[4 * q + 3] = z.y;
                }
                if (SPLIT) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        h0[j] = tanh_act(h0[j]);
                        h1[j] = tanh_act(h1[j]);
                    }
                    tc_store8<true>(a_hi, a_lo, row, 2 * c, h0);
                    tc_store8<true>(a_hi, a_lo, row, 2 * c + 1, h1);
                } else {
                    tc_tanh_store8(a_hi, row, 2 * c, h0);
                    tc_tanh_store8(a_hi, row, 2 * c + 1, h1);
                }
            }
        } else {
            float v[4];
            tc_ld4(t_lane, v);
#pragma unroll
            for (int k = 0; k < 3; ++k) y[k] = v[k] + T.b4[k];
        }
    }
    tc_fence_before();   // these accumulator reads precede the next call's MMAs (its barrier)
    return true;
}

}  // namespace cs
