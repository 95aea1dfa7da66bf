// The refraction surrogate network: 3 -> 64 -> 64 -> 64 -> 3 with tanh,
// BF16 weights on the tensor cores with FP32 accumulation.  Shared by the
// training translation unit and the photon kernel's fused inference.
#pragma once

#include <cuda_bf16.h>

#include "device_math.cuh"

namespace cs {

constexpr int kHid = 64;       // hidden width
constexpr int kNIn = 3;        // (h_e, cos(theta0), 1/lambda), affine-normalised to [-1, 1]
constexpr int kNOut = 3;       // (G_R, G_t, ln T), affine-normalised
constexpr int kNOutP = 8;      // output layer padded to one 8-wide MMA tile

// Flat FP32 parameter layout (W rows are output units):
//   W1[64][3] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[8][64] b4[8]
// (rows 3..7 of W4 and b4[3..7] stay zero)
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kNIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid * kHid;
constexpr int kOffW4 = kOffB3 + kHid;
constexpr int kOffB4 = kOffW4 + kNOutP * kHid;
constexpr int kNParams = kOffB4 + kNOutP;

// BF16 copies of the tensor-core weights, [n][k] (k contiguous)
constexpr int kBOffW2 = 0;
constexpr int kBOffW3 = kBOffW2 + kHid * kHid;
constexpr int kBOffW4 = kBOffW3 + kHid * kHid;
constexpr int kNBf16 = kBOffW4 + kNOutP * kHid;

// What the photon kernel needs to evaluate the network.
struct SurrogateView {
    const float* p;             // FP32 parameters (W1, biases; W2..W4 as trained masters)
    const __nv_bfloat16* wb;    // BF16 W2, W3, W4
    int split;                  // 1: hidden activations as hi + lo BF16 pairs (two MMAs)
    // input normalisation x = in_scale * v + in_shift for v = (height coordinate,
    // cos(theta0), 1/lambda_nm); the height coordinate is dz, or exp(-dz / H)
    // when height_scale H > 0
    float in_scale[3], in_shift[3];
    float inv_height_scale;   // 1 / H, or 0 for the linear coordinate
    // output de-normalisation y = out_half * o + out_mid for (G_R, G_t, ln T)
    float out_half[3], out_mid[3];
    // domain in which the network replaces the tables
    float dz_min, dz_max, mu_min;   // mu_min = cos of the largest zenith
    // bands around the atmosphere's layer boundaries, where the exact fields
    // jump with n(h_e): heights dz in [band_lo[i], band_hi[i]) use the tables
    int n_bands;
    float band_lo[kMaxLayers], band_hi[kMaxLayers];
};

__device__ __forceinline__ float height_coordinate(const SurrogateView& sv, float dz) {
    return sv.inv_height_scale > 0.0f ? ex2_approx(-dz * sv.inv_height_scale * 1.4426950408889634f) : dz;
}

__device__ __forceinline__ bool in_surrogate_domain(const SurrogateView& sv, float dz, float mu) {
    bool ok = dz >= sv.dz_min && dz <= sv.dz_max && mu >= sv.mu_min;
#pragma unroll
    for (int i = 0; i < kMaxLayers; ++i)
        if (i < sv.n_bands && dz >= sv.band_lo[i] && dz < sv.band_hi[i]) ok = false;
    return ok;
}

// The trained network's view (defined with the training code).
const SurrogateView* surrogate_view(const cs_surrogate* s);

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// D += A B for one m16n8k16 tile (BF16 inputs, FP32 accumulation).
__device__ __forceinline__ void mma_16816(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                          uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// tanh(x) = 1 - 2 / (exp(2x) + 1) from ex2 and rcp approximations: absolute
// error about 2e-7 (the hardware tanh approximation is ~5e-4 relative, too
// coarse for the network's error budget).  Used in training and inference.
__device__ __forceinline__ float tanh_act(float x) {
    const float e = ex2_approx(x * 2.8853900817779268f);   // exp(2x)
    return fmaf(-2.0f, rcp_approx(e + 1.0f), 1.0f);
}

// One hidden layer on 16 rows held in the C-fragment layout of m16n8 tiles:
// lane (g = lane / 4, q = lane % 4) holds rows g and g + 8, columns
// 8 j + 2 q + {0, 1} of each of the 8 column tiles j.  The same registers
// are the A fragments of the next layer, so activations never leave the warp.
// h_in/h_out: [8 tiles][4] floats.
template <bool SPLIT, bool TANH>
__device__ __forceinline__ void hidden_layer(const float (&h_in)[8][4], float (&h_out)[8][4],
                                             const __nv_bfloat16* __restrict__ W, const float* __restrict__ b,
                                             int n_tiles) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    uint32_t ahi[4][4], alo[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {   // k chunk kk covers input columns 16 kk .. 16 kk + 15
        const float* lo_t = h_in[2 * kk];
        const float* hi_t = h_in[2 * kk + 1];
        const float v[8] = {lo_t[0], lo_t[1], lo_t[2], lo_t[3], hi_t[0], hi_t[1], hi_t[2], hi_t[3]};
        // registers: {row g, k 2q..}, {row g+8, k 2q..}, {row g, k 8+2q..}, {row g+8, k 8+2q..}
        const int order[4][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float x0 = v[order[r][0]], x1 = v[order[r][1]];
            ahi[kk][r] = pack_bf16x2(x0, x1);
            if (SPLIT) {
                const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&ahi[kk][r]);
                alo[kk][r] = pack_bf16x2(x0 - __low2float(h), x1 - __high2float(h));
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j >= n_tiles) break;
        const float b0 = __ldg(b + 8 * j + 2 * q), b1 = __ldg(b + 8 * j + 2 * q + 1);
        float acc[4] = {b0, b1, b0, b1};
        const __nv_bfloat16* wrow = W + (size_t)(8 * j + g) * kHid + 2 * q;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint32_t w0 = __ldg(reinterpret_cast<const unsigned int*>(wrow + 16 * kk));
            const uint32_t w1 = __ldg(reinterpret_cast<const unsigned int*>(wrow + 16 * kk + 8));
            mma_16816(acc, ahi[kk][0], ahi[kk][1], ahi[kk][2], ahi[kk][3], w0, w1);
            if (SPLIT) mma_16816(acc, alo[kk][0], alo[kk][1], alo[kk][2], alo[kk][3], w0, w1);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) h_out[j][r] = TANH ? tanh_act(acc[r]) : acc[r];
    }
}

// The network on 16 rows whose normalised inputs are x_g (row g) and x_g8
// (row g + 8) in this lane.  Returns the normalised outputs of rows g and
// g + 8 for columns 2q, 2q + 1 in out[0..1] (row g) and out[2..3] (row g + 8).
template <bool SPLIT>
__device__ __forceinline__ void net16(const SurrogateView& sv, const float (&x_g)[3], const float (&x_g8)[3],
                                      float (&out)[4]) {
    const int lane = threadIdx.x & 31, q = lane & 3;
    const float* p = sv.p;
    float h1[8][4], h2[8][4];
    // layer 1 (3 inputs): FP32 on the CUDA cores
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int u = 8 * j + 2 * q + c;
            const float w0 = __ldg(p + kOffW1 + u * 3), w1 = __ldg(p + kOffW1 + u * 3 + 1),
                        w2 = __ldg(p + kOffW1 + u * 3 + 2), bb = __ldg(p + kOffB1 + u);
            h1[j][c] = tanh_act(fmaf(w2, x_g[2], fmaf(w1, x_g[1], fmaf(w0, x_g[0], bb))));
            h1[j][2 + c] = tanh_act(fmaf(w2, x_g8[2], fmaf(w1, x_g8[1], fmaf(w0, x_g8[0], bb))));
        }
    }
    hidden_layer<SPLIT, true>(h1, h2, sv.wb + kBOffW2, p + kOffB2, 8);
    hidden_layer<SPLIT, true>(h2, h1, sv.wb + kBOffW3, p + kOffB3, 8);
    hidden_layer<SPLIT, false>(h1, h2, sv.wb + kBOffW4, p + kOffB4, 1);
#pragma unroll
    for (int r = 0; r < 4; ++r) out[r] = h2[0][r];
}

// The network on the 32 photons of a warp, one per lane: x holds this lane's
// normalised inputs, y receives its normalised outputs.  Every lane must call.
template <bool SPLIT>
__device__ __forceinline__ void net32(const SurrogateView& sv, const float (&x)[3], float (&y)[3]) {
    const int lane = threadIdx.x & 31, g = lane >> 2;
#pragma unroll
    for (int grp = 0; grp < 2; ++grp) {   // rows of group grp are lanes 16 grp .. 16 grp + 15
        float xg[3], xg8[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            xg[k] = __shfl_sync(0xffffffffu, x[k], 16 * grp + g);
            xg8[k] = __shfl_sync(0xffffffffu, x[k], 16 * grp + g + 8);
        }
        float o[4];
        net16<SPLIT>(sv, xg, xg8, o);
        // row r of the group (lane 16 grp + r) sits in lane 4 (r % 8) + (column / 2)
        const int r = lane - 16 * grp;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int src = 4 * (r & 7) + (k >> 1);
            const float lo = __shfl_sync(0xffffffffu, o[k & 1], src);
            const float hi = __shfl_sync(0xffffffffu, o[2 + (k & 1)], src);
            if (r >= 0 && r < 16) y[k] = r < 8 ? lo : hi;
        }
    }
}

}  // namespace cs
