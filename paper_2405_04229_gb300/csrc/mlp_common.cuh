// The refraction surrogate network: 3 -> 64 -> 64 -> 64 -> 3 with tanh,
// BF16 weights on the tensor cores with FP32 accumulation.  Shared by the
// training translation unit (warp-level mma.sync GEMMs) and the inference
// (tcgen05, mlp_tc.cuh).
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

}  // namespace cs
