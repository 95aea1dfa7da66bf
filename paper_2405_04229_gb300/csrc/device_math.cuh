// Device-side building blocks of the photon kernels: the counter-based RNG,
// float-float helpers, the closed-form refractive index, a sin/cos of 2 pi u
// and approximate transcendental wrappers.
#pragma once

#include "common.cuh"

namespace cs {

constexpr float kInvC = (float)(1.0 / kC);

// Philox4x32-10 (Salmon et al., SC'11): per round two 32x32 -> 64 multiplies,
// the Weyl key schedule between rounds.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                        uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        // one 32 x 32 -> 64 multiply each (a single wide integer multiply-add)
        const unsigned long long p0 = 0xD2511F53ull * c0, p1 = 0xCD9E8D57ull * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// The same rounds with the key schedule precomputed (rk[2r], rk[2r + 1] = the
// round-r keys): kernel-parameter keys become constant operands of the XORs.
__device__ __forceinline__ uint4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const uint32_t* rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = 0xD2511F53ull * c0, p1 = 0xCD9E8D57ull * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r], n2 = hi0 ^ c3 ^ rk[2 * r + 1];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// 24-bit uniform in [0, 1), exact in FP32 and FP64
__device__ __forceinline__ float uniform24(uint32_t x) { return __uint2float_rn(x >> 8) * 0x1p-24f; }

// ---- float-float (error-free transformations) ------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// finiteness of a double from its exponent bits
__device__ __forceinline__ bool finite_f64(double d) {
    return ((unsigned long long)__double_as_longlong(d) & 0x7FF0000000000000ull) != 0x7FF0000000000000ull;
}

// hi = d rounded to the nearest float (ties to even), lo = d - hi rounded to
// float: the float-float split of a double, taken from its bits with integer
// operations (the FP64 pipe of this GPU is narrow).  The same values as
// hi = (float)d, lo = (float)(d - (double)hi); |d| outside [2^-74, 2^127)
// and non-finite values take that conversion path.
__device__ __forceinline__ void split_f64(double d, float& hi, float& lo) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((u >> 52) & 0x7FF);
    if (e < 949 || e > 1149) {
        hi = (float)d;
        lo = (float)(d - (double)hi);
        return;
    }
    const unsigned int sign = (unsigned int)(u >> 32) & 0x80000000u;
    const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    const unsigned int mh = (unsigned int)(m >> 29), rem = (unsigned int)m & 0x1FFFFFFFu;
    const unsigned int up = (rem > 0x10000000u || (rem == 0x10000000u && (mh & 1u))) ? 1u : 0u;
    hi = __uint_as_float(sign | ((((unsigned int)(e - 1023 + 127)) << 23) + mh + up));
    const int r = (int)rem - (up ? 0x20000000 : 0);
    const float scale = __uint_as_float((unsigned int)(e - 1075 + 127) << 23);   // 2^(e - 1075)
    const float l = __int2float_rn(r) * scale;
    lo = sign ? -l : l;
}

// floor(s + t) for |t| below one ulp of s
__device__ __forceinline__ int ff_floor(float s, float t) {
    const float f = floorf(s);
    int i = (int)f;
    if (t >= (f + 1.0f) - s) i += 1;
    else if (s == f && t < 0.0f) i -= 1;
    return i;
}

// (a_hi + a_lo) * m as float-float
__device__ __forceinline__ void ff_scale(float a_hi, float a_lo, float m, float& hi, float& lo) {
    hi = a_hi * m;
    lo = fmaf(a_hi, m, -hi) + a_lo * m;
    float s, e;
    two_sum(hi, lo, s, e);
    hi = s;
    lo = e;
}

// ---- approximate transcendental functions (PTX .approx forms) -------------
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sin and cos of 2 pi u for u in [0, 1): exact quadrant reduction of 4u and
// Taylor polynomials on |x| <= pi/4 (truncation below 3e-8).
__device__ __forceinline__ void sincos_2pi(float u, float& s, float& c) {
    const float v = 4.0f * u;                    // exact
    const float q = rintf(v);
    const float x = (v - q) * 1.57079632679489662f;   // |x| <= pi/4
    const float x2 = x * x;
    // the sine (odd) and cosine (even) Horner chains side by side, two lanes per
    // packed FP32 instruction: (1/9!, 1/8!), (-1/7!, -1/6!), (1/5!, 1/4!), (-1/3!, -1/2!)
    const float2 xx = make_float2(x2, x2);
    float2 p = __ffma2_rn(xx, make_float2(2.75573192e-6f, 2.48015873e-5f), make_float2(-1.98412698e-4f, -1.38888889e-3f));
    p = __ffma2_rn(xx, p, make_float2(8.33333333e-3f, 4.16666667e-2f));
    p = __ffma2_rn(xx, p, make_float2(-1.66666667e-1f, -0.5f));
    const float2 r = __ffma2_rn(make_float2(x * x2, x2), p, make_float2(x, 1.0f));
    const float sx = r.x, cx = r.y;
    const int qi = ((int)q) & 3;
    s = (qi == 0) ? sx : (qi == 1) ? cx : (qi == 2) ? -sx : -cx;
    c = (qi == 0) ? cx : (qi == 1) ? -sx : (qi == 2) ? -cx : sx;
}

// ---- refractive index n - 1 at dz above the observation level --------------
// closed form per layer (half-open layers [h_i, h_i+1)), FP32
__device__ __forceinline__ float delta_at(const AtmParams& a, float dz) {
    if (a.kind == CS_ATM_LAYERED) {
        if (dz >= a.top_rel) return 0.0f;
        // the layer's constants picked by selects over the unrolled layers (constant
        // operands, no indexed parameter loads)
        float D = a.lay_D[0], c2 = a.lay_c2[0];
#pragma unroll
        for (int k = 1; k < kMaxLayers; ++k)
            if (k < a.n_layers && dz >= a.lay_lo[k]) {
                D = a.lay_D[k];
                c2 = a.lay_c2[k];
            }
        return D * exp2f(c2 * dz);
    }
    if (a.kind == CS_ATM_LINEAR) return dz >= a.lin_top_rel ? a.lin_d1 : a.lin_d0 + a.lin_slope * dz;
    if (a.kind == CS_ATM_TABLE) {
        if (dz >= a.top_rel) return 0.0f;
        int lo = 0, hi = a.n_nodes - 1;   // interval: largest i < n - 1 with node_lo[i] <= dz
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(a.node_lo + mid) <= dz) lo = mid;
            else hi = mid;
        }
        return __ldg(a.node_d + lo) * exp2f(__ldg(a.node_c2 + lo) * (dz - __ldg(a.node_lo + lo)));
    }
    return a.hom_delta;
}

}  // namespace cs
