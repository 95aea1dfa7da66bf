// The exact refracted path evaluated per photon in FP32, for photons beyond
// the correction tables' domain (steeper than their largest zenith, or
// emitted above their top).  The method propagates every descending photon
// along the exact path (Sec. 3.4.3, Eq. 3.17-3.18: n(h) sin(theta(h)) is
// conserved; on the spherical shell of Sec. 3.3.4 Bouguer's n r sin(psi));
// the tables of Sec. 4.4.1 only make the common case cheap.
//
// The integrals over height are Gauss-Legendre sums (16 points) on
// sub-intervals cut at every breakpoint of n(h) (layer bottoms, the top,
// table nodes), no longer than 2 km, and shrinking geometrically (2 km,
// 200 m, 20 m) toward both ends of the path: a grazing emission makes the
// integrand steep at the top, a path nearly tangent to the ground sphere at
// the bottom.  Every integrand is written so that no FP32 subtraction of
// nearly equal numbers occurs: differences of indices are formed from n - 1,
// the spherical n r - K from small terms (below).  The routines are out of
// line and read the atmosphere through its device copy, so that the photon
// kernel's main path keeps its registers.
#pragma once

#include "device_math.cuh"

namespace cs {

// positive half of the 16-point Gauss-Legendre rule on [-1, 1] (nodes, weights)
static __constant__ float c_gl16_x[8] = {9.501250984e-02f, 2.816035508e-01f, 4.580167777e-01f, 6.178762444e-01f,
                                         7.554044084e-01f, 8.656312024e-01f, 9.445750231e-01f, 9.894009350e-01f};
static __constant__ float c_gl16_w[8] = {1.894506105e-01f, 1.826034150e-01f, 1.691565194e-01f, 1.495959888e-01f,
                                         1.246289713e-01f, 9.515851168e-02f, 6.225352394e-02f, 2.715245941e-02f};

// The next height above x (relative to h_obs) where n(h) is not smooth, or 3e38.
__device__ __forceinline__ float next_break(const AtmParams& a, float x) {
    float b = 3.0e38f;
    if (a.kind == CS_ATM_LAYERED) {
        for (int k = 1; k < a.n_layers; ++k)
            if (a.lay_lo[k] > x) b = fminf(b, a.lay_lo[k]);
        if (a.top_rel > x) b = fminf(b, a.top_rel);
    } else if (a.kind == CS_ATM_TABLE) {
        for (int k = 1; k < a.n_nodes - 1; ++k) {   // interval starts, ascending
            const float v = __ldg(a.node_lo + k);
            if (v > x) {
                b = v;
                break;
            }
        }
        if (a.top_rel > x) b = fminf(b, a.top_rel);
    } else if (a.kind == CS_ATM_LINEAR) {
        if (a.lin_top_rel > x) b = a.lin_top_rel;
    }
    return b;
}

// End of the sub-interval that starts at x on the way up to dz.
__device__ __forceinline__ float next_cut(const AtmParams& a, float x, float dz) {
    float c = fminf(x + fmaxf(2000.0f, dz * (1.0f / 128.0f)), dz);
    c = fminf(c, next_break(a, x));
    if (x < 20.0f) c = fminf(c, 20.0f);
    else if (x < 200.0f) c = fminf(c, 200.0f);
    else if (x < 2000.0f) c = fminf(c, 2000.0f);
    const float t2 = dz - 2000.0f, t1 = dz - 200.0f, t0 = dz - 20.0f;
    if (t2 > x) c = fminf(c, t2);
    else if (t1 > x) c = fminf(c, t1);
    else if (t0 > x) c = fminf(c, t0);
    return c;
}

// n - 1 on one piece between breakpoints: d(y) = a 2^(b (y - c)) (layers, table
// intervals, vacuum with a = 0) or a + b y (linear and homogeneous kinds).  The
// law is looked up once per sub-interval, at a point inside the piece.
struct PieceLaw {
    float a, b, c;
    int linear;
};
__device__ __forceinline__ PieceLaw piece_law(const AtmParams& ap, float y) {
    if (ap.kind == CS_ATM_LAYERED) {
        if (y >= ap.top_rel) return PieceLaw{0.0f, 0.0f, 0.0f, 1};
        int i = 0;
        for (int k = 1; k < ap.n_layers; ++k)
            if (y >= ap.lay_lo[k]) i = k;
        return PieceLaw{ap.lay_D[i], ap.lay_c2[i], 0.0f, 0};
    }
    if (ap.kind == CS_ATM_TABLE) {
        if (y >= ap.top_rel) return PieceLaw{0.0f, 0.0f, 0.0f, 1};
        int lo = 0, hi = ap.n_nodes - 1;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(ap.node_lo + mid) <= y) lo = mid;
            else hi = mid;
        }
        return PieceLaw{__ldg(ap.node_d + lo), __ldg(ap.node_c2 + lo), __ldg(ap.node_lo + lo), 0};
    }
    if (ap.kind == CS_ATM_LINEAR)
        return y >= ap.lin_top_rel ? PieceLaw{ap.lin_d1, 0.0f, 0.0f, 1} : PieceLaw{ap.lin_d0, ap.lin_slope, 0.0f, 1};
    return PieceLaw{ap.hom_delta, 0.0f, 0.0f, 1};
}
__device__ __forceinline__ float piece_delta(const PieceLaw& L, float y) {
    return L.linear ? fmaf(L.b, y, L.a) : L.a * exp2f(L.b * (y - L.c));
}

// One-sided limit of n - 1 from below at a breakpoint b > 0.
__device__ __forceinline__ float delta_below(const AtmParams& a, float b) {
    return delta_at(a, __int_as_float(__float_as_int(b) - 1));
}

// Planar exact path from dz above the observation level at zenith theta0
// (c0 = cos theta0 > 0) down to the observation level.  Returns the table
// fields {G_R, G_t, G_X, G_A} (normalised as the tables store them) and in
// `reaches` whether the path meets the ground: with the invariant
// s = n_e sin(theta0), q^2 = n^2 - s^2 = n_e^2 cos^2(theta0) + D,
// D = n^2 - n_e^2 = (d - d_e)(2 + d + d_e), must stay positive, which is
// checked at the ends of the pieces where n is monotone.  Integrands:
//   dR / sin(theta0) * cos(theta0) = -D / (q (n_e c0 + q))
//   c dt cos(theta0) = (n^2 c0 - q) / q = [c0^2 (2d + d^2 - d_e)(n^2 + n_e) - D] / (q (n^2 c0 + q))
//   X = 100 rho n / q,  A = exp(-h / H_A) n / q   (n = 1, q = c0 for the straight line)
__device__ __noinline__ float4 exact_fields_planar(const AtmParams* __restrict__ g, float dz, float c0, bool& reaches) {
    const AtmParams& ap = *g;
    const bool refr = ap.refraction != 0, trans = ap.transmission != 0;
    const float c2 = c0 * c0;
    const float de = refr ? delta_at(ap, dz) : 0.0f, ne = 1.0f + de;
    reaches = true;
    if (refr) {   // q^2 > 0 at the ground and on both sides of every breakpoint below dz
        auto q2_at = [&](float d) { return fmaf(ne * ne, c2, (d - de) * (2.0f + d + de)); };
        if (!(q2_at(delta_at(ap, 0.0f)) > 0.0f)) reaches = false;
        for (float b = next_break(ap, 0.0f); b < dz; b = next_break(ap, b))
            if (!(q2_at(delta_at(ap, b)) > 0.0f) || !(q2_at(delta_below(ap, b)) > 0.0f)) reaches = false;
        if (!reaches) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    float aR = 0.0f, aT = 0.0f, aX = 0.0f, aA = 0.0f;
    for (float xa = 0.0f; xa < dz;) {
        const float xb = next_cut(ap, xa, dz);
        const float mid = 0.5f * (xa + xb), half = 0.5f * (xb - xa);
        const PieceLaw law = piece_law(ap, mid);
        // unrolled: the points' special-function chains overlap (a few photons beyond the
        // tables leave one warp to integrate them, so latency, not issue, sets its time)
#pragma unroll
        for (int g = 0; g < 16; ++g) {
            const float gx = c_gl16_x[g & 7], y = (g < 8) ? fmaf(-half, gx, mid) : fmaf(half, gx, mid);
            const float wt = half * c_gl16_w[g & 7];
            const float d = piece_delta(law, y);
            if (refr) {
                const float n = 1.0f + d, n2 = n * n;
                const float D = (d - de) * (2.0f + d + de);
                const float q2 = fmaxf(fmaf(ne * ne, c2, D), 1e-30f);
                const float iq = rsqrtf(q2), q = q2 * iq;
                aR = fmaf(wt, -D * iq * rcp_approx(fmaf(ne, c0, q)), aR);
                aT = fmaf(wt, (c2 * (fmaf(d, d, 2.0f * d) - de) * (n2 + ne) - D) * iq * rcp_approx(fmaf(n2, c0, q)), aT);
                if (trans) {
                    aX = fmaf(wt, ap.rho_per_delta * d * n * iq, aX);
                    aA = fmaf(wt, ap.aer_hobs * ex2_approx(ap.aer_c2 * y) * n * iq, aA);
                }
            } else if (trans) {
                aX = fmaf(wt, ap.rho_per_delta * d, aX);
                aA = fmaf(wt, ap.aer_hobs * ex2_approx(ap.aer_c2 * y), aA);
            }
        }
        xa = xb;
    }
    if (!refr) return make_float4(0.0f, 0.0f, aX, aA);
    return make_float4(c2 * aR, aT, c0 * aX, c0 * aA);
}

// Spherical shell: n - 1 depends on the altitude y above the ground sphere
// r_g = R + h_obs; the photon starts at altitude dz with local zenith psi0
// (c0 = cos, s0 = sin).  With K = n_e r_e s0 (Bouguer) the path sweeps the
// central angle  int K / (r q) dy  and takes  c t = int n^2 r / q dy,
// q^2 = (n r - K)(n r + K).  The factor n r - K, a difference of two numbers
// near r_g, is formed from small terms: with om = 1 - s0 = c0^2 / (1 + s0),
//   n r - K = r_g om (1 + d_e) + dz om + r_g (d - d_e) + (y - dz) + d y - d_e dz s0.
// Refraction off: the straight line (n = 1, d = d_e = 0 in the geometry).
// The path meets the ground iff n r - K > 0 down to y = 0 (n r grows with r
// within each piece in any atmosphere with n - 1 below its scale height over
// the radius), checked at y = 0 and on both sides of every breakpoint.
__device__ __forceinline__ float sph_nrK(const AtmParams& ap, float y, float d, float de, float dz, float om,
                                         float s0) {
    const float rg = ap.rg;
    return fmaf(rg * om, 1.0f + de, dz * om) + fmaf(rg, d - de, y - dz) + fmaf(d, y, -de * dz * s0);
}

__device__ __noinline__ bool sph_reaches(const AtmParams* __restrict__ g, float dz, float c0, float s0) {
    const AtmParams& ap = *g;
    const float om = c0 * c0 / (1.0f + s0);
    if (!ap.refraction) return sph_nrK(ap, 0.0f, 0.0f, 0.0f, dz, om, s0) > 0.0f;
    const float de = delta_at(ap, dz);
    bool ok = sph_nrK(ap, 0.0f, delta_at(ap, 0.0f), de, dz, om, s0) > 0.0f;
    for (float b = next_break(ap, 0.0f); b < dz; b = next_break(ap, b))
        ok = ok && sph_nrK(ap, b, delta_at(ap, b), de, dz, om, s0) > 0.0f &&
             sph_nrK(ap, b, delta_below(ap, b), de, dz, om, s0) > 0.0f;
    return ok;
}

// Returns {Phi [rad], c t_path [m], G_X = X c0, G_A = A c0}; call only for
// paths that reach the ground (sph_reaches).
__device__ __noinline__ float4 exact_fields_sph(const AtmParams* __restrict__ g, float dz, float c0, float s0) {
    const AtmParams& ap = *g;
    const bool refr = ap.refraction != 0, trans = ap.transmission != 0;
    const float om = c0 * c0 / (1.0f + s0);
    const float de = refr ? delta_at(ap, dz) : 0.0f;
    const float re = ap.rg + dz, K = (1.0f + de) * re * s0;
    float aP = 0.0f, aT = 0.0f, aX = 0.0f, aA = 0.0f;
    for (float xa = 0.0f; xa < dz;) {
        const float xb = next_cut(ap, xa, dz);
        const float mid = 0.5f * (xa + xb), half = 0.5f * (xb - xa);
        const PieceLaw law = piece_law(ap, mid);
        // unrolled: the points' special-function chains overlap (a few photons beyond the
        // tables leave one warp to integrate them, so latency, not issue, sets its time)
#pragma unroll
        for (int g = 0; g < 16; ++g) {
            const float gx = c_gl16_x[g & 7], y = (g < 8) ? fmaf(-half, gx, mid) : fmaf(half, gx, mid);
            const float wt = half * c_gl16_w[g & 7];
            const float d = (refr || trans) ? piece_delta(law, y) : 0.0f;
            const float dg = refr ? d : 0.0f;   // n - 1 in the geometry
            const float r = ap.rg + y, nr = (1.0f + dg) * r;
            const float iq = rsqrtf(fmaxf(sph_nrK(ap, y, dg, de, dz, om, s0) * (nr + K), 1e-30f));
            aP = fmaf(wt, K * iq * rcp_approx(r), aP);
            aT = fmaf(wt, (1.0f + dg) * nr * iq, aT);
            if (trans) {
                aX = fmaf(wt, ap.rho_per_delta * d * nr * iq, aX);
                aA = fmaf(wt, ap.aer_hobs * ex2_approx(ap.aer_c2 * y) * nr * iq, aA);
            }
        }
        xa = xb;
    }
    return make_float4(aP, aT, c0 * aX, c0 * aA);
}

}  // namespace cs
