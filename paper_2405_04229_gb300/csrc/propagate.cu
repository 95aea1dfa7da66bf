// The fused generation + propagation kernel (thesis Sec. 5.3): per tile of
// segments a block imports and filters the segments, computes the sub-step
// yields, generates the photon bunches on their Cherenkov cones, drops
// upward photons, projects them to the observation level, applies the
// refraction/time correction tables and the transmission test, and bins
// them into the ground histogram and telescope counters.  The stages share
// data through shared memory and are separated by block barriers only.
//
// Precision plan: bulk arithmetic in FP32.  Each segment gets a local origin,
// the ground intercept G of its own straight line, computed once in
// float-float; a photon's ground point is G plus a residual proportional to
// the small angle between the photon and the segment, so FP32 rounding acts
// on that residual only.  FP64 is used per segment to split the input
// coordinates and for the absolute arrival times accumulated per telescope.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace cs {
namespace {

constexpr int kThreads = 256;
constexpr int kTile = kThreads;      // segments per tile, one per thread
constexpr int kSubCap = 1024;        // sub-steps per round
constexpr int kSubPerThread = kSubCap / kThreads;
constexpr float kInvC = (float)(1.0 / kC);

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al. 2011): two 32x32 multiplies per round, Weyl
// key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                        uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ float uniform24(uint32_t x) { return __uint2float_rn(x >> 8) * 0x1p-24f; }

// ---------------------------------------------------------------------------
// float-float helpers (error-free transformations)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// floor(s + t) for |t| below one ulp of s
__device__ __forceinline__ int ff_floor(float s, float t) {
    const float f = floorf(s);
    int i = (int)f;
    if (t >= (f + 1.0f) - s) i += 1;
    else if (s == f && t < 0.0f) i -= 1;
    return i;
}

// value (hi, lo) = (a_hi + a_lo) * m as float-float
__device__ __forceinline__ void ff_scale(float a_hi, float a_lo, float m, float& hi, float& lo) {
    hi = a_hi * m;
    lo = fmaf(a_hi, m, -hi) + a_lo * m;
    float s, e;
    two_sum(hi, lo, s, e);
    hi = s;
    lo = e;
}

// ---------------------------------------------------------------------------
// Refractive index n - 1 at height dz above the observation level (closed
// form per layer, FP32).  Layers are half-open [h_i, h_i+1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float delta_at(const AtmParams& a, float dz) {
    if (a.kind == CS_ATM_LAYERED) {
        if (dz >= a.top_rel) return 0.0f;
        int i = 0;
#pragma unroll
        for (int k = 1; k < kMaxLayers; ++k)
            if (k < a.n_layers && dz >= a.lay_lo[k]) i = k;
        return a.lay_D[i] * exp2f(a.lay_c2[i] * dz);
    }
    if (a.kind == CS_ATM_LINEAR) return dz >= a.lin_top_rel ? a.lin_d1 : a.lin_d0 + a.lin_slope * dz;
    return a.hom_delta;
}

// Per-tile shared memory: the imported segments (structure of arrays) and one
// round of sub-steps.
struct TileSmem {
    float Px[kTile], Py[kTile], Pz[kTile], inv1mPz[kTile];
    float Hs_hi[kTile], Hs_lo[kTile], LoverK[kTile];
    float g[kTile], z2[kTile], inv_betac[kTile];
    float Gx_hi[kTile], Gx_lo[kTile], Gy_hi[kTile], Gy_lo[kTile];   // ground intercept, frame [m]
    float Cx_hi[kTile], Cx_lo[kTile], Cy_hi[kTile], Cy_lo[kTile];   // ground intercept, hist cells
    double t0[kTile];
    int shower[kTile];
    int offK[kTile + 1];
    // sub-steps of the current round
    int q_seg[kSubCap];
    int q_k[kSubCap];
    float q_cos[kSubCap], q_sin[kSubCap], q_delta[kSubCap];
    int offN[kSubCap + 1];
    int wsum[kThreads / 32];
    unsigned int cnt[CS_N_COUNTERS];
};

// Exclusive block scan of one int per thread; returns the prefix, *total the sum.
__device__ __forceinline__ int block_scan(int v, int* wsum, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < kThreads / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kThreads / 32) wsum[lane] = s;
    }
    __syncthreads();
    const int pre = (wid ? wsum[wid - 1] : 0) + x - v;
    *total = wsum[kThreads / 32 - 1];
    __syncthreads();
    return pre;
}

__device__ __forceinline__ void emit_record(const OutParams& o, unsigned long long seg, int k, int i, float x,
                                            float y, float t_rel, float inv_l, int tel, int bin, int status) {
    const unsigned long long slot = atomicAdd(o.record_count, 1ULL);
    if (slot < o.record_capacity) {
        cs_record r;
        r.seg = seg;
        r.k = (uint32_t)k;
        r.i = (uint32_t)i;
        r.x = x;
        r.y = y;
        r.dt_ns = t_rel * 1e9f;
        r.lambda_nm = 1.0f / inv_l;
        r.tel = tel;
        r.bin = bin;
        r.status = (uint32_t)status;
        r.reserved = 0;
        o.records[slot] = r;
    }
}

__global__ void __launch_bounds__(kThreads)
propagate_kernel(const PropParams pp, const AtmParams ap, const DetParams dp, const OutParams op) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem& S = *reinterpret_cast<TileSmem*>(smem_raw);
    const int t = threadIdx.x;
    const unsigned int bu = (unsigned int)pp.bunch;
    const float inv_b = 1.0f / (float)pp.bunch;
    const bool want_records = op.records != nullptr;

    for (long long tile = blockIdx.x; tile * kTile < pp.n; tile += gridDim.x) {
        const long long base = tile * kTile;
        unsigned int cnt[CS_N_COUNTERS];
#pragma unroll
        for (int c = 0; c < CS_N_COUNTERS; ++c) cnt[c] = 0;

        // ---- stage 1: import and filter (Sec. 5.3.1) --------------------------
        int Kt = 0;
        const long long idx = base + t;
        if (idx < pp.n) {
            const double2* src = reinterpret_cast<const double2*>(pp.segs + idx);
            const double2 xy = __ldg(src), zt = __ldg(src + 1);
            const float4 dir = __ldg(reinterpret_cast<const float4*>(src + 2));
            const uint4 rest = __ldg(reinterpret_cast<const uint4*>(src + 3));
            const float g = __uint_as_float(rest.x), z = __uint_as_float(rest.y);
            const unsigned int shower = rest.z;
            const float n2 = dir.x * dir.x + dir.y * dir.y + dir.z * dir.z;
            const bool valid = isfinite(xy.x) && isfinite(xy.y) && isfinite(zt.x) && isfinite(zt.y) &&
                               isfinite(dir.x) && isfinite(dir.y) && isfinite(dir.z) && isfinite(dir.w) &&
                               dir.w > 0.0f && g > 0.0f && g < 1.0f && isfinite(z) && dir.z < 0.99f &&
                               fabsf(n2 - 1.0f) <= 1e-4f && shower < (unsigned int)dp.n_showers;
            if (!valid) {
                cnt[CS_CNT_INVALID_SEGMENTS] += 1;
            } else {
                const float inv_n = rsqrtf(n2);
                const float Px = dir.x * inv_n, Py = dir.y * inv_n, Pz = dir.z * inv_n;
                const float L = dir.w;
                Kt = max(1, (int)ceilf(L / pp.s_max));
                S.Px[t] = Px;
                S.Py[t] = Py;
                S.Pz[t] = Pz;
                S.inv1mPz[t] = 1.0f / (1.0f - Pz);
                S.LoverK[t] = L / (float)Kt;
                S.g[t] = g;
                S.z2[t] = z * z;
                S.inv_betac[t] = rsqrtf(1.0f - g) * kInvC;
                S.t0[t] = zt.y;
                S.shower[t] = (int)shower;
                // local origin: Hs = z0 - h_obs and G = S_xy - Hs P_xy / P_z (float-float)
                const double Hs = zt.x - ap.h_obs;
                const float Hs_hi = (float)Hs, Hs_lo = (float)(Hs - (double)Hs_hi);
                S.Hs_hi[t] = Hs_hi;
                S.Hs_lo[t] = Hs_lo;
                const float x_hi = (float)xy.x, x_lo = (float)(xy.x - (double)x_hi);
                const float y_hi = (float)xy.y, y_lo = (float)(xy.y - (double)y_hi);
                float Gxh = x_hi, Gxl = x_lo, Gyh = y_hi, Gyl = y_lo;
                if (Pz < -1e-3f) {
                    // slopes P_x / P_z as float-float via the FMA remainder
                    const float sx = Px / Pz, sy = Py / Pz;
                    const float sx_l = fmaf(-sx, Pz, Px) / Pz, sy_l = fmaf(-sy, Pz, Py) / Pz;
                    // Hs * slope as float-float
                    const float px = Hs_hi * sx, py = Hs_hi * sy;
                    const float px_l = fmaf(Hs_hi, sx, -px) + (Hs_hi * sx_l + Hs_lo * sx);
                    const float py_l = fmaf(Hs_hi, sy, -py) + (Hs_hi * sy_l + Hs_lo * sy);
                    float s, e;
                    two_sum(x_hi, -px, s, e);
                    two_sum(s, e + (x_lo - px_l), Gxh, Gxl);
                    two_sum(y_hi, -py, s, e);
                    two_sum(s, e + (y_lo - py_l), Gyh, Gyl);
                }
                S.Gx_hi[t] = Gxh;
                S.Gx_lo[t] = Gxl;
                S.Gy_hi[t] = Gyh;
                S.Gy_lo[t] = Gyl;
                if (dp.nx > 0) {
                    float s, e, hi, lo;
                    two_sum(Gxh, -dp.hx0_hi, s, e);
                    ff_scale(s, e + (Gxl - dp.hx0_lo), dp.inv_dx, hi, lo);
                    S.Cx_hi[t] = hi;
                    S.Cx_lo[t] = lo;
                    two_sum(Gyh, -dp.hy0_hi, s, e);
                    ff_scale(s, e + (Gyl - dp.hy0_lo), dp.inv_dy, hi, lo);
                    S.Cy_hi[t] = hi;
                    S.Cy_lo[t] = lo;
                }
            }
        }
        int S_tot;
        const int offk = block_scan(Kt, S.wsum, &S_tot);
        S.offK[t] = offk;
        if (t == kThreads - 1) S.offK[kTile] = S_tot;
        __syncthreads();

        for (int sub0 = 0; sub0 < S_tot; sub0 += kSubCap) {
            const int nsub = min(kSubCap, S_tot - sub0);
            // ---- stage 2: sub-step yields (Eq. 2.2-2.5, Sec. 4.2.1) -------------
            int Nloc[kSubPerThread];
            int lsum = 0;
#pragma unroll
            for (int r = 0; r < kSubPerThread; ++r) {
                const int q = t * kSubPerThread + r;
                int N = 0;
                if (q < nsub) {
                    const int qq = sub0 + q;
                    int lo = 0, hi = kTile;   // offK[lo] <= qq < offK[hi]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (S.offK[mid] <= qq) lo = mid;
                        else hi = mid;
                    }
                    const int sg = lo, k = qq - S.offK[sg];
                    const float dz_mid = S.Hs_hi[sg] + (S.Hs_lo[sg] + ((float)k + 0.5f) * S.LoverK[sg] * S.Pz[sg]);
                    const float d = delta_at(ap, dz_mid);
                    const float g = S.g[sg];
                    const float onepd = 1.0f + d;
                    // 1 - 1/(beta n)^2 without forming 1/(beta n)^2 (cancellation-free)
                    const float sin2 = (d * (2.0f + d) - onepd * onepd * g) / (onepd * onepd * (1.0f - g));
                    float nbar = 0.0f;
                    if (sin2 > 0.0f) nbar = ap.ft * S.z2[sg] * sin2 * S.LoverK[sg] * inv_b;
                    const unsigned long long gid = pp.seg_base + (unsigned long long)(base + sg);
                    const uint4 rc = philox((uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, 0xFFFFFFFFu,
                                            pp.key0, pp.key1);
                    const float uk = uniform24(rc.x);
                    const float fl = floorf(nbar);
                    N = (int)fl + (uk < nbar - fl ? 1 : 0);   // stochastic rounding
                    S.q_seg[q] = sg;
                    S.q_k[q] = k;
                    S.q_delta[q] = d;
                    S.q_cos[q] = sqrtf(fmaxf(1.0f - sin2, 0.0f));
                    S.q_sin[q] = sqrtf(fmaxf(sin2, 0.0f));
                }
                Nloc[r] = N;
                lsum += N;
            }
            int M;
            int run = block_scan(lsum, S.wsum, &M);
#pragma unroll
            for (int r = 0; r < kSubPerThread; ++r) {
                const int q = t * kSubPerThread + r;
                if (q < nsub) S.offN[q] = run;
                run += Nloc[r];
            }
            if (t == kThreads - 1) S.offN[nsub] = M;
            cnt[CS_CNT_EMITTED] += (unsigned int)lsum * bu;
            __syncthreads();

            // ---- stages 3-5: generate, filter, propagate, detect -----------------
            for (int p = t; p < M; p += kThreads) {
                int lo = 0, hi = nsub;   // offN[lo] <= p < offN[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (S.offN[mid] <= p) lo = mid;
                    else hi = mid;
                }
                const int q = lo;
                const int i = p - S.offN[q];
                const int sg = S.q_seg[q], k = S.q_k[q];
                const unsigned long long gid = pp.seg_base + (unsigned long long)(base + sg);
                const uint4 r4 = philox((uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, (uint32_t)i, pp.key0,
                                        pp.key1);
                const float u0 = uniform24(r4.x), u1 = uniform24(r4.y), u2 = uniform24(r4.z),
                            u3 = uniform24(r4.w);
                const float Px = S.Px[sg], Py = S.Py[sg], Pz = S.Pz[sg];
                // translation to a random point of the sub-step (Fig. 4.2c)
                const float ell = ((float)k + u0) * S.LoverK[sg];
                const float dz = S.Hs_hi[sg] + (S.Hs_lo[sg] + ell * Pz);
                // cone vector rotated into the track frame (Sec. 4.2): u = cos P + sin M e(phi)
                float sphi, cphi;
                sincospif(2.0f * u1, &sphi, &cphi);
                const float inv_l = ap.inv_l1_nm - u2 * ap.dinv_l_nm;   // 1/lambda^2 law
                const float ce = (Px * cphi + Py * sphi) * S.inv1mPz[sg];
                const float mx = Px * ce - cphi, my = Py * ce - sphi, mz = (Pz - 1.0f) * ce;
                const float ct = S.q_cos[q], st = S.q_sin[q];
                const float ux = ct * Px + st * mx, uy = ct * Py + st * my, uz = ct * Pz + st * mz;
                int status = CS_ST_LANDED, tel = -1, bin = -1;
                float x = 0.0f, y = 0.0f, t_rel = ell * S.inv_betac[sg];
                if (!(uz < 0.0f)) {
                    status = CS_ST_UPWARD;   // discarded before propagation (Sec. 5.3.4)
                } else if (dz < 0.0f) {
                    status = CS_ST_BELOW;
                } else {
                    const float inv_uz = -1.0f / uz;
                    const float w = (ux * ux + uy * uy) * inv_uz * inv_uz;   // tan^2(theta0)
                    if (ap.use_tables && (w > ap.tv.w_max || dz >= ap.tv.dz_max)) {
                        status = CS_ST_DOMAIN;
                    } else {
                        // straight line (Eq. 3.3) relative to the segment's ground intercept:
                        // I - G = dz (P_xy / P_z - u_xy / u_z), numerator sin(theta) (P x m)
                        float rx, ry;
                        if (Pz < -1e-3f) {
                            const float pmx = Pz * sphi - ce * Py, pmy = ce * Px - Pz * cphi;
                            const float fac = dz * st / (Pz * uz);
                            rx = -fac * pmy;
                            ry = fac * pmx;
                        } else {   // (near-)horizontal track: the origin is its start point
                            rx = ell * Px + dz * ux * inv_uz;
                            ry = ell * Py + dz * uy * inv_uz;
                        }
                        float path = dz * inv_uz;
                        float T = 1.0f;
                        if (ap.use_tables) {
                            // interpolation tracing (Sec. 4.4.1): bilinear in (h, tan^2 theta0)
                            const float fh = dz * ap.tv.inv_dh, fw = w * ap.tv.inv_dw;
                            const int j = min((int)fh, ap.tv.nh - 1);
                            const int m = min((int)fw, ap.tv.nw - 2);
                            const float fj = fh - (float)j, gm = fw - (float)m;
                            const float4* row = ap.tv.tab + ((size_t)j * ap.tv.nw + m) * 2;
                            const float4 v0 = __ldg(row), s0 = __ldg(row + 1), v1 = __ldg(row + 2),
                                         s1 = __ldg(row + 3);
                            const float a0 = 1.0f - gm;
                            const float GR = a0 * fmaf(fj, s0.x, v0.x) + gm * fmaf(fj, s1.x, v1.x);
                            const float Gt = a0 * fmaf(fj, s0.y, v0.y) + gm * fmaf(fj, s1.y, v1.y);
                            const float GX = a0 * fmaf(fj, s0.z, v0.z) + gm * fmaf(fj, s1.z, v1.z);
                            const float GA = a0 * fmaf(fj, s0.w, v0.w) + gm * fmaf(fj, s1.w, v1.w);
                            if (ap.refraction) {
                                const float c3 = GR * inv_uz * inv_uz * inv_uz;
                                rx += c3 * ux;
                                ry += c3 * uy;
                                path += Gt * inv_uz;
                            }
                            if (ap.transmission) {
                                const float il2 = inv_l * inv_l;
                                const float kR = ap.kR0 * il2 * il2;
                                const float kA = ap.kA0 * exp2f(ap.aer_alpha * log2f(ap.lamA_nm * inv_l));
                                T = exp2f(-(GX * kR + GA * kA) * inv_uz);
                            }
                        }
                        t_rel += path * kInvC;
                        {
                            float s, e;
                            two_sum(S.Gx_hi[sg], rx, s, e);
                            x = s + (e + S.Gx_lo[sg]);
                            two_sum(S.Gy_hi[sg], ry, s, e);
                            y = s + (e + S.Gy_lo[sg]);
                        }
                        if (ap.transmission && !(u3 < T)) {
                            status = CS_ST_ABSORBED;
                        } else {
                            const int sh = S.shower[sg];
                            // ground histogram: cell = floor(G_cells + r / d) in float-float
                            if (dp.nx > 0) {
                                float s, e;
                                two_sum(S.Cx_hi[sg], rx * dp.inv_dx, s, e);
                                const int ix = ff_floor(s, e + S.Cx_lo[sg]);
                                two_sum(S.Cy_hi[sg], ry * dp.inv_dy, s, e);
                                const int iy = ff_floor(s, e + S.Cy_lo[sg]);
                                if (ix >= 0 && ix < dp.nx && iy >= 0 && iy < dp.ny) {
                                    bin = iy * dp.nx + ix;
                                    atomicAdd(op.hist + ((size_t)sh * dp.ny * dp.nx + bin), (unsigned long long)bu);
                                }
                            }
                            // telescopes: distance from the centre to the arrival line < radius
                            if (dp.n_tel > 0 && x >= dp.bx0 && x < dp.bx1 && y >= dp.by0 && y < dp.by1) {
                                float ugx = ux, ugy = uy, ugz = uz;
                                if (ap.refraction) {   // n sin(theta) conserved, azimuth kept
                                    const float sc = (1.0f + S.q_delta[q]) / ap.n_obs;
                                    ugx = ux * sc;
                                    ugy = uy * sc;
                                    ugz = -sqrtf(fmaxf(1.0f - (ugx * ugx + ugy * ugy), 0.0f));
                                }
                                const float gxh = S.Gx_hi[sg], gxl = S.Gx_lo[sg], gyh = S.Gy_hi[sg],
                                            gyl = S.Gy_lo[sg];
                                float best_d2 = 3.0e38f;
                                auto test = [&](int it) {
                                    const float4 T4 = __ldg(dp.tel + it);
                                    const float2 TL = __ldg(dp.tel_lo + it);
                                    const float ddx = (T4.x - gxh) + ((TL.x - gxl) - rx);
                                    const float ddy = (T4.y - gyh) + ((TL.y - gyl) - ry);
                                    const float ddz = T4.z;
                                    const float along = ddx * ugx + ddy * ugy + ddz * ugz;
                                    const float d2 = ddx * ddx + ddy * ddy + ddz * ddz - along * along;
                                    if (d2 < T4.w * T4.w && d2 < best_d2) {
                                        best_d2 = d2;
                                        tel = it;
                                    }
                                };
                                if (ugx * ugx + ugy * ugy <= dp.hash_sin2_max) {
                                    const int cx = (int)((x - dp.gx0) * dp.inv_cell);
                                    const int cy = (int)((y - dp.gy0) * dp.inv_cell);
                                    if (cx >= 0 && cx < dp.gnx && cy >= 0 && cy < dp.gny) {
                                        const int c = cy * dp.gnx + cx;
                                        const int e0 = __ldg(dp.cell_start + c), e1 = __ldg(dp.cell_start + c + 1);
                                        for (int e = e0; e < e1; ++e) test(__ldg(dp.cell_tel + e));
                                    }
                                } else {
                                    for (int it = 0; it < dp.n_tel; ++it) test(it);
                                }
                                if (tel >= 0) {
                                    const size_t slot = (size_t)sh * dp.n_tel + tel;
                                    atomicAdd(op.tel_counts + slot, (unsigned long long)bu);
                                    if (op.tel_time)
                                        atomicAdd(op.tel_time + slot, (double)bu * (S.t0[sg] + (double)t_rel));
                                }
                            }
                        }
                    }
                }
                // bookkeeping of the photon's fate
                if (status == CS_ST_LANDED) {
                    if (bin >= 0) cnt[CS_CNT_HIST] += bu; else cnt[CS_CNT_MISSED_HIST] += bu;
                    if (tel >= 0) cnt[CS_CNT_TEL] += bu; else cnt[CS_CNT_MISSED_TEL] += bu;
                } else if (status == CS_ST_ABSORBED) {
                    cnt[CS_CNT_ABSORBED] += bu;
                } else {
                    cnt[CS_CNT_MISSED_HIST] += bu;
                    cnt[CS_CNT_MISSED_TEL] += bu;
                    if (status == CS_ST_UPWARD) cnt[CS_CNT_UPWARD] += bu;
                }
                if (want_records) emit_record(op, gid, k, i, x, y, t_rel, inv_l, tel, bin, status);
            }
            __syncthreads();
        }

        // ---- per-tile counter flush ----------------------------------------------
        if (t < CS_N_COUNTERS) S.cnt[t] = 0;
        __syncthreads();
#pragma unroll
        for (int c = 0; c < CS_N_COUNTERS; ++c) {
            unsigned int v = cnt[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((t & 31) == 0 && v) atomicAdd(&S.cnt[c], v);
        }
        __syncthreads();
        if (t < CS_N_COUNTERS && S.cnt[t]) atomicAdd(op.counters + t, (unsigned long long)S.cnt[t]);
        __syncthreads();
    }
}

__global__ void philox_kernel(const uint4* ctr, size_t n, uint32_t k0, uint32_t k1, uint4* out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const uint4 c = ctr[i];
        out[i] = philox(c.x, c.y, c.z, c.w, k0, k1);
    }
}

// Device buffers reused by host-pointer calls.
struct HostWorkspace {
    std::mutex mu;
    int device = -1;
    void* segs = nullptr; size_t segs_cap = 0;
    void* outs = nullptr; size_t outs_cap = 0;
    void* recs = nullptr; size_t recs_cap = 0;
};
HostWorkspace g_ws;

cudaError_t ensure(void** p, size_t* cap, size_t need) {
    if (*cap >= need) return cudaSuccess;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(p, need);
    if (e == cudaSuccess) *cap = need;
    return e;
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

cs_status launch(const cs_segment* d_segs, size_t n, const cs_atmosphere* atm, const cs_detector* det,
                 uint64_t seed, const cs_opts& o, const OutParams& op, cudaStream_t stream) {
    const DetParams& dp = det->p;
    if (!o.accumulate) {
        if (op.hist) CS_CUDA_TRY(cudaMemsetAsync(op.hist, 0, (size_t)dp.n_showers * dp.nx * dp.ny * 8, stream));
        if (op.tel_counts) CS_CUDA_TRY(cudaMemsetAsync(op.tel_counts, 0, (size_t)dp.n_showers * dp.n_tel * 8, stream));
        if (op.tel_time) CS_CUDA_TRY(cudaMemsetAsync(op.tel_time, 0, (size_t)dp.n_showers * dp.n_tel * 8, stream));
        CS_CUDA_TRY(cudaMemsetAsync(op.counters, 0, CS_N_COUNTERS * 8, stream));
        if (op.record_count) CS_CUDA_TRY(cudaMemsetAsync(op.record_count, 0, 8, stream));
    }
    if (n == 0) return CS_OK;
    PropParams pp;
    pp.segs = d_segs;
    pp.n = (long long)n;
    pp.seg_base = o.seg_base;
    pp.key0 = (uint32_t)seed;
    pp.key1 = (uint32_t)(seed >> 32);
    pp.bunch = o.bunch;
    pp.s_max = (float)o.s_max;
    const size_t smem = sizeof(TileSmem);
    static bool attr_done = false;
    if (!attr_done) {
        CS_CUDA_TRY(cudaFuncSetAttribute(propagate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_done = true;
    }
    const int per_sm = o.blocks_per_sm > 0 ? o.blocks_per_sm : 4;
    const long long tiles = ((long long)n + kTile - 1) / kTile;
    const long long grid = std::min<long long>(tiles, (long long)device_sm_count() * per_sm);
    propagate_kernel<<<(unsigned)grid, kThreads, smem, stream>>>(pp, atm->p, det->p, op);
    CS_CUDA_TRY(cudaGetLastError());
    return CS_OK;
}

}  // namespace
}  // namespace cs

using namespace cs;

extern "C" cs_status cs_propagate_ex(const cs_segment* segs, size_t n, const cs_atmosphere* atm,
                                     const cs_detector* det, uint64_t seed, const cs_opts* opts,
                                     cs_output* out, void* stream_) {
    if (!atm || !det || !out || !out->counters) return CS_ERR_INVALID_ARG;
    cs_opts o;
    if (opts) o = *opts; else cs_opts_default(&o);
    if (o.bunch < 1 || !(o.s_max > 0.0) || (n > 0 && !segs)) return CS_ERR_INVALID_ARG;
    if (det->p.nx > 0 && !out->hist) return CS_ERR_INVALID_ARG;
    if (det->p.n_tel > 0 && !out->tel_counts) return CS_ERR_INVALID_ARG;
    if (out->records && !out->record_count) return CS_ERR_INVALID_ARG;
    if (fabs(det->p.h_obs - atm->p.h_obs) > 1e-9 * fmax(1.0, fabs(atm->p.h_obs))) return CS_ERR_INVALID_ARG;
    if (n > (size_t)1 << 40) return CS_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_;
    const DetParams& dp = det->p;
    if (o.device_ptrs) {
        if (((uintptr_t)segs & 15) != 0) return CS_ERR_INVALID_ARG;
        OutParams op;
        op.hist = (unsigned long long*)out->hist;
        op.tel_counts = (unsigned long long*)out->tel_counts;
        op.tel_time = out->tel_time;
        op.counters = (unsigned long long*)out->counters;
        op.records = out->records;
        op.record_capacity = out->records ? out->record_capacity : 0;
        op.record_count = (unsigned long long*)out->record_count;
        return launch(segs, n, atm, det, seed, o, op, stream);
    }
    // host pointers: stage through the workspace
    std::lock_guard<std::mutex> lock(g_ws.mu);
    int dev = 0;
    CS_CUDA_TRY(cudaGetDevice(&dev));
    if (g_ws.device != dev) {   // buffers of another device are not reused
        g_ws.segs = g_ws.outs = g_ws.recs = nullptr;
        g_ws.segs_cap = g_ws.outs_cap = g_ws.recs_cap = 0;
        g_ws.device = dev;
    }
    const size_t hist_b = (size_t)dp.n_showers * dp.nx * dp.ny * 8, tel_b = (size_t)dp.n_showers * dp.n_tel * 8;
    const size_t o_hist = 0, o_tel = up256(hist_b), o_time = o_tel + up256(tel_b), o_cnt = o_time + up256(tel_b),
                 o_rc = o_cnt + 256, outs_b = o_rc + 256;
    CS_CUDA_TRY(ensure(&g_ws.segs, &g_ws.segs_cap, std::max<size_t>(n, 1) * sizeof(cs_segment)));
    CS_CUDA_TRY(ensure(&g_ws.outs, &g_ws.outs_cap, outs_b));
    const size_t rec_b = out->records ? out->record_capacity * sizeof(cs_record) : 0;
    if (rec_b) CS_CUDA_TRY(ensure(&g_ws.recs, &g_ws.recs_cap, rec_b));
    char* ob = (char*)g_ws.outs;
    OutParams op;
    op.hist = dp.nx > 0 ? (unsigned long long*)(ob + o_hist) : nullptr;
    op.tel_counts = dp.n_tel > 0 ? (unsigned long long*)(ob + o_tel) : nullptr;
    op.tel_time = (dp.n_tel > 0 && out->tel_time) ? (double*)(ob + o_time) : nullptr;
    op.counters = (unsigned long long*)(ob + o_cnt);
    op.records = out->records ? (cs_record*)g_ws.recs : nullptr;
    op.record_capacity = out->records ? out->record_capacity : 0;
    op.record_count = (unsigned long long*)(ob + o_rc);
    if (n) CS_CUDA_TRY(cudaMemcpyAsync(g_ws.segs, segs, n * sizeof(cs_segment), cudaMemcpyHostToDevice, stream));
    if (o.accumulate) {   // bring the caller's running totals in
        if (op.hist) CS_CUDA_TRY(cudaMemcpyAsync(op.hist, out->hist, hist_b, cudaMemcpyHostToDevice, stream));
        if (op.tel_counts) CS_CUDA_TRY(cudaMemcpyAsync(op.tel_counts, out->tel_counts, tel_b, cudaMemcpyHostToDevice, stream));
        if (op.tel_time) CS_CUDA_TRY(cudaMemcpyAsync(op.tel_time, out->tel_time, tel_b, cudaMemcpyHostToDevice, stream));
        CS_CUDA_TRY(cudaMemcpyAsync(op.counters, out->counters, CS_N_COUNTERS * 8, cudaMemcpyHostToDevice, stream));
        CS_CUDA_TRY(cudaMemsetAsync(op.record_count, 0, 8, stream));
    }
    cs_status st = launch((const cs_segment*)g_ws.segs, n, atm, det, seed, o, op, stream);
    if (st != CS_OK) return st;
    if (op.hist) CS_CUDA_TRY(cudaMemcpyAsync(out->hist, op.hist, hist_b, cudaMemcpyDeviceToHost, stream));
    if (op.tel_counts) CS_CUDA_TRY(cudaMemcpyAsync(out->tel_counts, op.tel_counts, tel_b, cudaMemcpyDeviceToHost, stream));
    if (op.tel_time) CS_CUDA_TRY(cudaMemcpyAsync(out->tel_time, op.tel_time, tel_b, cudaMemcpyDeviceToHost, stream));
    CS_CUDA_TRY(cudaMemcpyAsync(out->counters, op.counters, CS_N_COUNTERS * 8, cudaMemcpyDeviceToHost, stream));
    unsigned long long produced = 0;
    CS_CUDA_TRY(cudaMemcpyAsync(&produced, op.record_count, 8, cudaMemcpyDeviceToHost, stream));
    CS_CUDA_TRY(cudaStreamSynchronize(stream));
    if (out->record_count) *out->record_count = produced;
    if (out->records && produced) {
        const size_t ncopy = std::min<unsigned long long>(produced, out->record_capacity);
        CS_CUDA_TRY(cudaMemcpy(out->records, g_ws.recs, ncopy * sizeof(cs_record), cudaMemcpyDeviceToHost));
    }
    if (out->records && produced > out->record_capacity) return CS_ERR_CAPACITY;
    return CS_OK;
}

extern "C" cs_status cs_propagate(const cs_segment* segs, size_t n, const cs_atmosphere* atm,
                                  const cs_detector* det, uint64_t seed, cs_output* out) {
    return cs_propagate_ex(segs, n, atm, det, seed, nullptr, out, nullptr);
}

extern "C" cs_status cs_philox4x32_10(const uint32_t* ctr, size_t n, uint32_t key0, uint32_t key1, uint32_t* out,
                                      void* stream) {
    if ((n > 0 && (!ctr || !out)) || ((uintptr_t)ctr & 15) || ((uintptr_t)out & 15)) return CS_ERR_INVALID_ARG;
    cs_status st = check_device();
    if (st != CS_OK) return st;
    if (n == 0) return CS_OK;
    philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>((const uint4*)ctr, n, key0, key1,
                                                                                (uint4*)out);
    CS_CUDA_TRY(cudaGetLastError());
    return CS_OK;
}
