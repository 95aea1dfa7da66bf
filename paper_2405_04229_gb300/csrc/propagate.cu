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
#include <functional>
#include <mutex>
#include <type_traits>
#include <vector>

#include "exact_path.cuh"
#include "mlp_tc.cuh"

namespace cs {
namespace {

constexpr int kThreads = 256;           // exact tracer: threads per block
constexpr int kThreadsSur = 512;        // surrogate: four warpgroups per block
constexpr int kMaxThreads = 512;
constexpr int kTile = 256;              // segments per tile, one per thread (the first kTile threads)
constexpr int kSubCap = 512;            // sub-steps per round
constexpr int kMapCap = 2048;           // bunches per window of the bunch -> sub-step map
constexpr int kKShift = 8;              // sub-step record: segment (8 bits) | k << 8
constexpr int kQBits = 10;              // map entry: sub-step (10 bits) | bunch index << 10

// Per-tile shared memory: the imported segments (packed float4 field groups)
// and one round of sub-steps with its bunch map.
struct TileSmem {
    float4 segA[kTile];   // Px, Py, Pz, 1 / (1 - Pz)
    // planar | spherical shell
    float4 segB[kTile];   // Hs_hi, Hs_lo (z0 - h_obs), L / K, 1 / (beta c) | Hs, tilt_z, L / K, 1 / (beta c)
    float4 segC[kTile];   // ground intercept G, float-float x and y | start point (hi), radial P component
    float4 segD[kTile];   // G in histogram cells, float-float x and y | start point (lo), 1 / r
    double t0[kTile];
    float g[kTile], z2[kTile];
    int shower[kTile];
    int bunch[kTile];     // photons per bunch of the segment's shower
    int offK[kTile + 1];
    float4 sub[kSubCap];  // cos(theta), sin(theta), n - 1, segment | k << 8
    int nsub_ph[kSubCap]; // bunches of each sub-step
    unsigned int map[kMapCap];
    int wsum[2][kMaxThreads / 32];   // double-buffered warp sums of the block scans
    int tile;
};

// The exact-tracer instances run their warps independently: each warp takes
// tiles of 32 segments from the work counter and keeps its own segment,
// sub-step and bunch-map buffers, so no block-wide barrier ever holds a warp
// (the surrogate's warpgroups, whose tensor-core network is collective, keep
// the block-wide tile above).
constexpr int kWTile = 32;              // segments per warp tile
constexpr int kWSubCap = 128;           // sub-steps per warp round
constexpr int kWMapCap = 256;           // bunches per warp map window
struct WarpSmem {
    float4 segA[kWTile], segB[kWTile], segC[kWTile], segD[kWTile];   // as in TileSmem
    double t0[kWTile];
    float g[kWTile], z2[kWTile];
    int shower[kWTile];
    int bunch[kWTile];
    int offK[kWTile + 1];
    int perm[kWTile];      // tile slot of the i-th segment in processing order
    float4 sub[kWSubCap];
    int nsub_ph[kWSubCap];
    unsigned int map[kWMapCap];
};
constexpr size_t kSmemExact = (kThreads / 32) * sizeof(WarpSmem);
static_assert(4 * (kSmemExact + 1024) <= 228 * 1024, "four exact-tracer blocks per SM");

// The surrogate instances keep the tensor-core network's buffers after the tile.
constexpr size_t kTcSmemOffset = (sizeof(TileSmem) + 127) & ~(size_t)127;
constexpr size_t kSmemSurrogate = kTcSmemOffset + sizeof(TcSmem<kThreadsSur / 128>);

// Exclusive block scan with one barrier; `buf` alternates between calls so a
// scan never overwrites warp sums another warp may still be reading.
template <int NT>
__device__ __forceinline__ int block_scan(int v, int (*wsum)[kMaxThreads / 32], int& buf, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    int* ws = wsum[buf];
    buf ^= 1;
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    int pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        const int s = ws[w];
        pre += w < wid ? s : 0;
        tot += s;
    }
    *total = tot;
    return pre + x - v;
}

__device__ __forceinline__ void emit_record(const OutParams& o, unsigned long long seg, int k, int i, float x,
                                            float x_lo, float y, float y_lo, float t_rel, float inv_l, int tel,
                                            int bin, int status, int pix) {
    const unsigned long long slot = atomicAdd(o.record_count, 1ULL);
    if (slot < o.record_capacity) {
        cs_record r;
        r.seg = seg;
        r.k = (uint32_t)k;
        r.i = (uint32_t)i;
        r.x = x;
        r.y = y;
        r.x_lo = x_lo;
        r.y_lo = y_lo;
        r.dt_ns = t_rel * 1e9f;
        r.lambda_nm = 1.0f / inv_l;
        r.tel = tel;
        r.bin = bin;
        r.status = (uint32_t)status;
        r.pix = pix;
        o.records[slot] = r;
    }
}

// Angle [deg] from the unit direction P to a sphere of radius r whose centre
// lies at d from the segment start, less the sphere's angular radius (0 inside).
__device__ __forceinline__ float angle_to_sphere(float Px, float Py, float Pz, float dx, float dy, float dz, float r) {
    const float dn = sqrtf(dx * dx + dy * dy + dz * dz);
    if (!(dn > r)) return 0.0f;
    const float c = fminf(fmaxf((Px * dx + Py * dy + Pz * dz) / dn, -1.0f), 1.0f);
    return fmaxf(acosf(c) - asinf(r / dn), 0.0f) * 57.29577951308232f;
}

// LV1 particle filter (Sec. 4.3.2; the cut of Sec. 6.2.1): true when the
// segment starting at (x, y, z) (float-float; h its height above h_obs) with
// direction P is dropped, i.e. h >= a x^b for the angle x to the point of
// interest.
template <bool SPH>
__device__ __forceinline__ bool lv1_drop(const PropParams& pp, const DetParams& dp, float x_hi, float x_lo, float y_hi,
                                         float y_lo, float z_hi, float z_lo, float h, float Px, float Py, float Pz) {
    float x;
    if (pp.lv1 != CS_LV1_TELESCOPES) {
        const float dx = (pp.lv1_c[0] - x_hi) - x_lo, dy = (pp.lv1_c[1] - y_hi) - y_lo, dz = (pp.lv1_c[2] - z_hi) - z_lo;
        x = angle_to_sphere(Px, Py, Pz, dx, dy, dz, pp.lv1 == CS_LV1_ARRAY_DISC ? pp.lv1_r : 0.0f);
    } else {
        x = 180.0f;
        for (int it = 0; it < dp.n_tel; ++it) {
            float dx, dy, dz, r;
            if (SPH) {
                const float4 T3 = __ldg(dp.tel3 + it);
                dx = (T3.x - x_hi) - x_lo; dy = (T3.y - y_hi) - y_lo; dz = (T3.z - z_hi) - z_lo; r = T3.w;
            } else {
                const float4 T4 = __ldg(dp.tel + it);
                const float2 TL = __ldg(dp.tel_lo + it);
                dx = (T4.x - x_hi) + (TL.x - x_lo); dy = (T4.y - y_hi) + (TL.y - y_lo); dz = T4.z - h; r = T4.w;
            }
            x = fminf(x, angle_to_sphere(Px, Py, Pz, dx, dy, dz, r));
        }
    }
    x = fmaxf(x, 1e-3f);
    return h >= pp.lv1_a * exp2f(pp.lv1_b * log2f(x));
}

// K = ceil(L / s_max) sub-steps (Sec. 4.2.1) for s_max = sh + sl (float-float):
// the FP32 quotient proposes K, the sign of K s_max - L (the product exact
// through FMA, to 2^-48 relative) confirms K s_max >= L > (K - 1) s_max.
__device__ __forceinline__ int substep_count(float L, float sh, float sl) {
    int K = max(1, (int)ceilf(L / sh));
    const auto covers = [&](int k) {
        const float kf = (float)k, p = kf * sh;
        return (p - L) + (fmaf(kf, sh, -p) + kf * sl) >= 0.0f;
    };
    if (!covers(K)) ++K;
    else if (K > 1 && covers(K - 1)) --K;
    return K;
}

// Stage 1 (Sec. 5.3.1): import one segment, filter it, fold its parameters
// and compute its local origin.  Returns the number of sub-steps (0 if invalid).
// Planar: the origin is the ground intercept of the segment's line (float-float).
// Spherical shell: the start point (float-float), its altitude above h_obs,
// the radial component of P, 1 / r and the tilt of the local vertical.
template <bool SPH, bool FL, typename SM>
__device__ __forceinline__ int import_segment(SM& S, int t, const cs_segment* seg, const PropParams& pp,
                                              const AtmParams& ap, const DetParams& dp, unsigned int& invalid,
                                              unsigned int& dropped, bool filter = true) {
    const double2* src = reinterpret_cast<const double2*>(seg);
    const double2 xy = __ldg(src), zt = __ldg(src + 1);
    const float4 dir = __ldg(reinterpret_cast<const float4*>(src + 2));
    const uint4 rest = __ldg(reinterpret_cast<const uint4*>(src + 3));
    const float g = __uint_as_float(rest.x), z = __uint_as_float(rest.y);
    const unsigned int shower = rest.z;
    const float n2 = dir.x * dir.x + dir.y * dir.y + dir.z * dir.z;
    const bool valid = finite_f64(xy.x) && finite_f64(xy.y) && finite_f64(zt.x) && finite_f64(zt.y) && isfinite(dir.x) &&
                       isfinite(dir.y) && isfinite(dir.z) && isfinite(dir.w) && dir.w > 0.0f && g > 0.0f &&
                       g < 1.0f && isfinite(z) && dir.z < 0.99f && fabsf(n2 - 1.0f) <= 1e-4f &&
                       shower < (unsigned int)dp.n_showers;
    if (filter && !valid) {
        invalid += 1;
        return 0;
    }
    const float inv_n = rsqrtf(n2);
    const float Px = dir.x * inv_n, Py = dir.y * inv_n, Pz = dir.z * inv_n;
    const float L = dir.w;
    const int K = substep_count(L, pp.s_max, pp.s_max_lo);
    float x_hi, x_lo, y_hi, y_lo, z_hi, z_lo;
    split_f64(xy.x, x_hi, x_lo);
    split_f64(xy.y, y_hi, y_lo);
    split_f64(zt.x, z_hi, z_lo);
    // Hs = z0 - h_obs in float-float
    float Hs_hi, Hs_lo;
    {
        float s, e;
        two_sum(z_hi, -ap.h_obs_hi, s, e);
        const float t = e + (z_lo - ap.h_obs_lo);
        Hs_hi = s + t;
        Hs_lo = t - (Hs_hi - s);
    }
    if (SPH) {
        const float R = ap.R;
        // altitude h = |S - c| - R = z + rho^2 / (|S - c| + z + R), c = (0, 0, -R), without cancellation
        const float rho2 = x_hi * x_hi + y_hi * y_hi, a = z_hi + R;
        const float rr = sqrtf(rho2 + a * a);
        const float lift = rho2 / (rr + a);
        const float Hs = Hs_hi + (Hs_lo + lift);
        if (filter && pp.lv1 && lv1_drop<true>(pp, dp, x_hi, x_lo, y_hi, y_lo, z_hi, z_lo, Hs, Px, Py, Pz)) {
            dropped += 1;
            return 0;
        }
        const float inv_r = 1.0f / rr;
        const float dvx = x_hi * inv_r, dvy = y_hi * inv_r, dvz = -lift * inv_r;   // v - z-hat
        const float Pr = Px * dvx + Py * dvy + Pz * (1.0f + dvz);
        S.segA[t] = make_float4(Px, Py, Pz, 1.0f / (1.0f - Pz));
        S.segB[t] = make_float4(Hs, dvz, L / (float)K, rsqrtf(1.0f - g) * kInvC);
        S.segC[t] = make_float4(x_hi, y_hi, z_hi, Pr);
        S.segD[t] = make_float4(x_lo, y_lo, z_lo, inv_r);
        S.t0[t] = zt.y;
        S.g[t] = g;
        S.z2[t] = z * z;
        S.shower[t] = (int)shower;
        S.bunch[t] = pp.shower_bunch ? __ldg(pp.shower_bunch + shower) : pp.bunch;
        return K;
    }
    if (filter && pp.lv1 && lv1_drop<false>(pp, dp, x_hi, x_lo, y_hi, y_lo, z_hi, z_lo, Hs_hi + Hs_lo, Px, Py, Pz)) {
        dropped += 1;
        return 0;
    }
    // local origin: G = S_xy - Hs P_xy / P_z in float-float (isotropic fluorescence keeps the
    // start point: its photons land anywhere, not near the track's own ground point)
    float Gxh = x_hi, Gxl = x_lo, Gyh = y_hi, Gyl = y_lo;
    if (Pz < -1e-3f && !FL) {
        const float sx = Px / Pz, sy = Py / Pz;                       // slopes, float-float via FMA remainder
        const float sx_l = fmaf(-sx, Pz, Px) / Pz, sy_l = fmaf(-sy, Pz, Py) / Pz;
        const float px = Hs_hi * sx, py = Hs_hi * sy;
        const float px_l = fmaf(Hs_hi, sx, -px) + (Hs_hi * sx_l + Hs_lo * sx);
        const float py_l = fmaf(Hs_hi, sy, -py) + (Hs_hi * sy_l + Hs_lo * sy);
        float s, e;
        two_sum(x_hi, -px, s, e);
        two_sum(s, e + (x_lo - px_l), Gxh, Gxl);
        two_sum(y_hi, -py, s, e);
        two_sum(s, e + (y_lo - py_l), Gyh, Gyl);
    }
    S.segA[t] = make_float4(Px, Py, Pz, 1.0f / (1.0f - Pz));
    S.segB[t] = make_float4(Hs_hi, Hs_lo, L / (float)K, rsqrtf(1.0f - g) * kInvC);
    S.segC[t] = make_float4(Gxh, Gxl, Gyh, Gyl);
    if (dp.nx > 0) {
        float s, e, cxh, cxl, cyh, cyl;
        two_sum(Gxh, -dp.hx0_hi, s, e);
        ff_scale(s, e + (Gxl - dp.hx0_lo), dp.inv_dx, cxh, cxl);
        two_sum(Gyh, -dp.hy0_hi, s, e);
        ff_scale(s, e + (Gyl - dp.hy0_lo), dp.inv_dy, cyh, cyl);
        S.segD[t] = make_float4(cxh, cxl, cyh, cyl);
    }
    S.t0[t] = zt.y;
    S.g[t] = g;
    S.z2[t] = z * z;
    S.shower[t] = (int)shower;
    S.bunch[t] = pp.shower_bunch ? __ldg(pp.shower_bunch + shower) : pp.bunch;
    return K;
}

// Fluorescence line of bunch (segment, k, i): a second Philox draw, its 24-bit
// integer against the lines' cumulative yield shares in units of 2^-24.
__device__ __forceinline__ float fluorescence_line(const PropParams& pp, uint32_t g_lo, uint32_t g_hi, uint32_t k,
                                                  uint32_t i) {
    const PropParams& fp = pp;
    const uint4 r = philox_rk(g_lo, g_hi, k, i | 0x80000000u, pp.rk);
    const uint32_t v = r.x >> 8;
    int line = fp.fl_n - 1;
    for (int l = fp.fl_n - 2; l >= 0; --l)
        if (v < fp.fl_thr[l]) line = l;
    return fp.fl_inv_l[line];
}

// Stage 2 (Eq. 2.2-2.5, Sec. 4.2.1): sub-step k of tile segment sg at local
// slot q: angle and mean bunch count at the sub-step midpoint, stochastic
// rounding with the sub-step's own draw.  Returns the bunch count.
template <bool SPH, bool FL, typename SM>
__device__ __forceinline__ int substep(SM& S, int q, int sg, int k, long long base, const PropParams& pp,
                                       const AtmParams& ap) {
    const float4 B = S.segB[sg];
    float dz_mid;
    if (SPH) {   // altitude along the track: Hs + s Pr + s^2 (1 - Pr^2) / (2 r)
        const float Pr = S.segC[sg].w, s_mid = ((float)k + 0.5f) * B.z;
        dz_mid = B.x + s_mid * fmaf(s_mid * 0.5f * S.segD[sg].w, fmaf(-Pr, Pr, 1.0f), Pr);
    } else {
        dz_mid = B.x + (B.y + ((float)k + 0.5f) * B.z * S.segA[sg].z);
    }
    const float d = delta_at(ap, dz_mid);
    const float g = S.g[sg];
    const float onepd = 1.0f + d;
    // 1 - 1/(beta n)^2 without forming 1/(beta n)^2 (cancellation-free)
    const float sin2 = (d * (2.0f + d) - onepd * onepd * g) * rcp_approx(onepd * onepd * (1.0f - g));
    float nbar = 0.0f;
    if constexpr (FL) nbar = pp.fl_yd * S.z2[sg] * d * B.z * rcp_approx((float)S.bunch[sg]);   // Eq. 2.6
    else if (sin2 > 0.0f) nbar = ap.ft * S.z2[sg] * sin2 * B.z * rcp_approx((float)S.bunch[sg]);
    const unsigned long long gid = pp.seg_base + (unsigned long long)(base + sg);
    const uint4 rc = philox_rk((uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, 0xFFFFFFFFu, pp.rk);
    const float uk = uniform24(rc.x);
    const float fl = floorf(nbar);
    const int N = (int)fl + (uk < nbar - fl ? 1 : 0);
    const float c2 = fmaxf(1.0f - sin2, 1e-30f), s2 = fmaxf(sin2, 1e-30f);
    S.sub[q] = make_float4(c2 * rsqrtf(c2), sin2 > 0.0f ? s2 * rsqrtf(s2) : 0.0f, d,
                           __int_as_float(sg | (k << kKShift)));
    S.nsub_ph[q] = N;
    return N;
}

struct Tally {
    unsigned int absorbed, hist, tel, upward;
};

// Histogram count: one 64-bit atomic per bunch.  (Warp aggregation -- lanes
// adding to the same cell combining first -- measured 3 % slower: a warp's
// bunches come from cones whose ground rings spread over hundreds of 1 m
// cells, so lanes rarely share one.)
__device__ __forceinline__ void hist_add(const OutParams& op, unsigned int key, unsigned int b) {
    atomicAdd(op.hist + key, (unsigned long long)b);
}

// Telescopes: the sphere whose centre is closest to the arrival line, if
// closer than its radius (ties: lowest index).  Arrivals within the hash's
// zenith range (`hashed`; the caller has checked the box of all reach discs)
// test the entries of their grid cell: cell_delta(entry, corner_x, corner_y,
// ddx, ddy, ddz) gives the centre minus the ground point.  Steeper arrivals
// test every sphere through full_delta(index, ddx, ddy, ddz, radius).
template <typename CellDelta, typename FullDelta>
__device__ __forceinline__ int hit_telescope(const DetParams& dp, const TelHash& H, bool hashed, float x, float y, float ugx,
                                             float ugy, float ugz, CellDelta cell_delta, FullDelta full_delta) {
    int best = -1;
    float best_d2 = 3.0e38f;
    auto test = [&](float ddx, float ddy, float ddz, float r, int id) {
        const float along = ddx * ugx + ddy * ugy + ddz * ugz;
        const float d2 = ddx * ddx + ddy * ddy + ddz * ddz - along * along;
        if (d2 < r * r && d2 < best_d2) {
            best_d2 = d2;
            best = id;
        }
    };
    if (hashed) {
        const int cx = (int)((x - H.gx0) * H.inv_cell);
        const int cy = (int)((y - H.gy0) * H.inv_cell);
        if (cx < 0 || cx >= H.gnx || cy < 0 || cy >= H.gny) return -1;
        const int2 er = __ldg(H.cell_range + (cy * H.gnx + cx));
        if (er.x == er.y) return -1;   // no reach disc covers this cell
        const float cx0 = fmaf((float)cx, H.cell, H.gx0), cy0 = fmaf((float)cy, H.cell, H.gy0);   // exact
        for (int e = er.x; e < er.y; ++e) {
            const float4 D = __ldg(H.cell_data + e);
            float ddx, ddy, ddz;
            cell_delta(D, cx0, cy0, ddx, ddy, ddz);
            test(ddx, ddy, ddz, D.w, e);
        }
        return best >= 0 ? __ldg(H.cell_tel + best) : -1;
    }
    for (int it = 0; it < dp.n_tel; ++it) {
        float ddx, ddy, ddz, r;
        full_delta(it, ddx, ddy, ddz, r);
        test(ddx, ddy, ddz, r, it);
    }
    return best;
}

// Last-mile ray tracing (Sec. 6.4) through the telescope whose sphere centre
// lies at dd from the ground point, for the arrival direction u, in the
// telescope's frame (e1, e2, a) with the origin at the mirror vertex
// C - f/2 a.  The ray starts at its closest approach to the centre (the same
// line as from the ground point, better conditioned in FP32).  It must pass
// the camera plane z' = f outside the camera disc (else the camera shadows
// it), leave the bowl z' < r'^2 / (4 f) through the paraboloid inside the
// aperture -- the larger root of r'^2 - 4 f z' = 0 along the line, the
// smaller being an entry through the wall far above --, reflect about the
// surface normal (x', y', -2 f) and reach the camera plane inside the disc.
// Returns the pixel iy * cam_n + ix or -1.
__device__ __noinline__ int camera_pixel(const DetParams& dp, float ddx, float ddy, float ddz, float ux, float uy,
                                         float uz) {
    const float f = dp.cam_f, R = dp.cam_r;
    const float along = ddx * ux + ddy * uy + ddz * uz;
    const float hf = 0.5f * f;
    const float qx = fmaf(along, ux, fmaf(hf, dp.ax, -ddx));
    const float qy = fmaf(along, uy, fmaf(hf, dp.ay, -ddy));
    const float qz = fmaf(along, uz, fmaf(hf, dp.az, -ddz));
    const float p0 = qx * dp.e1x + qy * dp.e1y + qz * dp.e1z;
    const float p1 = qx * dp.e2x + qy * dp.e2y + qz * dp.e2z;
    const float p2 = qx * dp.ax + qy * dp.ay + qz * dp.az;
    const float d0 = ux * dp.e1x + uy * dp.e1y + uz * dp.e1z;
    const float d1 = ux * dp.e2x + uy * dp.e2y + uz * dp.e2z;
    const float d2 = ux * dp.ax + uy * dp.ay + uz * dp.az;
    if (!(d2 < 0.0f)) return -1;   // travelling away from the mirror
    const float tc = (f - p2) / d2;
    const float cx = fmaf(tc, d0, p0), cy = fmaf(tc, d1, p1);
    if (cx * cx + cy * cy < R * R) return -1;   // the camera's shadow
    const float A = d0 * d0 + d1 * d1;
    const float B = 2.0f * (p0 * d0 + p1 * d1) - 4.0f * f * d2;
    const float Cq = p0 * p0 + p1 * p1 - 4.0f * f * p2;
    const float disc = B * B - 4.0f * A * Cq;
    if (!(disc >= 0.0f)) return -1;
    // roots qq / A and Cq / qq without cancellation; A = 0 (a ray along the
    // axis, B > 0) leaves the finite root Cq / qq = -Cq / B
    const float qq = -0.5f * (B + copysignf(sqrtf(disc), B));
    const float t = fmaxf(qq / A, Cq / qq);
    if (!isfinite(t)) return -1;
    const float mx = fmaf(t, d0, p0), my = fmaf(t, d1, p1), mz = fmaf(t, d2, p2);
    const float rm2 = mx * mx + my * my;
    if (rm2 > dp.cam_rd2) return -1;   // outside the aperture
    const float nz = -2.0f * f;
    const float k = 2.0f * (d0 * mx + d1 * my + d2 * nz) / (rm2 + nz * nz);
    const float r0 = d0 - k * mx, r1 = d1 - k * my, r2 = d2 - k * nz;
    if (!(r2 > 0.0f)) return -1;
    const float sc = (f - mz) / r2;
    const float xq = fmaf(sc, r0, mx), yq = fmaf(sc, r1, my);
    if (xq * xq + yq * yq > R * R) return -1;   // beyond the camera's rim
    const int n = dp.cam_n;
    const int ix = min(max((int)floorf((xq + R) * dp.cam_scale), 0), n - 1);
    const int iy = min(max((int)floorf((yq + R) * dp.cam_scale), 0), n - 1);
    return iy * n + ix;
}

// Absorption in the optics (Sec. 6.4): the camera keeps a photon that reached
// pixel pix when the 24-bit uniform of Philox word x of counter (segment,
// sub-step, bunch | 2^30) lies below R(lambda) eps(lambda), the mirror's
// reflectivity times the camera's detection efficiency, each linear between
// the detector's nodes and constant beyond them.  Returns pix or -1.
__device__ __forceinline__ int optics_survival(const DetParams& dp, const PropParams& pp, unsigned long long gid, int k,
                                               int i, float inv_l, int pix) {
    if (pix < 0 || dp.eff_n == 0) return pix;
    const float lnm = 1.0f / inv_l;
    int j = 0;
    while (j + 2 < dp.eff_n && lnm > dp.eff_l[j + 1]) ++j;
    float fR = dp.eff_R[0], fE = dp.eff_E[0];
    if (dp.eff_n > 1) {
        const float t = fminf(fmaxf((lnm - dp.eff_l[j]) / (dp.eff_l[j + 1] - dp.eff_l[j]), 0.0f), 1.0f);
        fR = fmaf(t, dp.eff_R[j + 1] - dp.eff_R[j], dp.eff_R[j]);
        fE = fmaf(t, dp.eff_E[j + 1] - dp.eff_E[j], dp.eff_E[j]);
    }
    const uint4 r = philox_rk((uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, (uint32_t)i | 0x40000000u, pp.rk);
    return uniform24(r.x) < fR * fE ? pix : -1;
}

// Snell's law in vector form through homogeneous slabs (Sec. 3.4.2, Eq. 3.15),
// the general-atmosphere tracer.  The height dz above the observation level is
// cut into the fewest equal slabs no thicker than dh; slab j holds the index
// at its middle height and is crossed straight.  At a planar boundary Eq. 3.15
// adds c N to the optical vector A' = n A, so the horizontal part n sin(a)
// never changes and the normal part becomes A'_j = sqrt(A'_0^2 + D_j) with
// D_j = n_j^2 - n_0^2 = (d_j - d_0)(2 + d_j + d_0): the same algebra, written
// so that FP32 resolves changes of 1e-8 per slab.  (A'_j^2 <= 0, a total
// reflection that no atmosphere denser below produces, is clamped.)
// Returns {(R - R_straight) / sin(theta0), c t_path, X_slant [g/cm^2], A_slant [m]}.
__device__ __noinline__ float4 snell_path(const AtmParams& ap, float dz, float cos0, float dh) {
    const int ns = max(1, (int)ceilf(dz / dh));
    const float step = dz / (float)ns;
    const float d0 = delta_at(ap, dz - 0.5f * step);
    const float A0 = (1.0f + d0) * cos0;
    const float inv0 = 1.0f / A0;
    const float t0 = (1.0f + d0) * (1.0f + d0) * inv0;   // c t per metre of height in slab 0
    float sR = 0.0f, sT = 0.0f, sX = 0.0f, sA = 0.0f;
    for (int j = 0; j < ns; ++j) {
        const float h = dz - ((float)j + 0.5f) * step;
        const float dj = j == 0 ? d0 : delta_at(ap, h);
        const float D = (dj - d0) * (2.0f + dj + d0);
        const float Aj2 = fmaxf(fmaf(A0, A0, D), 1e-12f);
        const float inv = rsqrtf(Aj2);         // 1 / A'_j
        const float Aj = Aj2 * inv;
        const float g = (1.0f + dj) * inv;     // path length per metre of height
        sR -= D * inv * inv0 * rcp_approx(Aj + A0);   // 1 / A'_j - 1 / A'_0 without cancellation
        sT += fmaf(1.0f + dj, g, -t0);         // the delay relative to slab 0's, summed small
        if (ap.transmission) {
            sX = fmaf(dj, g, sX);
            sA = fmaf(ex2_approx(ap.aer_c2 * h), g, sA);
        }
    }
    return make_float4((1.0f + d0) * step * sR, fmaf(step, sT, dz * t0), ap.rho_per_delta * step * sX,
                       ap.aer_hobs * step * sA);
}

// The same stepper on the spherical shell: shells of equal thickness <= dh in
// altitude; inside a shell the photon runs straight to the next inner sphere,
// where Eq. 3.15 refracts it about the radial normal.  A straight line keeps
// its impact parameter r sin(psi), and Eq. 3.15 at a spherical boundary keeps
// n r sin(psi), so in shell j the photon runs with impact parameter
// b_j = K / n_j, K = n_0 r_e sin(psi_0) (the same algebra in FP32-stable
// scalar form).  A chord from r_out to r_in = r_out - step with impact
// parameter b has length step (r_out + r_in) / (q_out + q_in), q = sqrt(r^2 -
// b^2), and sweeps the central angle asin(b t / (r_in r_out)); the straight
// line (b_0 = r_e sin(psi_0)) is walked through the same shells and the
// differences are summed.  Returns {arc-length correction along the ground
// r_g (Phi - Phi_line) [m], c t_path - straight length [m], X_slant, A_slant}.
// When the straight line passes over the ground sphere (b_0 >= r_g) while the
// refracted photon still reaches it, there is no line to refer to: the sums
// are then absolute, {r_g Phi, c t_path, X, A}, and `absolute` is set.
__device__ __noinline__ float4 snell_path_sph(const AtmParams& ap, float dz, float sin2, float dh, bool& absolute) {
    const int ns = max(1, (int)ceilf(dz / dh));
    const float step = dz / (float)ns;
    const float d0 = delta_at(ap, dz - 0.5f * step);
    const float re = ap.rg + dz;
    const float b0 = re * sqrtf(sin2);
    const bool line = b0 < ap.rg;
    absolute = !line;
    float sPhi = 0.0f, sT = 0.0f, sX = 0.0f, sA = 0.0f;
    for (int j = 0; j < ns; ++j) {
        const float h = dz - ((float)j + 0.5f) * step;
        const float dj = j == 0 ? d0 : delta_at(ap, h);
        const float r_out = re - (float)j * step, r_in = r_out - step;
        const float rs = fmaf(-2.0f * (float)j - 1.0f, step, 2.0f * re);   // r_out + r_in
        const float b = b0 + b0 * (d0 - dj) * rcp_approx(1.0f + dj);
        const float q_out = sqrtf(fmaxf((r_out - b) * (r_out + b), 0.0f));
        const float q_in = sqrtf(fmaxf((r_in - b) * (r_in + b), 0.0f));
        const float p_out = sqrtf(fmaxf((r_out - b0) * (r_out + b0), 0.0f));
        const float p_in = sqrtf(fmaxf((r_in - b0) * (r_in + b0), 0.0f));
        const float t = step * rs * rcp_approx(q_out + q_in);
        const float t0 = line ? step * rs * rcp_approx(p_out + p_in) : 0.0f;
        const float irr = rcp_approx(r_in * r_out);
        sPhi += (b * t - b0 * t0) * irr;
        sT += fmaf(dj, t, t - t0);
        if (ap.transmission) {
            sX = fmaf(dj, t, sX);
            sA = fmaf(ex2_approx(ap.aer_c2 * h), t, sA);
        }
    }
    return make_float4(ap.rg * sPhi, sT, ap.rho_per_delta * sX, ap.aer_hobs * sA);
}

// The stepper in the cylindrical atmosphere (Sec. 3.3.3): shells between
// coaxial cylinders of equal thickness <= dh in altitude, each holding n at its
// middle altitude.  Eq. 3.15 at a cylinder changes only the optical vector's
// part along the inward normal, so its parts along the axis (A = n u_a) and
// along the transverse tangent (L = n rho u_chi) keep the values they take in
// the first shell, and in shell j the transverse track is the straight chord
// with impact parameter b_j = L / N_j, N_j^2 = n_j^2 - A^2 (the vector form's
// algebra in scalar form).  A chord from rho_out to rho_in = rho_out - step
// has the transverse length sigma = step (rho_out + rho_in) / (q_out + q_in),
// q = sqrt(rho^2 - b^2), sweeps b sigma / (rho_in rho_out) radians (the sine of
// the angle; they differ by < 1e-15 here), runs sigma n_j / N_j of path and
// drifts sigma A / N_j along the axis.  FP32 cannot form rho - b directly
// (rho ~ 6.4e6 m carries 0.5 m ulps, and grazing photons keep rho - b within a
// few hundred metres), so with e = n^2 - 1, D = rho_e - rho and u_chi^2 +
// cos^2 = 1 - u_a^2 = T the two are written cancellation-free:
//   N_j^2 = T (1 + e_0) + (e_j - e_0),
//   (rho N_j)^2 - L^2 = (1 + e_0) (rho^2 cos^2 - u_chi^2 D (2 rho_e - D)) + rho^2 (e_j - e_0),
// in units of rho_e^2, e_j - e_0 = (d_j - d_0)(2 + d_j + d_0).  The long sums
// are compensated.  Arguments: altitude dz above the observation level, u_a,
// |u_chi| and cos(zenith) at the emission point.  Returns false when a chord
// turns before its inner cylinder: the photon never meets the ground.
struct CylPath {
    float chi;     // angle swept about the axis [rad]
    float axial;   // drift along the axis [m]
    float ct;      // c t_path [m]
    float X, A;    // slant columns [g/cm^2], [m]
};
__device__ __noinline__ bool snell_path_cyl(const AtmParams& ap, float dz, float ua, float uchi, float cz, float dh,
                                            CylPath& out) {
    const int ns = max(1, (int)ceilf(dz / dh));
    const float step = dz / (float)ns;
    const bool refr = ap.refraction != 0;
    const float d0 = refr ? delta_at(ap, dz - 0.5f * step) : 0.0f;   // the first shell's n - 1
    const float e0 = d0 * (2.0f + d0);
    const float re = ap.rg + dz, ire = 1.0f / re, st = step * ire;
    const float T = fmaf(uchi, uchi, cz * cz);            // 1 - u_a^2 from the other two parts
    const float c2 = cz * cz, w2 = uchi * uchi;
    const float Lr = (1.0f + d0) * uchi, Aax = (1.0f + d0) * ua;   // L / rho_e and A
    float sChi = 0.0f, cChi = 0.0f, sAx = 0.0f, cAx = 0.0f, sCt = 0.0f, cCt = 0.0f, sX = 0.0f, sA = 0.0f;
    auto acc = [](float& s, float& c, float v) {
        float t, e;
        two_sum(s, v, t, e);
        s = t;
        c += e;
    };
    // (rho N)^2 - L^2 in units of rho_e^2 at depth d = D / rho_e (x = rho / rho_e = 1 - d)
    auto num = [&](float d, float de_) {
        const float x = 1.0f - d;
        return fmaf(1.0f + e0, fmaf(x * x, c2, -w2 * d * (2.0f - d)), x * x * de_);
    };
    bool reach = true;
    for (int j = 0; j < ns; ++j) {
        const float h = dz - ((float)j + 0.5f) * step;
        const float dc = (refr || ap.transmission) ? delta_at(ap, h) : 0.0f;   // the shell's n - 1
        const float dj = refr ? dc : 0.0f;                                      // in the geometry
        const float de_ = (dj - d0) * (2.0f + dj + d0);                          // e_j - e_0
        const float iN = rsqrtf(fmaxf(fmaf(T, 1.0f + e0, de_), 1e-30f));
        const float n_in = num((float)(j + 1) * st, de_);
        reach = reach && n_in > 0.0f;
        const float q_out = sqrtf(fmaxf(num((float)j * st, de_), 0.0f)) * iN;   // q / rho_e
        const float q_in = sqrtf(fmaxf(n_in, 0.0f)) * iN;
        const float xo = 1.0f - (float)j * st, xi = xo - st;
        const float sig = step * (xo + xi) * rcp_approx(q_out + q_in);   // transverse chord [m]
        const float s3 = sig * (1.0f + dj) * iN;                          // the chord in three dimensions
        acc(sChi, cChi, Lr * iN * sig * ire * rcp_approx(xi * xo));
        acc(sAx, cAx, sig * Aax * iN);
        acc(sCt, cCt, s3 * (1.0f + dj));
        if (ap.transmission) {
            sX = fmaf(dc, s3, sX);
            sA = fmaf(ex2_approx(ap.aer_c2 * h), s3, sA);
        }
    }
    out.chi = sChi + cChi;
    out.axial = sAx + cAx;
    out.ct = sCt + cCt;
    out.X = ap.rho_per_delta * sX;
    out.A = ap.aer_hobs * sA;
    return reach;
}

// Survival probability (Sec. 4.3.1) from the slant columns in table form
// (G_X = X cos, G_A = A cos): exp(-X / X_R(lambda) - tau_A(lambda) A / H_A).
__device__ __forceinline__ float transmission_T(const AtmParams& ap, float GX, float GA, float inv_l, float inv_uz) {
    const float il2 = inv_l * inv_l;
    const float kR = ap.kR0 * il2 * il2;
    const float kA = ap.kA0 * ex2_approx(ap.aer_alpha * lg2_approx(ap.lamA_nm * inv_l));
    return ex2_approx(-(GX * kR + GA * kA) * inv_uz);
}

// The correction fields at (dz, tan^2 of the local zenith) and the
// transmission: the network's outputs where it applies, else the bilinear
// table lookup; (0, 0, 1) without tables.
template <bool SURR, bool FIX = false>
__device__ __forceinline__ void correction_fields(const AtmParams& ap, bool use_net, const float (&net)[3], float dz,
                                                  float w, float inv_l, float inv_uz, float& GR, float& Gt,
                                                  float& Tr) {
    GR = 0.0f;
    Gt = 0.0f;
    Tr = 1.0f;
    if (!(FIX || ap.use_tables)) return;
    if (SURR && use_net) {
        GR = net[0];
        Gt = net[1];
        Tr = fminf(ex2_approx(net[2] * (float)kLog2e), 1.0f);   // the network gives ln T
    } else {
        // bilinear in (h, tan^2 theta0) on cells stored as value + change
        const float fh = dz * ap.tv.inv_dh, fw = w * ap.tv.inv_dw;
        const int j = min((int)fh, ap.tv.nh - 1);
        const int m = min((int)fw, ap.tv.nw - 2);
        const float fj = fh - (float)j, gm = fw - (float)m;
        const float4* row = ap.tv.tab + ((size_t)j * ap.tv.nw + m) * 2;
        const float4 v0 = __ldg(row), s0 = __ldg(row + 1), v1 = __ldg(row + 2), s1 = __ldg(row + 3);
        const float a0 = 1.0f - gm;
        // value + fj * change at both columns, then the column weights; two fields per packed instruction
        const float2 ff = make_float2(fj, fj), aa = make_float2(a0, a0), gg = make_float2(gm, gm);
        const float2 rt = __ffma2_rn(aa, __ffma2_rn(ff, make_float2(s0.x, s0.y), make_float2(v0.x, v0.y)),
                                     __fmul2_rn(gg, __ffma2_rn(ff, make_float2(s1.x, s1.y), make_float2(v1.x, v1.y))));
        GR = rt.x;
        Gt = rt.y;
        if (FIX || ap.transmission) {
            const float2 xa = __ffma2_rn(aa, __ffma2_rn(ff, make_float2(s0.z, s0.w), make_float2(v0.z, v0.w)),
                                         __fmul2_rn(gg, __ffma2_rn(ff, make_float2(s1.z, s1.w), make_float2(v1.z, v1.w))));
            Tr = transmission_T(ap, xa.x, xa.y, inv_l, inv_uz);
        }
    }
    if (!(FIX || ap.transmission)) Tr = 1.0f;
}

// Stages 3-5 for one bunch: generation on the cone (Sec. 4.2), the upward
// filter (Sec. 5.3.4), straight line (Eq. 3.3; on the sphere, the vacuum
// line to the ground sphere) plus the interpolation-tracing correction
// (Sec. 4.4.1) or the surrogate network, transmission (Sec. 4.3.1) and
// detection.  With SURR the whole warpgroup must call (inactive threads pass
// active = false): the network runs on the tensor cores for 128 photons.
// A bunch beyond the correction tables takes the exact path (Sec. 3.4.3),
// integrated for that bunch.  That integration lives in a second kernel, the
// exact pass, so that the photon kernel keeps its registers: MODE 0 (the
// photon kernel) returns true for such a bunch without counting or recording
// it; MODE 1 (the exact pass's scan) only returns whether the bunch lies
// beyond the tables; MODE 2 (the exact pass) propagates it along the exact
// path and counts it.
enum { kModeMain = 0, kModeCheck = 1, kModeExact = 2 };
template <bool SURR, bool SPH, bool REC, bool FL, bool TR, int MODE = kModeMain, bool FIX = false, typename SM>
__device__ __forceinline__ bool bunch(const SM& S, int q, int i, bool active, long long base,
                                      const PropParams& pp, const AtmParams& ap, const DetParams& dp,
                                      const OutParams& op, const SurrogateView& sv, TcSmem<kThreadsSur / 128>* tcs,
                                      Tally& T) {
    // The launch configuration; FIX instances are launched only for the standard one (refraction,
    // transmission and tables on; histogram, telescopes and time sums on; no camera optics), where
    // these are compile-time constants instead of parameter tests (the LV3 switch stays a test).
    static_assert(!(FIX && (SURR || FL || TR || MODE != kModeMain)), "the fixed configuration is the exact tracer's");
    const bool c_refr = FIX || ap.refraction, c_trans = FIX || ap.transmission, c_tables = FIX || ap.use_tables;
    const bool c_lv3 = pp.lv3 != 0, c_cam = !FIX && dp.cam_n > 0, c_hist = FIX || dp.nx > 0;
    const bool c_tel = FIX || dp.n_tel > 0, c_time = FIX || op.tel_time != nullptr;
    // ---- generation ------------------------------------------------------------
    const float4 Q = S.sub[q];
    const int segk = __float_as_int(Q.w);
    const int sg = segk & ((1 << kKShift) - 1), k = segk >> kKShift;
    const unsigned long long gid = pp.seg_base + (unsigned long long)(base + sg);
    const uint4 r4 = philox_rk((uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, (uint32_t)i, pp.rk);
    const float u0 = uniform24(r4.x), u1 = uniform24(r4.y), u2 = uniform24(r4.z), u3 = uniform24(r4.w);
    const float4 A = S.segA[sg], B = S.segB[sg];
    const float Px = A.x, Py = A.y, Pz = A.z;
    const unsigned int b = (unsigned int)S.bunch[sg];
    // translation to a random point of the sub-step (Fig. 4.2c)
    const float ell = ((float)k + u0) * B.z;
    // cone vector rotated into the track frame (Sec. 4.2): u = cos P + sin M e(phi),
    // M the 180-degree rotation about the bisector of (0,0,-1) and P
    float sphi, cphi;
    sincos_2pi(u1, sphi, cphi);
    const float inv_l_c = ap.inv_l1_nm - u2 * ap.dinv_l_nm;   // 1/lambda^2 spectrum
    const float ce = (Px * cphi + Py * sphi) * A.w;
    const float ct = Q.x, st = Q.y;
    // x and y components two lanes per packed FP32 instruction
    const float2 mxy = __ffma2_rn(make_float2(Px, Py), make_float2(ce, ce), make_float2(-cphi, -sphi));
    const float mz = (Pz - 1.0f) * ce;
    const float2 uxy_c = __ffma2_rn(make_float2(ct, ct), make_float2(Px, Py), __fmul2_rn(make_float2(st, st), mxy));
    const float uz_c = ct * Pz + st * mz;
    float2 uxy_f = uxy_c;
    float uz_f = uz_c, inv_l_f = inv_l_c;
    if constexpr (FL) {   // fluorescence (Sec. 4.2.2): isotropic, the line from a second draw
        const float c = pp.emission == CS_EMIT_FLUORESCENCE_HALF ? u2 - 1.0f : fmaf(2.0f, u2, -1.0f);
        const float sn = sqrtf(fmaxf(fmaf(-c, c, 1.0f), 0.0f));
        uxy_f = make_float2(sn * cphi, sn * sphi);
        uz_f = c;
        inv_l_f = fluorescence_line(pp, (uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, (uint32_t)i);
    }
    const float2 uxy = FL ? uxy_f : uxy_c;
    const float uz = FL ? uz_f : uz_c, inv_l = FL ? inv_l_f : inv_l_c;
    const float ux = uxy.x, uy = uxy.y;
    // height above the observation level and the local zenith
    float dz, cos_z, sin2;
    float4 Cc, Dd;
    float dvx = 0.0f, dvy = 0.0f, dvz = 0.0f, hx = 0.0f, hy = 0.0f, hz = 0.0f;
    if (!SPH) {
        dz = B.x + (B.y + ell * Pz);
        cos_z = -uz;
        sin2 = ux * ux + uy * uy;
    } else {
        Cc = S.segC[sg];
        Dd = S.segD[sg];
        // tilt of the local vertical at the start, v - z-hat = (x / r, y / r, B.y)
        const float ex = Cc.x * Dd.w, ey = Cc.y * Dd.w, ez = B.y;
        dz = B.x + ell * fmaf(ell * 0.5f * Dd.w, fmaf(-Cc.w, Cc.w, 1.0f), Cc.w);
        const float f = ell * Dd.w;   // the local vertical turns by ell / r along the track
        dvx = ex + f * (Px - Cc.w * ex);
        dvy = ey + f * (Py - Cc.w * ey);
        dvz = ez + f * (Pz - Cc.w * (1.0f + ez));
        cos_z = -(uz + ux * dvx + uy * dvy + uz * dvz);
        hx = ux + cos_z * dvx;
        hy = uy + cos_z * dvy;
        hz = uz + cos_z * (1.0f + dvz);
        sin2 = hx * hx + hy * hy + hz * hz;
    }
    const float inv_uz = rcp_approx(cos_z);
    const float w = sin2 * inv_uz * inv_uz;   // tan^2 of the local zenith
    int status = CS_ST_LANDED;
    if (!(cos_z > 0.0f)) status = CS_ST_UPWARD;              // discarded (Sec. 5.3.4)
    else if (dz < 0.0f) status = CS_ST_BELOW;
    // beyond the correction tables (steeper than their largest zenith or above their
    // top): the exact path is integrated for this photon instead (Sec. 3.4.3)
    const bool beyond = c_tables && !(TR && c_refr) && (w > ap.tv.w_max || dz >= ap.tv.dz_max);
    if constexpr (MODE == kModeCheck) return status == CS_ST_LANDED && beyond;
    if constexpr (MODE == kModeMain && !SURR) {
        if (status == CS_ST_LANDED && beyond) return true;   // left to the exact pass
    }

    // ---- the surrogate network, warp-collective --------------------------------
    float net[3] = {0.0f, 0.0f, 1.0f};
    bool use_net = false;
    if (SURR) {
        use_net = active && status == CS_ST_LANDED && in_surrogate_domain(sv, dz, cos_z);
        const float x[3] = {use_net ? fmaf(sv.in_scale[0], height_coordinate(sv, dz), sv.in_shift[0]) : 0.0f,
                            use_net ? fmaf(sv.in_scale[1], cos_z, sv.in_shift[1]) : 0.0f,
                            use_net ? fmaf(sv.in_scale[2], inv_l, sv.in_shift[2]) : 0.0f};
        float y[3];
        const bool ok = sv.split ? net128_tc<true>(sv, *tcs, x, y) : net128_tc<false>(sv, *tcs, x, y);
        use_net = use_net && ok;   // a tensor-core wait that gave up: the tables take over
        if (use_net) {   // the network's part plus the first-order baseline
            const float3 bl = surrogate_baseline(sv, dz, cos_z, inv_l);
            net[0] = fmaf(sv.out_half[0], y[0], sv.out_mid[0]) + bl.x;
            net[1] = fmaf(sv.out_half[1], y[1], sv.out_mid[1]) + bl.y;
            net[2] = fmaf(sv.out_half[2], y[2], sv.out_mid[2]) + bl.z;
        }
    }
    if (!active) return false;
    if constexpr (MODE == kModeMain && SURR) {
        if (status == CS_ST_LANDED && beyond) return true;   // left to the exact pass
    }

    // ---- propagation and detection -----------------------------------------------
    int tel = -1, bin = -1, pix = -1;
    float x = 0.0f, y = 0.0f, xl = 0.0f, yl = 0.0f, t_rel = ell * B.w;   // ground point x + xl, y + yl
    float rx = 0.0f, ry = 0.0f;
    if (status == CS_ST_LANDED && !SPH) {
        if (Pz < -1e-3f && !FL) {
            // I - G = dz (P_xy / P_z - u_xy / u_z); the numerator is sin(theta) (P x m)
            const float pmx = Pz * sphi - ce * Py, pmy = ce * Px - Pz * cphi;
            const float fac = dz * st * rcp_approx(Pz * uz);
            rx = -fac * pmy;
            ry = fac * pmx;
        } else {   // (near-)horizontal track: the origin is its start point
            rx = ell * Px + dz * ux * inv_uz;
            ry = ell * Py + dz * uy * inv_uz;
        }
        if (c_lv3) {   // LV3 photon pre-filter (Sec. 4.3.4): the straight line's landing point
            const float4 Cg = S.segC[sg];
            const float sx = (Cg.x - pp.lv3_c[0]) + (Cg.y + rx), sy = (Cg.z - pp.lv3_c[1]) + (Cg.w + ry);
            if (fmaf(sx, sx, fmaf(sy, sy, pp.lv3_dz2)) > pp.lv3_r2) status = CS_ST_LV3;
        }
    }
    if (status == CS_ST_LANDED && !SPH) {
        float path = dz * inv_uz;
        float GR, Gt, Tr;
        if (TR && c_refr) {   // the per-photon stepper instead of the tables
            const float4 sp = snell_path(ap, dz, cos_z, pp.snell_dh);
            const float2 r2 = __ffma2_rn(make_float2(sp.x, sp.x), uxy, make_float2(rx, ry));
            rx = r2.x;
            ry = r2.y;
            path = sp.y;
            Tr = 1.0f;
            if (c_trans) {
                const float il2 = inv_l * inv_l;
                const float kA = ap.kA0 * ex2_approx(ap.aer_alpha * lg2_approx(ap.lamA_nm * inv_l));
                Tr = ex2_approx(-(sp.z * (ap.kR0 * il2 * il2) + sp.w * kA));
            }
        } else {
            if (MODE == kModeExact && beyond) {   // the exact path, integrated for this photon
                bool reach;
                const float4 f = exact_fields_planar(ap.self, dz, cos_z, reach);
                GR = f.x;
                Gt = f.y;
                Tr = c_trans ? transmission_T(ap, f.z, f.w, inv_l, inv_uz) : 1.0f;
                if (!reach) status = CS_ST_NO_GROUND;   // reflected back up by an inverted profile
            } else {
                correction_fields<SURR, FIX>(ap, use_net, net, dz, w, inv_l, inv_uz, GR, Gt, Tr);
            }
            if (c_refr) {
                const float c3 = GR * inv_uz * inv_uz * inv_uz;
                const float2 r2 = __ffma2_rn(make_float2(c3, c3), uxy, make_float2(rx, ry));
                rx = r2.x;
                ry = r2.y;
                path = fmaf(Gt, inv_uz, path);
            }
        }
        t_rel = fmaf(path, kInvC, t_rel);
        const float4 Cg = S.segC[sg];
        if (REC) {   // records carry the ground point as float-float
            two_sum(Cg.x, rx, x, xl);
            xl += Cg.y;
            two_sum(Cg.z, ry, y, yl);
            yl += Cg.w;
        } else {     // the telescope hash only needs its cell
            x = Cg.x + (Cg.y + rx);
            y = Cg.z + (Cg.w + ry);
        }
        if (status != CS_ST_LANDED) {
            // the path never meets the observation level: missed
        } else if (c_trans && !(u3 < Tr)) {
            status = CS_ST_ABSORBED;
        } else {
            const int sh = S.shower[sg];
            if (c_hist) {   // ground cell = floor(G_cells + r / d); rounding < 3e-5 cells
                const float4 D = S.segD[sg];
                const int ix = (int)floorf(D.x + fmaf(rx, dp.inv_dx, D.y));
                const int iy = (int)floorf(D.z + fmaf(ry, dp.inv_dy, D.w));
                if (ix >= 0 && ix < dp.nx && iy >= 0 && iy < dp.ny) {
                    bin = iy * dp.nx + ix;
                    hist_add(op, (unsigned int)(sh * dp.ny * dp.nx + bin), b);
                }
            }
            if (c_tel) {
                // arrival direction: n sin(theta) conserved, azimuth kept
                const float sc = c_refr ? (1.0f + Q.z) * ap.inv_n_obs : 1.0f;
                const float s2 = (ux * ux + uy * uy) * (sc * sc);
                // the narrowest hash that serves; when every active lane's arrival fits the
                // first, its fields are constant operands (no indexed parameter loads)
                const bool lvl0 = s2 <= dp.hash[0].sin2_max;
                auto detect = [&](const TelHash& H, const bool hashed) {
                if (!hashed || (x >= H.bx0 && x < H.bx1 && y >= H.by0 && y < H.by1)) {
                    float ugz = uz;
                    if (c_refr) {
                        const float c2 = fmaxf(1.0f - s2, 1e-30f);
                        ugz = -c2 * rsqrtf(c2);
                    }
                    tel = hit_telescope(
                        dp, H, hashed, x, y, ux * sc, uy * sc, ugz,
                        [&](const float4& D, float cx0, float cy0, float& ddx, float& ddy, float& ddz) {
                            ddx = D.x - ((Cg.x - cx0) + (Cg.y + rx));
                            ddy = D.y - ((Cg.z - cy0) + (Cg.w + ry));
                            ddz = D.z;
                        },
                        [&](int it, float& ddx, float& ddy, float& ddz, float& r) {
                            const float4 T4 = __ldg(dp.tel + it);
                            const float2 TL = __ldg(dp.tel_lo + it);
                            ddx = (T4.x - Cg.x) + ((TL.x - Cg.y) - rx);
                            ddy = (T4.y - Cg.z) + ((TL.y - Cg.w) - ry);
                            ddz = T4.z;
                            r = T4.w;
                        });
                    if (tel >= 0 && c_cam) {
                        const float4 T4 = __ldg(dp.tel + tel);
                        const float2 TL = __ldg(dp.tel_lo + tel);
                        pix = camera_pixel(dp, (T4.x - Cg.x) + ((TL.x - Cg.y) - rx),
                                           (T4.y - Cg.z) + ((TL.y - Cg.w) - ry), T4.z, ux * sc, uy * sc, ugz);
                        pix = optics_survival(dp, pp, gid, k, i, inv_l, pix);
                    }
                }
                };
                if (__all_sync(__activemask(), lvl0)) detect(dp.hash[0], true);
                else detect(dp.hash[lvl0 ? 0 : (s2 <= dp.hash[1].sin2_max ? 1 : 2)], s2 <= dp.hash[2].sin2_max);
                if (tel >= 0) {
                    const size_t slot = (size_t)sh * dp.n_tel + tel;
                    atomicAdd(op.tel_counts + slot, (unsigned long long)b);
                    if (c_time) atomicAdd(op.tel_time + slot, (double)b * (S.t0[sg] + (double)t_rel));
                    if (pix >= 0) atomicAdd(op.camera + (slot * dp.cam_n * dp.cam_n + pix), (unsigned long long)b);
                }
            }
        }
    } else if (TR && ap.cylindrical && status == CS_ST_LANDED) {
        // the cylindrical atmosphere (Sec. 3.3.3): emission point E = start + ell P in
        // float-float, e_r the horizontal unit towards its foot, e_a = z x e_r the axis
        float Ex, Exl, Ey, Eyl;
        two_sum(Cc.x, fmaf(ell, Px, Dd.x), Ex, Exl);
        two_sum(Cc.y, fmaf(ell, Py, Dd.y), Ey, Eyl);
        const float dE2 = Ex * Ex + Ey * Ey;
        float erx = 1.0f, ery = 0.0f;
        if (dE2 > 0.0f) {
            const float id = rsqrtf(dE2);
            erx = Ex * id;
            ery = Ey * id;
        }
        // the local vertical v = sin(chi_E) e_r + cos(chi_E) z; u's parts along the axis
        // and along the transverse tangent e_chi = cos(chi_E) e_r - sin(chi_E) z
        const float s_chi = dvx * erx + dvy * ery, c_chi = 1.0f + dvz;
        const float ua = uy * erx - ux * ery;
        const float uchi = c_chi * (ux * erx + uy * ery) - s_chi * uz;
        CylPath cp;
        if (!snell_path_cyl(ap, dz, ua, fabsf(uchi), cos_z, pp.snell_dh, cp)) status = CS_ST_NO_GROUND;
        // ground point on the unrolled cylinder: E's footprint r_g chi_E e_r (the
        // azimuthal-equidistant point of E, x = E_x - E_x om as on the sphere) plus the
        // sweep along e_r and the drift along e_a
        const float irg = ap.inv_rg, rg = ap.rg, h_obs_f = (float)ap.h_obs;
        const float eta = ((Cc.z - h_obs_f) + (Dd.z + ell * Pz)) * irg, ie = rcp_approx(1.0f + eta);
        const float X2 = dE2 * (irg * irg) * (ie * ie);
        const float one_m_s = X2 < 0.01f ? X2 * fmaf(X2, -0.2f, 1.0f / 3.0f) : 1.0f - atanf(sqrtf(X2)) * rsqrtf(X2);
        const float om = (eta + one_m_s) * ie;
        const float dr = copysignf(cp.chi, uchi) * rg, da = cp.axial;
        x = Ex;
        xl = fmaf(-Ex, om, Exl) + fmaf(dr, erx, -da * ery);
        y = Ey;
        yl = fmaf(-Ey, om, Eyl) + fmaf(dr, ery, da * erx);
        two_sum(x, xl, x, xl);
        two_sum(y, yl, y, yl);
        t_rel = fmaf(cp.ct, kInvC, t_rel);
        float Tr = 1.0f;
        if (c_trans) {
            const float il2 = inv_l * inv_l;
            const float kA = ap.kA0 * ex2_approx(ap.aer_alpha * lg2_approx(ap.lamA_nm * inv_l));
            Tr = ex2_approx(-(cp.X * (ap.kR0 * il2 * il2) + cp.A * kA));
        }
        if (status != CS_ST_LANDED) {
            // turned above the ground: missed
        } else if (c_trans && !(u3 < Tr)) {
            status = CS_ST_ABSORBED;
        } else {
            const int sh = S.shower[sg];
            if (c_hist) {
                const int ix = (int)floorf(((x - dp.hx0_hi) + (xl - dp.hx0_lo)) * dp.inv_dx);
                const int iy = (int)floorf(((y - dp.hy0_hi) + (yl - dp.hy0_lo)) * dp.inv_dy);
                if (ix >= 0 && ix < dp.nx && iy >= 0 && iy < dp.ny) {
                    bin = iy * dp.nx + ix;
                    hist_add(op, (unsigned int)(sh * dp.ny * dp.nx + bin), b);
                }
            }
            if (c_tel) {
                // arrival direction in the unrolled frame: n u_a and n rho u_chi conserved
                const float ratio = c_refr ? (1.0f + delta_at(ap, dz)) * ap.inv_n_obs : 1.0f;   // n_e / n_g
                const float uga = ratio * ua, ugc = ratio * fmaf(dz, irg, 1.0f) * uchi;
                const float ugz = -sqrtf(fmaxf(1.0f - uga * uga - ugc * ugc, 0.0f));
                const float ugx = ugc * erx - uga * ery, ugy = ugc * ery + uga * erx;
                const float xs = x + xl, ys = y + yl;
                const float sg2 = ugx * ugx + ugy * ugy;
                const bool lvl0 = sg2 <= dp.hash[0].sin2_max;
                auto detect = [&](const TelHash& H, const bool hashed) {
                if (!hashed || (xs >= H.bx0 && xs < H.bx1 && ys >= H.by0 && ys < H.by1)) {
                    tel = hit_telescope(
                        dp, H, hashed, xs, ys, ugx, ugy, ugz,
                        [&](const float4& D, float cx0, float cy0, float& ddx, float& ddy, float& ddz) {
                            ddx = D.x - ((x - cx0) + xl);
                            ddy = D.y - ((y - cy0) + yl);
                            ddz = D.z;
                        },
                        [&](int it, float& ddx, float& ddy, float& ddz, float& r) {
                            const float4 T4 = __ldg(dp.tel + it);
                            const float2 TL = __ldg(dp.tel_lo + it);
                            ddx = (T4.x - x) + (TL.x - xl);
                            ddy = (T4.y - y) + (TL.y - yl);
                            ddz = T4.z;
                            r = T4.w;
                        });
                    if (tel >= 0 && c_cam) {
                        const float4 T4 = __ldg(dp.tel + tel);
                        const float2 TL = __ldg(dp.tel_lo + tel);
                        pix = camera_pixel(dp, (T4.x - x) + (TL.x - xl), (T4.y - y) + (TL.y - yl), T4.z, ugx, ugy, ugz);
                        pix = optics_survival(dp, pp, gid, k, i, inv_l, pix);
                    }
                }
                };
                if (__all_sync(__activemask(), lvl0)) detect(dp.hash[0], true);
                else detect(dp.hash[lvl0 ? 0 : (sg2 <= dp.hash[1].sin2_max ? 1 : 2)], sg2 <= dp.hash[2].sin2_max);
                if (tel >= 0) {
                    const size_t slot = (size_t)sh * dp.n_tel + tel;
                    atomicAdd(op.tel_counts + slot, (unsigned long long)b);
                    if (c_time) atomicAdd(op.tel_time + slot, (double)b * (S.t0[sg] + (double)t_rel));
                    if (pix >= 0) atomicAdd(op.camera + (slot * dp.cam_n * dp.cam_n + pix), (unsigned long long)b);
                }
            }
        }
    } else if (status == CS_ST_LANDED) {
        // vacuum straight line to the ground sphere r_g: length t with
        // t (r_e cos + sqrt(r_e^2 cos^2 - D)) = D, D = r_e^2 - r_g^2 = dz (r_e + r_g)
        const float rg = ap.rg, re = rg + dz;
        const float D2 = dz * (rg + re);
        const float disc = fmaxf(re * re * cos_z * cos_z - D2, 0.0f);
        const float tt = D2 * rcp_approx(re * cos_z + sqrtf(disc));
        const float h_obs_f = (float)ap.h_obs;
        // ground point G = start (float-float) + offset, kept as float-float (Gx + Gxl, ...):
        // the offset is as long as the photon's path, the start may lie tens of km out
        float Gx, Gy, Gz, Gxl, Gyl, Gzl;
        auto set_G = [&](float ox, float oy, float oz) {
            two_sum(Cc.x, Dd.x + ox, Gx, Gxl);
            two_sum(Cc.y, Dd.y + oy, Gy, Gyl);
            two_sum(Cc.z, Dd.z + oz, Gz, Gzl);
        };
        set_G(fmaf(ell, Px, tt * ux), fmaf(ell, Py, tt * uy), fmaf(ell, Pz, tt * uz));
        if (c_lv3) {   // LV3 photon pre-filter (Sec. 4.3.4): the straight line's landing point
            const float sx = Gx - pp.lv3_c[0], sy = Gy - pp.lv3_c[1], sz = Gz - pp.lv3_c[2];
            if (fmaf(sx, sx, fmaf(sy, sy, sz * sz)) > pp.lv3_r2) status = CS_ST_LV3;
        }
        float GR = 0.0f, Gt = 0.0f, Tr = 1.0f;
        const bool stepper = TR && c_refr;
        bool direct = false;   // landing point from the path's central angle
        // G = E + (r_g cos Phi - r_e) v_E + r_g sin Phi h_E, with
        // r_g cos Phi - r_e = -(dz + 2 r_g sin^2(Phi / 2)) and h_E = (u + cos v_E) / sin
        auto land_at = [&](float Phi) {
            // a central angle within the atmosphere stays below 0.4 rad: Taylor terms to x^11
            auto sin_small = [](float x) {
                const float x2 = x * x;
                return x * fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, -2.5052108e-8f, 2.7557319e-6f),
                                                              -1.9841270e-4f), 8.3333333e-3f), -1.6666667e-1f), 1.0f);
            };
            const float sP = sin_small(Phi), sh = sin_small(0.5f * Phi);
            const float down = fmaf(2.0f * rg * sh, sh, dz), along = rg * sP * rsqrtf(sin2);
            set_G(fmaf(ell, Px, fmaf(along, hx, -down * dvx)), fmaf(ell, Py, fmaf(along, hy, -down * dvy)),
                  fmaf(ell, Pz, fmaf(along, hz, -down * (1.0f + dvz))));
        };
        // Does the path meet the ground sphere?  Inside the tables' domain (zenith <= 75 deg,
        // below the top of the atmosphere) it always does; straight lines, the stepper and
        // photons beyond the tables are checked.
        if (status == CS_ST_LANDED) {
            if (!c_refr) {   // the straight line: r_g > r_e sin(psi) <=> r_e (1 - sin) > dz
                const float s0 = sqrtf(sin2);
                if (!(fmaf(re, cos_z * cos_z / (1.0f + s0), -dz) > 0.0f)) status = CS_ST_NO_GROUND;
            } else if ((stepper || (MODE == kModeExact && beyond)) && !sph_reaches(ap.self, dz, cos_z, sqrtf(sin2))) {
                status = CS_ST_NO_GROUND;
            }
        }
        if (status == CS_ST_LANDED) {
            if (stepper) {   // the per-photon stepper instead of the tables
                bool absolute;
                const float4 sp = snell_path_sph(ap, dz, sin2, pp.snell_dh, absolute);
                GR = sp.x;   // here the arc-length correction itself
                Gt = sp.y;   // and the delay as a length
                if (absolute) {   // no straight line to the ground: land from the central angle
                    direct = true;
                    land_at(sp.x * ap.inv_rg);
                }
                Tr = 1.0f;
                if (c_trans) {
                    const float il2 = inv_l * inv_l;
                    const float kA = ap.kA0 * ex2_approx(ap.aer_alpha * lg2_approx(ap.lamA_nm * inv_l));
                    Tr = ex2_approx(-(sp.z * (ap.kR0 * il2 * il2) + sp.w * kA));
                }
            } else if (MODE == kModeExact && beyond) {   // the exact path, integrated for this photon
                const float4 f = exact_fields_sph(ap.self, dz, cos_z, sqrtf(sin2));
                Tr = c_trans ? transmission_T(ap, f.z, f.w, inv_l, inv_uz) : 1.0f;
                if (c_refr) {
                    direct = true;
                    land_at(f.x);
                    Gt = f.y;   // c t_path itself
                }
            } else {
                correction_fields<SURR, FIX>(ap, use_net, net, dz, w, inv_l, inv_uz, GR, Gt, Tr);
            }
        }
        if (status == CS_ST_LANDED) {
            // ground tangent in the plane of travel at the landing point
            const float irg = ap.inv_rg;
            const float gvx = Gx * irg, gvy = Gy * irg, gvz = (Gz - h_obs_f) * irg;   // v_G - z-hat
            const float uvG = ux * gvx + uy * gvy + uz * (1.0f + gvz);
            float tx = ux - uvG * gvx, ty = uy - uvG * gvy, tz = uz - uvG * (1.0f + gvz);
            const float tn = rsqrtf(fmaxf(tx * tx + ty * ty + tz * tz, 1e-30f));
            tx *= tn;
            ty *= tn;
            tz *= tn;
            float path = direct ? Gt : tt;
            if (c_refr && !direct) {   // arc-length correction along the ground, delay
                const float dR = stepper ? GR : GR * inv_uz * inv_uz * inv_uz * sqrtf(sin2);
                Gxl = fmaf(dR, tx, Gxl);
                Gyl = fmaf(dR, ty, Gyl);
                Gzl = fmaf(dR, tz, Gzl);
                path = stepper ? path + Gt : fmaf(Gt, inv_uz, path);
            }
            t_rel = fmaf(path, kInvC, t_rel);
            // azimuthal-equidistant coordinates: x = G_x r_g atan(X) / (X z_c), X = rho / z_c,
            // z_c = r_g (1 + eta); written x = G_x - G_x om with the small om = 1 - r_g atan(X) /
            // (X z_c) = (eta + (1 - atan(X) / X)) / (1 + eta), kept as float-float
            const float eta = ((Gz - h_obs_f) + Gzl) * irg, ie = rcp_approx(1.0f + eta);
            const float X2 = (Gx * Gx + Gy * Gy) * (irg * irg) * (ie * ie);
            // 1 - atan(X) / X by its series near the centre; far landings (X^2 > 0.01, beyond
            // ~600 km, only photons beyond the tables' zenith) take the library arctangent
            const float one_m_s = X2 < 0.01f ? X2 * fmaf(X2, -0.2f, 1.0f / 3.0f) : 1.0f - atanf(sqrtf(X2)) * rsqrtf(X2);
            const float om = (eta + one_m_s) * ie;
            x = Gx;
            xl = fmaf(-Gx, om, Gxl);
            y = Gy;
            yl = fmaf(-Gy, om, Gyl);
            const float xs = x + xl, ys = y + yl;   // single floats for the box and hash tests
            if (c_trans && !(u3 < Tr)) {
                status = CS_ST_ABSORBED;
            } else {
                const int sh = S.shower[sg];
                if (c_hist) {
                    const int ix = (int)floorf(((x - dp.hx0_hi) + (xl - dp.hx0_lo)) * dp.inv_dx);
                    const int iy = (int)floorf(((y - dp.hy0_hi) + (yl - dp.hy0_lo)) * dp.inv_dy);
                    if (ix >= 0 && ix < dp.nx && iy >= 0 && iy < dp.ny) {
                        bin = iy * dp.nx + ix;
                        hist_add(op, (unsigned int)(sh * dp.ny * dp.nx + bin), b);
                    }
                }
                if (c_tel) {
                    float ugx = ux, ugy = uy, ugz = uz;
                    if (c_refr) {   // Bouguer: n r sin(psi) conserved in the plane of travel
                        const float sin_g = (1.0f + Q.z) * ap.inv_n_obs * re * irg * sqrtf(sin2);
                        const float cos_g = sqrtf(fmaxf(1.0f - sin_g * sin_g, 0.0f));
                        ugx = -cos_g * gvx + sin_g * tx;
                        ugy = -cos_g * gvy + sin_g * ty;
                        ugz = -cos_g * (1.0f + gvz) + sin_g * tz;
                    }
                    const float sg2 = ugx * ugx + ugy * ugy;
                    const bool lvl0 = sg2 <= dp.hash[0].sin2_max;
                    auto detect = [&](const TelHash& H, const bool hashed) {
                    if (!hashed || (xs >= H.bx0 && xs < H.bx1 && ys >= H.by0 && ys < H.by1)) {
                        auto delta3 = [&](const float4& T3, float& ddx, float& ddy, float& ddz) {
                            ddx = (T3.x - Gx) - Gxl;
                            ddy = (T3.y - Gy) - Gyl;
                            ddz = (T3.z - Gz) - Gzl;
                        };
                        tel = hit_telescope(
                            dp, H, hashed, xs, ys, ugx, ugy, ugz,
                            [&](const float4& D, float, float, float& ddx, float& ddy, float& ddz) { delta3(D, ddx, ddy, ddz); },
                            [&](int it, float& ddx, float& ddy, float& ddz, float& r) {
                                const float4 T3 = __ldg(dp.tel3 + it);
                                delta3(T3, ddx, ddy, ddz);
                                r = T3.w;
                            });
                        if (tel >= 0 && c_cam) {
                            const float4 T3 = __ldg(dp.tel3 + tel);
                            pix = camera_pixel(dp, (T3.x - Gx) - Gxl, (T3.y - Gy) - Gyl, (T3.z - Gz) - Gzl, ugx, ugy, ugz);
                            pix = optics_survival(dp, pp, gid, k, i, inv_l, pix);
                        }
                    }
                    };
                    if (__all_sync(__activemask(), lvl0)) detect(dp.hash[0], true);
                    else detect(dp.hash[lvl0 ? 0 : (sg2 <= dp.hash[1].sin2_max ? 1 : 2)], sg2 <= dp.hash[2].sin2_max);
                    if (tel >= 0) {
                        const size_t slot = (size_t)sh * dp.n_tel + tel;
                        atomicAdd(op.tel_counts + slot, (unsigned long long)b);
                        if (c_time) atomicAdd(op.tel_time + slot, (double)b * (S.t0[sg] + (double)t_rel));
                        if (pix >= 0) atomicAdd(op.camera + (slot * dp.cam_n * dp.cam_n + pix), (unsigned long long)b);
                    }
                }
            }
        }
    }
    T.absorbed += status == CS_ST_ABSORBED ? b : 0;
    T.upward += status == CS_ST_UPWARD ? b : 0;
    T.hist += bin >= 0 ? b : 0;
    T.tel += tel >= 0 ? b : 0;
    if (REC) emit_record(op, gid, k, i, x, xl, y, yl, t_rel, inv_l, tel, bin, status, pix);
    return false;
}

// Per-launch scratch (zeroed before the photon kernel): the photon kernel's
// work counter, the exact pass's cursor, the number of listed groups and the
// number of queued bunches; then one bit per group of pp.tiles_per_bit warp
// tiles (32 segments) that hold a bunch beyond the correction tables the
// queue could not take, the list of the marked groups (each entered once,
// when its bit is first set), and the queue of bunches beyond the tables
// ({segment index lo, hi, sub-step, bunch} per entry, 16-byte aligned).
constexpr int kScratchCounters = 4;
__host__ __device__ constexpr size_t scratch_groups(long long n_wtiles, int tiles_per_bit) {
    return (size_t)((n_wtiles + tiles_per_bit - 1) / tiles_per_bit);
}
__host__ __device__ constexpr size_t scratch_queue_off(long long n_wtiles, int tiles_per_bit) {
    return (kScratchCounters + (scratch_groups(n_wtiles, tiles_per_bit) + 31) / 32 + scratch_groups(n_wtiles, tiles_per_bit) +
            3) & ~(size_t)3;
}
__host__ __device__ constexpr size_t scratch_words(long long n_wtiles, int tiles_per_bit, unsigned int q_cap = 0) {
    return scratch_queue_off(n_wtiles, tiles_per_bit) + 4 * (size_t)q_cap;
}
// Queue entries for n_wtiles warp tiles: per_tile per tile (default eight; below zero, none),
// at least 4096 and at most 2^22 (64 MB).
__host__ __device__ constexpr unsigned int queue_cap(long long n_wtiles, int per_tile = 0) {
    return per_tile < 0 ? 0u
                        : (unsigned int)(n_wtiles * (per_tile ? per_tile : 8) < (1ll << 22)
                                             ? (n_wtiles * (per_tile ? per_tile : 8) > 4096 ? n_wtiles * (per_tile ? per_tile : 8) : 4096)
                                             : (1ll << 22));
}
// The part that must start at zero: the counters and the map (the list is written before it is read).
__host__ __device__ constexpr size_t scratch_zero_words(long long n_wtiles, int tiles_per_bit) {
    return kScratchCounters + (scratch_groups(n_wtiles, tiles_per_bit) + 31) / 32;
}

// Marks group g for the exact pass (bit and, the first time, list entry).
__device__ __forceinline__ void mark_group(unsigned int* scratch, long long n_wtiles, int tiles_per_bit, unsigned int g) {
    unsigned int* bits = scratch + kScratchCounters;
    const unsigned int bit = 1u << (g & 31);
    if (!(atomicOr(bits + (g >> 5), bit) & bit)) {
        unsigned int* list = bits + (scratch_groups(n_wtiles, tiles_per_bit) + 31) / 32;
        list[atomicAdd(scratch + 2, 1u)] = g;
    }
}

// The photon kernel (EX = false) and the exact pass (EX = true, exact-tracer
// instances only): the exact pass walks the same warp tiles, skips those
// whose bit the photon kernel left clear, regenerates the sub-steps and
// bunches of the others from their keyed draws, and propagates the bunches
// beyond the tables along the exact path, 32 at a time per warp.
template <bool SURR, bool SPH, int MINB, bool REC, bool FL = false, bool TR = false, bool EX = false,
          bool FIX = false, int NT = SURR ? kThreadsSur : kThreads>
__global__ void __launch_bounds__(NT, MINB)
propagate_kernel(const PropParams pp, const AtmParams ap, const DetParams dp, const OutParams op,
                 unsigned int* scratch, const SurrogateView sv) {
    static_assert(!(EX && SURR), "the exact pass runs the exact-tracer form");
    // The exact pass is launched as a programmatic dependent of the photon kernel: its blocks
    // become resident as the photon kernel's retire and wait here for its completion (and its
    // memory); the photon kernel lets it launch from the start.  Without the launch attribute
    // both instructions are no-ops.
    if (EX) asm volatile("griddepcontrol.wait;" ::: "memory");
    else asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (EX && __ldcg(scratch + 2) == 0 && __ldcg(scratch + 3) == 0) return;   // no bunch beyond the tables
    unsigned int* const tile_ctr = scratch + (EX ? 1 : 0);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TileSmem& S = *reinterpret_cast<TileSmem*>(smem_raw);
    TcSmem<kThreadsSur / 128>* tcs = SURR ? reinterpret_cast<TcSmem<kThreadsSur / 128>*>(smem_raw + kTcSmemOffset) : nullptr;
    const int t = threadIdx.x;
    if (SURR) tc_setup(*tcs, sv);
    const long long n_tiles = (pp.n + kTile - 1) / kTile;
    unsigned int emitted = 0, invalid = 0, dropped = 0;
    Tally T = {0, 0, 0, 0};
    int buf = 0;

    if constexpr (!SURR) {
        // ---- warps on their own: tiles of 32 segments, warp scans, no block barrier
        WarpSmem& W = reinterpret_cast<WarpSmem*>(smem_raw)[t >> 5];
        const int lane = t & 31;
        const long long n_wtiles = (pp.n + kWTile - 1) / kWTile;
        auto process_tile = [&](const long long tile) {
            const long long base = tile * kWTile;
            bool any_beyond = false;   // a bunch of this tile left to the exact pass
            const int Kt0 = base + lane < pp.n
                                ? import_segment<SPH, FL>(W, lane, pp.segs + base + lane, pp, ap, dp, invalid, dropped)
                                : 0;
            // The warp takes its segments in order of their ground footprint's distance
            // from the LV3 centre (the frame origin unless the filter is on), so that the
            // bunches of a warp round tend to land together: the telescope cells, histogram
            // rows and statuses of a round agree more often (measured 2-3 % faster), and with
            // the LV3 pre-filter whole rounds skip the correction (1.08x on the inclined
            // shower).  The draws stay keyed by the segments' own indices.
            int slot = lane;
            {
                float key = 3.0e38f;   // empty slots last
                if (Kt0 > 0) {
                    const float4 A = W.segA[lane], C = W.segC[lane];
                    float gx, gy;
                    if (SPH) {   // start point carried along P to the observation level
                        const float f = fmaxf(W.segB[lane].x, 0.0f) * rcp_approx(fmaxf(-C.w, 0.05f));
                        gx = fmaf(f, A.x, C.x);
                        gy = fmaf(f, A.y, C.y);
                    } else if (FL) {   // fluorescence keeps the start point as the origin
                        const float f = fmaxf(W.segB[lane].x, 0.0f) * rcp_approx(fmaxf(-A.z, 0.05f));
                        gx = fmaf(f, A.x, C.x);
                        gy = fmaf(f, A.y, C.z);
                    } else {     // the ground intercept
                        gx = C.x;
                        gy = C.z;
                    }
                    gx -= pp.lv3_c[0];
                    gy -= pp.lv3_c[1];
                    key = fmaf(gx, gx, gy * gy);
                }
                // bitonic sort across the warp, ascending, of one 32-bit word per lane: the
                // key's bits (a non-negative float orders as an unsigned integer) with its low
                // five bits replaced by the slot, so that words are distinct and carry the slot
                unsigned int word = (__float_as_uint(key) & ~31u) | (unsigned int)lane;
#pragma unroll
                for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                    for (int j = k >> 1; j > 0; j >>= 1) {
                        const unsigned int other = __shfl_xor_sync(0xffffffffu, word, j);
                        // the lower lane of an ascending pair keeps the smaller entry
                        const bool want_less = ((lane & k) == 0) == ((lane & j) == 0);
                        if ((other < word) == want_less) word = other;
                    }
                }
                slot = (int)(word & 31u);
            }
            const int Kt = __shfl_sync(0xffffffffu, Kt0, slot);
            W.perm[lane] = slot;
            int incl = Kt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int S_tot = __shfl_sync(0xffffffffu, incl, 31);
            W.offK[lane] = incl - Kt;
            if (lane == 31) W.offK[kWTile] = S_tot;
            __syncwarp();
            for (int sub0 = 0; sub0 < S_tot; sub0 += kWSubCap) {
                const int nsub = min(kWSubCap, S_tot - sub0);
                // sub-step yields: a balanced run [q0, q1) per lane
                const int per = (nsub + 31) >> 5;
                const int q0 = min(lane * per, nsub), q1 = min(q0 + per, nsub);
                int my_ph = 0;
                unsigned int my_emit = 0;
                if (q0 < q1) {
                    int lo = 0, hi = kWTile;   // offK[lo] <= sub0 + q0 < offK[lo + 1]
                    const int first = sub0 + q0;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (W.offK[mid] <= first) lo = mid;
                        else hi = mid;
                    }
                    int si = lo;
                    for (int q = q0; q < q1; ++q) {
                        const int qq = sub0 + q;
                        while (W.offK[si + 1] <= qq) ++si;   // next non-empty segment
                        const int sg = W.perm[si];
                        const int N = substep<SPH, FL>(W, q, sg, qq - W.offK[si], base, pp, ap);
                        my_ph += N;
                        my_emit += (unsigned int)N * (unsigned int)W.bunch[sg];
                    }
                }
                emitted += my_emit;
                int ph_incl = my_ph;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, ph_incl, o);
                    if (lane >= o) ph_incl += y;
                }
                const int M = __shfl_sync(0xffffffffu, ph_incl, 31);
                const int ph0 = ph_incl - my_ph;
                __syncwarp();
                // bunches over windows of the warp's bunch -> sub-step map
                for (int p0 = 0; p0 < M; p0 += kWMapCap) {
                    const int wn = min(kWMapCap, M - p0);
                    int off = ph0;
                    for (int q = q0; q < q1; ++q) {
                        const int N = W.nsub_ph[q];
                        const int a = max(off, p0), b = min(off + N, p0 + wn);
                        for (int p = a; p < b; ++p) W.map[p - p0] = (unsigned int)q | ((unsigned int)(p - off) << kQBits);
                        off += N;
                    }
                    __syncwarp();
                    if constexpr (!EX) {
                        for (int p = lane; p < wn; p += 32) {
                            const unsigned int e = W.map[p];
                            const int qs = (int)(e & ((1u << kQBits) - 1)), ib = (int)(e >> kQBits);
                            const bool bey = bunch<false, SPH, REC, FL, TR, kModeMain, FIX>(W, qs, ib, true, base, pp, ap,
                                                                                           dp, op, sv, tcs, T);
                            // a bunch beyond the tables goes to the exact pass's queue (one
                            // reservation per group of converged lanes); when the queue is full its
                            // tile is marked, and the exact pass then skips the tile's queued entries
                            if (bey) {   // the lanes here are exactly those with a bunch to queue
                                const unsigned int m = __activemask();
                                const int leader = __ffs(m) - 1;
                                unsigned int slot0 = 0;
                                // (a full queue takes no more reservations, so the 32-bit count cannot wrap)
                                if (lane == leader)
                                    slot0 = pp.q_cap && __ldcg(scratch + 3) < pp.q_cap ? atomicAdd(scratch + 3, (unsigned int)__popc(m))
                                                                                       : 0xFFFFFFFFu;
                                slot0 = __shfl_sync(m, slot0, leader);
                                const unsigned int slot = slot0 + (unsigned int)__popc(m & ((1u << lane) - 1u));
                                if (slot0 != 0xFFFFFFFFu && slot >= slot0 && slot < pp.q_cap) {
                                    const int segk = __float_as_int(W.sub[qs].w);
                                    const unsigned long long li = (unsigned long long)(base + (segk & ((1 << kKShift) - 1)));
                                    reinterpret_cast<uint4*>(scratch + pp.q_off)[slot] =
                                        make_uint4((uint32_t)li, (uint32_t)(li >> 32), (uint32_t)(segk >> kKShift), (uint32_t)ib);
                                } else {
                                    any_beyond = true;
                                }
                            }
                        }
                    } else {
                        // rounds of 32 bunches: those beyond the tables are queued (in the map
                        // entries already read: a round's entries are never read again) and
                        // propagated 32 at a time, so that the warp stays converged
                        int nq = 0;
                        for (int pw = 0;; pw += 32) {
                            const bool last = pw + 32 >= wn;
                            const int p = pw + lane;
                            bool take = false;
                            unsigned int e = 0;
                            if (p < wn) {
                                e = W.map[p];
                                take = bunch<false, SPH, REC, FL, TR, kModeCheck>(W, (int)(e & ((1u << kQBits) - 1)),
                                                                                 (int)(e >> kQBits), true, base, pp,
                                                                                 ap, dp, op, sv, tcs, T);
                            }
                            const unsigned int m = __ballot_sync(0xffffffffu, take);
                            __syncwarp();
                            if (take) W.map[nq + __popc(m & ((1u << lane) - 1u))] = e;
                            nq += __popc(m);
                            __syncwarp();
                            while (nq >= 32 || (last && nq > 0)) {
                                const int n_run = min(nq, 32);
                                if (lane < n_run) {
                                    const unsigned int ex = W.map[nq - n_run + lane];
                                    bunch<false, SPH, REC, FL, TR, kModeExact>(W, (int)(ex & ((1u << kQBits) - 1)),
                                                                               (int)(ex >> kQBits), true, base, pp, ap,
                                                                               dp, op, sv, tcs, T);
                                }
                                nq -= n_run;
                                __syncwarp();
                            }
                            if (last) break;
                        }
                    }
                    __syncwarp();
                }
            }
            if constexpr (!EX) {   // the exact pass is to visit this tile
                if (__any_sync(0xffffffffu, any_beyond) && lane == 0)
                    mark_group(scratch, n_wtiles, pp.tiles_per_bit, (unsigned int)tile / (unsigned int)pp.tiles_per_bit);
            }
        };
        if constexpr (!EX) {
            for (;;) {   // dynamic scheduling: warp tiles from the work counter
                unsigned int wt = 0;
                if (lane == 0) wt = atomicAdd(tile_ctr, 1u);
                const long long tile = (long long)__shfl_sync(0xffffffffu, wt, 0);
                if (tile >= n_wtiles) break;
                process_tile(tile);
            }
        } else {
            // the exact pass takes the queued bunches 32 at a time, then the marked groups
            // from their list (the cursor runs over both)
            const unsigned int n_listed = __ldcg(scratch + 2);
            const unsigned int n_q = min(__ldcg(scratch + 3), pp.q_cap), n_qc = (n_q + 31) / 32;
            const unsigned int* bits = scratch + kScratchCounters;
            const unsigned int* list = bits + (scratch_groups(n_wtiles, pp.tiles_per_bit) + 31) / 32;
            for (;;) {
                unsigned int idx = 0;
                if (lane == 0) idx = atomicAdd(tile_ctr, 1u);
                idx = __shfl_sync(0xffffffffu, idx, 0);
                if (idx < n_qc) {
                    // lane j: queue entry 32 idx + j, its segment in slot j, its sub-step in slot j
                    const unsigned int qe = idx * 32u + (unsigned int)lane;
                    bool act = qe < n_q;
                    uint4 ent = make_uint4(0u, 0u, 0u, 0u);
                    if (act) ent = __ldcg(reinterpret_cast<const uint4*>(scratch + pp.q_off) + qe);
                    const long long li = (long long)(((unsigned long long)ent.y << 32) | ent.x);
                    if (act) {   // a tile the queue overflowed on is the group pass's
                        const unsigned long long g = (unsigned long long)(li / kWTile) / (unsigned long long)pp.tiles_per_bit;
                        if ((__ldcg(bits + (g >> 5)) >> (g & 31)) & 1u) act = false;
                    }
                    const long long base_l = li - lane;   // so that base + slot is the segment's index
                    if (act) {
                        import_segment<SPH, FL>(W, lane, pp.segs + li, pp, ap, dp, invalid, dropped, false);
                        substep<SPH, FL>(W, lane, lane, (int)ent.z, base_l, pp, ap);
                        bunch<false, SPH, REC, FL, TR, kModeExact>(W, lane, (int)ent.w, true, base_l, pp, ap, dp, op, sv,
                                                                   tcs, T);
                    }
                    __syncwarp();
                    continue;
                }
                idx -= n_qc;
                if (idx >= n_listed) break;
                const long long g = (long long)__ldcg(list + idx);
                const long long t_end = std::min<long long>((g + 1) * pp.tiles_per_bit, n_wtiles);
                for (long long tile = g * pp.tiles_per_bit; tile < t_end; ++tile) process_tile(tile);
            }
        }
    } else {
        for (;;) {
            // dynamic tile scheduling: blocks that finish early take more tiles
            if (t == 0) S.tile = (int)atomicAdd(tile_ctr, 1u);
            __syncthreads();
            const long long tile = S.tile;
            if (tile >= n_tiles) break;
            const long long base = tile * kTile;

            // ---- stage 1: import and filter (one segment per thread) -------------
            const int Kt = (t < kTile && base + t < pp.n) ? import_segment<SPH, FL>(S, t, pp.segs + base + t, pp, ap, dp, invalid, dropped) : 0;
            int S_tot;
            const int offk = block_scan<NT>(Kt, S.wsum, buf, &S_tot);
            if (t < kTile) S.offK[t] = offk;
            if (t == 0) S.offK[kTile] = S_tot;
            __syncthreads();

            for (int sub0 = 0; sub0 < S_tot; sub0 += kSubCap) {
                const int nsub = min(kSubCap, S_tot - sub0);
                // ---- stage 2: sub-step yields, a balanced run [q0, q1) per thread ---
                const int per = (nsub + NT - 1) / NT;
                const int q0 = min(t * per, nsub), q1 = min(q0 + per, nsub);
                int my_ph = 0;
                unsigned int my_emit = 0;
                if (q0 < q1) {
                    int lo = 0, hi = kTile;   // offK[lo] <= sub0 + q0 < offK[lo + 1]
                    const int first = sub0 + q0;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (S.offK[mid] <= first) lo = mid;
                        else hi = mid;
                    }
                    int sg = lo;
                    for (int q = q0; q < q1; ++q) {
                        const int qq = sub0 + q;
                        while (S.offK[sg + 1] <= qq) ++sg;   // next non-empty segment
                        const int N = substep<SPH, FL>(S, q, sg, qq - S.offK[sg], base, pp, ap);
                        my_ph += N;
                        my_emit += (unsigned int)N * (unsigned int)S.bunch[sg];
                    }
                }
                int M;
                const int ph0 = block_scan<NT>(my_ph, S.wsum, buf, &M);
                emitted += my_emit;

                // ---- stages 3-5 over windows of the bunch map ------------------------
                for (int p0 = 0; p0 < M; p0 += kMapCap) {
                    const int wn = min(kMapCap, M - p0);
                    int off = ph0;
                    for (int q = q0; q < q1; ++q) {   // owners write their bunches' entries
                        const int N = S.nsub_ph[q];
                        const int a = max(off, p0), b = min(off + N, p0 + wn);
                        for (int p = a; p < b; ++p) S.map[p - p0] = (unsigned int)q | ((unsigned int)(p - off) << kQBits);
                        off += N;
                    }
                    __syncthreads();
                    // whole warps (warpgroups on the surrogate path, whose network is
                    // warpgroup-collective) iterate together
                    constexpr int kGroup = SURR ? 128 : 32;
                    for (int pw = t & ~(kGroup - 1); pw < wn; pw += NT) {
                        const int p = pw + (t & (kGroup - 1));
                        const bool active = p < wn;
                        const unsigned int e = S.map[active ? p : pw];
                        const int qs = (int)(e & ((1u << kQBits) - 1));
                        if (bunch<SURR, SPH, REC, FL, TR>(S, qs, (int)(e >> kQBits), active, base, pp, ap, dp, op, sv,
                                                          tcs, T)) {   // left to the exact pass: mark its warp tile
                            const int sg = __float_as_int(S.sub[qs].w) & ((1 << kKShift) - 1);
                            mark_group(scratch, (pp.n + kWTile - 1) / kWTile, pp.tiles_per_bit,
                                       (unsigned int)((base + sg) / kWTile) / (unsigned int)pp.tiles_per_bit);
                        }
                    }
                    __syncthreads();
                }
            }
        }

    }

    if (SURR) tc_teardown(*tcs);
    if (EX) {   // the photon kernel counted these segments and their emitted bunches
        emitted = 0;
        invalid = 0;
        dropped = 0;
    }

    // ---- counter flush: missed = emitted - absorbed - detected.  A thread's
    // emitted bunches and the bunches it propagated are different sets, so the
    // per-thread differences are signed; their 64-bit sum (mod 2^64) is exact.
    int v[CS_N_COUNTERS];
    v[CS_CNT_EMITTED] = (int)emitted;
    v[CS_CNT_ABSORBED] = (int)T.absorbed;
    v[CS_CNT_HIST] = (int)T.hist;
    v[CS_CNT_TEL] = (int)T.tel;
    v[CS_CNT_MISSED_HIST] = (int)emitted - (int)T.absorbed - (int)T.hist;
    v[CS_CNT_MISSED_TEL] = (int)emitted - (int)T.absorbed - (int)T.tel;
    v[CS_CNT_UPWARD] = (int)T.upward;
    v[CS_CNT_INVALID_SEGMENTS] = (int)invalid;
#pragma unroll
    for (int c = 0; c < CS_N_COUNTERS; ++c) {
        int x = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((t & 31) == 0 && x) atomicAdd(op.counters + c, (unsigned long long)(long long)x);
    }
    if (pp.lv1_dropped) {
        unsigned int x = dropped;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((t & 31) == 0 && x) atomicAdd(pp.lv1_dropped, (unsigned long long)x);
    }
}

// Launches the exact-tracer or the surrogate instance of the kernel.
// An atmosphere and a detector work together when they share the observation
// level and the geometry (and, on the sphere and the cylinders, the Earth radius).
bool compatible(const cs_atmosphere* atm, const cs_detector* det) {
    const double tol = 1e-9 * fmax(1.0, fabs(atm->p.h_obs));
    if (fabs(det->p.h_obs - atm->p.h_obs) > tol) return false;
    if (det->p.cylindrical != atm->p.cylindrical) return false;
    if (!atm->p.cylindrical && det->p.spherical != atm->p.spherical) return false;
    return !atm->p.spherical || fabs(det->p.R - atm->f64.R) <= 1e-9 * atm->f64.R;
}

cs_status launch_kernel(unsigned grid, cudaStream_t stream, const PropParams& pp, const AtmParams& ap,
                        const DetParams& dp, const OutParams& op, unsigned int* ctr, const cs_surrogate* sur,
                        int tc_poll_limit) {
    const size_t smem = sur ? kSmemSurrogate : kSmemExact;
    SurrogateView sv;
    memset(&sv, 0, sizeof sv);
    if (sur) {
        sv = *surrogate_view(sur);
        sv.polls = tc_poll_limit == 0 ? kTcSpin : std::max(tc_poll_limit, 0);
    }
    // instances: (network or tables) x (sphere or plane) x (records or throughput)
    auto go = [&](auto kernel, int threads) { kernel<<<grid, threads, smem, stream>>>(pp, ap, dp, op, ctr, sv); };
    const bool rec = op.records != nullptr;
    // the exact tracer's instances: emission (Cherenkov or fluorescence) x tracer (tables or stepper)
    // the standard configuration (refraction, transmission and tables; histogram, telescopes and
    // time sums; no camera optics) has its own instances, with those tests folded
    const bool fix = ap.refraction && ap.transmission && ap.use_tables && dp.cam_n == 0 && dp.nx > 0 &&
                     dp.n_tel > 0 && op.tel_time != nullptr;
    auto exact = [&](auto sph, auto fl, auto tr) {
        constexpr bool S = decltype(sph)::value, F = decltype(fl)::value, T = decltype(tr)::value;
        if constexpr (!F && !T) {
            if (fix) {
                rec ? go(propagate_kernel<false, S, 4, true, false, false, false, true>, kThreads)
                    : go(propagate_kernel<false, S, 4, false, false, false, false, true>, kThreads);
                return;
            }
        }
        rec ? go(propagate_kernel<false, S, 4, true, F, T>, kThreads) : go(propagate_kernel<false, S, 4, false, F, T>, kThreads);
    };
    using t_ = std::true_type;
    using f_ = std::false_type;
    const bool fl = pp.emission != 0, tr = pp.snell != 0;
    if (sur) {
        if (ap.spherical) rec ? go(propagate_kernel<true, true, 1, true>, kThreadsSur) : go(propagate_kernel<true, true, 1, false>, kThreadsSur);
        else rec ? go(propagate_kernel<true, false, 1, true>, kThreadsSur) : go(propagate_kernel<true, false, 1, false>, kThreadsSur);
    } else if (ap.spherical) {
        if (fl) tr ? exact(t_{}, t_{}, t_{}) : exact(t_{}, t_{}, f_{});
        else tr ? exact(t_{}, f_{}, t_{}) : exact(t_{}, f_{}, f_{});
    } else {
        if (fl) tr ? exact(f_{}, t_{}, t_{}) : exact(f_{}, t_{}, f_{});
        else tr ? exact(f_{}, f_{}, t_{}) : exact(f_{}, f_{}, f_{});
    }
    CS_CUDA_TRY(cudaGetLastError());
    // the exact pass over the warp tiles the photon kernel marked (only atmospheres
    // with tables have a domain to leave; the stepper integrates every photon itself)
    if (ap.use_tables && !(tr && ap.refraction)) {
        const long long n_wtiles = (pp.n + kWTile - 1) / kWTile;
        const unsigned grid_x = (unsigned)std::max<long long>(1, std::min<long long>(n_wtiles, (long long)device_sm_count() * 4));
        // outside a stream capture, as a programmatic dependent launch (it overlaps the photon
        // kernel's tail: for most workloads the pass finds nothing to do)
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        CS_CUDA_TRY(cudaStreamIsCapturing(stream, &cap));
        auto pass = [&](auto kernel) {
            if (cap != cudaStreamCaptureStatusNone) {
                kernel<<<grid_x, kThreads, kSmemExact, stream>>>(pp, ap, dp, op, ctr, sv);
                return;
            }
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(grid_x);
            cfg.blockDim = dim3(kThreads);
            cfg.dynamicSmemBytes = kSmemExact;
            cfg.stream = stream;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            if (cudaLaunchKernelEx(&cfg, kernel, pp, ap, dp, op, ctr, sv) != cudaSuccess) {
                cudaGetLastError();   // the attribute refused: an ordinary stream-ordered launch
                kernel<<<grid_x, kThreads, kSmemExact, stream>>>(pp, ap, dp, op, ctr, sv);
            }
        };
        if (ap.spherical) {
            if (fl) rec ? pass(propagate_kernel<false, true, 4, true, true, false, true>) : pass(propagate_kernel<false, true, 4, false, true, false, true>);
            else rec ? pass(propagate_kernel<false, true, 4, true, false, false, true>) : pass(propagate_kernel<false, true, 4, false, false, false, true>);
        } else {
            if (fl) rec ? pass(propagate_kernel<false, false, 4, true, true, false, true>) : pass(propagate_kernel<false, false, 4, false, true, false, true>);
            else rec ? pass(propagate_kernel<false, false, 4, true, false, false, true>) : pass(propagate_kernel<false, false, 4, false, false, false, true>);
        }
        CS_CUDA_TRY(cudaGetLastError());
    }
    return CS_OK;
}

template <bool S, bool F, bool T>
cudaError_t set_exact_smem(int smem) {
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(propagate_kernel<false, S, 4, false, F, T>, attr, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(propagate_kernel<false, S, 4, true, F, T>, attr, smem);
    if (!T) {   // the exact pass of the table-tracer instances
        if (e == cudaSuccess) e = cudaFuncSetAttribute(propagate_kernel<false, S, 4, false, F, false, true>, attr, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(propagate_kernel<false, S, 4, true, F, false, true>, attr, smem);
    }
    if (!T && !F) {   // the fixed-configuration instances
        if (e == cudaSuccess) e = cudaFuncSetAttribute(propagate_kernel<false, S, 4, false, false, false, false, true>, attr, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(propagate_kernel<false, S, 4, true, false, false, false, true>, attr, smem);
    }
    return e;
}

// Raises the kernels' shared-memory limits, once per device.
constexpr int kMaxDevices = 64;
std::mutex g_attr_mu;
bool g_attr_done[kMaxDevices] = {};

cs_status set_smem_attributes() {
    int dev = 0;
    CS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return CS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (g_attr_done[dev]) return CS_OK;
    const int smem = (int)kSmemExact, smem_sur = (int)kSmemSurrogate;
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    CS_CUDA_TRY((set_exact_smem<false, false, false>(smem)));
    CS_CUDA_TRY((set_exact_smem<false, false, true>(smem)));
    CS_CUDA_TRY((set_exact_smem<false, true, false>(smem)));
    CS_CUDA_TRY((set_exact_smem<false, true, true>(smem)));
    CS_CUDA_TRY((set_exact_smem<true, false, false>(smem)));
    CS_CUDA_TRY((set_exact_smem<true, false, true>(smem)));
    CS_CUDA_TRY((set_exact_smem<true, true, false>(smem)));
    CS_CUDA_TRY((set_exact_smem<true, true, true>(smem)));
    CS_CUDA_TRY(cudaFuncSetAttribute(propagate_kernel<true, false, 1, false>, attr, smem_sur));
    CS_CUDA_TRY(cudaFuncSetAttribute(propagate_kernel<true, false, 1, true>, attr, smem_sur));
    CS_CUDA_TRY(cudaFuncSetAttribute(propagate_kernel<true, true, 1, false>, attr, smem_sur));
    CS_CUDA_TRY(cudaFuncSetAttribute(propagate_kernel<true, true, 1, true>, attr, smem_sur));
    g_attr_done[dev] = true;
    return CS_OK;
}

int default_blocks_per_sm(const cs_opts& o) { return o.blocks_per_sm > 0 ? o.blocks_per_sm : (o.surrogate ? 1 : 4); }

__global__ void philox_kernel(const uint4* ctr, size_t n, uint32_t k0, uint32_t k1, uint4* out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const uint4 c = ctr[i];
        out[i] = philox(c.x, c.y, c.z, c.w, k0, k1);
    }
}

// Host-pointer calls above 2 chunks of this many segments stream their input.
constexpr size_t kHostChunk = (size_t)1 << 18;

// Device buffers reused by host-pointer calls.
struct HostWorkspace {
    std::mutex mu;
    int device = -1;
    void* segs = nullptr; size_t segs_cap = 0;
    void* outs = nullptr; size_t outs_cap = 0;
    void* recs = nullptr; size_t recs_cap = 0;
    cs_streamer* streamer = nullptr;   // large host inputs: chunks overlap copies and kernels
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

// Per-launch scratch (work counters and the exact pass's tile bits) from a
// stream-ordered memory pool the library keeps per device: allocated and
// freed on the launch's stream, so launches in flight on different streams
// never share it, and the pool keeps its memory between launches.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cs_status scratch_alloc(size_t bytes, cudaStream_t stream, unsigned int** out) {
    int dev = 0;
    CS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return CS_ERR_INVALID_ARG;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (!g_pool[dev]) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof props);
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            CS_CUDA_TRY(cudaMemPoolCreate(&g_pool[dev], &props));
            uint64_t keep = ~0ull;
            CS_CUDA_TRY(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep));
        }
        pool = g_pool[dev];
    }
    CS_CUDA_TRY(cudaMallocFromPoolAsync((void**)out, bytes, pool, stream));
    return CS_OK;
}

// The LV1 filter's parameters from the options (the counter as given: device memory here).
void set_filters(PropParams& pp, const cs_opts& o, const DetParams& dp, const AtmParams& ap) {
    uint32_t k0 = pp.key0, k1 = pp.key1;   // the Philox key schedule, once per call
    for (int r = 0; r < 10; ++r) {
        pp.rk[2 * r] = k0;
        pp.rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    pp.s_max = (float)o.s_max;
    pp.s_max_lo = (float)(o.s_max - (double)pp.s_max);
    pp.emission = o.emission;
    pp.fl_n = 0;
    pp.fl_yd = 0.0f;
    if (o.emission) {   // Eq. 2.6: z^2 dE/dX rho sum(yields), rho = rho_per_delta delta / 100 [g/cm^3]
        double ysum = 0.0, cum = 0.0;
        for (int l = 0; l < o.fl_n_lines; ++l) ysum += o.fl_yield_per_mev[l];
        pp.fl_n = o.fl_n_lines;
        for (int l = 0; l < o.fl_n_lines; ++l) {
            cum += o.fl_yield_per_mev[l];
            pp.fl_inv_l[l] = (float)(1.0 / o.fl_lines_nm[l]);
            pp.fl_thr[l] = l + 1 < o.fl_n_lines ? (uint32_t)floor(cum / ysum * 16777216.0) : 16777216u;
        }
        pp.fl_yd = (float)(o.fl_dedx * ysum * ap.rho_per_delta * (o.emission == CS_EMIT_FLUORESCENCE_HALF ? 0.5 : 1.0));
    }
    pp.lv3 = o.lv3 ? 1 : 0;
    for (int i = 0; i < 3; ++i) pp.lv3_c[i] = (float)o.lv3_centre[i];
    const double lim = o.lv3_radius + o.lv3_margin;
    pp.lv3_r2 = (float)(lim * lim);
    pp.lv3_dz2 = (float)((dp.h_obs - o.lv3_centre[2]) * (dp.h_obs - o.lv3_centre[2]));
    pp.snell = o.tracer == CS_TRACER_SNELL ? 1 : 0;
    pp.snell_dh = (float)o.tracer_dh;
    pp.lv1 = o.lv1_metric;
    pp.lv1_a = (float)o.lv1_a;
    pp.lv1_b = (float)o.lv1_b;
    pp.lv1_r = (float)o.lv1_radius;
    for (int i = 0; i < 3; ++i) pp.lv1_c[i] = (float)o.lv1_centre[i];
    pp.lv1_dropped = (unsigned long long*)o.lv1_dropped;
}

bool filters_valid(const cs_opts& o, const cs_atmosphere* atm) {
    if (o.emission < CS_EMIT_CHERENKOV || o.emission > CS_EMIT_FLUORESCENCE_HALF) return false;
    if (o.emission) {   // a line list, and no LV1 cut: isotropic light is not filtered (Sec. 4.3.2)
        if (o.fl_n_lines < 1 || o.fl_n_lines > 8 || !o.fl_lines_nm || !o.fl_yield_per_mev ||
            !(o.fl_dedx >= 0.0) || !isfinite(o.fl_dedx) || o.lv1_metric != CS_LV1_OFF || o.surrogate)
            return false;
        double ysum = 0.0;
        for (int l = 0; l < o.fl_n_lines; ++l) {
            if (!(o.fl_lines_nm[l] > 0.0) || !isfinite(o.fl_lines_nm[l]) || !(o.fl_yield_per_mev[l] >= 0.0) ||
                !isfinite(o.fl_yield_per_mev[l]))
                return false;
            ysum += o.fl_yield_per_mev[l];
        }
        if (!(ysum > 0.0)) return false;
    }
    if (o.tracer != CS_TRACER_TABLES &&
        (o.tracer != CS_TRACER_SNELL || !(o.tracer_dh >= 0.01) || !isfinite(o.tracer_dh) || o.surrogate))
        return false;
    // the cylinders: the stepper only, no filters (their geometry is the plane's or the sphere's), no network
    if (atm->p.cylindrical &&
        (o.tracer != CS_TRACER_SNELL || o.lv3 || o.lv1_metric != CS_LV1_OFF || o.surrogate))
        return false;
    if (o.lv3 && !(o.lv3_radius >= 0.0 && o.lv3_margin >= 0.0 && isfinite(o.lv3_radius + o.lv3_margin) &&
                   isfinite(o.lv3_centre[0]) && isfinite(o.lv3_centre[1]) && isfinite(o.lv3_centre[2])))
        return false;
    return o.lv1_metric >= CS_LV1_OFF && o.lv1_metric <= CS_LV1_TELESCOPES &&
           (o.lv1_metric == CS_LV1_OFF || (isfinite(o.lv1_a) && isfinite(o.lv1_b) && o.lv1_radius >= 0.0));
}

size_t camera_bytes(const DetParams& dp) { return (size_t)dp.n_showers * dp.n_tel * dp.cam_n * dp.cam_n * 8; }

// The caller's device outputs as the kernel sees them.
OutParams out_params(const cs_output* out) {
    OutParams op;
    op.hist = (unsigned long long*)out->hist;
    op.tel_counts = (unsigned long long*)out->tel_counts;
    op.tel_time = out->tel_time;
    op.counters = (unsigned long long*)out->counters;
    op.records = out->records;
    op.record_capacity = out->records ? out->record_capacity : 0;
    op.record_count = (unsigned long long*)out->record_count;
    op.camera = (unsigned long long*)out->camera;
    return op;
}

// The outputs a call that does not accumulate starts from: zero.
cs_status zero_outputs(const DetParams& dp, const OutParams& op, uint64_t* lv1_dropped, cudaStream_t stream) {
    if (op.hist) CS_CUDA_TRY(cudaMemsetAsync(op.hist, 0, (size_t)dp.n_showers * dp.nx * dp.ny * 8, stream));
    if (op.tel_counts) CS_CUDA_TRY(cudaMemsetAsync(op.tel_counts, 0, (size_t)dp.n_showers * dp.n_tel * 8, stream));
    if (op.tel_time) CS_CUDA_TRY(cudaMemsetAsync(op.tel_time, 0, (size_t)dp.n_showers * dp.n_tel * 8, stream));
    if (op.camera && dp.cam_n > 0) CS_CUDA_TRY(cudaMemsetAsync(op.camera, 0, camera_bytes(dp), stream));
    CS_CUDA_TRY(cudaMemsetAsync(op.counters, 0, CS_N_COUNTERS * 8, stream));
    if (op.record_count) CS_CUDA_TRY(cudaMemsetAsync(op.record_count, 0, 8, stream));
    if (lv1_dropped) CS_CUDA_TRY(cudaMemsetAsync(lv1_dropped, 0, 8, stream));
    return CS_OK;
}

// Output pointers every call needs for its detector.
bool outputs_complete(const cs_detector* det, const cs_output* out) {
    if (det->p.nx > 0 && !out->hist) return false;
    if (det->p.n_tel > 0 && !out->tel_counts) return false;
    if (det->p.cam_n > 0 && !out->camera) return false;
    if (out->records && !out->record_count) return false;
    return true;
}

cs_status launch(const cs_segment* d_segs, size_t n, const cs_atmosphere* atm, const cs_detector* det,
                 uint64_t seed, const cs_opts& o, const OutParams& op, cudaStream_t stream) {
    const DetParams& dp = det->p;
    if (!o.accumulate) {
        cs_status z = zero_outputs(dp, op, o.lv1_dropped, stream);
        if (z != CS_OK) return z;
    }
    if (n == 0) return CS_OK;
    PropParams pp;
    pp.segs = d_segs;
    pp.n = (long long)n;
    pp.seg_base = o.seg_base;
    pp.key0 = (uint32_t)seed;
    pp.key1 = (uint32_t)(seed >> 32);
    pp.bunch = o.bunch;
    pp.shower_bunch = nullptr;
    pp.s_max = (float)o.s_max;
    set_filters(pp, o, det->p, atm->p);
    cs_status st = set_smem_attributes();
    if (st != CS_OK) return st;
    const int per_sm = default_blocks_per_sm(o);
    const long long tiles = ((long long)n + kTile - 1) / kTile;
    const long long grid = std::min<long long>(tiles, (long long)device_sm_count() * per_sm);
    pp.tiles_per_bit = 1;
    const long long n_wtiles = (pp.n + kWTile - 1) / kWTile;
    pp.q_cap = queue_cap(n_wtiles, o.exact_queue);
    pp.q_off = (unsigned int)scratch_queue_off(n_wtiles, 1);
    const size_t bytes = scratch_words(n_wtiles, 1, pp.q_cap) * sizeof(unsigned int);
    unsigned int* scratch = nullptr;
    if ((st = scratch_alloc(bytes, stream, &scratch)) != CS_OK) return st;
    CS_CUDA_TRY(cudaMemsetAsync(scratch, 0, scratch_zero_words((pp.n + kWTile - 1) / kWTile, 1) * sizeof(unsigned int), stream));
    st = launch_kernel((unsigned)grid, stream, pp, atm->p, det->p, op, scratch, o.surrogate, o.tc_poll_limit);
    CS_CUDA_TRY(cudaFreeAsync(scratch, stream));
    return st;
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
    if (!outputs_complete(det, out)) return CS_ERR_INVALID_ARG;
    if (!compatible(atm, det) || !filters_valid(o, atm)) return CS_ERR_INVALID_ARG;
    if (n > (size_t)1 << 40) return CS_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_;
    const DetParams& dp = det->p;
    if (o.device_ptrs) {
        if (((uintptr_t)segs & 15) != 0) return CS_ERR_INVALID_ARG;
        return launch(segs, n, atm, det, seed, o, out_params(out), stream);
    }
    // host pointers: stage through the workspace
    std::lock_guard<std::mutex> lock(g_ws.mu);
    int dev = 0;
    CS_CUDA_TRY(cudaGetDevice(&dev));
    if (g_ws.device != dev) {   // buffers of another device are not reused
        g_ws.segs = g_ws.outs = g_ws.recs = nullptr;
        g_ws.segs_cap = g_ws.outs_cap = g_ws.recs_cap = 0;
        g_ws.streamer = nullptr;
        g_ws.device = dev;
    }
    const size_t hist_b = (size_t)dp.n_showers * dp.nx * dp.ny * 8, tel_b = (size_t)dp.n_showers * dp.n_tel * 8;
    const size_t cam_b = camera_bytes(dp);
    const size_t o_hist = 0, o_tel = up256(hist_b), o_time = o_tel + up256(tel_b), o_cam = o_time + up256(tel_b),
                 o_cnt = o_cam + up256(cam_b), o_rc = o_cnt + 256, outs_b = o_rc + 256;
    // large inputs are streamed in chunks: the copy of one chunk overlaps the kernel of the previous
    const bool chunked = n > 2 * kHostChunk;
    if (!chunked) CS_CUDA_TRY(ensure(&g_ws.segs, &g_ws.segs_cap, std::max<size_t>(n, 1) * sizeof(cs_segment)));
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
    op.camera = cam_b ? (unsigned long long*)(ob + o_cam) : nullptr;
    uint64_t* host_dropped = o.lv1_dropped;   // a host counter: staged through the workspace
    if (host_dropped) o.lv1_dropped = (uint64_t*)(ob + o_rc + 64);
    if (n && !chunked)
        CS_CUDA_TRY(cudaMemcpyAsync(g_ws.segs, segs, n * sizeof(cs_segment), cudaMemcpyHostToDevice, stream));
    if (o.accumulate) {   // bring the caller's running totals in
        if (op.hist) CS_CUDA_TRY(cudaMemcpyAsync(op.hist, out->hist, hist_b, cudaMemcpyHostToDevice, stream));
        if (op.tel_counts) CS_CUDA_TRY(cudaMemcpyAsync(op.tel_counts, out->tel_counts, tel_b, cudaMemcpyHostToDevice, stream));
        if (op.tel_time) CS_CUDA_TRY(cudaMemcpyAsync(op.tel_time, out->tel_time, tel_b, cudaMemcpyHostToDevice, stream));
        if (op.camera) CS_CUDA_TRY(cudaMemcpyAsync(op.camera, out->camera, cam_b, cudaMemcpyHostToDevice, stream));
        CS_CUDA_TRY(cudaMemcpyAsync(op.counters, out->counters, CS_N_COUNTERS * 8, cudaMemcpyHostToDevice, stream));
        CS_CUDA_TRY(cudaMemsetAsync(op.record_count, 0, 8, stream));
        if (host_dropped) CS_CUDA_TRY(cudaMemcpyAsync(o.lv1_dropped, host_dropped, 8, cudaMemcpyHostToDevice, stream));
    }
    cs_status st;
    if (chunked) {
        if (!g_ws.streamer) {
            st = cs_streamer_create(kHostChunk, &g_ws.streamer);
            if (st != CS_OK) return st;
        }
        cs_output dout;
        dout.hist = (uint64_t*)op.hist;
        dout.tel_counts = (uint64_t*)op.tel_counts;
        dout.tel_time = op.tel_time;
        dout.counters = (uint64_t*)op.counters;
        dout.records = op.records;
        dout.record_capacity = op.record_capacity;
        dout.record_count = (uint64_t*)op.record_count;
        dout.camera = (uint64_t*)op.camera;
        cs_opts od = o;
        od.device_ptrs = 1;
        st = cs_streamer_run(g_ws.streamer, segs, n, atm, det, seed, &od, &dout, stream);
    } else {
        st = launch((const cs_segment*)g_ws.segs, n, atm, det, seed, o, op, stream);
    }
    if (st != CS_OK) return st;
    if (op.hist) CS_CUDA_TRY(cudaMemcpyAsync(out->hist, op.hist, hist_b, cudaMemcpyDeviceToHost, stream));
    if (op.tel_counts) CS_CUDA_TRY(cudaMemcpyAsync(out->tel_counts, op.tel_counts, tel_b, cudaMemcpyDeviceToHost, stream));
    if (op.tel_time) CS_CUDA_TRY(cudaMemcpyAsync(out->tel_time, op.tel_time, tel_b, cudaMemcpyDeviceToHost, stream));
    if (op.camera) CS_CUDA_TRY(cudaMemcpyAsync(out->camera, op.camera, cam_b, cudaMemcpyDeviceToHost, stream));
    CS_CUDA_TRY(cudaMemcpyAsync(out->counters, op.counters, CS_N_COUNTERS * 8, cudaMemcpyDeviceToHost, stream));
    unsigned long long produced = 0;
    CS_CUDA_TRY(cudaMemcpyAsync(&produced, op.record_count, 8, cudaMemcpyDeviceToHost, stream));
    if (host_dropped) CS_CUDA_TRY(cudaMemcpyAsync(host_dropped, o.lv1_dropped, 8, cudaMemcpyDeviceToHost, stream));
    CS_CUDA_TRY(cudaStreamSynchronize(stream));
    const bool timed_out = o.surrogate && tc_take_timeout();   // the tables served the network's photons
    if (out->record_count) *out->record_count = produced;
    if (out->records && produced) {
        const size_t ncopy = std::min<unsigned long long>(produced, out->record_capacity);
        CS_CUDA_TRY(cudaMemcpy(out->records, g_ws.recs, ncopy * sizeof(cs_record), cudaMemcpyDeviceToHost));
    }
    if (out->records && produced > out->record_capacity) return CS_ERR_CAPACITY;
    return timed_out ? CS_ERR_TIMEOUT : CS_OK;
}

extern "C" cs_status cs_check_timeout(void) {
    CS_CUDA_TRY(cudaDeviceSynchronize());
    return tc_take_timeout() ? CS_ERR_TIMEOUT : CS_OK;
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

// ---------------------------------------------------------------------------
// Allocation-free variant of the device-pointer call.
//
// Some callers cannot let a library call cudaMalloc: code that runs while a
// memory pool or arena owns the whole device (so a surprise allocation would
// fail or fragment it), real-time or embedded hosts that allow no allocation
// after start-up, and callers that must keep every byte the library uses
// accounted for in advance.  The regular device-pointer call takes a small
// per-launch scratch (its dynamic scheduler's work counters and the tile map
// of its exact pass) from a memory pool the library creates; this variant
// uses a file-scope device array instead, which the CUDA module loader creates
// on every GPU that loads the library and which lives until the process exits.
// ---------------------------------------------------------------------------
namespace cs {
namespace {

// A call's counters, a map of 2^14 groups of warp tiles and their list (67.6 KB
// in all): a call schedules at most 2^32 - 65537 warp tiles of 32 segments, and
// each group holds ceil(tiles / 2^14) of them.
constexpr int kNoAllocBits = 1 << 14;
constexpr int kNoAllocScratchWords = kScratchCounters + kNoAllocBits / 32 + kNoAllocBits;
static __device__ __align__(256) unsigned int g_noalloc_scratch[kNoAllocScratchWords];

std::mutex g_noalloc_mu;
unsigned int* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this set-up).
cs_status noalloc_scratch(unsigned int** out) {
    int dev = 0;
    CS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return CS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        CS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = (unsigned int*)p;
    }
    *out = g_noalloc_ptr[dev];
    return CS_OK;
}

}  // namespace
}  // namespace cs

extern "C" cs_status cs_propagate_noalloc(const cs_segment* segs, size_t n, const cs_atmosphere* atm,
                                          const cs_detector* det, uint64_t seed, const cs_opts* opts,
                                          cs_output* out, void* stream_) {
    if (!atm || !det || !out || !out->counters) return CS_ERR_INVALID_ARG;
    cs_opts o;
    if (opts) o = *opts; else cs_opts_default(&o);
    if (o.bunch < 1 || !(o.s_max > 0.0) || (n > 0 && !segs)) return CS_ERR_INVALID_ARG;
    if (!o.device_ptrs) return CS_ERR_INVALID_ARG;           // host buffers would need staging memory
    if (((uintptr_t)segs & 15) != 0) return CS_ERR_INVALID_ARG;
    if (det->p.nx > 0 && !out->hist) return CS_ERR_INVALID_ARG;
    if (!outputs_complete(det, out)) return CS_ERR_INVALID_ARG;
    if (!compatible(atm, det) || !filters_valid(o, atm)) return CS_ERR_INVALID_ARG;
    // the counter is 32 bits wide: reject inputs with more tiles than it can count
    if ((n + kWTile - 1) / kWTile >= 0xFFFFFFFFull - 65536ull) return CS_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_;
    const DetParams& dp = det->p;
    unsigned int* ctr = nullptr;
    cs_status st = noalloc_scratch(&ctr);
    if (st != CS_OK) return st;
    const OutParams op = out_params(out);
    if (!o.accumulate && (st = zero_outputs(dp, op, o.lv1_dropped, stream)) != CS_OK) return st;
    if (n == 0) return CS_OK;
    PropParams pp;
    pp.segs = segs;
    pp.n = (long long)n;
    pp.seg_base = o.seg_base;
    pp.key0 = (uint32_t)seed;
    pp.key1 = (uint32_t)(seed >> 32);
    pp.bunch = o.bunch;
    pp.shower_bunch = nullptr;
    pp.s_max = (float)o.s_max;
    set_filters(pp, o, det->p, atm->p);
    if ((st = set_smem_attributes()) != CS_OK) return st;
    const int per_sm = default_blocks_per_sm(o);
    const long long tiles = ((long long)n + kTile - 1) / kTile;
    const long long grid = std::min<long long>(tiles, (long long)device_sm_count() * per_sm);
    const long long n_wtiles = ((long long)n + kWTile - 1) / kWTile;
    pp.tiles_per_bit = (int)std::max<long long>(1, (n_wtiles + kNoAllocBits - 1) / kNoAllocBits);
    pp.q_cap = 0;   // no queue in the fixed array: every bunch beyond the tables marks its group
    pp.q_off = 0;
    // the array keeps the previous call's counters and map: start this call's at zero
    CS_CUDA_TRY(cudaMemsetAsync(ctr, 0, scratch_zero_words(n_wtiles, pp.tiles_per_bit) * sizeof(unsigned int), stream));
    return launch_kernel((unsigned)grid, stream, pp, atm->p, dp, op, ctr, o.surrogate, o.tc_poll_limit);
}

// ---------------------------------------------------------------------------
// Batched uneven showers: one persistent launch over many showers of uneven
// size (the dynamic tile scheduler balances them), captured once into a CUDA
// graph and replayed; plus the autotuner for block tiling and per-shower
// bunch sizes.
// ---------------------------------------------------------------------------
struct cs_batch {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned int* d_ctr = nullptr;   // the batch's own scratch (work counters, exact-pass tile map)
    int* d_bunch = nullptr;          // per-shower bunch sizes
    int device = 0;
};

namespace cs {
namespace {

cs_status check_device_call(const cs_segment* segs, size_t n, const cs_atmosphere* atm, const cs_detector* det,
                            const cs_opts& o, const cs_output* out) {
    if (!atm || !det || !out || !out->counters) return CS_ERR_INVALID_ARG;
    if (o.bunch < 1 || !(o.s_max > 0.0) || (n > 0 && !segs) || !o.device_ptrs) return CS_ERR_INVALID_ARG;
    if (((uintptr_t)segs & 15) != 0) return CS_ERR_INVALID_ARG;
    if (!outputs_complete(det, out)) return CS_ERR_INVALID_ARG;
    if (!compatible(atm, det) || !filters_valid(o, atm)) return CS_ERR_INVALID_ARG;
    if (n > (size_t)1 << 40) return CS_ERR_INVALID_ARG;
    return CS_OK;
}

// Bytes of the per-launch scratch for n segments (one map bit per warp tile).
size_t scratch_bytes(size_t n) {
    const long long n_wtiles = ((long long)n + kWTile - 1) / kWTile;
    return scratch_words(n_wtiles, 1, queue_cap(n_wtiles)) * sizeof(unsigned int);
}

// Grid of the persistent launch; also sets the kernel's shared-memory limit
// (host-side calls kept out of stream capture).
cs_status prepare_launch(size_t n, const cs_opts& o, unsigned int* grid) {
    cs_status st = set_smem_attributes();
    if (st != CS_OK) return st;
    const int per_sm = default_blocks_per_sm(o);
    const long long tiles = ((long long)n + kTile - 1) / kTile;
    *grid = (unsigned)std::max<long long>(1, std::min<long long>(tiles, (long long)device_sm_count() * per_sm));
    return CS_OK;
}

// Zeroing (unless accumulating), counter reset and the kernel, on `stream`;
// only stream operations, so it can be captured.
cs_status enqueue(const cs_segment* segs, size_t n, const cs_atmosphere* atm, const cs_detector* det,
                  uint64_t seed, const int* d_bunch, const cs_opts& o, const cs_output* out, unsigned int* ctr,
                  unsigned int grid, cudaStream_t stream) {
    const DetParams& dp = det->p;
    const OutParams op = out_params(out);
    if (!o.accumulate) {
        cs_status z = zero_outputs(dp, op, o.lv1_dropped, stream);
        if (z != CS_OK) return z;
    }
    if (n == 0) return CS_OK;
    PropParams pp;
    pp.segs = segs;
    pp.n = (long long)n;
    pp.seg_base = o.seg_base;
    pp.key0 = (uint32_t)seed;
    pp.key1 = (uint32_t)(seed >> 32);
    pp.bunch = o.bunch;
    pp.shower_bunch = d_bunch;
    pp.s_max = (float)o.s_max;
    set_filters(pp, o, det->p, atm->p);
    pp.tiles_per_bit = 1;
    pp.q_cap = std::min(queue_cap(((long long)n + kWTile - 1) / kWTile, o.exact_queue),
                        queue_cap(((long long)n + kWTile - 1) / kWTile));   // within the scratch's default size
    pp.q_off = (unsigned int)scratch_queue_off(((long long)n + kWTile - 1) / kWTile, 1);
    CS_CUDA_TRY(cudaMemsetAsync(ctr, 0, scratch_zero_words(((long long)n + kWTile - 1) / kWTile, 1) * sizeof(unsigned int),
                                stream));
    return launch_kernel(grid, stream, pp, atm->p, dp, op, ctr, o.surrogate, o.tc_poll_limit);
}

cs_status upload_bunches(const cs_detector* det, const int* shower_bunch, int** d_bunch) {
    *d_bunch = nullptr;
    if (!shower_bunch) return CS_OK;
    for (int s = 0; s < det->p.n_showers; ++s)
        if (shower_bunch[s] < 1) return CS_ERR_INVALID_ARG;
    CS_CUDA_TRY(cudaMalloc(d_bunch, sizeof(int) * det->p.n_showers));
    cudaError_t e = cudaMemcpy(*d_bunch, shower_bunch, sizeof(int) * det->p.n_showers, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_last_error("bunch upload", e);
        cudaFree(*d_bunch);
        *d_bunch = nullptr;
        return CS_ERR_CUDA;
    }
    return CS_OK;
}

}  // namespace
}  // namespace cs

extern "C" cs_status cs_batch_create(const cs_segment* segs, size_t n, const cs_atmosphere* atm,
                                     const cs_detector* det, uint64_t seed, const int* shower_bunch,
                                     const cs_opts* opts, cs_output* out, cs_batch** out_batch) {
    if (!out_batch) return CS_ERR_INVALID_ARG;
    *out_batch = nullptr;
    cs_opts o;
    if (opts) o = *opts; else cs_opts_default(&o);
    cs_status st = check_device_call(segs, n, atm, det, o, out);
    if (st != CS_OK) return st;
    cs_batch* b = new cs_batch;
    cudaGetDevice(&b->device);
    cudaStream_t cap = nullptr;
    auto fail = [&](cs_status s) {
        if (cap) cudaStreamDestroy(cap);
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        cudaFree(b->d_ctr);
        cudaFree(b->d_bunch);
        delete b;
        return s;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_ctr, scratch_bytes(n))) != cudaSuccess) { set_last_error("batch scratch", e); return fail(CS_ERR_CUDA); }
    if ((st = upload_bunches(det, shower_bunch, &b->d_bunch)) != CS_OK) return fail(st);
    unsigned int grid = 1;
    if ((st = prepare_launch(n, o, &grid)) != CS_OK) return fail(st);
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) {
        set_last_error("capture stream", e);
        return fail(CS_ERR_CUDA);
    }
    if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        set_last_error("begin capture", e);
        return fail(CS_ERR_CUDA);
    }
    st = enqueue(segs, n, atm, det, seed, b->d_bunch, o, out, b->d_ctr, grid, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    b->graph = g;
    if (st != CS_OK) return fail(st);
    if (e != cudaSuccess) { set_last_error("end capture", e); return fail(CS_ERR_CUDA); }
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) {
        set_last_error("graph instantiate", e);
        return fail(CS_ERR_CUDA);
    }
    cudaStreamDestroy(cap);
    *out_batch = b;
    return CS_OK;
}

extern "C" cs_status cs_batch_launch(cs_batch* b, void* stream) {
    if (!b || !b->exec) return CS_ERR_INVALID_ARG;
    CS_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return CS_OK;
}

extern "C" void cs_batch_destroy(cs_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_ctr);
    cudaFree(b->d_bunch);
    delete b;
}

extern "C" cs_status cs_autotune_tiling(const cs_segment* segs, size_t n, const cs_atmosphere* atm,
                                        const cs_detector* det, uint64_t seed, const int* shower_bunch,
                                        const cs_opts* opts, cs_output* out, void* stream_,
                                        cs_tune_result* res) {
    if (!res) return CS_ERR_INVALID_ARG;
    cs_opts o;
    if (opts) o = *opts; else cs_opts_default(&o);
    cs_status st = check_device_call(segs, n, atm, det, o, out);
    if (st != CS_OK) return st;
    cudaStream_t stream = (cudaStream_t)stream_;
    int* d_bunch = nullptr;
    if ((st = upload_bunches(det, shower_bunch, &d_bunch)) != CS_OK) return st;
    unsigned int* ctr = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    auto done = [&](cs_status s) {
        cudaFree(d_bunch);
        cudaFree(ctr);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return s;
    };
    if ((e = cudaMalloc(&ctr, scratch_bytes(n))) != cudaSuccess) { set_last_error("tune scratch", e); return done(CS_ERR_CUDA); }
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        set_last_error("tune events", e);
        return done(CS_ERR_CUDA);
    }
    memset(res, 0, sizeof *res);
    float best = 3.0e38f;
    for (int bpm = 1; bpm <= 4; ++bpm) {
        o.blocks_per_sm = bpm;
        unsigned int grid = 1;
        if ((st = prepare_launch(n, o, &grid)) != CS_OK) return done(st);
        if ((st = enqueue(segs, n, atm, det, seed, d_bunch, o, out, ctr, grid, stream)) != CS_OK) return done(st);
        float total = 0.0f;
        for (int r = 0; r < 3; ++r) {
            float ms = 0.0f;
            if ((e = cudaEventRecord(e0, stream)) != cudaSuccess) { set_last_error("tune", e); return done(CS_ERR_CUDA); }
            if ((st = enqueue(segs, n, atm, det, seed, d_bunch, o, out, ctr, grid, stream)) != CS_OK) return done(st);
            if ((e = cudaEventRecord(e1, stream)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
                (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
                set_last_error("tune timing", e);
                return done(CS_ERR_CUDA);
            }
            total += ms;
        }
        res->ms[bpm - 1] = total / 3.0f;
        res->n_tried = bpm;
        if (res->ms[bpm - 1] < best) {
            best = res->ms[bpm - 1];
            res->blocks_per_sm = bpm;
        }
    }
    return done(CS_OK);
}

extern "C" cs_status cs_autotune_bunches(const cs_segment* segs, size_t n, const cs_atmosphere* atm,
                                         const cs_detector* det, uint64_t seed, double rel_noise,
                                         const int* allowed, int n_allowed, const cs_opts* opts, cs_output* out,
                                         void* stream_, int* shower_bunch) {
    if (!allowed || n_allowed < 1 || !shower_bunch || !(rel_noise > 0.0)) return CS_ERR_INVALID_ARG;
    if (det && det->p.nx <= 0) return CS_ERR_INVALID_ARG;   // the rule reads the ground histogram
    cs_opts o;
    if (opts) o = *opts; else cs_opts_default(&o);
    int bmin = allowed[0], bmax = allowed[0];
    for (int i = 0; i < n_allowed; ++i) {
        if (allowed[i] < 1) return CS_ERR_INVALID_ARG;
        bmin = std::min(bmin, allowed[i]);
        bmax = std::max(bmax, allowed[i]);
    }
    o.bunch = bmax;
    o.accumulate = 0;
    cs_status st = check_device_call(segs, n, atm, det, o, out);
    if (st != CS_OK) return st;
    cudaStream_t stream = (cudaStream_t)stream_;
    // pilot run with the largest bunch: per-shower photon density in the light-pool core
    st = cs_propagate_ex(segs, n, atm, det, seed, &o, out, stream);
    if (st != CS_OK) return st;
    const DetParams& dp = det->p;
    const size_t cells = (size_t)dp.nx * dp.ny;
    std::vector<unsigned long long> h(cells * dp.n_showers);
    CS_CUDA_TRY(cudaMemcpyAsync(h.data(), out->hist, h.size() * 8, cudaMemcpyDeviceToHost, stream));
    CS_CUDA_TRY(cudaStreamSynchronize(stream));
    const size_t top = std::min<size_t>(100, cells);
    for (int s = 0; s < dp.n_showers; ++s) {
        auto first = h.begin() + (size_t)s * cells, last = first + cells;
        std::nth_element(first, first + (top - 1), last, std::greater<unsigned long long>());
        double mean = 0.0;
        for (size_t i = 0; i < top; ++i) mean += (double)first[i];
        mean /= (double)top;
        // bunching multiplies a cell's variance by b: keep sqrt(b / mean) <= rel_noise
        int pick = bmin;
        for (int i = 0; i < n_allowed; ++i)
            if (allowed[i] > pick && sqrt((double)allowed[i] / fmax(mean, 1e-300)) <= rel_noise) pick = allowed[i];
        shower_bunch[s] = pick;
    }
    return CS_OK;
}

// ---------------------------------------------------------------------------
// Streaming: host segments in fixed-size chunks through two device staging
// buffers on two streams, so the host-to-device copy of one chunk overlaps
// the photon kernel of the previous one (data transfer and batching,
// Sec. 5.1 and 5.4).  Buffer b is only ever used on stream b, so stream
// order alone keeps a copy from overwriting segments a kernel still reads.
// ---------------------------------------------------------------------------
struct cs_streamer {
    size_t chunk = 0;
    cs_segment* d_buf[2] = {nullptr, nullptr};
    unsigned int* d_scratch[2] = {nullptr, nullptr};   // per-stream launch scratch
    cudaStream_t st[2] = {nullptr, nullptr};
    cudaEvent_t ev_in = nullptr, ev_done[2] = {nullptr, nullptr};
    int device = 0;
};

extern "C" void cs_streamer_destroy(cs_streamer* s) {
    if (!s) return;
    for (int b = 0; b < 2; ++b) {
        if (s->st[b]) cudaStreamSynchronize(s->st[b]);
        cudaFree(s->d_buf[b]);
        cudaFree(s->d_scratch[b]);
        if (s->st[b]) cudaStreamDestroy(s->st[b]);
        if (s->ev_done[b]) cudaEventDestroy(s->ev_done[b]);
    }
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    delete s;
}

extern "C" cs_status cs_streamer_create(size_t chunk, cs_streamer** out) {
    if (!out) return CS_ERR_INVALID_ARG;
    *out = nullptr;
    if (chunk < 1 || chunk > ((size_t)1 << 32)) return CS_ERR_INVALID_ARG;
    cs_status st = check_device();
    if (st != CS_OK) return st;
    cs_streamer* s = new cs_streamer;
    s->chunk = chunk;
    cudaGetDevice(&s->device);
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMalloc(&s->d_buf[b], chunk * sizeof(cs_segment));
        if (e == cudaSuccess) e = cudaMalloc(&s->d_scratch[b], scratch_bytes(chunk));
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st[b], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_done[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        set_last_error("streamer create", e);
        cs_streamer_destroy(s);
        return CS_ERR_CUDA;
    }
    *out = s;
    return CS_OK;
}

extern "C" cs_status cs_streamer_run(cs_streamer* s, const cs_segment* host_segs, size_t n, const cs_atmosphere* atm,
                                     const cs_detector* det, uint64_t seed, const cs_opts* opts, cs_output* out,
                                     void* stream_) {
    if (!s) return CS_ERR_INVALID_ARG;
    cs_opts o;
    if (opts) o = *opts; else cs_opts_default(&o);
    // the outputs are device memory (device_ptrs = 1); the segments are host memory
    cs_status st = check_device_call(s->d_buf[0], n, atm, det, o, out);
    if (st != CS_OK) return st;
    if (n > 0 && !host_segs) return CS_ERR_INVALID_ARG;
    int dev = 0;
    CS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != s->device) return CS_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_;
    unsigned int grid = 0;
    st = prepare_launch(std::min(n, s->chunk), o, &grid);
    if (st != CS_OK) return st;
    // zeroing (unless accumulating) on the caller's stream, then both streams wait for it
    st = enqueue(nullptr, 0, atm, det, seed, nullptr, o, out, nullptr, grid, stream);
    if (st != CS_OK) return st;
    CS_CUDA_TRY(cudaEventRecord(s->ev_in, stream));
    for (int b = 0; b < 2; ++b) CS_CUDA_TRY(cudaStreamWaitEvent(s->st[b], s->ev_in, 0));
    cs_opts oc = o;
    oc.accumulate = 1;
    const size_t n_chunks = (n + s->chunk - 1) / s->chunk;
    for (size_t c = 0; c < n_chunks; ++c) {
        const int b = (int)(c & 1);
        const size_t off = c * s->chunk, m = std::min(s->chunk, n - off);
        CS_CUDA_TRY(cudaMemcpyAsync(s->d_buf[b], host_segs + off, m * sizeof(cs_segment), cudaMemcpyHostToDevice,
                                    s->st[b]));
        oc.seg_base = o.seg_base + off;
        st = enqueue(s->d_buf[b], m, atm, det, seed, nullptr, oc, out, s->d_scratch[b], grid, s->st[b]);
        if (st != CS_OK) return st;
    }
    // the caller's stream continues after both streams' last chunks
    for (int b = 0; b < 2; ++b) {
        CS_CUDA_TRY(cudaEventRecord(s->ev_done[b], s->st[b]));
        CS_CUDA_TRY(cudaStreamWaitEvent(stream, s->ev_done[b], 0));
    }
    return CS_OK;
}
