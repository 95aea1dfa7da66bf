// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cherenkov.h"

namespace cs {

constexpr double kC = 299792458.0;          // m/s
constexpr double kAlpha = 7.2973525693e-3;  // fine-structure constant
constexpr double kPi = 3.14159265358979323846;
constexpr double kLog2e = 1.4426950408889634;
constexpr int kMaxLayers = 8;
constexpr int kHashLevels = 3;   // telescope hash levels (zenith reach 45, 75, 82 deg)
constexpr int kMaxNodes = 128;     // tabulated atmosphere
constexpr double kTableRhoRef = 1.225e-3;   // [g/cm^3]: density = kTableRhoRef (n - 1) / kappa

// Correction table: per node two float4 {value at h_j from above, change to
// h_j+1 from below}; the four fields are
//   G_R = dR cos^3(theta0) / sin(theta0)   (dR: displacement minus straight line)
//   G_t = c dt cos(theta0)                 (dt: optical minus vacuum straight-line time)
//   G_X = X_slant cos(theta0)              [g/cm^2]
//   G_A = A_slant cos(theta0)              [m], aerosol-weighted path
// on rows h_obs + j dh and columns tan^2(theta0) = m dw (Sec. 4.4.1).
struct TableView {
    const float4* tab;   // [nh][nw][2]
    int nh, nw;
    float inv_dh, inv_dw;
    float dz_max;        // emission heights above h_obs + dz_max are out of domain
    float w_max;         // tan^2 of the domain's maximum zenith
};

// Everything a kernel needs about the atmosphere, passed by value.
struct AtmParams {
    int kind;            // CS_ATM_*
    int spherical;       // 1: spherical shell (Earth centre at (0, 0, -R)); also set for the cylinders
    int cylindrical;     // 1: coaxial cylinders per photon (traced by the stepper only)
    float R, rg, inv_rg; // Earth radius, r_g = R + h_obs [m], 1 / r_g
    int n_layers;
    int refraction;
    int transmission;
    int use_tables;      // refraction || transmission
    // delta(h) = n - 1 at a height dz = h - h_obs above the observation level:
    // layer i (dz >= lay_lo[i]) has delta = lay_D[i] * exp2(lay_c2[i] * dz)
    float lay_lo[kMaxLayers];
    float lay_D[kMaxLayers];
    float lay_c2[kMaxLayers];
    float top_rel;       // vacuum above h_top - h_obs
    float lin_d0, lin_slope, lin_top_rel, lin_d1;   // linear kind, relative to h_obs
    float hom_delta;
    // tabulated kind: interval i starts at node_lo[i] (relative to h_obs; the
    // first also serves below it) with n - 1 = node_d[i] exp2(node_c2[i] (dz - node_lo[i]))
    int n_nodes;
    const float* node_lo;   // device: node_lo, node_d, node_c2 (n_nodes - 1 each)
    const float* node_d;
    const float* node_c2;
    float n_obs;         // n(h_obs)
    float inv_n_obs;
    double h_obs;
    float h_obs_hi, h_obs_lo;   // h_obs as float-float
    float inv_l1_nm, dinv_l_nm;  // 1/lambda_min and 1/lambda_min - 1/lambda_max [1/nm]
    float ft;            // 2 pi alpha (1/lambda_min - 1/lambda_max) [1/m]
    // transmission: exponent in log2 units = (G_X kR + G_A kA) / |u_z|
    float kR0;           // log2(e) lambda0_R^4 / X0_R [nm^4 cm^2/g]
    float kA0;           // log2(e) tau0 / H_A [1/m]
    // the Snell stepper's slant columns: X [g/cm^2] per metre = rho_per_delta * delta,
    // exp(-h / H_A) = aer_hobs * exp2(aer_c2 * dz)
    float rho_per_delta, aer_hobs, aer_c2;
    float lamA_nm;       // aerosol reference wavelength [nm]
    float aer_alpha;
    TableView tv;
    const AtmParams* self;   // device copy of these parameters (for out-of-line routines)
};

// A uniform grid hash over the telescopes' reach discs for arrivals up to a
// zenith: the grid origin and the cell size are whole metres, so cell corners
// are exact in FP32; cell c lists the entries [cell_range[c].x, cell_range[c].y).
struct TelHash {
    float gx0, gy0, cell, inv_cell;
    int gnx, gny;
    const int2* cell_range;
    const int* cell_tel;      // telescope index of each entry (ascending within a cell)
    const float4* cell_data;  // planar: {x - corner_x, y - corner_y, z - h_obs, radius}; spherical: tel3
    float sin2_max;           // arrivals steeper than this need a wider hash or the full list
    float bx0, bx1, by0, by1; // bounding box of all reach discs
};

struct DetParams {
    int n_showers;
    int spherical;        // telescope layout and histogram in azimuthal-equidistant coordinates
    int cylindrical;      // layout and histogram on the unrolled ground cylinder (flat data, like the plane's)
    double R;
    float h_obs_f;        // observation level the telescopes were placed for
    double h_obs;
    int nx, ny;           // 0: no histogram
    float hx0_hi, hx0_lo, hy0_hi, hy0_lo;   // histogram corner as float-float [m]
    float inv_dx, inv_dy;
    int n_tel;
    const float4* tel;    // {x_hi, y_hi, z - h_obs, radius}
    const float2* tel_lo; // {x_lo, y_lo}
    const float4* tel3;   // spherical: centre in frame coordinates and radius
    // three hashes: hash[0] for arrivals up to 45 deg (small cells, mostly empty),
    // hash[1] up to 75 deg (the tables' domain), hash[2] up to 82 deg (the photons
    // beyond the tables, in the exact pass); steeper arrivals test every sphere
    TelHash hash[kHashLevels];
    // last-mile optics: mirror focal length, (aperture radius)^2, camera radius,
    // pixels per metre on the camera, and the telescope frame (axis a, e1 = a x z-hat, e2 = a x e1)
    int cam_n;
    float cam_f, cam_rd2, cam_r, cam_scale;
    float ax, ay, az, e1x, e1y, e1z, e2x, e2y, e2z;
    // absorption in the optics: R(lambda), eps(lambda) linear between eff_n nodes [1/nm in eff_il]
    int eff_n;
    float eff_l[16], eff_R[16], eff_E[16];
};

struct OutParams {
    unsigned long long* hist;
    unsigned long long* tel_counts;
    double* tel_time;
    unsigned long long* counters;
    cs_record* records;
    unsigned long long record_capacity;
    unsigned long long* record_count;
    unsigned long long* camera;   // n_showers x n_tel x cam_n^2, or null
};

struct PropParams {
    const cs_segment* segs;
    long long n;
    unsigned long long seg_base;
    uint32_t key0, key1;
    int bunch;                 // photons per bunch when shower_bunch is null
    const int* shower_bunch;   // per-shower bunch sizes (device), or null
    float s_max, s_max_lo;     // sub-step length as float-float
    // LV1 particle filter: drop when y >= lv1_a x^lv1_b (x in degrees)
    int lv1;                   // CS_LV1_*
    float lv1_a, lv1_b, lv1_r;
    float lv1_c[3];            // array centre, frame coordinates
    unsigned long long* lv1_dropped;   // device counter or null
    // LV3 photon pre-filter: drop when the straight line lands farther than
    // sqrt(lv3_r2) from lv3_c (planar: lv3_dz2 = (h_obs - centre z)^2)
    int lv3;
    float lv3_c[3];
    float lv3_r2, lv3_dz2;
    // Snell vector stepper instead of the tables: slabs no thicker than snell_dh
    int snell;
    float snell_dh;
    // fluorescence (CS_EMIT_*): mean bunches per metre = fl_yd z^2 delta(h) / b; line l
    // (1 / lambda in fl_inv_l) when the second draw's 24 bits are below fl_thr[l]
    int emission;
    int fl_n;
    float fl_yd;
    float fl_inv_l[8];
    uint32_t fl_thr[8];
    uint32_t rk[20];   // Philox key schedule: round r uses rk[2r], rk[2r + 1]
    int tiles_per_bit; // warp tiles (32 segments) per bit of the exact pass's tile map
    unsigned int q_cap; // entries of the exact pass's bunch queue (0: tile map only)
    unsigned int q_off; // its offset in the scratch, in 32-bit words (a multiple of 4)
};

// The atmosphere in FP64, as the table builder integrates it.
struct AtmF64 {
    int kind, n_layers;
    double lay_h[kMaxLayers], lay_a[kMaxLayers], lay_b[kMaxLayers], lay_c[kMaxLayers];
    double h_top, kappa, rho0;
    double lin_h0, lin_h1, lin_n0, lin_n1, hom_delta;
    double h_obs, H_A;
    int refraction;
    int spherical;          // 1: spherical shell, Earth radius R
    double R;
    int n_nodes;            // tabulated kind: n - 1 log-linear between nodes
    double node_h[kMaxNodes], node_d[kMaxNodes];
};


// ---- host-side helpers ------------------------------------------------------
void set_last_error(const char* where, cudaError_t e);
cs_status check_device();
int device_sm_count();

}  // namespace cs

struct cs_atmosphere;
namespace cs {
struct __align__(16) Fields4 {   // {G_R, G_t, G_X, G_A} in FP64
    double x, y, z, w;
};
// Exact FP64 {G_R, G_t, G_X, G_A} at samples {h_e [m], theta0 [rad]} (device arrays).
cs_status exact_fields(const cs_atmosphere* atm, const double2* d_in, size_t n, Fields4* d_out, cudaStream_t stream);
// FP64 vertical integrals from h_obs up to each height h [m] (device arrays):
// {int (n - 1) dh, n(h) - 1, int 100 rho dh [g/cm^2], int exp(-h / H_A) dh}.
cs_status column_fields(const cs_atmosphere* atm, const double* d_h, size_t n, Fields4* d_out, cudaStream_t stream);
}  // namespace cs

struct cs_atmosphere {
    cs::AtmParams p;
    cs::AtmParams* d_params;   // device copy of p (owned)
    float4* d_tab;         // device table (owned)
    float* d_nodes;        // tabulated kind: interval laws (owned)
    double h0, dh, dw;
    int device;
    cs::AtmF64 f64;        // the FP64 description the tables were built from
    double rayl_X0, rayl_lambda0, aer_tau0, aer_lambda0, aer_alpha, aer_H;
    double lambda_min, lambda_max;
};

struct cs_detector {
    cs::DetParams p;
    void* d_mem;           // one device allocation holding all arrays (owned)
    int device;
};

#define CS_CUDA_TRY(call)                                     \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) {                              \
            cs::set_last_error(#call, e_);                    \
            return CS_ERR_CUDA;                               \
        }                                                     \
    } while (0)
