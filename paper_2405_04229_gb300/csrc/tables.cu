// Atmosphere handle: closed-form refractive index parameters for the hot
// path and the FP64-built correction tables of the interpolation tracer
// (thesis Sec. 4.4.1).  The tables hold, per emission height and zenith, the
// difference between the exact refracted path (Eq. 3.17-3.18) and the
// straight line of Eq. 3.3, the time delay, and the slant columns used by
// the transmission stage (Sec. 4.3.1).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "common.cuh"

namespace cs {
namespace {

constexpr int kGL = 16;            // Gauss-Legendre points per sub-interval
constexpr double kSubMax = 2000.0; // maximum sub-interval length [m]

__constant__ double c_gl_x[kGL];
__constant__ double c_gl_w[kGL];

// Gauss-Legendre rule on [-1, 1]: roots of P_n by Newton's method started
// from the asymptotic guess, weights 2 / ((1 - x^2) P_n'(x)^2).
void legendre_rule(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double r = cos(kPi * (4.0 * i + 3.0) / (4.0 * n + 2.0));
        double deriv = 0.0;
        for (int iter = 0; iter < 64; ++iter) {
            double pm1 = 0.0, p = 1.0;
            for (int k = 1; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * r * p - (k - 1.0) * pm1) / k;
                pm1 = p;
                p = pk;
            }
            deriv = n * (pm1 - r * p) / (1.0 - r * r);
            double step = p / deriv;
            r -= step;
            if (fabs(step) <= 1e-17) break;
        }
        x[i] = r;
        w[i] = 2.0 / ((1.0 - r * r) * deriv * deriv);
    }
}

// layer of h; at a boundary `below` selects the lower layer (limit from below)
__device__ __host__ inline int layer_index(const AtmF64& a, double h, bool below) {
    int i = 0;
    for (int k = 1; k < a.n_layers; ++k)
        if (below ? (h > a.lay_h[k]) : (h >= a.lay_h[k])) i = k;
    return i;
}

__device__ inline void delta_rho(const AtmF64& a, double h, bool below, double* delta, double* rho) {
    if (a.kind == CS_ATM_LAYERED) {
        bool vac = below ? (h > a.h_top) : (h >= a.h_top);
        if (vac) { *delta = 0.0; *rho = 0.0; return; }
        int i = layer_index(a, h, below);
        double r = (i == a.n_layers - 1) ? a.lay_b[i] / a.lay_c[i]
                                         : a.lay_b[i] / a.lay_c[i] * exp(-h * 100.0 / a.lay_c[i]);
        *rho = r;
        *delta = a.kappa * r / a.rho0;
    } else if (a.kind == CS_ATM_TABLE) {
        const int n = a.n_nodes;
        bool vac = below ? (h > a.node_h[n - 1]) : (h >= a.node_h[n - 1]);
        if (vac) { *delta = 0.0; *rho = 0.0; return; }
        int i = 0;
        while (i + 2 < n && h >= a.node_h[i + 1]) ++i;
        const double k = log(a.node_d[i + 1] / a.node_d[i]) / (a.node_h[i + 1] - a.node_h[i]);
        *delta = a.node_d[i] * exp(k * (h - a.node_h[i]));
        *rho = kTableRhoRef * *delta / a.kappa;
    } else if (a.kind == CS_ATM_LINEAR) {
        *rho = 0.0;
        bool above_top = below ? (h > a.lin_h1) : (h >= a.lin_h1);
        *delta = above_top ? a.lin_n1 - 1.0
                           : (a.lin_n0 - 1.0) - (h - a.lin_h0) / (a.lin_h1 - a.lin_h0) * (a.lin_n0 - a.lin_n1);
    } else {
        *rho = 0.0;
        *delta = a.hom_delta;
    }
}

// The four integrals from h_obs up to h_e for zenith theta0 (cos0, sin0),
// normalised as described in common.cuh.
__device__ void node_fields(const AtmF64& a, double h_e, bool below, double cos0, double sin0,
                            double out[4]) {
    double de, rho_e;
    delta_rho(a, h_e, below, &de, &rho_e);
    const double ne = 1.0 + de, s = ne * sin0;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    // breakpoints: layer bottoms, table nodes and the top strictly inside (h_obs, h_e)
    double cuts[kMaxNodes + 3];
    int nc = 0;
    cuts[nc++] = a.h_obs;
    if (a.kind == CS_ATM_LAYERED) {
        for (int k = 1; k < a.n_layers; ++k)
            if (a.lay_h[k] > a.h_obs && a.lay_h[k] < h_e) cuts[nc++] = a.lay_h[k];
        if (a.h_top > a.h_obs && a.h_top < h_e) cuts[nc++] = a.h_top;
    } else if (a.kind == CS_ATM_LINEAR) {
        if (a.lin_h1 > a.h_obs && a.lin_h1 < h_e) cuts[nc++] = a.lin_h1;
    } else if (a.kind == CS_ATM_TABLE) {
        for (int k = 1; k < a.n_nodes; ++k)
            if (a.node_h[k] > a.h_obs && a.node_h[k] < h_e) cuts[nc++] = a.node_h[k];
    }
    cuts[nc++] = h_e;
    // spherical shell: r = R + h, Bouguer's invariant K = n_e r_e sin(psi0); the
    // straight-line reference has K0 = r_e sin(psi0) and q0 = sqrt(r^2 - K0^2)
    const double re = a.R + h_e, K0 = re * sin0;
    for (int piece = 0; piece + 1 < nc; ++piece) {
        const double lo = cuts[piece], hi = cuts[piece + 1];
        const int nsub = (int)ceil((hi - lo) / kSubMax);
        const double step = (hi - lo) / nsub;
        for (int sub = 0; sub < nsub; ++sub) {
            const double mid = lo + (sub + 0.5) * step, half = 0.5 * step;
            for (int g = 0; g < kGL; ++g) {
                const double h = mid + half * c_gl_x[g], wt = half * c_gl_w[g];
                double d, rho;
                delta_rho(a, h, false, &d, &rho);
                const double n = 1.0 + d;
                if (!a.spherical) {
                    if (a.refraction) {
                        const double q = sqrt(n * n - s * s);
                        acc[0] += wt * (de - d) * (2.0 + de + d) / (q * (ne * cos0 + q));
                        acc[1] += wt * (n * n * cos0 - q) / q;
                        acc[2] += wt * 100.0 * rho * n / q;
                        acc[3] += wt * exp(-h / a.H_A) * n / q;
                    } else {
                        acc[2] += wt * 100.0 * rho;
                        acc[3] += wt * exp(-h / a.H_A);
                    }
                } else {
                    const double r = a.R + h;
                    const double q0 = sqrt(r * r - K0 * K0);
                    if (a.refraction) {
                        const double q = sqrt(n * n * r * r - ne * ne * K0 * K0);
                        // central angle minus the straight line's, divided by sin(psi0):
                        // K0 r (n_e^2 - n^2) / (q q0 (n_e q0 + q)) / sin(psi0)
                        acc[0] += wt * re * r * (de - d) * (2.0 + de + d) / (q * q0 * (ne * q0 + q));
                        acc[1] += wt * (n * n * r / q - r / q0);
                        acc[2] += wt * 100.0 * rho * n * r / q;
                        acc[3] += wt * exp(-h / a.H_A) * n * r / q;
                    } else {
                        acc[2] += wt * 100.0 * rho * r / q0;
                        acc[3] += wt * exp(-h / a.H_A) * r / q0;
                    }
                }
            }
        }
    }
    if (a.spherical) {
        // G_R = (arc length correction on the ground sphere) cos^3 / sin, G_t = c dt cos,
        // G_X = X cos, G_A = A cos
        out[0] = a.refraction ? (a.R + a.h_obs) * cos0 * cos0 * cos0 * acc[0] : 0.0;
        out[1] = a.refraction ? cos0 * acc[1] : 0.0;
        out[2] = cos0 * acc[2];
        out[3] = cos0 * acc[3];
        return;
    }
    if (a.refraction) {
        out[0] = cos0 * cos0 * acc[0];
        out[1] = acc[1];
        out[2] = cos0 * acc[2];
        out[3] = cos0 * acc[3];
    } else {
        out[0] = 0.0;
        out[1] = 0.0;
        out[2] = acc[2];
        out[3] = acc[3];
    }
}

// One thread per (row, column): fields at row j approached from above.
__global__ void build_rows_kernel(AtmF64 a, int nh, int nw, double dh, double dw, double* F) {
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= nh * nw) return;
    const int j = node / nw, m = node % nw;
    const double w = m * dw, cos0 = 1.0 / sqrt(1.0 + w), sin0 = sqrt(w) * cos0;
    double out[4];
    node_fields(a, a.h_obs + j * dh, false, cos0, sin0, out);
    for (int f = 0; f < 4; ++f) F[(size_t)node * 4 + f] = out[f];
}

// Fields at the listed rows approached from below (rows on layer boundaries).
__global__ void build_below_kernel(AtmF64 a, const int* rows, int nb, int nw, double dh, double dw,
                                   double* Fb) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * nw) return;
    const int b = t / nw, m = t % nw;
    const double w = m * dw, cos0 = 1.0 / sqrt(1.0 + w), sin0 = sqrt(w) * cos0;
    double out[4];
    node_fields(a, a.h_obs + rows[b] * dh, true, cos0, sin0, out);
    for (int f = 0; f < 4; ++f) Fb[(size_t)t * 4 + f] = out[f];
}

// Cell form: value at h_j (from above) and change to h_j+1 (from below).
__global__ void assemble_kernel(const double* F, const double* Fb, const int* below_slot, int nh, int nw,
                                float4* tab) {
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= nh * nw) return;
    const int j = node / nw, m = node % nw;
    const double* v = F + (size_t)node * 4;
    double up[4];
    if (j + 1 < nh) {
        const int slot = below_slot[j + 1];
        const double* src = slot >= 0 ? Fb + ((size_t)slot * nw + m) * 4 : F + ((size_t)(j + 1) * nw + m) * 4;
        for (int f = 0; f < 4; ++f) up[f] = src[f];
    } else {
        for (int f = 0; f < 4; ++f) up[f] = v[f];
    }
    tab[(size_t)node * 2 + 0] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
    tab[(size_t)node * 2 + 1] = make_float4((float)(up[0] - v[0]), (float)(up[1] - v[1]),
                                            (float)(up[2] - v[2]), (float)(up[3] - v[3]));
}

// Vertical integrals from h_obs up to each height h (one thread per height):
// {int (n - 1) dh [m], n(h) - 1 (from above), int 100 rho dh [g/cm^2],
//  int exp(-h / H_A) dh [m]}, by the same Gauss-Legendre pieces as the tables.
__global__ void column_kernel(AtmF64 a, const double* h_in, size_t n, Fields4* out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double h = h_in[i];
    double de, rho_e;
    delta_rho(a, h, false, &de, &rho_e);
    double cuts[kMaxNodes + 3];
    int nc = 0;
    cuts[nc++] = a.h_obs;
    if (a.kind == CS_ATM_LAYERED) {
        for (int k = 1; k < a.n_layers; ++k)
            if (a.lay_h[k] > a.h_obs && a.lay_h[k] < h) cuts[nc++] = a.lay_h[k];
        if (a.h_top > a.h_obs && a.h_top < h) cuts[nc++] = a.h_top;
    } else if (a.kind == CS_ATM_LINEAR) {
        if (a.lin_h1 > a.h_obs && a.lin_h1 < h) cuts[nc++] = a.lin_h1;
    } else if (a.kind == CS_ATM_TABLE) {
        for (int k = 1; k < a.n_nodes; ++k)
            if (a.node_h[k] > a.h_obs && a.node_h[k] < h) cuts[nc++] = a.node_h[k];
    }
    cuts[nc++] = h;
    double sI = 0.0, sX = 0.0, sA = 0.0;
    for (int piece = 0; piece + 1 < nc; ++piece) {
        const double lo = cuts[piece], hi = cuts[piece + 1];
        const int nsub = (int)ceil((hi - lo) / kSubMax);
        const double step = (hi - lo) / nsub;
        for (int sub = 0; sub < nsub; ++sub) {
            const double mid = lo + (sub + 0.5) * step, half = 0.5 * step;
            for (int g = 0; g < kGL; ++g) {
                const double y = mid + half * c_gl_x[g], wt = half * c_gl_w[g];
                double d, rho;
                delta_rho(a, y, false, &d, &rho);
                sI += wt * d;
                sX += wt * 100.0 * rho;
                sA += wt * exp(-y / a.H_A);
            }
        }
    }
    out[i] = Fields4{sI, de, sX, sA};
}

// One thread per sample: the exact FP64 fields at (h_e, theta0).
__global__ void exact_fields_kernel(AtmF64 a, const double2* in, size_t n, Fields4* out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double h_e = in[i].x, th = in[i].y;
    const double cos0 = cos(th), sin0 = sin(th);
    double f[4];
    node_fields(a, h_e, false, cos0, sin0, f);
    out[i] = Fields4{f[0], f[1], f[2], f[3]};
}

bool divides(double len, double dh) {
    double r = len / dh;
    return fabs(r - nearbyint(r)) < 1e-9 * fmax(1.0, fabs(r));
}

}  // namespace
}  // namespace cs

using namespace cs;

extern "C" cs_status cs_atmosphere_create(const cs_atmosphere_desc* d, cs_atmosphere** out) {
    if (!d || !out) return CS_ERR_INVALID_ARG;
    *out = nullptr;
    if (d->kind < CS_ATM_LAYERED || d->kind > CS_ATM_TABLE) return CS_ERR_INVALID_ARG;
    if (!(d->lambda_min > 0.0) || !(d->lambda_max > d->lambda_min)) return CS_ERR_INVALID_ARG;
    if (!isfinite(d->h_obs)) return CS_ERR_INVALID_ARG;
    const double theta_max = d->theta_max > 0.0 ? d->theta_max : 75.0 * kPi / 180.0;
    if (!(theta_max < 89.0 * kPi / 180.0)) return CS_ERR_INVALID_ARG;
    const double dh = d->table_dh > 0.0 ? d->table_dh : 20.0;
    const int nw = d->table_nw > 0 ? d->table_nw : 48;
    if (nw < 2 || nw > 4096) return CS_ERR_INVALID_ARG;

    AtmF64 a;
    memset(&a, 0, sizeof a);
    a.kind = d->kind;
    a.h_obs = d->h_obs;
    a.refraction = d->refraction ? 1 : 0;
    // the cylinders keep the sphere's frame (altitude of the emission point, local vertical)
    a.spherical = d->geometry == CS_GEOM_SPHERICAL || d->geometry == CS_GEOM_CYLINDRICAL ? 1 : 0;
    a.R = d->earth_radius > 0.0 ? d->earth_radius : 6370000.0;
    if (d->geometry != CS_GEOM_PLANAR && d->geometry != CS_GEOM_SPHERICAL && d->geometry != CS_GEOM_CYLINDRICAL)
        return CS_ERR_INVALID_ARG;
    a.H_A = d->aer_H > 0.0 ? d->aer_H : 1200.0;
    double table_top;
    if (d->kind == CS_ATM_LAYERED) {
        if (d->n_layers < 1 || d->n_layers > kMaxLayers) return CS_ERR_INVALID_ARG;
        if (!d->layer_h || !d->layer_a || !d->layer_b || !d->layer_c) return CS_ERR_INVALID_ARG;
        a.n_layers = d->n_layers;
        for (int i = 0; i < d->n_layers; ++i) {
            a.lay_h[i] = d->layer_h[i];
            a.lay_a[i] = d->layer_a[i];
            a.lay_b[i] = d->layer_b[i];
            a.lay_c[i] = d->layer_c[i];
            if (!(a.lay_c[i] > 0.0) || !(a.lay_b[i] > 0.0)) return CS_ERR_INVALID_ARG;
            if (i > 0 && !(a.lay_h[i] > a.lay_h[i - 1])) return CS_ERR_INVALID_ARG;
        }
        a.h_top = d->h_top;
        a.kappa = d->kappa;
        if (!(a.h_top > a.lay_h[a.n_layers - 1]) || !(a.kappa > 0.0)) return CS_ERR_INVALID_ARG;
        if (!(d->h_obs < a.h_top)) return CS_ERR_INVALID_ARG;
        a.rho0 = a.lay_b[0] / a.lay_c[0];
        table_top = a.h_top;
        for (int i = 1; i < a.n_layers; ++i)
            if (a.lay_h[i] > d->h_obs && !divides(a.lay_h[i] - d->h_obs, dh)) return CS_ERR_INVALID_ARG;
    } else if (d->kind == CS_ATM_LINEAR) {
        a.lin_h0 = d->lin_h0; a.lin_h1 = d->lin_h1; a.lin_n0 = d->lin_n0; a.lin_n1 = d->lin_n1;
        if (!(a.lin_h1 > a.lin_h0) || !(a.lin_n0 >= 1.0) || !(a.lin_n1 >= 1.0)) return CS_ERR_INVALID_ARG;
        if (!(d->h_obs < a.lin_h1)) return CS_ERR_INVALID_ARG;
        if (d->transmission) return CS_ERR_INVALID_ARG;   // no density for this kind
        table_top = a.lin_h1;
        if (!divides(a.lin_h1 - d->h_obs, dh)) return CS_ERR_INVALID_ARG;
    } else if (d->kind == CS_ATM_TABLE) {
        if (d->table_n < 2 || d->table_n > kMaxNodes || !d->table_h || !d->table_delta) return CS_ERR_INVALID_ARG;
        a.n_nodes = d->table_n;
        for (int i = 0; i < d->table_n; ++i) {
            a.node_h[i] = d->table_h[i];
            a.node_d[i] = d->table_delta[i];
            if (!isfinite(a.node_h[i]) || !(a.node_d[i] > 0.0) || !isfinite(a.node_d[i])) return CS_ERR_INVALID_ARG;
            if (i > 0 && !(a.node_h[i] > a.node_h[i - 1])) return CS_ERR_INVALID_ARG;
        }
        a.kappa = d->kappa > 0.0 ? d->kappa : 2.9e-4;
        a.h_top = a.node_h[a.n_nodes - 1];
        if (!(d->h_obs < a.h_top)) return CS_ERR_INVALID_ARG;
        table_top = a.h_top;
    } else {
        a.hom_delta = d->hom_delta;
        if (!(a.hom_delta >= 0.0)) return CS_ERR_INVALID_ARG;
        if (d->transmission) return CS_ERR_INVALID_ARG;
        table_top = d->h_obs + 100000.0;
    }
    cs_status st = check_device();
    if (st != CS_OK) return st;

    cs_atmosphere* h = new cs_atmosphere;
    memset(h, 0, sizeof *h);
    cudaGetDevice(&h->device);
    if (d->kind == CS_ATM_TABLE) {   // interval laws for the FP32 hot path, relative to h_obs
        const int m = a.n_nodes - 1;
        std::vector<float> nodes(3 * (size_t)m);
        for (int i = 0; i < m; ++i) {
            const double k = log(a.node_d[i + 1] / a.node_d[i]) / (a.node_h[i + 1] - a.node_h[i]);
            nodes[i] = (float)(a.node_h[i] - d->h_obs);
            nodes[m + i] = (float)a.node_d[i];
            nodes[2 * m + i] = (float)(k * kLog2e);
        }
        if (cudaMalloc(&h->d_nodes, nodes.size() * sizeof(float)) != cudaSuccess ||
            cudaMemcpy(h->d_nodes, nodes.data(), nodes.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(h->d_nodes);
            delete h;
            return CS_ERR_CUDA;
        }
        h->p.node_lo = h->d_nodes;
        h->p.node_d = h->d_nodes + m;
        h->p.node_c2 = h->d_nodes + 2 * m;
    }
    h->f64 = a;
    h->rayl_X0 = d->rayl_X0;
    h->rayl_lambda0 = d->rayl_lambda0;
    h->aer_tau0 = d->aer_tau0;
    h->aer_lambda0 = d->aer_lambda0;
    h->aer_alpha = d->aer_alpha;
    h->aer_H = a.H_A;
    h->lambda_min = d->lambda_min;
    h->lambda_max = d->lambda_max;
    AtmParams& p = h->p;
    p.kind = d->kind;
    p.spherical = a.spherical;
    p.cylindrical = d->geometry == CS_GEOM_CYLINDRICAL ? 1 : 0;
    p.R = (float)a.R;
    p.rg = (float)(a.R + d->h_obs);
    p.inv_rg = (float)(1.0 / (a.R + d->h_obs));
    p.n_layers = a.n_layers;
    p.refraction = a.refraction;
    p.transmission = d->transmission ? 1 : 0;
    // the cylinders' stepper integrates every photon's fields itself
    p.use_tables = (p.refraction || p.transmission) && !p.cylindrical ? 1 : 0;
    p.h_obs = d->h_obs;
    if (d->kind == CS_ATM_LAYERED) {
        for (int i = 0; i < a.n_layers; ++i) {
            p.lay_lo[i] = (float)(a.lay_h[i] - d->h_obs);
            if (i == a.n_layers - 1) {
                p.lay_D[i] = (float)(a.kappa * (a.lay_b[i] / a.lay_c[i]) / a.rho0);
                p.lay_c2[i] = 0.0f;
            } else {
                p.lay_D[i] = (float)(a.kappa * (a.lay_b[i] / a.lay_c[i]) * exp(-100.0 * d->h_obs / a.lay_c[i]) / a.rho0);
                p.lay_c2[i] = (float)(-100.0 * kLog2e / a.lay_c[i]);
            }
        }
        p.lay_lo[0] = -1e30f;   // the lowest law extends downwards
        p.top_rel = (float)(a.h_top - d->h_obs);
        int iobs = layer_index(a, d->h_obs, false);
        double rho_obs = (iobs == a.n_layers - 1) ? a.lay_b[iobs] / a.lay_c[iobs]
                                                  : a.lay_b[iobs] / a.lay_c[iobs] * exp(-100.0 * d->h_obs / a.lay_c[iobs]);
        p.n_obs = (float)(1.0 + a.kappa * rho_obs / a.rho0);
    } else if (d->kind == CS_ATM_LINEAR) {
        double slope = -(a.lin_n0 - a.lin_n1) / (a.lin_h1 - a.lin_h0);
        p.lin_d0 = (float)((a.lin_n0 - 1.0) + slope * (d->h_obs - a.lin_h0));
        p.lin_slope = (float)slope;
        p.lin_top_rel = (float)(a.lin_h1 - d->h_obs);
        p.lin_d1 = (float)(a.lin_n1 - 1.0);
        p.n_obs = 1.0f + p.lin_d0;
    } else if (d->kind == CS_ATM_TABLE) {
        p.n_nodes = a.n_nodes;
        p.top_rel = (float)(a.h_top - d->h_obs);
        double d_obs = 0.0;
        {
            int i = 0;
            while (i + 2 < a.n_nodes && d->h_obs >= a.node_h[i + 1]) ++i;
            const double k = log(a.node_d[i + 1] / a.node_d[i]) / (a.node_h[i + 1] - a.node_h[i]);
            d_obs = a.node_d[i] * exp(k * (d->h_obs - a.node_h[i]));
        }
        p.n_obs = (float)(1.0 + d_obs);
    } else {
        p.hom_delta = (float)a.hom_delta;
        p.n_obs = (float)(1.0 + a.hom_delta);
    }
    p.inv_n_obs = 1.0f / p.n_obs;
    p.h_obs_hi = (float)d->h_obs;
    p.h_obs_lo = (float)(d->h_obs - (double)p.h_obs_hi);
    const double l1_nm = d->lambda_min * 1e9, l2_nm = d->lambda_max * 1e9;
    p.inv_l1_nm = (float)(1.0 / l1_nm);
    p.dinv_l_nm = (float)(1.0 / l1_nm - 1.0 / l2_nm);
    p.ft = (float)(2.0 * kPi * kAlpha * (1.0 / d->lambda_min - 1.0 / d->lambda_max));
    // density per unit n - 1, in g/cm^2 per metre: the stepper's columns and the fluorescence yield
    p.rho_per_delta = a.kind == CS_ATM_LAYERED ? (float)(100.0 * a.rho0 / a.kappa)
                    : a.kind == CS_ATM_TABLE   ? (float)(100.0 * kTableRhoRef / a.kappa)
                                               : 0.0f;
    if (p.transmission) {
        if (!(d->rayl_X0 > 0.0) || !(d->rayl_lambda0 > 0.0) || !(d->aer_lambda0 > 0.0)) {
            cudaFree(h->d_nodes);
            delete h;
            return CS_ERR_INVALID_ARG;
        }
        const double lR = d->rayl_lambda0 * 1e9;
        p.kR0 = (float)(kLog2e * lR * lR * lR * lR / d->rayl_X0);
        p.kA0 = (float)(kLog2e * d->aer_tau0 / a.H_A);
        p.aer_hobs = (float)exp(-d->h_obs / a.H_A);
        p.aer_c2 = (float)(-kLog2e / a.H_A);
        p.lamA_nm = (float)(d->aer_lambda0 * 1e9);
        p.aer_alpha = (float)d->aer_alpha;
    }

    const int nh = (int)ceil((table_top - d->h_obs) / dh - 1e-9) + 1;
    const double w_max = tan(theta_max) * tan(theta_max);
    const double dw = w_max / (nw - 1);
    h->h0 = d->h_obs;
    h->dh = dh;
    h->dw = dw;
    p.tv.nh = nh;
    p.tv.nw = nw;
    p.tv.inv_dh = (float)(1.0 / dh);
    p.tv.inv_dw = (float)(1.0 / dw);
    p.tv.dz_max = (float)(table_top - d->h_obs);
    p.tv.w_max = (float)w_max;

    // ---- FP64 table build on the device ------------------------------------
    double glx[kGL], glw[kGL];
    legendre_rule(kGL, glx, glw);
    std::vector<int> below_slot(nh, -1), brows;
    if (d->kind == CS_ATM_LAYERED) {
        for (int i = 1; i < a.n_layers; ++i) {
            double r = (a.lay_h[i] - d->h_obs) / dh;
            if (a.lay_h[i] > d->h_obs && r < nh) {
                int row = (int)nearbyint(r);
                below_slot[row] = (int)brows.size();
                brows.push_back(row);
            }
        }
    }
    const size_t nodes = (size_t)nh * nw;
    double *dF = nullptr, *dFb = nullptr;
    int *dslot = nullptr, *drows = nullptr;
    cudaError_t e = cudaSuccess;
    auto fail = [&](const char* where) {
        set_last_error(where, e);
        cudaFree(dF); cudaFree(dFb); cudaFree(dslot); cudaFree(drows); cudaFree(h->d_tab); cudaFree(h->d_nodes);
        cudaFree(h->d_params);
        delete h;
        return CS_ERR_CUDA;
    };
    if ((e = cudaMemcpyToSymbol(c_gl_x, glx, sizeof glx)) != cudaSuccess) return fail("gl nodes");
    if ((e = cudaMemcpyToSymbol(c_gl_w, glw, sizeof glw)) != cudaSuccess) return fail("gl weights");
    if ((e = cudaMalloc(&dF, nodes * 4 * sizeof(double))) != cudaSuccess) return fail("table scratch");
    if ((e = cudaMalloc(&dFb, (brows.size() + 1) * nw * 4 * sizeof(double))) != cudaSuccess) return fail("table scratch");
    if ((e = cudaMalloc(&dslot, nh * sizeof(int))) != cudaSuccess) return fail("table scratch");
    if ((e = cudaMalloc(&drows, (brows.size() + 1) * sizeof(int))) != cudaSuccess) return fail("table scratch");
    if ((e = cudaMalloc(&h->d_tab, nodes * 2 * sizeof(float4))) != cudaSuccess) return fail("table");
    if ((e = cudaMemcpy(dslot, below_slot.data(), nh * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) return fail("copy");
    if (!brows.empty() &&
        (e = cudaMemcpy(drows, brows.data(), brows.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail("copy");
    const int T = 128;
    build_rows_kernel<<<(unsigned)((nodes + T - 1) / T), T>>>(a, nh, nw, dh, dw, dF);
    if (!brows.empty())
        build_below_kernel<<<(unsigned)((brows.size() * nw + T - 1) / T), T>>>(a, drows, (int)brows.size(), nw, dh, dw, dFb);
    assemble_kernel<<<(unsigned)((nodes + T - 1) / T), T>>>(dF, dFb, dslot, nh, nw, h->d_tab);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail("table kernels");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail("table build");
    cudaFree(dF); cudaFree(dFb); cudaFree(dslot); cudaFree(drows);
    p.tv.tab = h->d_tab;
    if ((e = cudaMalloc(&h->d_params, sizeof(AtmParams))) != cudaSuccess) return fail("parameters");
    p.self = h->d_params;
    if ((e = cudaMemcpy(h->d_params, &p, sizeof(AtmParams), cudaMemcpyHostToDevice)) != cudaSuccess) return fail("parameters");
    *out = h;
    return CS_OK;
}

namespace cs {
cs_status column_fields(const cs_atmosphere* atm, const double* d_h, size_t n, Fields4* d_out, cudaStream_t stream) {
    if (n == 0) return CS_OK;
    column_kernel<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(atm->f64, d_h, n, d_out);
    CS_CUDA_TRY(cudaGetLastError());
    return CS_OK;
}

cs_status exact_fields(const cs_atmosphere* atm, const double2* d_in, size_t n, Fields4* d_out, cudaStream_t stream) {
    if (n == 0) return CS_OK;
    exact_fields_kernel<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(atm->f64, d_in, n, d_out);
    CS_CUDA_TRY(cudaGetLastError());
    return CS_OK;
}
}  // namespace cs

extern "C" void cs_atmosphere_destroy(cs_atmosphere* atm) {
    if (!atm) return;
    cudaFree(atm->d_tab);
    cudaFree(atm->d_nodes);
    cudaFree(atm->d_params);
    delete atm;
}

extern "C" cs_status cs_atmosphere_table_info(const cs_atmosphere* atm, int* nh, int* nw, double* h0,
                                              double* dh, double* dw) {
    if (!atm) return CS_ERR_INVALID_ARG;
    if (nh) *nh = atm->p.tv.nh;
    if (nw) *nw = atm->p.tv.nw;
    if (h0) *h0 = atm->h0;
    if (dh) *dh = atm->dh;
    if (dw) *dw = atm->dw;
    return CS_OK;
}

extern "C" cs_status cs_atmosphere_copy_table(const cs_atmosphere* atm, float* host_dst, size_t n_floats) {
    if (!atm || !host_dst) return CS_ERR_INVALID_ARG;
    const size_t need = (size_t)atm->p.tv.nh * atm->p.tv.nw * 8;
    if (n_floats < need) return CS_ERR_INVALID_ARG;
    CS_CUDA_TRY(cudaMemcpy(host_dst, atm->d_tab, need * sizeof(float), cudaMemcpyDeviceToHost));
    return CS_OK;
}
