/*
 * FP64 CPU oracle for Cherenkov photon generation and propagation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no source,
 * header, table or helper with the CUDA path; the two are independent
 * implementations of the same method and are compared photon by photon.
 *
 * Everything here is plain, unblocked FP64 and follows the thesis
 * (D. Baack, "Optical Photon Emission in Extended Airshowers", 2023):
 *
 *   photon yield          Sec. 2.2.1, Eq. 2.2-2.5 (Frank-Tamm, threshold,
 *                         location-dependent Cherenkov angle)
 *   random numbers        Sec. 3.1 (counter-based Philox, Salmon et al. 2011)
 *   atmosphere            Sec. 3.3.1-3.3.2 (homogeneous, planar layered),
 *                         Sec. 6.3.1 (linear test profile)
 *   straight line         Sec. 3.4.1, Eq. 3.1-3.3
 *   Snell vector stepper  Sec. 3.4.2, Eq. 3.6-3.15
 *   refraction invariant  Sec. 3.4.3, Eq. 3.17-3.18 (n sin(theta) = const),
 *                         linear profile Eq. 3.19-3.23 and Appendix A.1
 *   photon generation     Sec. 4.2 (cone vector, Euler-Rodrigues 180-degree
 *                         rotation about the bisector, translation along the
 *                         track) and Sec. 4.2.1 (sub-stepping)
 *   absorption            Sec. 2.3.2 and Sec. 4.3.1 (survival test r < p)
 *   correction target     Sec. 4.4.1 (the exact path that the correction
 *                         tables approximate)
 *   spherical shell       Sec. 3.3.4 (Bouguer's invariant n r sin(psi),
 *                         azimuthal-equidistant ground coordinates)
 *   cylindrical model     Sec. 3.3.3 (coaxial cylinders per photon, the
 *                         axial and angular invariants, unrolled ground)
 *   tabulated atmosphere  Sec. 3.3 (a user's n(h) table, log-linear)
 *   Snell stepper as a    Sec. 3.4.2 on slabs and on spherical shells, with
 *   propagation method    delay and slant columns
 *   fluorescence          Sec. 2.2.2, Eq. 2.6 and Sec. 4.2.2 (isotropic or
 *                         half-sphere line emission)
 *   LV1 / LV3 filters     Sec. 4.3.2, 4.3.4, 6.2.1, 6.2.2
 *   mirror and camera     Sec. 6.4 (last-mile ray tracing)
 *
 * Where the thesis is silent the oracle takes the documented readings
 * (layer parameters, transmission constants, stochastic rounding of the
 * photon count, sub-step midpoint for the angle, edge bands).
 *
 * The refraction integrals are evaluated per photon by adaptive
 * Gauss-Legendre quadrature split at every layer boundary; a second,
 * independent path evaluates the same integrals in closed form per
 * exponential layer, and a third (the thesis's own Snell stepper) must
 * converge to both.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_C_LIGHT 299792458.0           /* m/s */
#define ORC_ALPHA   7.2973525693e-3       /* fine-structure constant (CODATA 2018) */
#define ORC_PI      3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).                 */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {               /* Weyl key schedule between rounds */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 24-bit uniform in [0, 1): exact in both FP32 and FP64. */
static double orc_uniform(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------ */
/* Atmosphere (Sec. 3.3).                                             */
/* ------------------------------------------------------------------ */
enum { ORC_ATM_LAYERED = 0, ORC_ATM_LINEAR = 1, ORC_ATM_HOMOGENEOUS = 2, ORC_ATM_TABLE = 3 };
#define ORC_MAX_NODES 128

typedef struct {
    int kind;
    int n_layers;          /* layered kind: number of layers (<= 8)               */
    int last_linear;       /* layered kind: top layer has T linear in h            */
    int pad;
    double layer_h[8];     /* layer bottoms [m], ascending; layer_h[0] is the ground */
    double a[8], b[8], c[8];  /* T(h) = a + b exp(-h/c) [g/cm^2], c in cm          */
    double h_top;          /* top of the atmosphere [m]; vacuum above              */
    double kappa;          /* n - 1 = kappa * rho(h) / rho(0)                       */
    double lin_h0, lin_h1; /* linear kind: n = n0 at h0 falling to n1 at h1        */
    double lin_n0, lin_n1;
    double hom_delta;      /* homogeneous kind: n - 1                              */
    /* table kind (a user's n(h) table, Sec. 3.3): n - 1 at ascending node
     * heights, log-linear between nodes (each interval one exponential), the
     * first interval's law continued below the first node, vacuum at and
     * above the last node (the top); density rho = rho_ref (n - 1) / kappa */
    int n_nodes;
    int pad2;
    double node_h[ORC_MAX_NODES];
    double node_d[ORC_MAX_NODES];
    double rho_ref;        /* [g/cm^3] */
} orc_atm;

/* Table kind: the interval [node_h[i], node_h[i+1]) holding h (the first
 * interval below the first node) and its exponential rate k = d ln(n-1)/dh. */
static int orc_node_interval(const orc_atm* a, double h, double* k)
{
    int i = 0;
    while (i + 2 < a->n_nodes && h >= a->node_h[i + 1]) ++i;
    *k = log(a->node_d[i + 1] / a->node_d[i]) / (a->node_h[i + 1] - a->node_h[i]);
    return i;
}

static double orc_table_delta(const orc_atm* a, double h)
{
    if (h >= a->node_h[a->n_nodes - 1]) return 0.0;
    double k;
    int i = orc_node_interval(a, h, &k);
    return a->node_d[i] * exp(k * (h - a->node_h[i]));
}

/* Table kind: integral of n - 1 over [lo, hi] below the top, interval by interval. */
static double orc_table_delta_integral(const orc_atm* a, double lo, double hi)
{
    double top = a->node_h[a->n_nodes - 1], sum = 0.0;
    if (hi > top) hi = top;
    for (int i = 0; i + 1 < a->n_nodes; ++i) {
        double l0 = (i == 0) ? -1e30 : a->node_h[i];
        double l1 = a->node_h[i + 1];
        double p = fmax(lo, l0), q = fmin(hi, l1);
        if (q <= p) continue;
        double k = log(a->node_d[i + 1] / a->node_d[i]) / (a->node_h[i + 1] - a->node_h[i]);
        double ep = exp(k * (p - a->node_h[i])), eq = exp(k * (q - a->node_h[i]));
        sum += (k != 0.0) ? a->node_d[i] * (eq - ep) / k : a->node_d[i] * (q - p);
    }
    return sum;
}

static int orc_layer_of(const orc_atm* a, double h)
{
    int i = 0;
    while (i + 1 < a->n_layers && h >= a->layer_h[i + 1]) ++i;   /* half-open [h_i, h_i+1) */
    return i;
}

/* Vertical column depth above h [g/cm^2]. */
double orc_atm_T(const orc_atm* a, double h)
{
    if (a->kind == ORC_ATM_TABLE)
        return 100.0 * a->rho_ref / a->kappa * orc_table_delta_integral(a, h, a->node_h[a->n_nodes - 1]);
    if (a->kind != ORC_ATM_LAYERED) return 0.0;
    if (h >= a->h_top) return 0.0;
    int i = orc_layer_of(a, h);
    double hc = h * 100.0;
    if (a->last_linear && i == a->n_layers - 1) return a->a[i] - a->b[i] * hc / a->c[i];
    return a->a[i] + a->b[i] * exp(-hc / a->c[i]);
}

/* Density rho = -dT/dh [g/cm^3]. */
double orc_atm_rho(const orc_atm* a, double h)
{
    if (a->kind == ORC_ATM_TABLE) return a->rho_ref * orc_table_delta(a, h) / a->kappa;
    if (a->kind != ORC_ATM_LAYERED) return 0.0;
    if (h >= a->h_top) return 0.0;
    int i = orc_layer_of(a, h);
    if (a->last_linear && i == a->n_layers - 1) return a->b[i] / a->c[i];
    return a->b[i] / a->c[i] * exp(-h * 100.0 / a->c[i]);
}

/* Layer i's own column law evaluated at h (no layer lookup). */
static double orc_T_layer(const orc_atm* a, int i, double h)
{
    double hc = h * 100.0;
    if (a->last_linear && i == a->n_layers - 1) return a->a[i] - a->b[i] * hc / a->c[i];
    return a->a[i] + a->b[i] * exp(-hc / a->c[i]);
}

/* Vertical column between lo < hi, i.e. the integral of rho: the sum over
 * layers of each layer's column law differenced at its clipped ends (the
 * piecewise fit is continuous only to about 1e-3 g/cm^2 at the boundaries). */
double orc_column(const orc_atm* a, double lo, double hi)
{
    if (a->kind == ORC_ATM_TABLE) return 100.0 * a->rho_ref / a->kappa * orc_table_delta_integral(a, lo, hi);
    if (a->kind != ORC_ATM_LAYERED) return 0.0;
    double X = 0.0;
    for (int i = 0; i < a->n_layers; ++i) {
        double l0 = (i == 0) ? -1e30 : a->layer_h[i];
        double l1 = (i + 1 < a->n_layers) ? a->layer_h[i + 1] : a->h_top;
        double p = fmax(lo, l0), q = fmin(hi, l1);
        if (q > p) X += orc_T_layer(a, i, p) - orc_T_layer(a, i, q);
    }
    return X;
}

static double orc_rho0(const orc_atm* a) { return a->b[0] / a->c[0]; }   /* rho at h = 0 */

/* Reduced refractive index n(h) - 1. */
double orc_atm_delta(const orc_atm* a, double h)
{
    switch (a->kind) {
    case ORC_ATM_LAYERED:
        return a->kappa * orc_atm_rho(a, h) / orc_rho0(a);
    case ORC_ATM_TABLE:
        return orc_table_delta(a, h);
    case ORC_ATM_LINEAR: {
        if (h >= a->lin_h1) return a->lin_n1 - 1.0;
        double f = (h - a->lin_h0) / (a->lin_h1 - a->lin_h0);
        return (a->lin_n0 - 1.0) - f * (a->lin_n0 - a->lin_n1);
    }
    default:
        return a->hom_delta;
    }
}

static double orc_n(const orc_atm* a, double h) { return 1.0 + orc_atm_delta(a, h); }

/* Heights in (lo, hi) where n(h) is not smooth; returns their count. */
static int orc_breakpoints(const orc_atm* a, double lo, double hi, double* bp)
{
    int m = 0;
    if (a->kind == ORC_ATM_LAYERED) {
        for (int i = 1; i < a->n_layers; ++i)
            if (a->layer_h[i] > lo && a->layer_h[i] < hi) bp[m++] = a->layer_h[i];
        if (a->h_top > lo && a->h_top < hi) bp[m++] = a->h_top;
    } else if (a->kind == ORC_ATM_LINEAR) {
        if (a->lin_h1 > lo && a->lin_h1 < hi) bp[m++] = a->lin_h1;
    } else if (a->kind == ORC_ATM_TABLE) {
        for (int i = 1; i < a->n_nodes; ++i)
            if (a->node_h[i] > lo && a->node_h[i] < hi) bp[m++] = a->node_h[i];
    }
    return m;
}

/* ------------------------------------------------------------------ */
/* Adaptive Gauss-Legendre quadrature.                                */
/* ------------------------------------------------------------------ */
#define ORC_GL_N 10
static double g_gl_x[ORC_GL_N], g_gl_w[ORC_GL_N];
static int g_gl_ready = 0;

/* Nodes and weights of the n-point Gauss-Legendre rule by Newton iteration
 * on the Legendre polynomial P_n (three-term recurrence). */
void orc_gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));   /* initial guess for root i */
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p_prev = 1.0, p = z;                     /* P_0, P_1 */
            for (int k = 2; k <= n; ++k) {
                double p_next = ((2.0 * k - 1.0) * z * p - (k - 1.0) * p_prev) / k;
                p_prev = p; p = p_next;
            }
            dp = n * (z * p - p_prev) / (z * z - 1.0);      /* P_n'(z) */
            double dz = p / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static void orc_gl_init(void)
{
    if (!g_gl_ready) {
        orc_gauss_legendre(ORC_GL_N, g_gl_x, g_gl_w);
        g_gl_ready = 1;
    }
}

/* Fill the rule once at load time so concurrent callers only read it. */
__attribute__((constructor)) static void orc_load(void) { orc_gl_init(); }

typedef double (*orc_fn)(double h, const void* ctx);

static double orc_gl(orc_fn f, const void* ctx, double lo, double hi)
{
    double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo), s = 0.0;
    for (int i = 0; i < ORC_GL_N; ++i) s += g_gl_w[i] * f(mid + half * g_gl_x[i], ctx);
    return s * half;
}

static double orc_adapt(orc_fn f, const void* ctx, double lo, double hi, double whole,
                        double rtol, int depth)
{
    double mid = 0.5 * (lo + hi);
    double left = orc_gl(f, ctx, lo, mid), right = orc_gl(f, ctx, mid, hi);
    double both = left + right;
    if (!isfinite(both)) return both;   /* a path that never reaches the lower limit: no refinement helps */
    if (depth >= 40 || fabs(both - whole) <= rtol * fabs(both) + 1e-300) return both;
    return orc_adapt(f, ctx, lo, mid, left, rtol, depth + 1) +
           orc_adapt(f, ctx, mid, hi, right, rtol, depth + 1);
}

/* Integral of f over [lo, hi], split at the atmosphere's breakpoints. */
static double orc_integrate(const orc_atm* a, orc_fn f, const void* ctx, double lo, double hi,
                            double rtol)
{
    orc_gl_init();
    double bp[ORC_MAX_NODES + 16];
    int m = orc_breakpoints(a, lo, hi, bp);
    double edges[ORC_MAX_NODES + 18];
    edges[0] = lo;
    for (int i = 0; i < m; ++i) edges[i + 1] = bp[i];
    edges[m + 1] = hi;
    double total = 0.0;
    for (int i = 0; i <= m; ++i) {
        double piece_lo = edges[i], piece_hi = edges[i + 1];
        if (piece_hi <= piece_lo) continue;
        /* Start from a few equal sub-intervals so a single rule never spans
         * many scale heights. */
        int nsub = 1 + (int)((piece_hi - piece_lo) / 2000.0);
        double step = (piece_hi - piece_lo) / nsub;
        for (int j = 0; j < nsub; ++j) {
            double s0 = piece_lo + j * step, s1 = (j + 1 == nsub) ? piece_hi : s0 + step;
            total += orc_adapt(f, ctx, s0, s1, orc_gl(f, ctx, s0, s1), rtol, 0);
        }
    }
    return total;
}

/* ------------------------------------------------------------------ */
/* Exact planar refraction integrals (Eq. 3.17-3.18).                 */
/*                                                                    */
/* With the invariant n(h) sin(theta(h)) = s = n(h_e) sin(theta0), a  */
/* photon that descends dh moves horizontally by s / sqrt(n^2 - s^2)  */
/* dh and spends n^2 / (c sqrt(n^2 - s^2)) dh of time (path length    */
/* n / sqrt(n^2 - s^2) dh at speed c / n).                            */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_atm* atm;
    double s;      /* Snell invariant */
    double H_A;    /* aerosol scale height [m] */
} orc_rctx;

static double orc_q(const orc_rctx* r, double h, double* n_out)
{
    double n = orc_n(r->atm, h);
    *n_out = n;
    return sqrt(n * n - r->s * r->s);
}
static double orc_fR(double h, const void* p)
{
    const orc_rctx* r = (const orc_rctx*)p; double n; double q = orc_q(r, h, &n);
    return r->s / q;
}
static double orc_fT(double h, const void* p)
{
    const orc_rctx* r = (const orc_rctx*)p; double n; double q = orc_q(r, h, &n);
    return n * n / q / ORC_C_LIGHT;
}
static double orc_fX(double h, const void* p)
{
    const orc_rctx* r = (const orc_rctx*)p; double n; double q = orc_q(r, h, &n);
    return 100.0 * orc_atm_rho(r->atm, h) * n / q;     /* dh in cm -> g/cm^2 */
}
static double orc_fA(double h, const void* p)
{
    const orc_rctx* r = (const orc_rctx*)p; double n; double q = orc_q(r, h, &n);
    return exp(-h / r->H_A) * n / q;
}

/* out = {R [m], t_path [s], X_slant [g/cm^2], A_slant [m]} for a photon
 * emitted at h_e with zenith theta0 that descends to h_obs. */
void orc_refract_quad(const orc_atm* a, double h_obs, double h_e, double theta0, double H_A,
                      double rtol, double out[4])
{
    orc_rctx r = { a, orc_n(a, h_e) * sin(theta0), H_A };
    out[0] = orc_integrate(a, orc_fR, &r, h_obs, h_e, rtol);
    out[1] = orc_integrate(a, orc_fT, &r, h_obs, h_e, rtol);
    out[2] = orc_integrate(a, orc_fX, &r, h_obs, h_e, rtol);
    out[3] = orc_integrate(a, orc_fA, &r, h_obs, h_e, rtol);
}

/* Straight-line propagation (Sec. 3.4.1, Eq. 3.3): same outputs with the
 * atmosphere neglected for the geometry and the time (vacuum light speed);
 * the column integrals follow the straight path. */
void orc_straight(const orc_atm* a, double h_obs, double h_e, double theta0, double H_A,
                  double out[4])
{
    double cz = cos(theta0), dz = h_e - h_obs;
    out[0] = dz * tan(theta0);
    out[1] = dz / cz / ORC_C_LIGHT;
    out[2] = orc_column(a, h_obs, h_e) / cz;
    out[3] = H_A * (exp(-h_obs / H_A) - exp(-h_e / H_A)) / cz;
}

/* ------------------------------------------------------------------ */
/* Second, independent path: the same integrals in closed form.       */
/*                                                                    */
/* Exponential layer n = 1 + D exp(-h/H): dh = -H dn / (n - 1), and   */
/*   int dn / ((n-1) q)  = -(1/k) ln[(n - s^2 + k q) / (n - 1)],       */
/*   int n dn / q        = q,                                          */
/*   int dn / q          = ln(n + q),                                  */
/* with q = sqrt(n^2 - s^2), k = sqrt(1 - s^2).  In such a layer       */
/* rho = (n - 1) rho0 / kappa, so the column integral is H (rho0 /     */
/* kappa) [q].  Constant-n layers are straight lines.  The linear kind */
/* (dn/dh = -c1) integrates to arcosh forms (Eq. 3.20-3.23, App. A.1). */
/* ------------------------------------------------------------------ */
static double orc_F(double n, double s)
{
    double k = sqrt(1.0 - s * s), q = sqrt(n * n - s * s);
    return -log((n - s * s + k * q) / (n - 1.0)) / k;
}

/* out = {R, t_path, X_slant}; aerosol has no closed form in general. */
int orc_refract_closed(const orc_atm* a, double h_obs, double h_e, double theta0, double out[3])
{
    double s = orc_n(a, h_e) * sin(theta0);
    double R = 0.0, T = 0.0, X = 0.0;
    if (a->kind == ORC_ATM_HOMOGENEOUS) {
        double n = 1.0 + a->hom_delta, q = sqrt(n * n - s * s), dz = h_e - h_obs;
        out[0] = dz * s / q; out[1] = dz * n * n / q / ORC_C_LIGHT; out[2] = 0.0;
        return 0;
    }
    if (a->kind == ORC_ATM_LINEAR) {
        if (h_e > a->lin_h1) return -1;
        double c1 = (a->lin_n0 - a->lin_n1) / (a->lin_h1 - a->lin_h0);
        double n_lo = orc_n(a, h_obs), n_hi = orc_n(a, h_e);
        double q_lo = sqrt(n_lo * n_lo - s * s), q_hi = sqrt(n_hi * n_hi - s * s);
        out[0] = s / c1 * (acosh(n_lo / s) - acosh(n_hi / s));
        double G_lo = 0.5 * (n_lo * q_lo + s * s * log(n_lo + q_lo));
        double G_hi = 0.5 * (n_hi * q_hi + s * s * log(n_hi + q_hi));
        out[1] = (G_lo - G_hi) / (c1 * ORC_C_LIGHT);
        out[2] = 0.0;
        return 0;
    }
    if (a->kind == ORC_ATM_TABLE) {
        /* each interval is an exponential layer with its own scale height */
        double top = a->node_h[a->n_nodes - 1];
        if (h_e >= top) return -1;
        for (int i = 0; i + 1 < a->n_nodes; ++i) {
            double lo = (i == 0) ? h_obs : fmax(h_obs, a->node_h[i]);
            double hi = fmin(h_e, a->node_h[i + 1]);
            if (hi <= lo) continue;
            double k = log(a->node_d[i + 1] / a->node_d[i]) / (a->node_h[i + 1] - a->node_h[i]);
            double n_lo = 1.0 + a->node_d[i] * exp(k * (lo - a->node_h[i]));
            double n_hi = 1.0 + a->node_d[i] * exp(k * (hi - a->node_h[i]));
            double q_lo = sqrt(n_lo * n_lo - s * s), q_hi = sqrt(n_hi * n_hi - s * s);
            if (k == 0.0) {   /* constant n: a straight line */
                R += (hi - lo) * s / q_lo;
                T += (hi - lo) * n_lo * n_lo / q_lo / ORC_C_LIGHT;
                X += 100.0 * a->rho_ref / a->kappa * (n_lo - 1.0) * (hi - lo) * n_lo / q_lo;
                continue;
            }
            double H = -1.0 / k;
            double F_lo = orc_F(n_lo, s), F_hi = orc_F(n_hi, s);
            R += H * s * (F_lo - F_hi);
            T += H / ORC_C_LIGHT * ((q_lo - q_hi) + (log(n_lo + q_lo) - log(n_hi + q_hi)) + (F_lo - F_hi));
            X += 100.0 * H * (a->rho_ref / a->kappa) * (q_lo - q_hi);
        }
        out[0] = R; out[1] = T; out[2] = X;
        return 0;
    }
    /* layered */
    double rho0 = orc_rho0(a);
    for (int i = 0; i < a->n_layers; ++i) {
        double lo = a->layer_h[i];
        double hi = (i + 1 < a->n_layers) ? a->layer_h[i + 1] : a->h_top;
        if (lo < h_obs) lo = h_obs;
        if (hi > h_e) hi = h_e;
        if (hi <= lo) continue;
        if (a->last_linear && i == a->n_layers - 1) {
            double rho = a->b[i] / a->c[i];
            double n = 1.0 + a->kappa * rho / rho0, q = sqrt(n * n - s * s);
            R += (hi - lo) * s / q;
            T += (hi - lo) * n * n / q / ORC_C_LIGHT;
            X += 100.0 * rho * (hi - lo) * n / q;
            continue;
        }
        double H = a->c[i] / 100.0;                     /* scale height [m] */
        double D = a->kappa * (a->b[i] / a->c[i]) / rho0; /* n - 1 at h = 0 of this layer's law */
        double n_lo = 1.0 + D * exp(-lo / H), n_hi = 1.0 + D * exp(-hi / H);
        double q_lo = sqrt(n_lo * n_lo - s * s), q_hi = sqrt(n_hi * n_hi - s * s);
        double F_lo = orc_F(n_lo, s), F_hi = orc_F(n_hi, s);
        /* int_lo^hi f(h) dh = H int_{n_hi}^{n_lo} f / (n - 1) dn */
        R += H * s * (F_lo - F_hi);
        T += H / ORC_C_LIGHT * ((q_lo - q_hi) + (log(n_lo + q_lo) - log(n_hi + q_hi)) + (F_lo - F_hi));
        X += 100.0 * H * (rho0 / a->kappa) * (q_lo - q_hi);
    }
    out[0] = R; out[1] = T; out[2] = X;
    return 0;
}

/* ------------------------------------------------------------------ */
/* The thesis's numerical tracer: Snell's law in vector form at the   */
/* boundaries of homogeneous slabs (Eq. 3.15).  The height range is   */
/* cut into the fewest equal slabs no thicker than dh; slab j holds   */
/* the index at its middle height; the photon crosses it straight and */
/* refracts at its lower boundary.                                    */
/* out = {R, t_path, X_slant [g/cm^2], A_slant [m]}.                  */
/* ------------------------------------------------------------------ */
void orc_snell_path(const orc_atm* a, double h_obs, double h_e, double theta0, double dh, double H_A,
                    double out[4])
{
    /* 2-D: direction (horizontal, vertical); N = (0, -1) is the downward normal */
    double dir_x = sin(theta0), dir_z = -cos(theta0);
    double x = 0.0, t = 0.0, X = 0.0, A = 0.0;
    int nsteps = (int)ceil((h_e - h_obs) / dh - 1e-9);
    if (nsteps < 1) nsteps = 1;
    double step = (h_e - h_obs) / nsteps;
    double n1 = orc_n(a, h_e - 0.5 * step);
    for (int j = 0; j < nsteps; ++j) {
        /* straight through slab j with index n1 */
        const double h_mid = h_e - (j + 0.5) * step;
        double path = step / (-dir_z);
        x += path * dir_x;
        t += path * n1 / ORC_C_LIGHT;
        X += 100.0 * orc_atm_rho(a, h_mid) * path;
        A += exp(-h_mid / H_A) * path;
        if (j + 1 == nsteps) break;
        double n2 = orc_n(a, h_mid - step);
        /* optical vectors A' = n A; A2' = A1' + (sqrt(n2^2 - n1^2 + n1^2 cos^2 a1) - n1 cos a1) N */
        double cos_a1 = -dir_z;                       /* A1 . N with N = (0, -1) */
        double c = sqrt(n2 * n2 - n1 * n1 + n1 * n1 * cos_a1 * cos_a1) - n1 * cos_a1;
        double Ax = n1 * dir_x, Az = n1 * dir_z - c;  /* + c N = (0, -c) */
        dir_x = Ax / n2; dir_z = Az / n2;
        n1 = n2;
    }
    out[0] = x; out[1] = t; out[2] = X; out[3] = A;
}

/* The same stepper on the spherical shell: shells of equal thickness <= dh in
 * altitude, each holding n at its middle altitude; inside a shell the photon
 * runs straight to the next inner sphere, where Eq. 3.15 refracts it about the
 * radial normal.  Worked in the plane of travel: p = (x, y) with the Earth's
 * centre at the origin and the emission point at (0, R + h_e); direction at
 * local zenith psi0 towards +x.  out = {central angle, t_path, X_slant, A_slant}. */
void orc_snell_path_sph(const orc_atm* a, double R, double h_obs, double h_e, double psi0, double dh, double H_A,
                        double out[4])
{
    double px = 0.0, py = R + h_e;
    double dx = sin(psi0), dy = -cos(psi0);
    double t = 0.0, X = 0.0, A = 0.0;
    int nsteps = (int)ceil((h_e - h_obs) / dh - 1e-9);
    if (nsteps < 1) nsteps = 1;
    const double step = (h_e - h_obs) / nsteps;
    double n1 = orc_n(a, h_e - 0.5 * step);
    for (int j = 0; j < nsteps; ++j) {
        const double h_mid = h_e - (j + 0.5) * step;
        const double r_in = R + h_e - (j + 1) * step;
        /* first crossing of |p + s d| = r_in: s^2 + 2 (p.d) s + |p|^2 - r_in^2 = 0 */
        const double pd = px * dx + py * dy, c = px * px + py * py - r_in * r_in;
        const double disc = pd * pd - c;
        const double sq = sqrt(fmax(disc, 0.0));
        const double sl = c / (-pd + sq);           /* the smaller root, without cancellation */
        px += sl * dx; py += sl * dy;
        t += sl * n1 / ORC_C_LIGHT;
        X += 100.0 * orc_atm_rho(a, h_mid) * sl;
        A += exp(-h_mid / H_A) * sl;
        if (j + 1 == nsteps) break;
        const double n2 = orc_n(a, h_mid - step);
        /* Eq. 3.15 with N the inward normal at the crossing */
        const double r = sqrt(px * px + py * py), Nx = -px / r, Ny = -py / r;
        const double cos_a1 = dx * Nx + dy * Ny;
        const double cc = sqrt(n2 * n2 - n1 * n1 + n1 * n1 * cos_a1 * cos_a1) - n1 * cos_a1;
        const double Ax = n1 * dx + cc * Nx, Ay = n1 * dy + cc * Ny;
        dx = Ax / n2; dy = Ay / n2;
        n1 = n2;
    }
    out[0] = atan2(px, py); out[1] = t; out[2] = X; out[3] = A;
}

/* {R, t_path} of the stepper (the pins' entry point). */
void orc_snell_stepper(const orc_atm* a, double h_obs, double h_e, double theta0, double dh,
                       double out[2])
{
    double o4[4];
    orc_snell_path(a, h_obs, h_e, theta0, dh, 1200.0, o4);
    out[0] = o4[0]; out[1] = o4[1];
}

/* ------------------------------------------------------------------ */
/* Spherical-shell atmosphere (Sec. 3.3.4): n depends on the altitude */
/* h = r - R_E only, and Bouguer's law n(r) r sin(psi) = K holds      */
/* along the path (the spherical form of Eq. 3.17).  A photon that    */
/* descends from r_e to the ground sphere r_g sweeps the central      */
/* angle  int K / (r sqrt(n^2 r^2 - K^2)) dr  and spends              */
/* int n^2 r / (c sqrt(n^2 r^2 - K^2)) dr  of time.                   */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_atm* atm;
    double K, R, H_A;
} orc_sctx;

static double orc_sq(const orc_sctx* c, double h, double* n_out, double* r_out)
{
    double n = orc_n(c->atm, h), r = c->R + h;
    *n_out = n; *r_out = r;
    return sqrt(n * n * r * r - c->K * c->K);
}
static double orc_sPhi(double h, const void* p)
{
    const orc_sctx* c = (const orc_sctx*)p; double n, r; double q = orc_sq(c, h, &n, &r);
    return c->K / (r * q);
}
static double orc_sT(double h, const void* p)
{
    const orc_sctx* c = (const orc_sctx*)p; double n, r; double q = orc_sq(c, h, &n, &r);
    return n * n * r / q / ORC_C_LIGHT;
}
static double orc_sX(double h, const void* p)
{
    const orc_sctx* c = (const orc_sctx*)p; double n, r; double q = orc_sq(c, h, &n, &r);
    return 100.0 * orc_atm_rho(c->atm, h) * n * r / q;
}
static double orc_sA(double h, const void* p)
{
    const orc_sctx* c = (const orc_sctx*)p; double n, r; double q = orc_sq(c, h, &n, &r);
    return exp(-h / c->H_A) * n * r / q;
}

static double orc_sX_straight(double h, const void* p)
{
    const orc_sctx* c = (const orc_sctx*)p; double r = c->R + h;
    return 100.0 * orc_atm_rho(c->atm, h) * r / sqrt(r * r - c->K * c->K);
}
static double orc_sA_straight(double h, const void* p)
{
    const orc_sctx* c = (const orc_sctx*)p; double r = c->R + h;
    return exp(-h / c->H_A) * r / sqrt(r * r - c->K * c->K);
}

/* out = {central angle Phi [rad], t_path [s], X_slant [g/cm^2], A_slant [m]}
 * for a photon at altitude h_e with local zenith psi0 descending to h_obs;
 * refraction = 0 gives the vacuum straight line (n = 1 for the geometry and
 * the time, the columns along that line). */
void orc_sph_path(const orc_atm* a, double R, double h_obs, double h_e, double psi0, double H_A, int refraction,
                  double rtol, double out[4])
{
    double n_e = refraction ? orc_n(a, h_e) : 1.0;
    orc_sctx c = { a, n_e * (R + h_e) * sin(psi0), R, H_A };
    if (refraction) {
        out[0] = orc_integrate(a, orc_sPhi, &c, h_obs, h_e, rtol);
        out[1] = orc_integrate(a, orc_sT, &c, h_obs, h_e, rtol);
        out[2] = orc_integrate(a, orc_sX, &c, h_obs, h_e, rtol);
        out[3] = orc_integrate(a, orc_sA, &c, h_obs, h_e, rtol);
    } else {
        /* straight line: r(s)^2 = r_e^2 - 2 r_e cos(psi0) s + s^2 meets r_g */
        double re = R + h_e, rg = R + h_obs, K = re * sin(psi0);
        double len = sqrt(re * re - K * K) - sqrt(rg * rg - K * K);
        out[0] = asin(K / rg) - asin(K / re);
        out[1] = len / ORC_C_LIGHT;
        /* columns along the straight line (n = 1 in the geometry) */
        orc_sctx v = { a, K, R, H_A };
        out[2] = orc_integrate(a, orc_sX_straight, &v, h_obs, h_e, rtol);
        out[3] = orc_integrate(a, orc_sA_straight, &v, h_obs, h_e, rtol);
    }
}

/* Azimuthal-equidistant coordinates about the array centre (the point of the
 * ground sphere above the Earth's centre) of a point G (frame coordinates,
 * Earth centre at (0, 0, -R)); rg = R + h_obs. */
static void orc_ae(double R, double rg, const double G[3], double* x, double* y)
{
    double rho = sqrt(G[0] * G[0] + G[1] * G[1]);
    double alpha = atan2(rho, G[2] + R);
    if (rho > 0.0) { *x = rg * alpha * G[0] / rho; *y = rg * alpha * G[1] / rho; }
    else { *x = 0.0; *y = 0.0; }
}

/* Frame coordinates of the point at altitude h_obs + dz above AE (x, y). */
void orc_ae_inverse(double R, double h_obs, double x, double y, double dz, double out[3])
{
    double rg = R + h_obs, s = sqrt(x * x + y * y), alpha = s / rg, r = rg + dz;
    double cx = s > 0.0 ? x / s : 1.0, cy = s > 0.0 ? y / s : 0.0;
    out[0] = r * sin(alpha) * cx;
    out[1] = r * sin(alpha) * cy;
    out[2] = r * cos(alpha) - R;
}

/* ------------------------------------------------------------------ */
/* Cylindrical atmosphere (Sec. 3.3.3).  The model adds to the         */
/* altitude the horizontal distance d of the emission point E from the */
/* array centre: the index gradient leans from the vertical by the     */
/* angle chi_E, tan(chi_E) = d / (R + z_E), inside the vertical plane   */
/* through the centre and E, and keeps that plane's azimuth along the  */
/* whole path.  Reading: n depends on the distance rho from the        */
/* horizontal axis through the Earth's centre normal to that plane     */
/* (altitude rho - R), i.e. the atmosphere is a set of coaxial         */
/* cylinders chosen per photon.  With e_r the horizontal unit from the */
/* centre towards E's foot (the x axis when d = 0) and e_a = z x e_r   */
/* along the axis, two invariants follow from the symmetry:            */
/*   n u_a = A            (translation along the axis),               */
/*   n rho u_chi = L      (rotation about it),                         */
/* u_chi the component along the transverse tangent e_chi.  The path's */
/* projection on the transverse plane is the ray of the planar index   */
/* N = sqrt(n^2 - A^2) with Bouguer's N rho sin(psi) = L, and per      */
/* unit of altitude it sweeps   dchi = L / (rho q),                     */
/* runs the length   ds = n rho / q   and drifts   da = A rho / q       */
/* along the axis, q = sqrt(N^2 rho^2 - L^2).  The ground is the       */
/* cylinder rho = R + h_obs, unrolled onto the plane of the array: its */
/* point (chi, a) has the coordinates (R + h_obs) chi e_r + a e_a, and */
/* a direction keeps its components along the unrolled e_chi, e_a and  */
/* the normal.  With u_a = 0 the photon stays in the plane through the */
/* Earth's centre and the model is the spherical shell's.              */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_atm* atm;
    double A, L, R, H_A;       /* L >= 0 */
    int refraction;            /* 0: n = 1 in the geometry (the straight line) */
} orc_cctx;

static double orc_cq(const orc_cctx* c, double h, double* n_out, double* r_out)
{
    double n = c->refraction ? orc_n(c->atm, h) : 1.0, r = c->R + h;
    *n_out = n; *r_out = r;
    return sqrt((n * n - c->A * c->A) * r * r - c->L * c->L);
}
static double orc_cChi(double h, const void* p)
{
    const orc_cctx* c = (const orc_cctx*)p; double n, r; double q = orc_cq(c, h, &n, &r);
    return c->L / (r * q);
}
static double orc_cT(double h, const void* p)
{
    const orc_cctx* c = (const orc_cctx*)p; double n, r; double q = orc_cq(c, h, &n, &r);
    return n * n * r / q / ORC_C_LIGHT;
}
static double orc_cAx(double h, const void* p)
{
    const orc_cctx* c = (const orc_cctx*)p; double n, r; double q = orc_cq(c, h, &n, &r);
    return c->A * r / q;
}
static double orc_cX(double h, const void* p)
{
    const orc_cctx* c = (const orc_cctx*)p; double n, r; double q = orc_cq(c, h, &n, &r);
    return 100.0 * orc_atm_rho(c->atm, h) * n * r / q;
}
static double orc_cAer(double h, const void* p)
{
    const orc_cctx* c = (const orc_cctx*)p; double n, r; double q = orc_cq(c, h, &n, &r);
    return exp(-h / c->H_A) * n * r / q;
}

/* out = {chi swept [rad], t_path [s], axial drift [m], X_slant [g/cm^2], A_slant [m]}
 * for a photon at altitude h_e whose direction has the component u_a along the
 * axis and u_chi >= 0 along the transverse tangent (the rest points down the
 * radius); refraction = 0 gives the vacuum straight line. */
void orc_cyl_path(const orc_atm* a, double R, double h_obs, double h_e, double u_a, double u_chi, double H_A,
                  int refraction, double rtol, double out[5])
{
    const double n_e = refraction ? orc_n(a, h_e) : 1.0;
    orc_cctx c = { a, n_e * u_a, n_e * (R + h_e) * u_chi, R, H_A, refraction };
    out[0] = orc_integrate(a, orc_cChi, &c, h_obs, h_e, rtol);
    out[1] = orc_integrate(a, orc_cT, &c, h_obs, h_e, rtol);
    out[2] = orc_integrate(a, orc_cAx, &c, h_obs, h_e, rtol);
    out[3] = orc_integrate(a, orc_cX, &c, h_obs, h_e, rtol);
    out[4] = orc_integrate(a, orc_cAer, &c, h_obs, h_e, rtol);
}

/* The Snell stepper (Sec. 3.4.2, Eq. 3.15) in the cylindrical atmosphere, in
 * three dimensions: shells between coaxial cylinders of equal thickness
 * <= dh in altitude, each holding n at its middle altitude; inside a shell
 * the photon runs straight to the next inner cylinder, where Eq. 3.15
 * refracts it about the inward normal (towards the axis, no axial part).
 * Coordinates: transverse (x, y) with the axis at the origin and E at
 * (0, R + h_e), axial a; direction (u_chi, u_rho, u_a), u_rho < 0.
 * out = {chi swept, t_path, axial drift, X_slant, A_slant}. */
void orc_snell_path_cyl(const orc_atm* a, double R, double h_obs, double h_e, double u_chi, double u_rho,
                        double u_a, double dh, double H_A, int refraction, double out[5])
{
    double px = 0.0, py = R + h_e, pa = 0.0;
    double dx = u_chi, dy = u_rho, da = u_a;
    double t = 0.0, X = 0.0, A = 0.0;
    int nsteps = (int)ceil((h_e - h_obs) / dh - 1e-9);
    if (nsteps < 1) nsteps = 1;
    const double step = (h_e - h_obs) / nsteps;
    double n1 = refraction ? orc_n(a, h_e - 0.5 * step) : 1.0;
    for (int j = 0; j < nsteps; ++j) {
        const double h_mid = h_e - (j + 0.5) * step;
        const double r_in = R + h_e - (j + 1) * step;
        /* first crossing of |(px, py) + s (dx, dy)| = r_in */
        const double tt = dx * dx + dy * dy, pd = px * dx + py * dy, c = px * px + py * py - r_in * r_in;
        const double disc = pd * pd - tt * c;
        const double sl = c / (-pd + sqrt(fmax(disc, 0.0)));   /* the smaller root, without cancellation */
        px += sl * dx; py += sl * dy; pa += sl * da;
        t += sl * n1 / ORC_C_LIGHT;
        X += 100.0 * orc_atm_rho(a, h_mid) * sl;
        A += exp(-h_mid / H_A) * sl;
        if (j + 1 == nsteps) break;
        const double n2 = refraction ? orc_n(a, h_mid - step) : 1.0;
        const double r = sqrt(px * px + py * py), Nx = -px / r, Ny = -py / r;   /* inward normal */
        const double cos_a1 = dx * Nx + dy * Ny;
        const double cc = sqrt(n2 * n2 - n1 * n1 + n1 * n1 * cos_a1 * cos_a1) - n1 * cos_a1;
        dx = (n1 * dx + cc * Nx) / n2;
        dy = (n1 * dy + cc * Ny) / n2;
        da = n1 * da / n2;
        n1 = n2;
    }
    out[0] = atan2(px, py); out[1] = t; out[2] = pa; out[3] = X; out[4] = A;
}

/* Reach condition in the cylindrical atmosphere: the smallest value of
 * (N rho - L) / L over [h_obs, h_e], N = sqrt(n^2 - A^2) (n = 1 for the
 * straight line).  Within a piece between breakpoints phi = (n^2 - A^2) rho^2
 * has at most one turning point and it is a minimum only if phi' rises through
 * zero (on exponential pieces phi'/(2 rho) = n^2 - A^2 + n n' rho grows with
 * rho; on linear and constant ones it does not), so phi is unimodal there and a
 * golden-section search finds its smallest value, ends included.  Positive:
 * the path reaches the ground. */
static double orc_cyl_phi(const orc_atm* a, int refr, double R, double A, double h)
{
    const double n = refr ? orc_n(a, h) : 1.0, r = R + h;
    return (n * n - A * A) * r * r;
}
double orc_cyl_reach_margin(const orc_atm* a, int refr, double R, double h_obs, double h_e, double u_a, double u_chi)
{
    const double n_e = refr ? orc_n(a, h_e) : 1.0;
    const double A = n_e * u_a, L = n_e * (R + h_e) * fabs(u_chi);
    if (!(L > 0.0)) return 1.0;
    double edges[ORC_MAX_NODES + 18];
    int m = 0;
    edges[m++] = h_obs;
    double bp[ORC_MAX_NODES + 16];
    const int nb = refr ? orc_breakpoints(a, h_obs, h_e, bp) : 0;
    for (int i = 0; i < nb; ++i) edges[m++] = bp[i];
    edges[m++] = h_e;
    const double g = 0.5 * (sqrt(5.0) - 1.0);
    double best = 1e300;
    for (int p = 0; p + 1 < m; ++p) {
        /* the piece's interior, 1e-9 relative inside its ends (the one-sided limits) */
        double lo = edges[p], hi = edges[p + 1];
        const double eps = 1e-9 * fmax(1.0, fmax(fabs(lo), fabs(hi)));
        if (p > 0) lo += eps;
        hi -= eps;
        if (!(hi > lo)) continue;
        double v = fmin(orc_cyl_phi(a, refr, R, A, lo), orc_cyl_phi(a, refr, R, A, hi));
        double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
        double f1 = orc_cyl_phi(a, refr, R, A, x1), f2 = orc_cyl_phi(a, refr, R, A, x2);
        for (int it = 0; it < 200 && hi - lo > 1e-7; ++it) {
            if (f1 < f2) { hi = x2; x2 = x1; f2 = f1; x1 = hi - g * (hi - lo); f1 = orc_cyl_phi(a, refr, R, A, x1); }
            else { lo = x1; x1 = x2; f1 = f2; x2 = lo + g * (hi - lo); f2 = orc_cyl_phi(a, refr, R, A, x2); }
        }
        v = fmin(v, fmin(f1, f2));
        const double m_ = (sqrt(fmax(v, 0.0)) - L) / L;
        if (m_ < best) best = m_;
    }
    return best;
}

/* ------------------------------------------------------------------ */
/* Full photon generation and propagation.                            */
/* ------------------------------------------------------------------ */
typedef struct {               /* input segment, 64 bytes */
    double x0, y0, z0;         /* start point [m] */
    double t0;                 /* time at the start point [s] */
    float ux, uy, uz;          /* direction */
    float length;              /* [m] */
    float inv_gamma2;          /* 1 / gamma^2 */
    float charge;              /* z */
    uint32_t shower_id;
    uint32_t flags;
} orc_segment;

typedef struct {
    double h_obs;
    double lambda1, lambda2;   /* band [m] */
    double s_max;              /* sub-step length [m] */
    int bunch;
    int refraction;            /* 0: straight line, 1: exact planar refraction */
    int transmission;          /* 0: off, 1: Rayleigh + aerosol */
    double rayl_X0, rayl_lambda0;                 /* X_R(l) = X0 (l / l0)^4          */
    double aer_tau0, aer_lambda0, aer_alpha, aer_H; /* tau_A(l) = tau0 (l / l0)^-alpha */
    uint64_t seed;
    uint64_t seg_base;         /* global index of segs[0] */
    int n_showers;
    int hist_nx, hist_ny;
    int n_tel;
    double hist_x0, hist_y0, hist_dx, hist_dy;
    const double* tel;         /* n_tel x {x, y, z, r} */
    /* edge bands used only to flag photons for the parity comparison */
    double band_pos, band_count, band_T, band_h, band_w;
    double quad_rtol;
    int spherical;             /* 1: spherical-shell atmosphere, Earth centre at (0, 0, -earth_radius) */
    int cylindrical;           /* 1 (with spherical = 1): the cylindrical atmosphere of Sec. 3.3.3, ground
                                * and detector in the unrolled ground cylinder's coordinates */
    double earth_radius;
    /* LV1 particle filter (Sec. 4.3.2, 6.2.1): a segment whose start lies y above
     * h_obs and whose direction makes the angle x [deg] with the point of interest
     * is dropped, before any photon is generated, when y >= a x^b */
    int lv1_metric;            /* 0 off, 1 array centre, 2 disc of radius lv1_radius about it, 3 telescope spheres */
    int pad3;
    double lv1_a, lv1_b;
    double lv1_centre[3];
    double lv1_radius;
    double band_lv1;           /* relative band of y about a x^b flagged for the parity comparison */
    /* last-mile optics (Sec. 6.4): each telescope a parabolic mirror (diameter mirror_d,
     * focal length focal_f, vertex focal_f / 2 behind the sphere centre along the optical
     * axis pointing at (point_zenith, point_azimuth)), a flat camera disc of radius
     * camera_r at the focus that also shadows the mirror, cam_n x cam_n pixels */
    double mirror_d, focal_f, camera_r, point_zenith, point_azimuth;
    int cam_n;
    int pad4;
    /* LV3 photon pre-filter (Sec. 4.3.4, 6.2.2): before the refraction correction a
     * photon is dropped when its vacuum straight line lands farther than
     * lv3_radius + lv3_margin from lv3_centre (3-D distance in the frame) */
    int lv3;
    int pad5;
    double lv3_centre[3];
    double lv3_radius, lv3_margin;
    /* propagation method with refraction on: 0 the exact path (quadrature), 1 the Snell
     * vector stepper (Sec. 3.4.2, Eq. 3.15) through slabs no thicker than tracer_dh */
    int tracer;
    int pad6;
    double tracer_dh;
    /* emission (Sec. 2.2.2, 4.2.2): 0 Cherenkov; 1 fluorescence, isotropic; 2 fluorescence into
     * the downward half sphere with half the photons.  Fluorescence yield (Eq. 2.6) per metre:
     * z^2 fl_dedx [MeV cm^2/g] rho [g/cm^3] 100 sum_l fl_yield[l] [photons/MeV], lines fl_lines_nm */
    int emission;
    int fl_n_lines;
    double fl_lines_nm[8];
    double fl_yield[8];
    double fl_dedx;
    /* absorption in the last-mile optics (Sec. 6.4): a photon that reaches a camera pixel
     * survives the mirror's reflectivity R(lambda) and the camera's detection efficiency
     * eps(lambda) with probability R eps, each linear between eff_n nodes (eff_l [nm],
     * ascending; constant beyond the end nodes); eff_n = 0: no absorption.  The draw is
     * the Philox word x of counter (segment, sub-step, bunch index | 2^30). */
    int eff_n;
    int pad7;
    double eff_l[16], eff_R[16], eff_E[16];
} orc_config;

/* ORC_ST_NO_GROUND: a descending photon whose path never meets the observation level
 * (on the spherical shell it passes over the ground sphere and leaves the atmosphere;
 * in the plane, a profile whose index drops below the Snell invariant reflects it) */
enum { ORC_ST_LANDED = 0, ORC_ST_UPWARD = 1, ORC_ST_BELOW = 2, ORC_ST_NO_GROUND = 3,
       ORC_ST_ABSORBED = 4, ORC_ST_LV3 = 5, ORC_ST_SUBSTEP_FLAG = 15 };
/* ORC_FL_SEGMENT: the segment's sub-step count K = ceil(L / s_max) lies within rounding
 * of a whole number, so an FP32 evaluation may take the other count and every bunch of
 * the segment is undetermined; ORC_FL_GROUND: the photon lies within the band of the
 * condition that decides whether its path meets the observation level */
enum { ORC_FL_COUNT = 1, ORC_FL_ABSORB = 2, ORC_FL_HIST_EDGE = 4, ORC_FL_TEL_EDGE = 8,
       ORC_FL_GROUND = 16, ORC_FL_BELOW = 32, ORC_FL_UPWARD = 64, ORC_FL_LAYER = 128, ORC_FL_LV1 = 256,
       ORC_FL_LV3 = 512, ORC_FL_SEGMENT = 1024, ORC_FL_OPTICS = 2048 };

typedef struct {
    uint64_t seg;
    uint32_t k, i;
    double x, y;               /* ground position [m] (landed and absorbed photons) */
    double dt;                 /* arrival time minus segment t0 [s] */
    double lambda;             /* [m] */
    double ex, ey, h_e;        /* emission point [m] */
    double ux, uy, uz;         /* emission direction */
    double theta0, T, nbar;
    int32_t status, tel, bin;
    uint32_t flags;
    int32_t pix;               /* camera pixel iy * cam_n + ix, or -1 */
    int32_t pad;
} orc_record;

typedef struct {
    uint64_t* hist;            /* n_showers x ny x nx (photons) */
    uint64_t* tel_counts;      /* n_showers x n_tel (photons) */
    double* tel_time;          /* n_showers x n_tel: sum of photons x absolute arrival time [s] */
    uint64_t counters[8];      /* emitted, absorbed, hist, tel, missed_hist, missed_tel, upward, invalid_segments */
    orc_record* records;
    size_t capacity;
    size_t count;
    uint64_t lv1_dropped;      /* segments removed by the LV1 filter */
    uint64_t* camera;          /* n_showers x n_tel x cam_n x cam_n (photons), or NULL */
} orc_output;

static double orc_floor_dist(double v)     /* distance of v to the nearest integer */
{
    double f = v - floor(v);
    return f < 0.5 ? f : 1.0 - f;
}

static void orc_push(orc_output* o, const orc_record* r)
{
    if (o->records && o->count < o->capacity) o->records[o->count] = *r;
    o->count++;
}

static int orc_segment_valid(const orc_segment* s, int n_showers)
{
    if (!isfinite(s->x0) || !isfinite(s->y0) || !isfinite(s->z0) || !isfinite(s->t0)) return 0;
    if (!isfinite(s->ux) || !isfinite(s->uy) || !isfinite(s->uz)) return 0;
    if (!(s->length > 0.0f) || !isfinite(s->length)) return 0;
    if (!(s->inv_gamma2 > 0.0f) || !(s->inv_gamma2 < 1.0f)) return 0;
    if (!isfinite(s->charge)) return 0;
    if (!(s->uz < 0.99f)) return 0;              /* bisector rotation needs P != (0,0,1) */
    double n2 = (double)s->ux * s->ux + (double)s->uy * s->uy + (double)s->uz * s->uz;
    if (fabs(n2 - 1.0) > 1e-4) return 0;
    if ((int64_t)s->shower_id >= n_showers) return 0;
    return 1;
}

/* Last-mile ray tracing through one telescope (Sec. 6.4).  The photon line
 * G + t u (G on the ground, u its arrival direction) is followed in the
 * telescope's frame (e1, e2, a; origin the mirror vertex V = C - f/2 a): it
 * must cross the camera plane z' = f outside the camera disc (else the camera
 * shadows it), meet the paraboloid z' = (x'^2 + y'^2) / (4 f) inside the
 * aperture, reflect about the surface normal (x', y', -2 f) and reach the
 * camera plane inside the disc.  Returns the pixel iy * n + ix or -1; sets
 * *edge when a decision lies within `band` [m] of a rim or a pixel edge. */
static int orc_camera_pixel_xy(const orc_config* cfg, const double C[3], const double G[3], const double u[3],
                               double band, int* edge, double xy[2]);

static int orc_camera_pixel(const orc_config* cfg, const double C[3], const double G[3], const double u[3],
                            double band, int* edge)
{
    double xy[2];
    return orc_camera_pixel_xy(cfg, C, G, u, band, edge, xy);
}

/* For the pins: the pixel (or -1) and the camera-plane point of one ray. */
int orc_camera_trace(const orc_config* cfg, const double C[3], const double G[3], const double u[3], double xy[2])
{
    int edge = 0;
    return orc_camera_pixel_xy(cfg, C, G, u, 0.0, &edge, xy);
}

static int orc_camera_pixel_xy(const orc_config* cfg, const double C[3], const double G[3], const double u[3],
                               double band, int* edge, double xy[2])
{
    const double f = cfg->focal_f, R = cfg->camera_r, rd = 0.5 * cfg->mirror_d;
    const double th = cfg->point_zenith, ph = cfg->point_azimuth;
    const double a[3] = { sin(th) * cos(ph), sin(th) * sin(ph), cos(th) };
    double e1[3] = { a[1], -a[0], 0.0 };                 /* a x z-hat */
    double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1]);
    if (n1 < 1e-12) { e1[0] = 1.0; e1[1] = 0.0; } else { e1[0] /= n1; e1[1] /= n1; }
    const double e2[3] = { a[1] * e1[2] - a[2] * e1[1], a[2] * e1[0] - a[0] * e1[2], a[0] * e1[1] - a[1] * e1[0] };
    double q[3], p[3], d[3];
    for (int c = 0; c < 3; ++c) q[c] = G[c] - (C[c] - 0.5 * f * a[c]);
    p[0] = q[0] * e1[0] + q[1] * e1[1] + q[2] * e1[2];
    p[1] = q[0] * e2[0] + q[1] * e2[1] + q[2] * e2[2];
    p[2] = q[0] * a[0] + q[1] * a[1] + q[2] * a[2];
    d[0] = u[0] * e1[0] + u[1] * e1[1] + u[2] * e1[2];
    d[1] = u[0] * e2[0] + u[1] * e2[1] + u[2] * e2[2];
    d[2] = u[0] * a[0] + u[1] * a[1] + u[2] * a[2];
    if (!(d[2] < 0.0)) return -1;                        /* travelling away from the mirror */
    /* the camera's shadow */
    double tc = (f - p[2]) / d[2];
    double rc = hypot(p[0] + tc * d[0], p[1] + tc * d[1]);
    if (fabs(rc - R) < band) *edge = 1;
    if (rc < R) return -1;
    /* the mirror: F(t) = A t^2 + B t + Cq = r'^2 - 4 f z' is negative inside the
     * bowl; a ray travelling down leaves the bowl through the mirror at the
     * larger root (the smaller one is an entry through the wall far above) */
    double A = d[0] * d[0] + d[1] * d[1];
    double B = 2.0 * (p[0] * d[0] + p[1] * d[1]) - 4.0 * f * d[2];
    double Cq = p[0] * p[0] + p[1] * p[1] - 4.0 * f * p[2];
    double t;
    if (A < 1e-300) t = -Cq / B;
    else {
        double disc = B * B - 4.0 * A * Cq;
        if (disc < 0.0) return -1;
        double qq = -0.5 * (B + (B >= 0.0 ? sqrt(disc) : -sqrt(disc)));
        double t1 = qq / A, t2 = Cq / qq;
        t = fmax(t1, t2);
    }
    double m[3] = { p[0] + t * d[0], p[1] + t * d[1], p[2] + t * d[2] };
    double rm = hypot(m[0], m[1]);
    if (fabs(rm - rd) < band) *edge = 1;
    if (rm > rd) return -1;
    /* reflection */
    double N[3] = { m[0], m[1], -2.0 * f };
    double nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    for (int c = 0; c < 3; ++c) N[c] /= nn;
    double dn = d[0] * N[0] + d[1] * N[1] + d[2] * N[2];
    double r[3] = { d[0] - 2.0 * dn * N[0], d[1] - 2.0 * dn * N[1], d[2] - 2.0 * dn * N[2] };
    if (!(r[2] > 0.0)) return -1;
    double t2c = (f - m[2]) / r[2];
    double xq = m[0] + t2c * r[0], yq = m[1] + t2c * r[1];
    xy[0] = xq; xy[1] = yq;
    double rq = hypot(xq, yq);
    if (fabs(rq - R) < band) *edge = 1;
    if (rq > R) return -1;
    const int n = cfg->cam_n;
    double fx = (xq + R) / (2.0 * R) * n, fy = (yq + R) / (2.0 * R) * n;
    double pitch = 2.0 * R / n;
    if (orc_floor_dist(fx) * pitch < band || orc_floor_dist(fy) * pitch < band) *edge = 1;
    int ix = (int)floor(fx), iy = (int)floor(fy);
    ix = ix < 0 ? 0 : (ix >= n ? n - 1 : ix);
    iy = iy < 0 ? 0 : (iy >= n ? n - 1 : iy);
    return iy * n + ix;
}

/* Angle [deg] between the unit direction P and the direction from S towards a
 * sphere of radius r about C, less the sphere's angular radius (0 inside). */
static double orc_angle_to_sphere(const double S[3], const double P[3], const double C[3], double r)
{
    double d[3] = { C[0] - S[0], C[1] - S[1], C[2] - S[2] };
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(dn > r)) return 0.0;
    double c = (P[0] * d[0] + P[1] * d[1] + P[2] * d[2]) / dn;
    double a = acos(fmax(-1.0, fmin(1.0, c))) - asin(r / dn);
    return fmax(a, 0.0) * 180.0 / ORC_PI;
}

/* The LV1 cut parameter x [deg] of a segment starting at S with direction P. */
static double orc_lv1_x(const orc_config* cfg, const double S[3], const double P[3])
{
    if (cfg->lv1_metric == 1) return orc_angle_to_sphere(S, P, cfg->lv1_centre, 0.0);
    if (cfg->lv1_metric == 2) return orc_angle_to_sphere(S, P, cfg->lv1_centre, cfg->lv1_radius);
    double best = 180.0;
    for (int it = 0; it < cfg->n_tel; ++it) {
        const double* T4 = cfg->tel + 4 * it;
        double Tc[3] = { T4[0], T4[1], T4[2] };
        if (cfg->spherical) orc_ae_inverse(cfg->earth_radius, cfg->h_obs, T4[0], T4[1], T4[2] - cfg->h_obs, Tc);
        best = fmin(best, orc_angle_to_sphere(S, P, Tc, T4[3]));
    }
    return best;
}

/* Piecewise-linear curve through n nodes (x ascending), constant beyond the ends. */
static double orc_lerp_curve(const double* x, const double* y, int n, double v)
{
    if (v <= x[0]) return y[0];
    if (v >= x[n - 1]) return y[n - 1];
    int i = 0;
    while (v > x[i + 1]) ++i;
    return y[i] + (y[i + 1] - y[i]) * (v - x[i]) / (x[i + 1] - x[i]);
}

/* Relative margin by which a descending photon emitted at h_e with (local)
 * zenith sine sin_z clears the turning-point condition: the smallest of
 * (n(h) r(h) - K) / K over [h_obs, h_e], with K = n(h_e) r(h_e) sin_z and
 * r = R + h on the spherical shell (r = 1 in the plane; n = 1 for the straight
 * line).  Within each piece between breakpoints n(h) is monotone (exponential,
 * linear or constant) and, on the shell, n r grows with r wherever
 * (n - 1) < H / r (the scale height over the radius, ~1e-3 against n - 1 <
 * 3e-4 here), so the smallest value lies at a piece end; both one-sided limits
 * are taken at a breakpoint.  Positive: the path reaches the ground. */
static double orc_reach_margin(const orc_atm* a, const orc_config* cfg, double h_e, double sin_z)
{
    const int refr = cfg->refraction;
    const double R = cfg->earth_radius;
    double rr_e = cfg->spherical ? R + h_e : 1.0;
    const double K = (refr ? orc_n(a, h_e) : 1.0) * rr_e * sin_z;
    if (!(K > 0.0)) return 1.0;
    double hs[ORC_MAX_NODES + 20];
    int m = 0;
    hs[m++] = cfg->h_obs;
    double bp[ORC_MAX_NODES + 16];
    int nb = refr ? orc_breakpoints(a, cfg->h_obs, h_e, bp) : 0;
    for (int i = 0; i < nb; ++i) {
        hs[m++] = bp[i];
        hs[m++] = bp[i] - 1e-9 * fmax(1.0, fabs(bp[i]));   /* the limit from below */
    }
    double best = 1e300;
    for (int i = 0; i < m; ++i) {
        const double r = cfg->spherical ? R + hs[i] : 1.0;
        const double v = ((refr ? orc_n(a, hs[i]) : 1.0) * r - K) / K;
        if (v < best) best = v;
    }
    return best;
}

int orc_propagate(const orc_segment* segs, size_t n_segs, const orc_atm* atm,
                  const orc_config* cfg, orc_output* out)
{
    const double inv_l1 = 1.0 / cfg->lambda1, inv_l2 = 1.0 / cfg->lambda2;
    /* Frank-Tamm (Eq. 2.2/2.4) integrated over the band with mu_r = 1 and
     * no dispersion: dN/dx = 2 pi alpha z^2 (1/l1 - 1/l2) sin^2(theta). */
    const double ft = 2.0 * ORC_PI * ORC_ALPHA * (inv_l1 - inv_l2);
    const double b = (double)cfg->bunch;
    const uint32_t key[2] = { (uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32) };
    const double n_obs = orc_n(atm, cfg->h_obs);
    /* the cylinders are laid out per photon from the spherical frame; the LV3 filter's
     * straight-line landing point is defined on the plane and the sphere only */
    if (cfg->cylindrical && (!cfg->spherical || cfg->lv3)) return 2;

    for (size_t is = 0; is < n_segs; ++is) {
        const orc_segment* sg = &segs[is];
        const uint64_t gid = cfg->seg_base + is;
        if (!orc_segment_valid(sg, cfg->n_showers)) { out->counters[7]++; continue; }

        double un = sqrt((double)sg->ux * sg->ux + (double)sg->uy * sg->uy + (double)sg->uz * sg->uz);
        const double P[3] = { sg->ux / un, sg->uy / un, sg->uz / un };
        const double L = sg->length, g = sg->inv_gamma2, z = sg->charge;
        const double beta = sqrt(1.0 - g);
        /* Sub-stepping (Sec. 4.2.1): K = ceil(L / s_max) sub-steps of equal length, the
         * exact ceiling of the quotient of the two stored numbers.  The rounded quotient
         * proposes K; the residual K s_max - L, whose sign one fused multiply-add gives
         * exactly, confirms K s_max >= L > (K - 1) s_max.  A length within 1e-13
         * (relative) of a whole number of sub-steps, without lying exactly on one, is
         * flagged: a rounding of s_max at that level moves the count, and every bunch of
         * the segment with it. */
        const double s_max = cfg->s_max, Lq = L / s_max;
        int K = Lq <= 1.0 ? 1 : (int)ceil(Lq);
        if (fma((double)K, s_max, -L) < 0.0) ++K;
        else if (K > 1 && fma((double)(K - 1), s_max, -L) >= 0.0) --K;
        const double res = fma(nearbyint(Lq), s_max, -L);
        const int seg_flag = (res != 0.0 && fabs(res) < 1e-13 * L) ? ORC_FL_SEGMENT : 0;
        const int shower = (int)sg->shower_id;
        if (seg_flag) {
            orc_record fr; memset(&fr, 0, sizeof fr);
            fr.seg = gid; fr.k = 0xFFFFFFFFu; fr.i = 0xFFFFFFFFu;
            fr.status = ORC_ST_SUBSTEP_FLAG; fr.flags = ORC_FL_SEGMENT;
            fr.tel = -1; fr.bin = -1; fr.pix = -1;
            orc_push(out, &fr);
        }

        /* LV1 particle filter (Sec. 4.3.2; the two-parameter cut of Sec. 6.2.1) */
        int lv1_near = 0;
        if (cfg->lv1_metric) {
            const double S[3] = { sg->x0, sg->y0, sg->z0 };
            double y = sg->z0 - cfg->h_obs;
            if (cfg->spherical) {
                double zr = sg->z0 + cfg->earth_radius;
                y = sqrt(sg->x0 * sg->x0 + sg->y0 * sg->y0 + zr * zr) - cfg->earth_radius - cfg->h_obs;
            }
            double x = fmax(orc_lv1_x(cfg, S, P), 1e-3);
            double thr = cfg->lv1_a * pow(x, cfg->lv1_b);
            lv1_near = fabs(y - thr) < cfg->band_lv1 * fmax(fabs(thr), 1.0);
            if (y >= thr) {
                out->lv1_dropped++;
                if (lv1_near) {   /* the kernel may keep it: its sub-steps may appear */
                    for (int k = 0; k < K; ++k) {
                        orc_record fr; memset(&fr, 0, sizeof fr);
                        fr.seg = gid; fr.k = (uint32_t)k; fr.i = 0xFFFFFFFFu;
                        fr.status = ORC_ST_SUBSTEP_FLAG; fr.flags = ORC_FL_COUNT | ORC_FL_LV1;
                        fr.tel = -1; fr.bin = -1; fr.pix = -1;
                        orc_push(out, &fr);
                    }
                }
                continue;
            }
        }

        /* Euler-Rodrigues rotation by 180 degrees about the bisector A of
         * D = (0,0,-1) and P: M = 2 A A^T - 1 (Sec. 4.2), A normalised. */
        double A[3] = { P[0], P[1], P[2] - 1.0 };
        double an = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
        A[0] /= an; A[1] /= an; A[2] /= an;
        double M[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) M[r][c] = 2.0 * A[r] * A[c] - (r == c ? 1.0 : 0.0);

        for (int k = 0; k < K; ++k) {
            /* Sub-step k (Sec. 4.2.1): n and the angle at its midpoint, whose
             * altitude on the spherical shell is its distance from the Earth's
             * centre minus R_E (Sec. 3.3.4). */
            const double s_mid = (k + 0.5) / K * L;
            double h_mid = sg->z0 + s_mid * P[2];
            if (cfg->spherical) {
                const double mx = sg->x0 + s_mid * P[0], my = sg->y0 + s_mid * P[1];
                const double mz = h_mid + cfg->earth_radius;
                h_mid = sqrt(mx * mx + my * my + mz * mz) - cfg->earth_radius;
            }
            double n_k = orc_n(atm, h_mid);
            int mid_layer_flag = 0;       /* angle and yield may come from the other layer's law */
            if (atm->kind == ORC_ATM_LAYERED)
                for (int li = 1; li < atm->n_layers; ++li)
                    if (fabs(h_mid - atm->layer_h[li]) < cfg->band_h) mid_layer_flag = 1;
            double sin2 = 1.0 - 1.0 / (beta * beta * n_k * n_k);    /* Eq. 2.3 */
            double nbar = sin2 > 0.0 ? ft * z * z * sin2 * (L / K) / b : 0.0;  /* threshold */
            if (cfg->emission) {   /* fluorescence (Eq. 2.6): deposited energy times the lines' yields */
                double ysum = 0.0;
                for (int l = 0; l < cfg->fl_n_lines; ++l) ysum += cfg->fl_yield[l];
                nbar = z * z * cfg->fl_dedx * orc_atm_rho(atm, h_mid) * 100.0 * ysum * (L / K) / b;
                if (cfg->emission == 2) nbar *= 0.5;
            }
            uint32_t ctr_c[4] = { (uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, 0xFFFFFFFFu };
            uint32_t rc[4];
            orc_philox4x32_10(ctr_c, key, rc);
            double uk = orc_uniform(rc[0]);
            double fl = floor(nbar);
            int N = (int)fl + (uk < nbar - fl ? 1 : 0);               /* stochastic rounding */
            int count_flag = orc_floor_dist(nbar - uk) < cfg->band_count || mid_layer_flag;
            if (count_flag) {
                orc_record fr; memset(&fr, 0, sizeof fr);
                fr.seg = gid; fr.k = (uint32_t)k; fr.i = 0xFFFFFFFFu;
                fr.status = ORC_ST_SUBSTEP_FLAG; fr.nbar = nbar; fr.flags = ORC_FL_COUNT;
                fr.tel = -1; fr.bin = -1; fr.pix = -1;
                orc_push(out, &fr);
            }
            if (N == 0) continue;
            double cos_t = 1.0 / (beta * n_k), sin_t = sqrt(sin2);

            for (int i = 0; i < N; ++i) {
                uint32_t ctr[4] = { (uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, (uint32_t)i };
                uint32_t r4[4];
                orc_philox4x32_10(ctr, key, r4);
                double u0 = orc_uniform(r4[0]), u1 = orc_uniform(r4[1]);
                double u2 = orc_uniform(r4[2]), u3 = orc_uniform(r4[3]);

                orc_record rec; memset(&rec, 0, sizeof rec);
                rec.pix = -1;
                rec.seg = gid; rec.k = (uint32_t)k; rec.i = (uint32_t)i;
                rec.tel = -1; rec.bin = -1; rec.nbar = nbar;
                rec.flags |= seg_flag;
                if (count_flag && i == N - 1) rec.flags |= ORC_FL_COUNT;
                if (mid_layer_flag) rec.flags |= ORC_FL_LAYER;
                if (lv1_near) rec.flags |= ORC_FL_COUNT | ORC_FL_LV1;   /* the kernel may drop the segment */

                /* translation to a random point of the sub-step (Fig. 4.2c) */
                double ell = (k + u0) / K * L;
                double E[3] = { sg->x0 + ell * P[0], sg->y0 + ell * P[1], sg->z0 + ell * P[2] };
                double t_emit_rel = ell / (beta * ORC_C_LIGHT);
                /* cone vector (Sec. 4.2) and wavelength from the 1/lambda^2 law */
                double phi = 2.0 * ORC_PI * u1;
                double inv_l = inv_l1 - u2 * (inv_l1 - inv_l2);
                rec.lambda = 1.0 / inv_l;
                double p[3] = { cos(phi) * sin_t, sin(phi) * sin_t, -cos_t };
                double u[3];
                for (int r = 0; r < 3; ++r) u[r] = M[r][0] * p[0] + M[r][1] * p[1] + M[r][2] * p[2];
                if (cfg->emission) {
                    /* fluorescence (Sec. 4.2.2): isotropic, cos(zenith) uniform over the sphere
                     * or the downward half sphere; the line from a second draw, its 24-bit
                     * integer against the lines' cumulative shares in units of 2^-24 */
                    const double c = cfg->emission == 2 ? u2 - 1.0 : 2.0 * u2 - 1.0;
                    const double sc = sqrt(fmax(1.0 - c * c, 0.0));
                    u[0] = sc * cos(phi); u[1] = sc * sin(phi); u[2] = c;
                    uint32_t ctr2[4] = { (uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, (uint32_t)i | 0x80000000u };
                    uint32_t r2[4];
                    orc_philox4x32_10(ctr2, key, r2);
                    double ysum = 0.0, cum = 0.0;
                    for (int l = 0; l < cfg->fl_n_lines; ++l) ysum += cfg->fl_yield[l];
                    const uint32_t v = r2[0] >> 8;
                    int line = cfg->fl_n_lines - 1;
                    for (int l = 0; l + 1 < cfg->fl_n_lines; ++l) {
                        cum += cfg->fl_yield[l];
                        if (v < (uint32_t)floor(cum / ysum * 16777216.0)) { line = l; break; }
                    }
                    rec.lambda = cfg->fl_lines_nm[line] * 1e-9;
                }
                rec.ux = u[0]; rec.uy = u[1]; rec.uz = u[2];
                out->counters[0] += (uint64_t)cfg->bunch;

                /* local vertical and altitude of the emission point */
                const double R = cfg->earth_radius;
                double vloc[3] = { 0.0, 0.0, 1.0 }, h_e = E[2];
                if (cfg->spherical) {
                    double d[3] = { E[0], E[1], E[2] + R };
                    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    for (int c = 0; c < 3; ++c) vloc[c] = d[c] / r;
                    h_e = r - R;
                    double G0[3] = { E[0], E[1], E[2] };
                    orc_ae(R, R + cfg->h_obs, G0, &rec.ex, &rec.ey);   /* footprint of E */
                } else {
                    rec.ex = E[0]; rec.ey = E[1];
                }
                rec.h_e = h_e;
                const double cos_z = -(u[0] * vloc[0] + u[1] * vloc[1] + u[2] * vloc[2]);   /* cos(local zenith) */

                if (fabs(cos_z) < cfg->band_w) rec.flags |= ORC_FL_UPWARD;
                if (fabs(h_e - cfg->h_obs) < cfg->band_h) rec.flags |= ORC_FL_BELOW;
                if ((cfg->refraction || cfg->transmission) && atm->kind == ORC_ATM_LAYERED) {
                    for (int li = 1; li < atm->n_layers; ++li)
                        if (fabs(h_e - atm->layer_h[li]) < cfg->band_h) rec.flags |= ORC_FL_LAYER;
                }
                if (!(cos_z > 0.0)) {                   /* not descending: discarded (Sec. 5.3.4) */
                    rec.status = ORC_ST_UPWARD;
                    out->counters[4] += cfg->bunch; out->counters[5] += cfg->bunch;
                    out->counters[6] += cfg->bunch;
                    orc_push(out, &rec);
                    continue;
                }
                if (h_e < cfg->h_obs) {                 /* emitted below the observation level */
                    rec.status = ORC_ST_BELOW;
                    out->counters[4] += cfg->bunch; out->counters[5] += cfg->bunch;
                    orc_push(out, &rec);
                    continue;
                }
                double theta0 = acos(cos_z);
                rec.theta0 = theta0;
                double sin_z = sin(theta0);
                /* cylindrical atmosphere: the photon's axis frame (e_r towards E's foot,
                 * e_a = z x e_r, e_chi the transverse tangent at E) and its components */
                double c_er[3] = { 1.0, 0.0, 0.0 }, c_ea[3] = { 0.0, 1.0, 0.0 }, c_ua = 0.0, c_uchi = 0.0;
                if (cfg->cylindrical) {
                    const double dE = sqrt(E[0] * E[0] + E[1] * E[1]);
                    if (dE > 0.0) { c_er[0] = E[0] / dE; c_er[1] = E[1] / dE; }
                    c_ea[0] = -c_er[1]; c_ea[1] = c_er[0];
                    /* vloc = sin(chi_E) e_r + cos(chi_E) z, e_chi = cos(chi_E) e_r - sin(chi_E) z */
                    const double s_chi = vloc[0] * c_er[0] + vloc[1] * c_er[1], c_chi = vloc[2];
                    c_ua = u[0] * c_ea[0] + u[1] * c_ea[1];
                    c_uchi = c_chi * (u[0] * c_er[0] + u[1] * c_er[1]) - s_chi * u[2];
                }
                /* Does the path meet the observation level?  Along the exact path the
                 * invariant (Eq. 3.17; Bouguer's n r sin(psi) on the shell; in the cylinders
                 * N rho sin(psi) with N = sqrt(n^2 - A^2)) must stay below n (h) (n r, N rho)
                 * all the way down; the straight line of Eq. 3.3 is the n = 1 case. */
                {
                    double margin = cfg->cylindrical
                                    ? orc_cyl_reach_margin(atm, cfg->refraction, R, cfg->h_obs, h_e, c_ua, c_uchi)
                                    : orc_reach_margin(atm, cfg, h_e, sin_z);
                    if (fabs(margin) < cfg->band_w) rec.flags |= ORC_FL_GROUND;
                    if (!(margin > 0.0)) {
                        rec.status = ORC_ST_NO_GROUND;
                        out->counters[4] += cfg->bunch; out->counters[5] += cfg->bunch;
                        orc_push(out, &rec);
                        continue;
                    }
                }
                /* LV3 photon pre-filter (Sec. 4.3.4, 6.2.2): the vacuum straight line's
                 * landing point S decides, before any correction is looked up */
                if (cfg->lv3) {
                    double S[3];
                    if (!cfg->spherical) {
                        const double t = (h_e - cfg->h_obs) / cos_z;
                        S[0] = E[0] + t * u[0]; S[1] = E[1] + t * u[1]; S[2] = cfg->h_obs;
                    } else {   /* first crossing of |E + t u - (0, 0, -R)| = R + h_obs */
                        const double d[3] = { E[0], E[1], E[2] + R }, rg = R + cfg->h_obs;
                        const double b = d[0] * u[0] + d[1] * u[1] + d[2] * u[2];
                        const double c = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - rg * rg;
                        const double disc = b * b - c;
                        if (disc < 0.0) rec.flags |= ORC_FL_LV3;   /* the line passes over the ground */
                        const double t = -b - sqrt(fmax(disc, 0.0));
                        for (int c3 = 0; c3 < 3; ++c3) S[c3] = E[c3] + t * u[c3];
                    }
                    const double dx = S[0] - cfg->lv3_centre[0], dy = S[1] - cfg->lv3_centre[1],
                                 dz = S[2] - cfg->lv3_centre[2];
                    const double dist = sqrt(dx * dx + dy * dy + dz * dz), lim = cfg->lv3_radius + cfg->lv3_margin;
                    if (fabs(dist - lim) < cfg->band_pos) rec.flags |= ORC_FL_LV3;
                    if (dist > lim) {
                        rec.status = ORC_ST_LV3;
                        out->counters[4] += cfg->bunch; out->counters[5] += cfg->bunch;
                        orc_push(out, &rec);
                        continue;
                    }
                }

                /* horizontal unit of u in the local frame (the plane of travel) */
                double hv[3] = { u[0] + cos_z * vloc[0], u[1] + cos_z * vloc[1], u[2] + cos_z * vloc[2] };
                double hn = sqrt(hv[0] * hv[0] + hv[1] * hv[1] + hv[2] * hv[2]);
                if (hn > 0.0) { hv[0] /= hn; hv[1] /= hn; hv[2] /= hn; }
                else { hv[0] = 1.0; hv[1] = 0.0; hv[2] = 0.0; }

                double path[4], G3[3], ug[3], gx, gy;
                if (!cfg->spherical) {
                    if (cfg->refraction && cfg->tracer == 1) {
                        orc_snell_path(atm, cfg->h_obs, h_e, theta0, cfg->tracer_dh, cfg->aer_H, path);
                        /* the slab count and the slab holding a jump of n are decisions too */
                        const double q = (h_e - cfg->h_obs) / cfg->tracer_dh;
                        if (fabs(q - nearbyint(q)) < 1e-3) rec.flags |= ORC_FL_LAYER;
                        int ns = (int)ceil(q - 1e-9); if (ns < 1) ns = 1;
                        const double step = (h_e - cfg->h_obs) / ns;
                        double jumps[9]; int nj = 0;
                        if (atm->kind == ORC_ATM_LAYERED) {
                            for (int li = 1; li < atm->n_layers; ++li) jumps[nj++] = atm->layer_h[li];
                            jumps[nj++] = atm->h_top;
                        }
                        for (int k2 = 0; k2 < nj; ++k2) {
                            if (!(jumps[k2] > cfg->h_obs && jumps[k2] < h_e)) continue;
                            const double f = (h_e - jumps[k2]) / step - 0.5;   /* midpoints at integer f */
                            if (fabs(f - nearbyint(f)) * step < 0.01) rec.flags |= ORC_FL_LAYER;
                        }
                    } else if (cfg->refraction) {
                        orc_refract_quad(atm, cfg->h_obs, h_e, theta0, cfg->aer_H, cfg->quad_rtol, path);
                    } else {
                        orc_straight(atm, cfg->h_obs, h_e, theta0, cfg->aer_H, path);
                    }
                    /* ground point: E_xy + R along the horizontal unit of u */
                    gx = E[0] + path[0] * hv[0];
                    gy = E[1] + path[0] * hv[1];
                    G3[0] = gx; G3[1] = gy; G3[2] = cfg->h_obs;
                    /* arrival direction: zenith from the invariant, azimuth kept */
                    if (cfg->refraction) {
                        double sg_ = orc_n(atm, h_e) * sin_z / n_obs, cg = sqrt(1.0 - sg_ * sg_);
                        ug[0] = sg_ * hv[0]; ug[1] = sg_ * hv[1]; ug[2] = -cg;
                    } else { ug[0] = u[0]; ug[1] = u[1]; ug[2] = u[2]; }
                } else if (cfg->cylindrical) {
                    /* the transverse path sweeps chi, the axial drift follows from A; both are
                     * laid out on the unrolled ground cylinder, where the arrival direction keeps
                     * its components along e_chi, e_a and the normal */
                    double cp[5];
                    if (cfg->refraction && cfg->tracer == 1) {
                        orc_snell_path_cyl(atm, R, cfg->h_obs, h_e, fabs(c_uchi), -cos_z, c_ua, cfg->tracer_dh, cfg->aer_H,
                                           1, cp);
                        const double q = (h_e - cfg->h_obs) / cfg->tracer_dh;
                        if (fabs(q - nearbyint(q)) < 1e-3) rec.flags |= ORC_FL_LAYER;
                        int ns = (int)ceil(q - 1e-9); if (ns < 1) ns = 1;
                        const double step = (h_e - cfg->h_obs) / ns;
                        if (atm->kind == ORC_ATM_LAYERED) {
                            for (int li = 1; li <= atm->n_layers; ++li) {
                                const double hb = li < atm->n_layers ? atm->layer_h[li] : atm->h_top;
                                if (!(hb > cfg->h_obs && hb < h_e)) continue;
                                const double f = (h_e - hb) / step - 0.5;
                                if (fabs(f - nearbyint(f)) * step < 0.01) rec.flags |= ORC_FL_LAYER;
                            }
                        }
                    } else {
                        orc_cyl_path(atm, R, cfg->h_obs, h_e, c_ua, fabs(c_uchi), cfg->aer_H, cfg->refraction,
                                     cfg->quad_rtol, cp);
                    }
                    const double rg = R + cfg->h_obs, chi_E = atan2(sqrt(E[0] * E[0] + E[1] * E[1]), E[2] + R);
                    const double chi_g = chi_E + (c_uchi < 0.0 ? -cp[0] : cp[0]);
                    gx = rg * chi_g * c_er[0] + cp[2] * c_ea[0];
                    gy = rg * chi_g * c_er[1] + cp[2] * c_ea[1];
                    G3[0] = gx; G3[1] = gy; G3[2] = cfg->h_obs;
                    path[0] = cp[0]; path[1] = cp[1]; path[2] = cp[3]; path[3] = cp[4];
                    const double n_e = cfg->refraction ? orc_n(atm, h_e) : 1.0, n_g = cfg->refraction ? n_obs : 1.0;
                    const double ga = n_e * c_ua / n_g, gchi = n_e * (R + h_e) * c_uchi / (n_g * rg);
                    const double grho = -sqrt(fmax(1.0 - ga * ga - gchi * gchi, 0.0));
                    for (int c = 0; c < 2; ++c) ug[c] = gchi * c_er[c] + ga * c_ea[c];
                    ug[2] = grho;
                } else {
                    /* the path stays in the plane (centre, E, u): rotate the vertical by the
                     * central angle Phi towards hv; Bouguer's invariant gives the arrival zenith */
                    if (cfg->refraction && cfg->tracer == 1) {
                        orc_snell_path_sph(atm, R, cfg->h_obs, h_e, theta0, cfg->tracer_dh, cfg->aer_H, path);
                        const double q = (h_e - cfg->h_obs) / cfg->tracer_dh;
                        if (fabs(q - nearbyint(q)) < 1e-3) rec.flags |= ORC_FL_LAYER;
                        int ns = (int)ceil(q - 1e-9); if (ns < 1) ns = 1;
                        const double step = (h_e - cfg->h_obs) / ns;
                        if (atm->kind == ORC_ATM_LAYERED) {
                            for (int li = 1; li <= atm->n_layers; ++li) {
                                const double hb = li < atm->n_layers ? atm->layer_h[li] : atm->h_top;
                                if (!(hb > cfg->h_obs && hb < h_e)) continue;
                                const double f = (h_e - hb) / step - 0.5;
                                if (fabs(f - nearbyint(f)) * step < 0.01) rec.flags |= ORC_FL_LAYER;
                            }
                        }
                    } else {
                        orc_sph_path(atm, R, cfg->h_obs, h_e, theta0, cfg->aer_H, cfg->refraction, cfg->quad_rtol, path);
                    }
                    const double rg = R + cfg->h_obs, Phi = path[0];
                    double vG[3], hG[3];
                    for (int c = 0; c < 3; ++c) {
                        vG[c] = cos(Phi) * vloc[c] + sin(Phi) * hv[c];
                        hG[c] = -sin(Phi) * vloc[c] + cos(Phi) * hv[c];
                        G3[c] = rg * vG[c];
                    }
                    G3[2] -= R;
                    orc_ae(R, rg, G3, &gx, &gy);
                    const double n_e = cfg->refraction ? orc_n(atm, h_e) : 1.0, n_g = cfg->refraction ? n_obs : 1.0;
                    const double sg_ = n_e * (R + h_e) * sin_z / (n_g * rg), cg = sqrt(1.0 - sg_ * sg_);
                    for (int c = 0; c < 3; ++c) ug[c] = -cg * vG[c] + sg_ * hG[c];
                }
                rec.x = gx; rec.y = gy;
                double t_arr = sg->t0 + t_emit_rel + path[1];
                rec.dt = t_emit_rel + path[1];

                if (cfg->transmission) {
                    double lam = rec.lambda;
                    double XR = cfg->rayl_X0 * pow(lam / cfg->rayl_lambda0, 4.0);
                    double tauA = cfg->aer_tau0 * pow(lam / cfg->aer_lambda0, -cfg->aer_alpha);
                    double T = exp(-path[2] / XR - tauA * path[3] / cfg->aer_H);
                    rec.T = T;
                    if (fabs(u3 - T) < cfg->band_T) rec.flags |= ORC_FL_ABSORB;
                    if (!(u3 < T)) {
                        rec.status = ORC_ST_ABSORBED;
                        out->counters[1] += cfg->bunch;
                        orc_push(out, &rec);
                        continue;
                    }
                } else rec.T = 1.0;
                rec.status = ORC_ST_LANDED;

                /* ground histogram (planar coordinates, or azimuthal-equidistant on the sphere) */
                if (cfg->hist_nx > 0) {
                    double fx = (gx - cfg->hist_x0) / cfg->hist_dx, fy = (gy - cfg->hist_y0) / cfg->hist_dy;
                    double ix = floor(fx), iy = floor(fy);
                    double ex_d = fmin(fx - ix, ix + 1.0 - fx) * cfg->hist_dx;
                    double ey_d = fmin(fy - iy, iy + 1.0 - fy) * cfg->hist_dy;
                    int near_x = fx > -1.0 && fx < cfg->hist_nx + 1.0 && fy > -1.0 && fy < cfg->hist_ny + 1.0;
                    if (near_x && (ex_d < cfg->band_pos || ey_d < cfg->band_pos)) rec.flags |= ORC_FL_HIST_EDGE;
                    if (ix >= 0 && ix < cfg->hist_nx && iy >= 0 && iy < cfg->hist_ny) {
                        int bin = (int)iy * cfg->hist_nx + (int)ix;
                        rec.bin = bin;
                        out->hist[((size_t)shower * cfg->hist_ny * cfg->hist_nx) + bin] += cfg->bunch;
                        out->counters[2] += cfg->bunch;
                    } else out->counters[4] += cfg->bunch;
                } else out->counters[4] += cfg->bunch;

                /* telescopes: distance from the sphere centre to the arrival line */
                int best = -1; double best_d = 0.0;
                for (int it = 0; it < cfg->n_tel; ++it) {
                    const double* T4 = cfg->tel + 4 * it;
                    double Tc[3] = { T4[0], T4[1], T4[2] };
                    if (cfg->spherical && !cfg->cylindrical) orc_ae_inverse(R, cfg->h_obs, T4[0], T4[1], T4[2] - cfg->h_obs, Tc);
                    double d0 = Tc[0] - G3[0], d1 = Tc[1] - G3[1], d2 = Tc[2] - G3[2];
                    double along = d0 * ug[0] + d1 * ug[1] + d2 * ug[2];
                    double dist2 = d0 * d0 + d1 * d1 + d2 * d2 - along * along;
                    double dist = sqrt(fmax(dist2, 0.0));
                    if (fabs(dist - T4[3]) < cfg->band_pos) rec.flags |= ORC_FL_TEL_EDGE;
                    if (dist < T4[3]) {
                        if (best >= 0 && fabs(dist - best_d) < cfg->band_pos) rec.flags |= ORC_FL_TEL_EDGE;
                        if (best < 0 || dist < best_d) { best = it; best_d = dist; }
                    }
                }
                rec.pix = -1;
                if (best >= 0 && cfg->cam_n > 0) {
                    const double* T4 = cfg->tel + 4 * best;
                    double Tc[3] = { T4[0], T4[1], T4[2] };
                    if (cfg->spherical && !cfg->cylindrical) orc_ae_inverse(R, cfg->h_obs, T4[0], T4[1], T4[2] - cfg->h_obs, Tc);
                    int edge = 0;
                    rec.pix = orc_camera_pixel(cfg, Tc, G3, ug, cfg->band_pos, &edge);
                    if (edge) rec.flags |= ORC_FL_TEL_EDGE;
                    if (rec.pix >= 0 && cfg->eff_n > 0) {   /* mirror reflectivity x camera efficiency */
                        const double lnm = rec.lambda * 1e9;
                        const double P = orc_lerp_curve(cfg->eff_l, cfg->eff_R, cfg->eff_n, lnm) *
                                         orc_lerp_curve(cfg->eff_l, cfg->eff_E, cfg->eff_n, lnm);
                        uint32_t ctr3[4] = { (uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, (uint32_t)i | 0x40000000u };
                        uint32_t r3[4];
                        orc_philox4x32_10(ctr3, key, r3);
                        const double uo = orc_uniform(r3[0]);
                        if (fabs(uo - P) < cfg->band_T) rec.flags |= ORC_FL_OPTICS;
                        if (!(uo < P)) rec.pix = -1;   /* absorbed in the optics: no camera photon */
                    }
                    if (rec.pix >= 0 && out->camera)
                        out->camera[((size_t)shower * cfg->n_tel + best) * cfg->cam_n * cfg->cam_n + rec.pix] += cfg->bunch;
                }
                if (best >= 0) {
                    rec.tel = best;
                    out->tel_counts[(size_t)shower * cfg->n_tel + best] += cfg->bunch;
                    out->tel_time[(size_t)shower * cfg->n_tel + best] += cfg->bunch * t_arr;
                    out->counters[3] += cfg->bunch;
                } else out->counters[5] += cfg->bunch;
                orc_push(out, &rec);
            }
        }
    }
    return 0;
}

/* Sizes of the structs, so the Python side can check its mirror layout. */
size_t orc_sizeof_segment(void) { return sizeof(orc_segment); }
size_t orc_sizeof_record(void) { return sizeof(orc_record); }
size_t orc_sizeof_config(void) { return sizeof(orc_config); }
size_t orc_sizeof_atm(void) { return sizeof(orc_atm); }

/* ------------------------------------------------------------------ */
/* Surrogate network (no thesis counterpart): a tanh MLP              */
/* din -> dh -> dh -> dh -> dout in FP64, MSE loss and Adam.          */
/* Parameters are one flat array: W1 (dh x din), b1, W2 (dh x dh),    */
/* b2, W3 (dh x dh), b3, W4 (dout x dh), b4; W rows are output units. */
/* ------------------------------------------------------------------ */
size_t orc_mlp_n_params(int din, int dh, int dout)
{
    return (size_t)dh * din + dh + 2 * ((size_t)dh * dh + dh) + (size_t)dout * dh + dout;
}

static void orc_dense(const double* W, const double* b, const double* x, int nin, int nout, double* z)
{
    for (int o = 0; o < nout; ++o) {
        double s = b[o];
        for (int i = 0; i < nin; ++i) s += W[(size_t)o * nin + i] * x[i];
        z[o] = s;
    }
}

/* y (B x dout); acts, if given, receives the three hidden layers' outputs
 * (B x 3 x dh). */
void orc_mlp_forward(const double* theta, int din, int dh, int dout, const double* x, int B, double* y,
                     double* acts)
{
    const double* W1 = theta;
    const double* b1 = W1 + (size_t)dh * din;
    const double* W2 = b1 + dh;
    const double* b2 = W2 + (size_t)dh * dh;
    const double* W3 = b2 + dh;
    const double* b3 = W3 + (size_t)dh * dh;
    const double* W4 = b3 + dh;
    const double* b4 = W4 + (size_t)dout * dh;
    double* h1 = malloc(sizeof(double) * dh);
    double* h2 = malloc(sizeof(double) * dh);
    double* h3 = malloc(sizeof(double) * dh);
    for (int r = 0; r < B; ++r) {
        orc_dense(W1, b1, x + (size_t)r * din, din, dh, h1);
        for (int j = 0; j < dh; ++j) h1[j] = tanh(h1[j]);
        orc_dense(W2, b2, h1, dh, dh, h2);
        for (int j = 0; j < dh; ++j) h2[j] = tanh(h2[j]);
        orc_dense(W3, b3, h2, dh, dh, h3);
        for (int j = 0; j < dh; ++j) h3[j] = tanh(h3[j]);
        orc_dense(W4, b4, h3, dh, dout, y + (size_t)r * dout);
        if (acts) {
            memcpy(acts + ((size_t)r * 3 + 0) * dh, h1, sizeof(double) * dh);
            memcpy(acts + ((size_t)r * 3 + 1) * dh, h2, sizeof(double) * dh);
            memcpy(acts + ((size_t)r * 3 + 2) * dh, h3, sizeof(double) * dh);
        }
    }
    free(h1); free(h2); free(h3);
}

/* Loss L = (1/B) sum_r sum_o (y_ro - t_ro)^2 and its gradient with respect
 * to every parameter (same flat layout), by the chain rule layer by layer. */
double orc_mlp_loss_grad(const double* theta, int din, int dh, int dout, const double* x, const double* t,
                         int B, double* grad)
{
    const size_t np = orc_mlp_n_params(din, dh, dout);
    const double* W2 = theta + (size_t)dh * din + dh;
    const double* W3 = W2 + (size_t)dh * dh + dh;
    const double* W4 = W3 + (size_t)dh * dh + dh;
    double* gW1 = grad;
    double* gb1 = gW1 + (size_t)dh * din;
    double* gW2 = gb1 + dh;
    double* gb2 = gW2 + (size_t)dh * dh;
    double* gW3 = gb2 + dh;
    double* gb3 = gW3 + (size_t)dh * dh;
    double* gW4 = gb3 + dh;
    double* gb4 = gW4 + (size_t)dout * dh;
    memset(grad, 0, sizeof(double) * np);
    double* y = malloc(sizeof(double) * (size_t)B * dout);
    double* acts = malloc(sizeof(double) * (size_t)B * 3 * dh);
    orc_mlp_forward(theta, din, dh, dout, x, B, y, acts);
    double loss = 0.0;
    double* dy = malloc(sizeof(double) * dout);
    double* dz3 = malloc(sizeof(double) * dh);
    double* dz2 = malloc(sizeof(double) * dh);
    double* dz1 = malloc(sizeof(double) * dh);
    for (int r = 0; r < B; ++r) {
        const double* h1 = acts + ((size_t)r * 3 + 0) * dh;
        const double* h2 = acts + ((size_t)r * 3 + 1) * dh;
        const double* h3 = acts + ((size_t)r * 3 + 2) * dh;
        const double* xr = x + (size_t)r * din;
        for (int o = 0; o < dout; ++o) {
            double e = y[(size_t)r * dout + o] - t[(size_t)r * dout + o];
            loss += e * e / B;
            dy[o] = 2.0 * e / B;
        }
        for (int o = 0; o < dout; ++o) {            /* output layer */
            gb4[o] += dy[o];
            for (int j = 0; j < dh; ++j) gW4[(size_t)o * dh + j] += dy[o] * h3[j];
        }
        for (int j = 0; j < dh; ++j) {              /* through tanh of layer 3 */
            double s = 0.0;
            for (int o = 0; o < dout; ++o) s += dy[o] * W4[(size_t)o * dh + j];
            dz3[j] = s * (1.0 - h3[j] * h3[j]);
        }
        for (int j = 0; j < dh; ++j) {
            gb3[j] += dz3[j];
            for (int i = 0; i < dh; ++i) gW3[(size_t)j * dh + i] += dz3[j] * h2[i];
        }
        for (int i = 0; i < dh; ++i) {
            double s = 0.0;
            for (int j = 0; j < dh; ++j) s += dz3[j] * W3[(size_t)j * dh + i];
            dz2[i] = s * (1.0 - h2[i] * h2[i]);
        }
        for (int j = 0; j < dh; ++j) {
            gb2[j] += dz2[j];
            for (int i = 0; i < dh; ++i) gW2[(size_t)j * dh + i] += dz2[j] * h1[i];
        }
        for (int i = 0; i < dh; ++i) {
            double s = 0.0;
            for (int j = 0; j < dh; ++j) s += dz2[j] * W2[(size_t)j * dh + i];
            dz1[i] = s * (1.0 - h1[i] * h1[i]);
        }
        for (int j = 0; j < dh; ++j) {
            gb1[j] += dz1[j];
            for (int i = 0; i < din; ++i) gW1[(size_t)j * din + i] += dz1[j] * xr[i];
        }
    }
    free(y); free(acts); free(dy); free(dz3); free(dz2); free(dz1);
    return loss;
}

/* One Adam step (Kingma & Ba 2015) with bias correction; `step` counts from 1. */
void orc_adam(double* theta, const double* grad, double* m, double* v, size_t n, double lr, double beta1,
              double beta2, double eps, int step)
{
    const double c1 = 1.0 - pow(beta1, step), c2 = 1.0 - pow(beta2, step);
    for (size_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        theta[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
