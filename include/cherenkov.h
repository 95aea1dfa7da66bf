/*
 * cherenkov.h - C ABI of the GB300 (sm_103a) Cherenkov photon library.
 *
 * The library generates Cherenkov photons (or bunches of photons) along
 * charged track segments and propagates them through a layered atmosphere
 * to an observation level, where they are binned into ground histograms and
 * hit-tested against telescope spheres.  It follows D. Baack, "Optical
 * Photon Emission in Extended Airshowers" (TU Dortmund, 2023):
 *
 *   yield and angle      Sec. 2.2.1, Eq. 2.2-2.5
 *   random numbers       Sec. 3.1 (counter-based Philox)
 *   atmosphere           Sec. 3.3 and Sec. 4.1
 *   straight line        Sec. 3.4.1, Eq. 3.3
 *   exact refraction     Sec. 3.4.3, Eq. 3.17-3.18
 *   photon generation    Sec. 4.2 and 4.2.1
 *   absorption           Sec. 4.3.1
 *   correction tables    Sec. 4.4.1 ("interpolation tracing")
 *   GPU pipeline         Sec. 5.3 (import, generate, filter, propagate, store)
 *   Snell vector stepper Sec. 3.4.2, Eq. 3.15 (the general-atmosphere tracer)
 *   fluorescence         Sec. 2.2.2, Eq. 2.6 and Sec. 4.2.2
 *   LV1 / LV3 filters    Sec. 4.3.2, 4.3.4 and 6.2
 *   mirror and camera    Sec. 6.4 (last-mile ray tracing)
 *
 * Conventions.  Lengths in metres, times in seconds, heights above sea level
 * on the z axis, the detector frame's origin at the array centre.  All calls
 * return a cs_status; no C++ exception crosses this boundary.  Handles are
 * immutable after creation and may be shared between host threads and CUDA
 * streams; the calls themselves are not re-entrant on one output buffer.
 * A call that fails with CS_ERR_CUDA leaves a message in cs_last_error().
 */
#ifndef CHERENKOV_H
#define CHERENKOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cs_status {
    CS_OK = 0,
    CS_ERR_INVALID_ARG = 1,   /* a NULL pointer, a size or a parameter out of range */
    CS_ERR_CUDA = 2,          /* a CUDA runtime call failed; see cs_last_error() */
    CS_ERR_CAPACITY = 3,      /* more photon records than record_capacity (counts stay valid) */
    CS_ERR_TIMEOUT = 4,       /* a bounded device wait gave up */
    CS_ERR_DOMAIN = 5,        /* a table or network was asked outside its domain */
    CS_ERR_NO_DEVICE = 6      /* no CUDA device of compute capability 10.3 */
} cs_status;

/* Human-readable name of a status code (static storage). */
const char* cs_status_string(cs_status s);
/* Message of the last CS_ERR_CUDA on the calling thread (static storage). */
const char* cs_last_error(void);

/* ------------------------------------------------------------------------
 * Charged track segment, 64 bytes, array-of-structs at the boundary.
 *
 * The thesis's GPU segment (Sec. 5.3.1) carries position, direction, mass,
 * energy, charge and age; mass and energy are folded here into 1/gamma^2
 * (the thesis folds them into a "light yield parameter"), and a length is
 * carried because a segment is a start point plus a straight step.
 * A segment is skipped and counted as invalid if any field is not finite,
 * length <= 0, inv_gamma2 is not in (0, 1), uz >= 0.99, |u|^2 differs from
 * 1 by more than 1e-4, or shower_id >= the detector's n_showers.
 * ---------------------------------------------------------------------- */
typedef struct cs_segment {
    double x0, y0, z0;   /* start point [m] */
    double t0;           /* time at the start point [s] (e.g. since the first interaction) */
    float ux, uy, uz;    /* unit direction of motion */
    float length;        /* [m] */
    float inv_gamma2;    /* 1 / gamma^2 of the particle */
    float charge;        /* charge number z (only z^2 enters) */
    uint32_t shower_id;  /* selects the per-shower histogram and telescope counters */
    uint32_t flags;      /* reserved, 0 */
} cs_segment;

/* ------------------------------------------------------------------------
 * Atmosphere.
 * ---------------------------------------------------------------------- */
enum {
    CS_GEOM_PLANAR = 0,      /* n depends on z only, ground is the plane z = h_obs (Sec. 3.3.2) */
    CS_GEOM_SPHERICAL = 1,   /* n depends on the altitude |x - c| - R_E, c = (0, 0, -R_E); the ground is the
                                sphere of radius R_E + h_obs (Sec. 3.3.4) */
    CS_GEOM_CYLINDRICAL = 2  /* Sec. 3.3.3: the index gradient leans in zenith only, inside the vertical
                                plane through the array centre and the emission point E.  Per photon the
                                atmosphere is a set of cylinders coaxial with the horizontal line through
                                c normal to that plane (e_a = z x e_r, e_r the horizontal unit from the
                                centre towards E's foot, the x axis when E lies above the centre); n
                                depends on the distance rho from that axis (altitude rho - R_E).  The
                                ground is the cylinder rho = R_E + h_obs, unrolled onto the array's plane:
                                its point at angle chi from the centre's vertical and axial offset a has
                                the coordinates (R_E + h_obs) chi e_r + a e_a, and arrival directions keep
                                their components along the unrolled tangent, axis and normal.  Traced by
                                the Snell stepper only (cs_opts.tracer = CS_TRACER_SNELL; the correction
                                tables serve the plane and the sphere), without the LV1/LV3 filters or a
                                surrogate; the detector must use this geometry too */
};

enum {
    CS_ATM_LAYERED = 0,      /* CORSIKA-style layers: T(h) = a + b exp(-h/c), top layer linear */
    CS_ATM_LINEAR = 1,       /* n falls linearly from lin_n0 at lin_h0 to lin_n1 at lin_h1 (Sec. 6.3.1) */
    CS_ATM_HOMOGENEOUS = 2,  /* constant n = 1 + hom_delta (Sec. 3.3.1) */
    CS_ATM_TABLE = 3         /* a user's n(h) table (Sec. 3.3): n - 1 at ascending node heights,
                                log-linear between nodes, the first interval's law below the first
                                node, vacuum at and above the last node (the top); density
                                1.225e-3 g/cm^3 * (n - 1) / kappa for the transmission stage */
};

typedef struct cs_atmosphere_desc {
    int kind;                    /* CS_ATM_* */
    int n_layers;                /* layered: 1..8 */
    const double* layer_h;       /* layered: layer bottoms [m], ascending (host, n_layers) */
    const double* layer_a;       /* layered: a_i [g/cm^2] */
    const double* layer_b;       /* layered: b_i [g/cm^2] */
    const double* layer_c;       /* layered: c_i [cm]; the top layer has T = a - b h / c */
    double h_top;                /* layered: top of the atmosphere [m]; vacuum above */
    double kappa;                /* layered: n - 1 = kappa rho(h) / rho(0), e.g. 2.9e-4 */
    double lin_h0, lin_h1, lin_n0, lin_n1;   /* linear kind */
    double hom_delta;            /* homogeneous kind: n - 1 */
    double h_obs;                /* observation level [m] */
    double lambda_min, lambda_max;   /* wavelength band [m], e.g. 300e-9 .. 600e-9 */
    int refraction;              /* 0: straight line (Eq. 3.3); 1: exact planar refraction via tables */
    int transmission;            /* 0: off; 1: Rayleigh + exponential aerosol survival test */
    double rayl_X0, rayl_lambda0;    /* Rayleigh length X_R = X0 (lambda / lambda0)^4 [g/cm^2] */
    double aer_tau0, aer_lambda0, aer_alpha, aer_H;  /* aerosol depth tau0 (lambda/lambda0)^-alpha per scale height aer_H [m] */
    double theta_max;            /* table domain: largest tabulated zenith [rad]; steeper photons (and
                                    photons emitted above the table top) take the exact path, integrated
                                    per photon by the exact pass; 0 = 75 deg */
    int table_nw;                /* 0 = default number of tan^2(theta) columns */
    double table_dh;             /* 0 = default row spacing [m]; must divide the layer bottoms - h_obs */
    int geometry;                /* CS_GEOM_PLANAR, CS_GEOM_SPHERICAL or CS_GEOM_CYLINDRICAL */
    double earth_radius;         /* spherical, cylindrical: R_E [m]; 0 = 6,370 km */
    int table_n;                 /* CS_ATM_TABLE: 2 .. 128 nodes */
    const double* table_h;       /* CS_ATM_TABLE: node heights [m], strictly ascending; host, read during
                                    the call only */
    const double* table_delta;   /* CS_ATM_TABLE: n - 1 at the nodes, > 0 */
} cs_atmosphere_desc;

typedef struct cs_atmosphere cs_atmosphere;

/* Builds the atmosphere on the current CUDA device: its FP64 refraction,
 * time-delay, slant-column and aerosol tables (Sec. 4.4.1) are integrated on
 * the GPU in FP64 and stored as FP32.  The descriptor's arrays are read
 * during the call only.  Errors: CS_ERR_INVALID_ARG for inconsistent
 * parameters, CS_ERR_CUDA / CS_ERR_NO_DEVICE for device failures. */
cs_status cs_atmosphere_create(const cs_atmosphere_desc* desc, cs_atmosphere** out);
void cs_atmosphere_destroy(cs_atmosphere* atm);

/* Shape of the correction table: rows h_obs + j dh (j < nh), columns
 * tan^2(theta0) = m dw (m < nw). */
cs_status cs_atmosphere_table_info(const cs_atmosphere* atm, int* nh, int* nw, double* h0,
                                   double* dh, double* dw);
/* Copies the table to host memory: nh * nw * 8 floats, row-major, per node
 * {G_R, G_t, G_X, G_A at h_j from above, the same four at h_j+1 from below
 * minus those at h_j}.  For a photon emitted at h_j with (local) zenith
 * theta0: G_R = D cos^3(theta0) / sin(theta0), D the ground displacement of
 * the refracted path beyond the straight line (on the sphere: the arc length
 * on the ground sphere); G_t = c dt cos(theta0), dt its delay beyond the
 * straight line; G_X = X cos(theta0), X the slant density column [g/cm^2]
 * along the path; G_A = A cos(theta0), A = the path integral of
 * exp(-h / aer_H) [m]. */
cs_status cs_atmosphere_copy_table(const cs_atmosphere* atm, float* host_dst, size_t n_floats);

/* ------------------------------------------------------------------------
 * Detector: per-shower ground histograms and telescope spheres.
 * ---------------------------------------------------------------------- */
typedef struct cs_detector_desc {
    int n_showers;               /* >= 1: number of per-shower output slots */
    double h_obs;                /* observation level [m]; must equal the atmosphere's at propagation */
    int hist_nx, hist_ny;        /* 0 = no histogram */
    double hist_x0, hist_y0;     /* lower-left corner [m] */
    double hist_dx, hist_dy;     /* cell size [m] */
    int n_tel;                   /* 0 = no telescopes */
    const double* tel_xyzr;      /* host, n_tel x {x, y, z, radius} [m] */
    int geometry;                /* CS_GEOM_SPHERICAL: histogram and telescope (x, y) are azimuthal-
                                    equidistant ground coordinates about the array centre (0, 0, h_obs),
                                    telescope z is the height above the ground sphere plus h_obs;
                                    CS_GEOM_CYLINDRICAL: (x, y) are the unrolled ground cylinder's
                                    coordinates and z the height above it plus h_obs, every photon tested
                                    in its own cylinder's unrolled frame; must match the atmosphere */
    double earth_radius;         /* spherical, cylindrical: R_E [m]; 0 = 6,370 km */
    /* Last-mile optics (Sec. 6.4), cam_n > 0 to enable: every telescope is a parabolic mirror of
     * diameter mirror_d and focal length focal_f whose vertex lies focal_f / 2 behind the sphere
     * centre along the optical axis (pointing at zenith point_zenith, azimuth point_azimuth [rad],
     * frame coordinates), with a flat camera disc of radius camera_r at the focus that also shadows
     * the mirror; photons reaching the camera are binned into cam_n x cam_n square pixels over the
     * camera's square (pixel iy * cam_n + ix, x along a x z-hat, y along a x x).  Every sphere must
     * hold its instrument: radius >= sqrt((mirror_d / 2)^2 + (focal_f / 2)^2). */
    double mirror_d, focal_f, camera_r;
    double point_zenith, point_azimuth;
    int cam_n;
    /* Absorption in those optics (Sec. 6.4): a photon that reaches a camera pixel survives the
     * mirror's reflectivity R(lambda) and the camera's photon detection efficiency eps(lambda)
     * with probability R eps, each linear between eff_n <= 16 nodes (eff_lambda_nm [nm]
     * ascending, values in [0, 1]; constant beyond the end nodes); a photon that does not
     * survive still counts as a telescope hit but adds nothing to the camera image.  The
     * survival draw is Philox word x of counter (segment, sub-step, bunch index | 2^30).
     * eff_n = 0 (default): no absorption. */
    int eff_n;
    const double* eff_lambda_nm;
    const double* eff_mirror;
    const double* eff_camera;
} cs_detector_desc;

typedef struct cs_detector cs_detector;

/* The detector of the thesis's pipeline (Sec. 5.3 "store"; Sec. 6.2 bounding
 * spheres of the telescopes; App. B.3 the detector layouts): copies the layout to
 * the device and builds its telescope grid hash.  A photon hits telescope i if its
 * arrival line passes within radius_i of the sphere's centre; the closest centre
 * wins, then the lowest index.  Errors: CS_ERR_INVALID_ARG (NULL or inconsistent
 * description), CS_ERR_CUDA. */
cs_status cs_detector_create(const cs_detector_desc* desc, cs_detector** out);
void cs_detector_destroy(cs_detector* det);

/* ------------------------------------------------------------------------
 * Outputs.  All counts are in photons (each bunch adds its bunch size).
 * ---------------------------------------------------------------------- */
enum {
    CS_CNT_EMITTED = 0, CS_CNT_ABSORBED = 1, CS_CNT_HIST = 2, CS_CNT_TEL = 3,
    CS_CNT_MISSED_HIST = 4, CS_CNT_MISSED_TEL = 5, CS_CNT_UPWARD = 6,
    CS_CNT_INVALID_SEGMENTS = 7,      /* in segments, not photons */
    CS_N_COUNTERS = 8
};
/* Conservation: emitted = absorbed + hist + missed_hist = absorbed + tel + missed_tel. */

/* Bunch statuses.  CS_ST_NO_GROUND: a descending bunch whose exact path never
 * meets the observation level (on the spherical shell it passes over the ground
 * sphere, Bouguer's n r sin(psi) exceeding n r at the ground; in the plane an
 * inverted n(h) profile turns it back up); it counts as missed.  Every other
 * descending bunch emitted above the observation level is propagated: inside the
 * correction tables' domain by the tables, beyond it (steeper zenith, or emitted
 * above the tables' top) by the exact path integrated for that bunch. */
enum { CS_ST_LANDED = 0, CS_ST_UPWARD = 1, CS_ST_BELOW = 2, CS_ST_NO_GROUND = 3, CS_ST_ABSORBED = 4, CS_ST_LV3 = 5 };

/* Optional per-bunch record (parity mode), 56 bytes.  Records are written in
 * no particular order; (seg, k, i) identifies a bunch uniquely.  The ground
 * position is a float-float pair (x + x_lo, y + y_lo): a single float would
 * round it to ~2 mm at 30 km from the frame origin, coarser than the
 * per-photon bar for photons that travel a short way far out. */
typedef struct cs_record {
    uint64_t seg;        /* global segment index (seg_base + position in the input) */
    uint32_t k;          /* sub-step index */
    uint32_t i;          /* bunch index within the sub-step */
    float x, y;          /* ground position [m] (landed and absorbed bunches), leading part */
    float dt_ns;         /* arrival time minus the segment's t0 [ns] */
    float lambda_nm;     /* wavelength [nm] */
    int32_t tel;         /* telescope hit or -1 */
    int32_t bin;         /* histogram cell iy * nx + ix or -1 */
    uint32_t status;     /* CS_ST_* */
    int32_t pix;         /* camera pixel iy * cam_n + ix of the telescope hit, or -1 */
    float x_lo, y_lo;    /* trailing parts of the ground position [m] */
} cs_record;

typedef struct cs_output {
    uint64_t* hist;          /* n_showers x hist_ny x hist_nx, or NULL if no histogram */
    uint64_t* tel_counts;    /* n_showers x n_tel, or NULL if no telescopes */
    double* tel_time;        /* n_showers x n_tel: sum over hits of bunch size x absolute arrival
                                time [s], accumulated in FP64; NULL allowed */
    uint64_t* counters;      /* CS_N_COUNTERS */
    cs_record* records;      /* NULL: throughput mode (no per-bunch output) */
    uint64_t record_capacity;
    uint64_t* record_count;  /* 1 element: records produced (may exceed the capacity) */
    uint64_t* camera;        /* n_showers x n_tel x cam_n x cam_n camera images (photons), or NULL;
                                required when the detector has optics */
} cs_output;

typedef struct cs_surrogate cs_surrogate;

typedef struct cs_opts {
    int bunch;               /* photons per bunch, >= 1 */
    double s_max;            /* maximum sub-step length [m] (Sec. 4.2.1), > 0 */
    uint64_t seg_base;       /* global index of segs[0]; keys the random draws */
    int device_ptrs;         /* 0: segs and all output arrays are host memory; 1: device memory */
    int accumulate;          /* 0: outputs are zeroed before the call; 1: added to */
    int block_threads;       /* 0 = default */
    int blocks_per_sm;       /* 0 = default */
    const cs_surrogate* surrogate;  /* NULL: exact tracer (tables); else the network replaces the
                                       refraction/time/transmission lookups inside its domain */
    /* LV1 particle filter (Sec. 4.3.2, with the two-parameter cut of Sec. 6.2.1): a
     * segment whose start lies y [m] above h_obs (on the sphere: altitude) and whose
     * direction makes the angle x [deg] (clamped to >= 1e-3) with the point of
     * interest is dropped before any photon is generated when y >= lv1_a x^lv1_b.
     * The cut is fitted per detector (the package's lv1.fit_cut). */
    int lv1_metric;          /* CS_LV1_OFF (default), CS_LV1_ARRAY_CENTRE, CS_LV1_ARRAY_DISC,
                                CS_LV1_TELESCOPES */
    double lv1_a, lv1_b;
    double lv1_centre[3];    /* array centre in the frame [m] (centre and disc metrics) */
    double lv1_radius;       /* disc radius [m] (disc metric) */
    uint64_t* lv1_dropped;   /* NULL or one counter in the outputs' memory kind: dropped segments are
                                added (zeroed first unless accumulate) */
    /* LV3 photon pre-filter (Sec. 4.3.4, 6.2.2): after the straight line and before the
     * refraction correction, a photon whose vacuum straight line lands farther than
     * lv3_radius + lv3_margin from lv3_centre (3-D distance, frame coordinates; on the
     * plane the landing point lies at h_obs) is dropped: status CS_ST_LV3, counted as
     * missed by the histogram and the telescopes, no lookup, transmission or detection.
     * Detector counts are unchanged when the disc holds the histogram and the telescope
     * spheres and the margin covers the largest correction displacement. */
    int lv3;                 /* 0 (default) off, 1 on */
    double lv3_centre[3];
    double lv3_radius, lv3_margin;   /* >= 0 [m] */
    /* Propagation method when the atmosphere refracts: CS_TRACER_TABLES (default) looks
     * the correction up in the FP64-built tables (interpolation tracing, Sec. 4.4.1);
     * CS_TRACER_SNELL traces every photon through homogeneous slabs (on the spherical
     * shell: shells; in the cylindrical atmosphere: coaxial cylinders) of thickness
     * <= tracer_dh [m], >= 0.01 m, with Snell's law in vector form (Sec. 3.4.2, Eq. 3.15)
     * and accumulates its delay and slant columns on the way (the general-atmosphere
     * fallback; the exact path only: CS_ERR_INVALID_ARG with a surrogate).  Ignored when
     * the atmosphere does not refract, except in the cylindrical atmosphere, which it
     * traces always (with n = 1 in the geometry when refraction is off). */
    int tracer;
    double tracer_dh;
    /* Emission (Sec. 2.2.2, 4.2.2): CS_EMIT_CHERENKOV (default), or nitrogen fluorescence,
     * isotropic (CS_EMIT_FLUORESCENCE) or into the downward half sphere with half the photons
     * (CS_EMIT_FLUORESCENCE_HALF).  Fluorescence yield (Eq. 2.6) per metre of track:
     * z^2 fl_dedx [MeV cm^2/g] rho(h) [g/cm^3] 100 sum_l fl_yield_per_mev[l], rho from the
     * atmosphere's density law (zero for the linear and homogeneous kinds); each bunch takes
     * line l with probability fl_yield_per_mev[l] / sum (up to 8 lines, fl_lines_nm [nm]).
     * Every propagation method, filter and detector applies, except the LV1 cut
     * (CS_ERR_INVALID_ARG): isotropic light cannot be filtered by direction. */
    int emission;
    int fl_n_lines;
    const double* fl_lines_nm;
    const double* fl_yield_per_mev;
    double fl_dedx;
    /* Polls of each tensor-core completion wait of the surrogate network before the
     * kernel gives up on it: 0 (default) = 2^20; < 0 = no poll at all (the wait gives up at
     * once, which exercises the give-up path).  A warpgroup whose wait gives up stops using
     * the network: its photons take the correction tables, so the counts stay valid, and
     * the call reports CS_ERR_TIMEOUT (host-pointer calls directly, device-pointer and
     * streamed calls through cs_check_timeout). */
    int tc_poll_limit;
    /* Bunches beyond the correction tables are queued by the photon kernel for the exact pass:
     * entries per warp tile of 32 segments (0 = default 8; at least 4096 and at most 2^22
     * entries in all, and at most the default in the batched and streamed calls; < 0 = no
     * queue).  When the queue is full the remaining such bunches mark their warp tile, which
     * the exact pass then regenerates whole; the results are the same either way. */
    int exact_queue;
} cs_opts;

enum { CS_EMIT_CHERENKOV = 0, CS_EMIT_FLUORESCENCE = 1, CS_EMIT_FLUORESCENCE_HALF = 2 };

enum { CS_TRACER_TABLES = 0, CS_TRACER_SNELL = 1 };

/* The LV1 filter's point of interest: x is the angle from the segment's
 * direction to the array centre, to a sphere of lv1_radius about it (0 inside),
 * or the smallest such angle to the telescope spheres (a loop over all
 * telescopes per segment: for arrays of up to a few hundred). */
enum {
    CS_LV1_OFF = 0,
    CS_LV1_ARRAY_CENTRE = 1,
    CS_LV1_ARRAY_DISC = 2,
    CS_LV1_TELESCOPES = 3
};

/* Defaults: bunch 1, s_max 1 m, seg_base 0, host pointers, no accumulation, no
 * LV1 or LV3 filter, the table tracer (tracer_dh 10 m for the Snell stepper). */
void cs_opts_default(cs_opts* opts);

/* Synchronises the current device and reports whether a tensor-core wait of the
 * surrogate network gave up in a propagation call (device-pointer, batched or
 * streamed) since the last check: CS_ERR_TIMEOUT if so (the flag is cleared; the
 * affected photons took the correction tables, so that call's counts are valid),
 * CS_OK otherwise, CS_ERR_CUDA if the synchronisation fails.  Host-pointer calls
 * check this themselves. */
cs_status cs_check_timeout(void);

/* Generates and propagates the photons of n segments (Sec. 5.3 pipeline).
 * Random draws are keyed by (seed, global segment index, sub-step, bunch),
 * so any split of the input into calls gives identical totals.
 * Host-pointer mode copies segs to the device, runs, copies the outputs
 * back and synchronises.  Device-pointer mode enqueues everything on
 * `stream` (a cudaStream_t, NULL = legacy default stream) and returns
 * without synchronising; outputs must not be read before the stream is.
 * Errors: CS_ERR_INVALID_ARG (NULL handles/outputs, bad options),
 * CS_ERR_CAPACITY (host mode only: more records than the capacity),
 * CS_ERR_CUDA. */
cs_status cs_propagate(const cs_segment* segs, size_t n, const cs_atmosphere* atm,
                       const cs_detector* det, uint64_t seed, cs_output* out);
cs_status cs_propagate_ex(const cs_segment* segs, size_t n, const cs_atmosphere* atm,
                          const cs_detector* det, uint64_t seed, const cs_opts* opts,
                          cs_output* out, void* stream);

/* ------------------------------------------------------------------------
 * Batched uneven showers: many showers of uneven size in one persistent
 * launch (warps take tiles of 32 segments -- blocks tiles of 256 with the
 * surrogate -- from a work counter until the batch is done), captured once
 * into a CUDA graph and replayed.  The thesis
 * batches tens of thousands of tracks per kernel call (Sec. 5.1, 5.4).
 * ---------------------------------------------------------------------- */
typedef struct cs_batch cs_batch;

/* Captures [output zeroing unless opts->accumulate, work-counter reset,
 * kernel] for these device buffers into a graph.  Device pointers only
 * (opts->device_ptrs must be 1).  shower_bunch: host array of n_showers
 * bunch sizes (>= 1), or NULL to use opts->bunch for every shower.  The
 * buffers must stay valid and are re-read at every launch.  Errors:
 * CS_ERR_INVALID_ARG, CS_ERR_CUDA. */
cs_status cs_batch_create(const cs_segment* segs, size_t n, const cs_atmosphere* atm, const cs_detector* det,
                          uint64_t seed, const int* shower_bunch, const cs_opts* opts, cs_output* out,
                          cs_batch** out_batch);
/* Replays the captured graph on `stream` (cudaStream_t). */
cs_status cs_batch_launch(cs_batch* batch, void* stream);
void cs_batch_destroy(cs_batch* batch);

/* ------------------------------------------------------------------------
 * Streaming host segments: chunks of `chunk` segments are copied to the
 * device through two staging buffers on two library-owned streams, so the
 * copy of chunk c overlaps the photon kernel of chunk c - 1 (the thesis's
 * data transfer and batching, Sec. 5.1 and 5.4).  Every chunk's draws are
 * keyed by its global segment index, so the result equals one call over all
 * segments.
 * ---------------------------------------------------------------------- */
typedef struct cs_streamer cs_streamer;

/* Allocates two device buffers of `chunk` segments (1 <= chunk <= 2^32) and
 * two streams on the current device.  Errors: CS_ERR_INVALID_ARG,
 * CS_ERR_CUDA. */
cs_status cs_streamer_create(size_t chunk, cs_streamer** out);
/* Propagates n segments from host memory `host_segs` (page-locked memory for
 * the copies to overlap the kernels; pageable memory works without overlap).
 * The outputs in `out` are device memory and opts->device_ptrs must be 1;
 * they are zeroed first on `stream` unless opts->accumulate.  Chunk c is
 * keyed from opts->seg_base + c * chunk.  Enqueues only: the work starts
 * after what is already queued on `stream` (cudaStream_t, NULL = legacy
 * default stream) and `stream` waits for all of it, so read the outputs
 * after synchronising `stream`.  Calls on one streamer must not overlap
 * (they share its buffers).  Errors: CS_ERR_INVALID_ARG (NULL arguments,
 * host outputs, another device), CS_ERR_CUDA. */
cs_status cs_streamer_run(cs_streamer* s, const cs_segment* host_segs, size_t n, const cs_atmosphere* atm,
                          const cs_detector* det, uint64_t seed, const cs_opts* opts, cs_output* out,
                          void* stream);
/* Waits for the streamer's work and frees it. */
void cs_streamer_destroy(cs_streamer* s);

typedef struct cs_tune_result {
    int blocks_per_sm;   /* fastest resident blocks per SM (256 threads each) */
    int n_tried;
    float ms[8];         /* mean kernel time per tried setting, index blocks_per_sm - 1 */
} cs_tune_result;

/* Times 1..4 resident blocks per SM on this batch (3 timed runs each after a
 * warm-up, CUDA events on `stream`) and returns the fastest.  Overwrites the
 * outputs.  Device pointers only. */
cs_status cs_autotune_tiling(const cs_segment* segs, size_t n, const cs_atmosphere* atm, const cs_detector* det,
                             uint64_t seed, const int* shower_bunch, const cs_opts* opts, cs_output* out,
                             void* stream, cs_tune_result* result);

/* Per-shower bunch sizes: a pilot run with the largest allowed bunch gives
 * each shower's mean photon count c over its 100 densest ground cells;
 * bunching multiplies a cell's variance by b, so the shower gets the largest
 * allowed b with sqrt(b / c) <= rel_noise (else the smallest allowed).  Needs
 * a ground histogram; overwrites the outputs; shower_bunch is a host array of
 * n_showers.  Device pointers only. */
cs_status cs_autotune_bunches(const cs_segment* segs, size_t n, const cs_atmosphere* atm, const cs_detector* det,
                              uint64_t seed, double rel_noise, const int* allowed, int n_allowed,
                              const cs_opts* opts, cs_output* out, void* stream, int* shower_bunch);

/* ------------------------------------------------------------------------
 * Learned surrogate of the refraction integral (no thesis counterpart; the
 * thesis's interpolation tracer of Sec. 4.4.1 is what it replaces).  A tanh
 * MLP 3 -> 64 -> 64 -> 64 -> 3 maps (emission height, cos(zenith),
 * 1/wavelength) to the displacement field G_R, the delay field G_t and the
 * transmission T.  Training samples have uniform height in [h_min, h_max],
 * uniform zenith in [0, theta_max] and uniform wavelength in the atmosphere's
 * band (minus bands around the layer boundaries, where n(h) and hence the
 * exact fields are discontinuous), labelled by the FP64 quadrature of the
 * exact path.  The network learns the fields less their first-order
 * expansion in n - 1 (I = int (n - 1) dh over [h_obs, h_e], H = h_e - h_obs,
 * mu = cos(zenith): G_R = d_e H - I, G_t = 2 I - d_e H + (d_e H - I) / mu^2,
 * ln T from the vertical slant columns over mu), which is added back at
 * inference from a table of the FP64 vertical integrals.  Hidden layers run
 * on the tensor cores (BF16 weights, FP32 accumulation); the 3-input layer
 * runs in FP32.  Outside its domain the photon kernel uses the tables.
 * ---------------------------------------------------------------------- */
typedef struct cs_surrogate_config {
    int n_train;             /* training samples (default 2^20) */
    int n_heldout;           /* held-out samples (default 2^16) */
    int batch;               /* mini-batch (default 32768) */
    int epochs;              /* passes over the training set (default 1600) */
    uint64_t seed;
    double lr, lr_min;       /* Adam learning rate (default 1e-2), cosine-decayed to lr_min (1e-5) */
    double h_min, h_max;     /* emission heights [m] (default 2 km .. 30 km) */
    double theta_max;        /* largest zenith [rad] (default 60 deg) */
    int split_activations;   /* 1: hidden activations enter the MMAs as BF16 hi + lo pairs after an accurate
                                tanh; 0: as single BF16 values through the hardware's packed BF16 tanh
                                (default: fewer instructions and MMAs; the network only adds a correction
                                to the first-order baseline) */
    double boundary_band;    /* half-width [m] of the bands around layer boundaries left to the tables
                                (the exact fields jump there with n(h_e)); default 500 m */
    double height_scale;     /* > 0: the height enters as exp(-(h - h_obs) / height_scale) (default
                                8 km, the fields are nearly linear in this density-like coordinate);
                                0: linear in h */
} cs_surrogate_config;

typedef struct cs_surrogate_stats {
    double heldout_p99[3];   /* held-out 99th percentile |error|: displacement [m], delay [s], transmission */
    double heldout_max[3];   /* held-out maximum |error|, same order */
    double final_loss;       /* MSE of the last mini-batch (normalised targets) */
    int steps;
    double train_seconds;
} cs_surrogate_stats;

void cs_surrogate_config_default(cs_surrogate_config* cfg);
/* Samples, labels and trains on the device of `atm` (which must have
 * refraction on); errors against the held-out set go to *stats. */
cs_status cs_surrogate_train(const cs_atmosphere* atm, const cs_surrogate_config* cfg, cs_surrogate** out,
                             cs_surrogate_stats* stats);
void cs_surrogate_destroy(cs_surrogate* s);
/* Runs the network (the photon kernel's inference code) on device float4
 * inputs {h_e - h_obs [m], cos(theta0), 1/lambda [1/nm], unused}; writes
 * float4 {G_R [m], G_t [m], T, 0}.  16-byte aligned device pointers. */
cs_status cs_surrogate_eval(const cs_surrogate* s, const float* d_in, size_t n, float* d_out, void* stream);
/* The same on the network's own part: float4 {G_R, G_t, ln T} less the
 * first-order baseline (the de-normalised network outputs), for checking the
 * tensor-core arithmetic against a plain forward pass. */
cs_status cs_surrogate_eval_network(const cs_surrogate* s, const float* d_in, size_t n, float* d_out, void* stream);
/* Host copies of the parameters as inference uses them (flat FP32, the
 * tensor-core weights already rounded to BF16; layout W1[64][3] b1[64]
 * W2[64][64] b2 W3[64][64] b3 W4[8][64] b4[8]), the training statistics, and
 * 15 normalisation floats (input scale[3], shift[3], output half-range[3],
 * mid[3], dz_min, dz_max, cos(theta_max)).  Any pointer may be NULL. */
cs_status cs_surrogate_info(const cs_surrogate* s, float* params, size_t n_params, cs_surrogate_stats* stats,
                            float* norm);
/* One forward and backward pass of the training path on B rows (host
 * arrays: params in the layout above, x and t B x 3 normalised): the loss
 * (1/B) sum (y - t)^2 and its gradient (host, same layout).  For checking
 * the tensor-core training kernels against a reference. */
cs_status cs_mlp_loss_grad(const float* params, const float* x, const float* t, int B, float* grad, float* loss);

/* Allocation-free form of the device-pointer call (the thesis has no
 * counterpart; this is a library service).  For callers that cannot let the
 * library allocate device memory: code running while a memory pool or arena
 * owns the device, real-time or embedded hosts that allow no allocation after
 * start-up, callers that must account for every byte in advance.  It does
 * what cs_propagate_ex does with opts->device_ptrs = 1 (opts must say so;
 * host pointers are rejected with CS_ERR_INVALID_ARG), but its only scratch,
 * the dynamic scheduler's work counters and the exact pass's map and list of
 * warp tiles with bunches beyond the correction tables (no bunch queue: the
 * exact pass regenerates the marked tiles), lives in a 67.6 KB array
 * that the library declares statically on every device that loads it (held
 * until the process exits) instead of in memory the library allocates.  It
 * calls no cudaMalloc, cudaFree or pool allocation.
 * Limits and rules: 32-bit counters, so inputs needing 2^32 - 65537 or more
 * warp tiles of 32 segments (about 1.37e11 segments) are rejected with
 * CS_ERR_INVALID_ARG; the map holds 2^14 groups, each of ceil(tiles / 2^14)
 * warp tiles.  The first call on a device looks up the array's device address,
 * so make that first call before any stream capture.  Every call reuses the
 * same array and clears it on its stream before the kernels; two calls whose
 * work overlaps on the GPU (different streams, or different host threads) race
 * on it and give wrong results, so serialise them. */
cs_status cs_propagate_noalloc(const cs_segment* segs, size_t n, const cs_atmosphere* atm,
                               const cs_detector* det, uint64_t seed, const cs_opts* opts,
                               cs_output* out, void* stream);

/* Philox4x32-10 (Salmon et al. 2011) on the device, for bit-exact checks:
 * out[4 j .. 4 j + 3] = philox(ctr[4 j .. 4 j + 3], key).  Device pointers,
 * enqueued on `stream`. */
cs_status cs_philox4x32_10(const uint32_t* ctr, size_t n, uint32_t key0, uint32_t key1,
                           uint32_t* out, void* stream);

/* Number of SMs of the current device (for grid sizing by callers). */
cs_status cs_device_sm_count(int* n_sm);

#ifdef __cplusplus
}
#endif
#endif /* CHERENKOV_H */
