/* helios_oracle.h - FP64 CPU oracle of the per-pulse beam-scene interaction.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference the
 * CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference arm of bench.py may load it.  It shares no source,
 * header, table or helper with the CUDA library (include/helios.h and
 * paper_2101_09154_gb300/csrc never include this file, and this file never
 * includes theirs).
 *
 * Every quantity is computed in IEEE double precision.  Inputs arrive as the
 * same FP32 arrays the GPU receives and are promoted on entry.
 */
#ifndef HELIOS_ORACLE_H
#define HELIOS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double prf_hz;
    double divergence_rad;       /* full angle at the 1/e^2 points (Sec. 3.4, Fig. subrays) */
    int32_t quality;             /* beamSampleQuality q: number of subray rings */
    int32_t pulse_shape;         /* 0 Gaussian (FWHM), 1 Eq. beam_time (t/tau)^2 e^{-t/tau} */
    double wavelength_m, beam_waist_m, focus_m;
    double peak_power_w, receiver_diam_m, eta_sys, eta_atm;
    double pulse_fwhm_ns, pulse_length_ns, bin_ns;
    int32_t n_bins, max_echoes;
    double echo_threshold_rel, range_noise_sigma_m;
    int32_t deflector, grid_n_az, grid_n_el, n_fibres;   /* n_fibres: deflector 4 */
    double scan_freq_hz, scan_angle_max_rad, head_rate_rad_s, el_min_rad, el_max_rad;
} or_scanner;

typedef struct {
    int32_t platform;            /* 0 static, 1 linear path */
    int32_t quality;             /* -1: the scanner's */
    uint32_t leg_id;
    int32_t pad0;
    double start[3], end[3];
    double speed_mps;
    double attitude_rpy[3];
    double t0;
    int64_t n_pulses;
    double platform_noise_m;     /* sigma of the per-pulse platform position noise (Sec. 3.7) */
} or_leg;

/* One voxel grid (Sec. 3.5.4).  Voxel (x,y,z) spans origin + [x,x+1)*cell etc. */
typedef struct {
    double origin[3];
    double cell;
    int32_t dims[3];             /* nx, ny, nz */
    int32_t opaque;              /* non-transmissive voxels (Sec. 3.5.4) */
    const float* density;        /* [nz][ny][nx] plant area density */
    double G;                    /* sigma = G * density (no leaf-angle table) */
    double leaf_refl;
    const float* lad;            /* [lad_n] leaf-angle table G(mu) at mu_i = i/(n-1), mu =
                                    |vertical component| of the subray (Eq. extinction, Table
                                    ladlut), linear in between; NULL: the constant G */
    int32_t lad_n, pad;
} or_grid_in;

/* A scene: triangles of all meshes, and voxel grids whose boxes have disjoint
 * interiors.  Voxel ids: n_tri + (voxels of the earlier grids) + (z*ny + y)*nx + x. */
typedef struct {
    int64_t n_tri;
    const float* tri;            /* [n_tri][3][3] vertex coordinates */
    const float* refl;           /* [n_tri] Lambertian reflectance */
    int32_t n_grids, pad0;       /* at most OR_MAX_GRIDS */
    const or_grid_in* grids;
} or_scene_in;

#define OR_MAX_GRIDS 4096

typedef struct or_scene or_scene;

typedef struct {
    int32_t* window_bin;         /* [n]        first bin index m of the window, OR_NO_WINDOW: no return */
    double* waveform;            /* [n][n_bins] */
    int32_t* echo_count;         /* [n] */
    int32_t* echo_bin;           /* [n][K]     bin within the window */
    double* echo_amp;            /* [n][K] */
    double* echo_range;          /* [n][K]     with range noise */
    double* echo_range_clean;    /* [n][K]     without noise */
    int64_t* echo_object;        /* [n][K]     primitive id (tri, or n_tri + voxel) */
    double* echo_width;          /* [n][K]     fitted Gaussian sigma (ns); NULL: no fit */
    int64_t* subray_hit;         /* [n][S]     event primitive, -1 none */
    double* subray_range;        /* [n][S] */
    uint32_t* flags;             /* [n]        OR_F_* */
    uint32_t* subray_flags;      /* [n][S]     OR_F_* raised by each subray, or NULL */
    int64_t* echo_object_alt;    /* [n][K]     the runner-up object when within 1e-4 of the
                                    echo object's contribution (OR_F_OBJ), else -1; or NULL */
} or_out;

#define OR_NO_WINDOW   INT32_MIN
#define OR_MAX_ECHOES  64         /* largest max_echoes or_scan accepts */

/* parity flags: conditions under which an FP32 result may legitimately differ */
#define OR_F_EDGE      (1u << 0)  /* a candidate triangle within eps of an edge */
#define OR_F_TIE       (1u << 1)  /* two hits within eps in t */
#define OR_F_VOX       (1u << 2)  /* a transmission decision within eps */
#define OR_F_WIN       (1u << 3)  /* window start within eps of a bin boundary */
#define OR_F_ECHO      (1u << 4)  /* a local-max / threshold decision within tolerance */
#define OR_F_OBJ       (1u << 5)  /* echo object argmax near-tie */
#define OR_F_OVERFLOW  (1u << 8)  /* more echoes than max_echoes */
#define OR_F_NOHIT     (1u << 9)  /* no subray returned */
#define OR_F_FIT       (1u << 10) /* an echo-width fit step decided within tolerance */
#define OR_F_FORCED_BAD (1u << 11) /* a given subray event that no flagged decision allows */

#define OR_FREE_HIT    (-2)       /* force_hit entry: the oracle decides the event */

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_uniform24(uint32_t w);
int or_subray_count(int q);
int or_subray_angles(int q, double theta_r, int s, double* alpha, double* phi);
void or_onb(const double n[3], double u[3], double v[3]);
void or_pulse_ray(const or_scanner* sn, const or_leg* lg, int64_t k, uint64_t seed, double o[3],
                  double d[3]);
void or_subray_dir(const or_scanner* sn, int q, int s, const double d[3], double ds[3]);
double or_beam_width(const or_scanner* sn, double R);
double or_subray_intensity(const or_scanner* sn, double R, double alpha);
double or_pulse_shape(const or_scanner* sn, double t_ns);
/* Echo width (Sec. 3.4, optional output): Gaussian fit to W[0..nb) around the
 * echo at bin p over bins p -/+ ceil(2 sigma_b), sigma_b the emitted pulse's
 * sigma in bins; 10 Levenberg-Marquardt iterations from (W[p], p, sigma_b).
 * Returns the fitted sigma in bins; *near_tie is set when an accept/reject
 * decision on a step of more than 1e-5 s was within 1e-6 of the window's
 * energy (sum of W^2). */
double or_echo_width(const double* W, int nb, int p, double sigma_b, int* near_tie);
double or_triangle_power(const or_scanner* sn, double Is, double R, double refl, double cos_inc);
/* Echoes of one waveform W[0..nb) (Sec. 3.4, local maxima above a threshold):
 * bin b is an echo when W[b] > W[b-1], W[b] >= W[b+1] (W is 0 outside the
 * window), W[b] > 0 and W[b] >= thr_rel * max W.  The first K in bin order go
 * to bins[0..K); *overflow = 1 when there were more; *near = 1 when such a
 * decision was within 1e-4 max W.  Returns the number written. */
int or_echo_peaks(const double* W, int nb, double thr_rel, int K, int32_t* bins, int* overflow,
                  int* near);
/* Echo object: of n returns (power P, range R, primitive id) in summation
 * order, the id with the largest contribution P p(tb - 2R/c) at time tb_ns,
 * the first on equal values; *near = 1 when the two largest are within 1e-4. */
int64_t or_echo_object(const or_scanner* sn, int64_t n, const double* P, const double* R,
                       const int64_t* id, double tb_ns, int* near);

or_scene* or_scene_build(const or_scene_in* in);
void or_scene_free(or_scene* sc);
int64_t or_scene_bvh_nodes(const or_scene* sc);

/* closest hit; returns id (-1 none), t, |cos incidence|, parity flags */
int64_t or_intersect(const or_scene* sc, const double o[3], const double d[3],
                     double* t, double* cos_inc, uint32_t* flags);
int64_t or_intersect_brute(const or_scene* sc, const double o[3], const double d[3],
                           double* t, double* cos_inc);
/* voxels crossed with positive length before t_hi: ids, t_in, t_out; returns count */
int64_t or_march(const or_scene* sc, const double o[3], const double d[3], double t_hi,
                 int64_t cap, int64_t* vid, double* t_in, double* t_out);

/* the returns (range, power, primitive) of one subray from origin o along unit ds */
int64_t or_trace_returns(const or_scene* sc, const or_scanner* sn, const double o[3],
                         const double ds[3], double alpha, int mode, uint64_t seed, uint32_t leg_id,
                         int64_t pulse, int s, int64_t cap, double* R, double* P, int64_t* id,
                         uint32_t* flags);

/* mode 0 stochastic, 1 expected.  fixed_window (nullable) holds the window
 * start per pulse.  force_hit (nullable, [n][S]) gives a subray's event in
 * place of the oracle's search where it is not OR_FREE_HIT: a triangle id,
 * n_tri + voxel (stochastic mode: the voxel the subray stopped in) or -1 (no
 * event); this re-runs a pulse with the choices an FP32 path made on subrays
 * the oracle flagged, and OR_F_FORCED_BAD marks a choice that no flagged
 * decision allows.  n_threads <= 0: all online cores.  Returns -1 (nothing
 * written) when max_echoes is outside 1..OR_MAX_ECHOES. */
int or_scan(const or_scene* sc, const or_scanner* sn, const or_leg* lg,
            const int64_t* pulses, int64_t n, int mode, uint64_t seed,
            const int32_t* fixed_window, const int64_t* force_hit, const or_out* out,
            int n_threads);

/* adjoint of the expected-mode waveform: g = dL/dW [n][n_bins], window held
 * fixed.  Accumulates into d_refl [n_tri] and d_density [nz*ny*nx]. */
int or_adjoint(const or_scene* sc, const or_scanner* sn, const or_leg* lg,
               const int64_t* pulses, int64_t n, const double* g, const int32_t* window,
               double* d_refl, double* d_density, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
