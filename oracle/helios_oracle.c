/* helios_oracle.c - FP64 CPU oracle of the per-pulse beam-scene interaction
 * (HELIOS++, Winiwarter et al.).  TEST INFRASTRUCTURE ONLY: see helios_oracle.h.
 *
 * The method is a simulation, so this file is the algorithm itself, step by
 * step, in the paper's order:
 *   1. pulse k: platform pose (Sec. 3.2) and deflector angle (Sec. 3.3);
 *   2. subrays: a centre ray plus rings i = 1..q of floor(2*pi*i) rays (Sec. 3.4);
 *   3. intersection: nearest triangle (Sec. 5.1) and transmissive voxels with
 *      s = -ln(R)/sigma (Sec. 3.5.4, Eq. intersection_dist; Sec. 5.2);
 *   4. power: Gaussian beam weight (Eq. beamdiv, Eq. beamdiv_w) times the laser
 *      radar equation (Eq. ladlut_intensity) with a Lambertian target;
 *   5. waveform: the sum of the subrays' shifted pulse shapes (Sec. 3.4);
 *   6. echoes: local maxima above a threshold (Sec. 3.4), range noise (Sec. 3.7).
 * Readings where the paper is silent or garbled are stated at each step.
 *
 * The nearest-triangle search uses a plain median-split BVH so that large
 * scenes finish; or_intersect_brute() is the all-triangle definition the BVH
 * is checked against.  Nothing here is blocked, fused or reordered beyond
 * that.
 */
#include "helios_oracle.h"

#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_PI 3.14159265358979323846
#define OR_C 299792458.0 /* speed of light, Sec. 3.4 */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11: "Parallel random      */
/* numbers: as easy as 1, 2, 3").  Replaces the seeded sequential RNG of      */
/* Sec. 3.7 with a counter-based one, so draws do not depend on thread order. */
/* ------------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint32_t h0, l0, h1, l1;
        mulhilo32(M0, x0, &h0, &l0);
        mulhilo32(M1, x2, &h1, &l1);
        uint32_t y0 = h1 ^ x1 ^ k0, y1 = l1, y2 = h0 ^ x3 ^ k1, y3 = l0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* a uniform in (0,1): (top 23 bits + 1/2) * 2^-23, i.e. odd multiples of 2^-24,
 * exactly representable in FP32 too (so both precisions draw the same number) */
double or_uniform24(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Counter (128 bits) of one draw: word 0 = pulse bits 0-31; word 1 = pulse bits
 * 32-43, stream (2 bits) at bit 12, subray or echo index (9 bits) at bit 14,
 * voxel id bits 32-39 at bit 23; word 2 = voxel id bits 0-31; word 3 = leg id.
 * Key = the seed's low and high words.  Pulses < 2^44, voxel ids < 2^40. */
static void draw(uint64_t seed, uint32_t leg, int64_t pulse, uint32_t stream, uint32_t idx,
                 uint64_t sub, uint32_t out[4]) {
    const uint64_t p = (uint64_t)pulse;
    uint32_t c[4] = {(uint32_t)p,
                     ((uint32_t)(p >> 32) & 0xFFFu) | ((stream & 3u) << 12) | ((idx & 0x1FFu) << 14) |
                         (((uint32_t)(sub >> 32) & 0xFFu) << 23),
                     (uint32_t)sub, leg};
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(c, k, out);
}

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static void sub3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2];
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static double eps_rel(double t) { return 1e-6 * (t > 1.0 ? t : 1.0); }

/* ------------------------------------------------------------------------ */
/* 2. subrays (Sec. 3.4): centre + rings i=1..q with floor(2*pi*i) subrays.   */
/* Reading: ring i sits at angle (i/q)*theta_r, theta_r = divergence/2 (the  */
/* half angle at 1/e^2), azimuths 2*pi*j/n_i starting at 0.                  */
/* ------------------------------------------------------------------------ */
static int ring_n(int i) { return (int)floor(2.0 * OR_PI * (double)i); }

int or_subray_count(int q) {
    int s = 1;
    for (int i = 1; i <= q; ++i) s += ring_n(i);
    return s;
}

int or_subray_angles(int q, double theta_r, int s, double* alpha, double* phi) {
    *alpha = 0.0;
    *phi = 0.0;
    if (s == 0) return 0;
    int idx = s - 1;
    for (int i = 1; i <= q; ++i) {
        int n = ring_n(i);
        if (idx < n) {
            *alpha = ((double)i / (double)q) * theta_r;
            *phi = 2.0 * OR_PI * (double)idx / (double)n;
            return 0;
        }
        idx -= n;
    }
    return -1;
}

/* Orthonormal basis around a unit vector: Duff et al., "Building an
 * Orthonormal Basis, Revisited", JCGT 6(1), 2017. */
void or_onb(const double n[3], double u[3], double v[3]) {
    double sign = copysign(1.0, n[2]);
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    u[0] = 1.0 + sign * n[0] * n[0] * a;
    u[1] = sign * b;
    u[2] = -sign * n[0];
    v[0] = b;
    v[1] = sign + n[1] * n[1] * a;
    v[2] = -n[1];
}

void or_subray_dir(const or_scanner* sn, int q, int s, const double d[3], double ds[3]) {
    double alpha, phi, u[3], v[3];
    or_subray_angles(q, 0.5 * sn->divergence_rad, s, &alpha, &phi);
    or_onb(d, u, v);
    double ca = cos(alpha), sa = sin(alpha), cp = cos(phi), sp = sin(phi);
    for (int a = 0; a < 3; ++a) ds[a] = ca * d[a] + sa * (cp * u[a] + sp * v[a]);
}

/* ------------------------------------------------------------------------ */
/* 1. pulse k: time, platform position (Sec. 3.2) and beam direction        */
/* (Sec. 3.3).  The deflector laws are a reading (the paper only describes   */
/* the patterns): polygon = sawtooth, swinging = sine (denser at extrema).   */
/* ------------------------------------------------------------------------ */
static void rot_rpy(const double rpy[3], const double in[3], double out[3]) {
    double cr = cos(rpy[0]), sr = sin(rpy[0]);
    double cp = cos(rpy[1]), sp = sin(rpy[1]);
    double cy = cos(rpy[2]), sy = sin(rpy[2]);
    double x = in[0], y = in[1], z = in[2];
    /* roll about x */
    double y1 = y * cr - z * sr, z1 = y * sr + z * cr;
    /* pitch about y */
    double x2 = x * cp + z1 * sp, z2 = -x * sp + z1 * cp;
    /* yaw about z */
    out[0] = x2 * cy - y1 * sy;
    out[1] = x2 * sy + y1 * cy;
    out[2] = z2;
}

void or_pulse_ray(const or_scanner* sn, const or_leg* lg, int64_t k, uint64_t seed, double o[3],
                  double d[3]) {
    double elapsed = (double)k / sn->prf_hz;
    double t = lg->t0 + elapsed;
    double rpy[3] = {lg->attitude_rpy[0], lg->attitude_rpy[1], lg->attitude_rpy[2]};
    o[0] = lg->start[0]; o[1] = lg->start[1]; o[2] = lg->start[2];
    if (lg->platform == 1) {
        double D[3];
        sub3(lg->end, lg->start, D);
        double L = norm3(D);
        if (L > 0.0) {
            double s = lg->speed_mps * elapsed;
            if (s > L) s = L;
            for (int a = 0; a < 3; ++a) o[a] = lg->start[a] + s * (D[a] / L);
            rpy[2] += atan2(D[1], D[0]); /* heading towards the next waypoint */
        }
    }
    /* platform noise (Sec. 3.7): N(0, sigma) on each axis, Box-Muller on the
     * Philox draw of stream 2 for this pulse */
    if (lg->platform_noise_m > 0.0) {
        uint32_t w[4];
        draw(seed, lg->leg_id, k, 2, 0, 0, w);
        double u1 = or_uniform24(w[0]), u2 = or_uniform24(w[1]);
        double u3 = or_uniform24(w[2]), u4 = or_uniform24(w[3]);
        double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u3));
        o[0] += lg->platform_noise_m * r1 * cos(2.0 * OR_PI * u2);
        o[1] += lg->platform_noise_m * r1 * sin(2.0 * OR_PI * u2);
        o[2] += lg->platform_noise_m * r2 * cos(2.0 * OR_PI * u4);
    }
    double dp[3];
    double amax = sn->scan_angle_max_rad;
    switch (sn->deflector) {
    case 0: { /* rotating polygon mirror: sawtooth across track */
        double ph = sn->scan_freq_hz * t;
        ph -= floor(ph);
        double th = -amax + 2.0 * amax * ph;
        dp[0] = 0.0; dp[1] = sin(th); dp[2] = -cos(th);
        break;
    }
    case 1: { /* oscillating mirror: sinusoidal across track */
        double th = amax * sin(2.0 * OR_PI * sn->scan_freq_hz * t);
        dp[0] = 0.0; dp[1] = sin(th); dp[2] = -cos(th);
        break;
    }
    case 2: { /* static TLS grid: pulse k = i*n_el + j */
        int64_t i = k / sn->grid_n_el, j = k % sn->grid_n_el;
        double az = 2.0 * OR_PI * (double)i / (double)sn->grid_n_az;
        double el = sn->el_min_rad;
        if (sn->grid_n_el > 1)
            el = sn->el_min_rad + (sn->el_max_rad - sn->el_min_rad) * (double)j / (double)(sn->grid_n_el - 1);
        dp[0] = cos(el) * cos(az); dp[1] = cos(el) * sin(az); dp[2] = sin(el);
        break;
    }
    case 4: { /* fibre-optic line (reading): pulse k leaves fibre k mod n, the
               * fibres fanned evenly across track over [-max, max] */
        int64_t n = sn->n_fibres > 0 ? sn->n_fibres : 1;
        int64_t i = k % n;
        double th = n > 1 ? -amax + 2.0 * amax * (double)i / (double)(n - 1) : 0.0;
        dp[0] = 0.0; dp[1] = sin(th); dp[2] = -cos(th);
        break;
    }
    case 5: { /* Palmer (slanted rotating mirror): a cone at max off nadir,
               * azimuth 2 pi frac(f t) */
        double ph = sn->scan_freq_hz * t;
        ph -= floor(ph);
        double az = 2.0 * OR_PI * ph;
        dp[0] = sin(amax) * cos(az); dp[1] = sin(amax) * sin(az); dp[2] = -cos(amax);
        break;
    }
    case 3:
    default: { /* rotating head: azimuth = rate*t, polygon mirror in elevation */
        double az = sn->head_rate_rad_s * t;
        double ph = sn->scan_freq_hz * t;
        ph -= floor(ph);
        double el = -amax + 2.0 * amax * ph;
        dp[0] = cos(el) * cos(az); dp[1] = cos(el) * sin(az); dp[2] = sin(el);
        break;
    }
    }
    rot_rpy(rpy, dp, d);
}

/* ------------------------------------------------------------------------ */
/* 4. power.  Eq. beamdiv: I = I0 exp(-2 r^2 / w^2).  Eq. beamdiv_w is       */
/* garbled (no "1 +", no focus offset); reading: the Gaussian-beam width     */
/* w(R) = w0 sqrt(1 + (lambda (R - R0) / (pi w0^2))^2), w0 = lambda/(pi      */
/* theta_r) unless given.  r is the subray's offset R tan(alpha).           */
/* ------------------------------------------------------------------------ */
double or_beam_width(const or_scanner* sn, double R) {
    double lam = sn->wavelength_m;
    double w0 = sn->beam_waist_m > 0.0 ? sn->beam_waist_m : lam / (OR_PI * 0.5 * sn->divergence_rad);
    double z = lam * (R - sn->focus_m) / (OR_PI * w0 * w0);
    return w0 * sqrt(1.0 + z * z);
}

double or_subray_intensity(const or_scanner* sn, double R, double alpha) {
    double r = R * tan(alpha);
    double w = or_beam_width(sn, R);
    return sn->peak_power_w * exp(-2.0 * r * r / (w * w));
}

/* Eq. ladlut_intensity with the extended-Lambertian cross-section
 * sigma = pi rho R^2 beta^2 cos(theta): P = I Dr^2 eta_sys eta_atm rho cos / (4 R^2). */
double or_triangle_power(const or_scanner* sn, double Is, double R, double refl, double cos_inc) {
    double Dr = sn->receiver_diam_m;
    return Is * Dr * Dr * sn->eta_sys * sn->eta_atm * refl * cos_inc / (4.0 * R * R);
}

/* 5. pulse shape: Gaussian (FWHM) or Eq. beam_time, t in ns */
double or_pulse_shape(const or_scanner* sn, double t) {
    if (sn->pulse_shape == 0) {
        double s = sn->pulse_fwhm_ns / (2.0 * sqrt(2.0 * log(2.0)));
        return exp(-t * t / (2.0 * s * s));
    }
    double tau = sn->pulse_length_ns / 1.75;
    if (t < 0.0) return 0.0;
    double x = t / tau;
    return x * x * exp(-x);
}

/* ------------------------------------------------------------------------ */
/* scene: triangles (FP64 copies) + median-split BVH + optional voxel grid  */
/* ------------------------------------------------------------------------ */
typedef struct {
    double lo[3], hi[3];
    int64_t left, right; /* children, or -1 for a leaf */
    int64_t start, count;
} bnode;

struct or_grid {
    double g0[3], gc;
    int32_t gd[3];
    int opaque;
    const float* dens;
    double G, leaf_refl;
    const float* lad;
    int64_t lad_n;
    int64_t vox_off;      /* voxels of the earlier grids */
};

struct or_scene {
    int64_t n_tri;
    double* tv;       /* [n][9] */
    const float* refl;
    int64_t* order;
    double* cen;      /* [n][3] */
    bnode* nodes;
    int64_t n_nodes, cap_nodes;
    double eps_box;
    int n_grid;
    struct or_grid* grid;
};

static void tri_bounds(const double* v, double lo[3], double hi[3]) {
    for (int a = 0; a < 3; ++a) {
        double m = v[a], M = v[a];
        for (int k = 1; k < 3; ++k) {
            if (v[3 * k + a] < m) m = v[3 * k + a];
            if (v[3 * k + a] > M) M = v[3 * k + a];
        }
        lo[a] = m; hi[a] = M;
    }
}

/* quickselect: reorder idx[lo..hi) so that element `mid` is in sorted position by key */
static void select_nth(int64_t* idx, const double* cen, int axis, int64_t lo, int64_t hi, int64_t mid) {
    hi -= 1;
    while (hi > lo) {
        double pivot = cen[3 * idx[(lo + hi) / 2] + axis];
        int64_t i = lo, j = hi;
        while (i <= j) {
            while (cen[3 * idx[i] + axis] < pivot) ++i;
            while (cen[3 * idx[j] + axis] > pivot) --j;
            if (i <= j) {
                int64_t t = idx[i]; idx[i] = idx[j]; idx[j] = t;
                ++i; --j;
            }
        }
        if (mid <= j) hi = j;
        else if (mid >= i) lo = i;
        else return;
    }
}

static int64_t build_rec(or_scene* sc, int64_t start, int64_t end) {
    int64_t id = sc->n_nodes++;
    bnode* nd = &sc->nodes[id];
    double clo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, chi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int a = 0; a < 3; ++a) { nd->lo[a] = DBL_MAX; nd->hi[a] = -DBL_MAX; }
    for (int64_t i = start; i < end; ++i) {
        int64_t t = sc->order[i];
        double lo[3], hi[3];
        tri_bounds(&sc->tv[9 * t], lo, hi);
        for (int a = 0; a < 3; ++a) {
            if (lo[a] < nd->lo[a]) nd->lo[a] = lo[a];
            if (hi[a] > nd->hi[a]) nd->hi[a] = hi[a];
            double c = sc->cen[3 * t + a];
            if (c < clo[a]) clo[a] = c;
            if (c > chi[a]) chi[a] = c;
        }
    }
    int axis = 0;
    double ext = chi[0] - clo[0];
    for (int a = 1; a < 3; ++a)
        if (chi[a] - clo[a] > ext) { ext = chi[a] - clo[a]; axis = a; }
    nd->start = start;
    nd->count = end - start;
    nd->left = nd->right = -1;
    if (end - start <= 4 || ext <= 0.0) return id;
    int64_t mid = (start + end) / 2;
    select_nth(sc->order, sc->cen, axis, start, end, mid);
    int64_t l = build_rec(sc, start, mid);
    int64_t r = build_rec(sc, mid, end);
    nd = &sc->nodes[id];
    nd->left = l;
    nd->right = r;
    return id;
}

or_scene* or_scene_build(const or_scene_in* in) {
    or_scene* sc = (or_scene*)calloc(1, sizeof(or_scene));
    int64_t n = in->n_tri;
    sc->n_tri = n;
    sc->refl = in->refl;
    sc->tv = (double*)malloc(sizeof(double) * 9 * (n > 0 ? n : 1));
    sc->cen = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    sc->order = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    double smax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 9; ++k) {
            sc->tv[9 * i + k] = (double)in->tri[9 * i + k];
            if (fabs(sc->tv[9 * i + k]) > smax) smax = fabs(sc->tv[9 * i + k]);
        }
        for (int a = 0; a < 3; ++a)
            sc->cen[3 * i + a] = (sc->tv[9 * i + a] + sc->tv[9 * i + 3 + a] + sc->tv[9 * i + 6 + a]) / 3.0;
        sc->order[i] = i;
    }
    sc->cap_nodes = 2 * (n > 0 ? n : 1);
    sc->nodes = (bnode*)malloc(sizeof(bnode) * sc->cap_nodes);
    sc->n_nodes = 0;
    if (n > 0) build_rec(sc, 0, n);
    sc->n_grid = in->n_grids < 0 ? 0 : (in->n_grids > OR_MAX_GRIDS ? OR_MAX_GRIDS : in->n_grids);
    sc->grid = (struct or_grid*)calloc(sc->n_grid > 0 ? sc->n_grid : 1, sizeof(struct or_grid));
    int64_t off = 0;
    for (int i = 0; i < sc->n_grid; ++i) {
        const or_grid_in* gi = &in->grids[i];
        struct or_grid* g = &sc->grid[i];
        for (int a = 0; a < 3; ++a) { g->g0[a] = gi->origin[a]; g->gd[a] = gi->dims[a]; }
        g->gc = gi->cell;
        g->opaque = gi->opaque;
        g->dens = gi->density;
        g->G = gi->G;
        g->leaf_refl = gi->leaf_refl;
        g->lad = gi->lad;
        g->lad_n = gi->lad ? gi->lad_n : 0;
        g->vox_off = off;
        off += (int64_t)g->gd[0] * g->gd[1] * g->gd[2];
        for (int a = 0; a < 3; ++a) {
            double e = fabs(g->g0[a]) + g->gd[a] * g->gc;
            if (e > smax) smax = e;
        }
    }
    /* boxes are widened so that near misses (within eps of an edge) are found */
    sc->eps_box = 4e-6 * (smax + 1.0);
    return sc;
}

void or_scene_free(or_scene* sc) {
    if (!sc) return;
    free(sc->tv); free(sc->cen); free(sc->order); free(sc->nodes); free(sc->grid);
    free(sc);
}

int64_t or_scene_bvh_nodes(const or_scene* sc) { return sc->n_nodes; }

/* ------------------------------------------------------------------------ */
/* 3a. ray-triangle in FP64: plane hit t, and the smallest signed in-plane   */
/* distance of the hit point to the three edge lines (positive inside).     */
/* ------------------------------------------------------------------------ */
static int tri_eval(const double* v, const double o[3], const double d[3],
                    double* t_out, double* smin_out, double* cos_out) {
    double e1[3], e2[3], n[3], w[3];
    sub3(&v[3], &v[0], e1);
    sub3(&v[6], &v[0], e2);
    cross3(e1, e2, n);
    double nn = norm3(n);
    if (nn == 0.0) return 0;
    double den = dot3(n, d);
    if (den == 0.0) return 0;
    sub3(&v[0], o, w);
    double t = dot3(n, w) / den;
    if (!(t > 0.0)) return 0;
    double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
    double smin = DBL_MAX;
    for (int k = 0; k < 3; ++k) {
        const double* a = &v[3 * k];
        const double* b = &v[3 * ((k + 1) % 3)];
        double ab[3], ap[3], c[3];
        sub3(b, a, ab);
        sub3(p, a, ap);
        cross3(ab, ap, c);
        double s = dot3(c, n) / (nn * norm3(ab));
        if (s < smin) smin = s;
    }
    *t_out = t;
    *smin_out = smin;
    *cos_out = fabs(den) / nn;
    return 1;
}

static int box_enter(const double lo[3], const double hi[3], double eps, const double o[3],
                     const double d[3], double tmax, double* tenter) {
    double t0 = 0.0, t1 = tmax;
    for (int a = 0; a < 3; ++a) {
        double l = lo[a] - eps, h = hi[a] + eps;
        if (d[a] == 0.0) {
            if (o[a] < l || o[a] > h) return 0;
            continue;
        }
        double ta = (l - o[a]) / d[a], tb = (h - o[a]) / d[a];
        if (ta > tb) { double x = ta; ta = tb; tb = x; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    *tenter = t0;
    return 1;
}

typedef struct { double t, smin; int64_t id; } cand_t;

/* clear_only = 0: the closest hit (edge points count as inside) with parity
 * flags; clear_only = 1: the closest hit whose point is at least eps inside
 * its triangle (no FP32 evaluation could miss it). */
static int64_t intersect_impl(const or_scene* sc, const double o[3], const double d[3],
                              int clear_only, double* t_hit, double* cos_hit, uint32_t* flags) {
    *t_hit = INFINITY;
    *cos_hit = 0.0;
    if (sc->n_tri == 0) return -1;
    int64_t stack[256];
    int sp = 0;
    cand_t cands[64];
    int nc = 0;
    int overflow = 0;
    double best_t = INFINITY, best_cos = 0.0, best_s = 0.0;
    int64_t best = -1;
    stack[sp++] = 0;
    while (sp > 0) {
        const bnode* nd = &sc->nodes[stack[--sp]];
        double bound = isinf(best_t) ? INFINITY : best_t + eps_rel(best_t) + sc->eps_box;
        double te;
        if (!box_enter(nd->lo, nd->hi, sc->eps_box, o, d, bound, &te)) continue;
        if (nd->left < 0) {
            for (int64_t i = nd->start; i < nd->start + nd->count; ++i) {
                int64_t id = sc->order[i];
                double t, smin, c;
                if (!tri_eval(&sc->tv[9 * id], o, d, &t, &smin, &c)) continue;
                double e = eps_rel(t);
                if (smin < -e) continue;
                if (nc < 64) cands[nc++] = (cand_t){t, smin, id};
                else overflow = 1;
                if (smin >= (clear_only ? e : 0.0) && (t < best_t || (t == best_t && id < best))) {
                    best_t = t; best = id; best_cos = c; best_s = smin;
                }
            }
        } else {
            if (sp + 2 > 256) { overflow = 1; continue; }
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
    uint32_t f = 0;
    double eb = isinf(best_t) ? 0.0 : eps_rel(best_t);
    if (best >= 0 && best_s < eb) f |= OR_F_EDGE;
    for (int i = 0; i < nc; ++i) {
        if (cands[i].id == best) continue;
        if (best >= 0 && cands[i].t > best_t + eb) continue;
        double e = eps_rel(cands[i].t);
        if (fabs(cands[i].smin) < e) f |= OR_F_EDGE;
        else if (cands[i].smin >= 0.0 && best >= 0 && cands[i].t - best_t <= eb) f |= OR_F_TIE;
    }
    if (overflow) f |= OR_F_TIE;
    if (flags) *flags |= f;
    *t_hit = best_t;
    *cos_hit = best_cos;
    return best;
}

int64_t or_intersect(const or_scene* sc, const double o[3], const double d[3],
                     double* t_hit, double* cos_hit, uint32_t* flags) {
    return intersect_impl(sc, o, d, 0, t_hit, cos_hit, flags);
}

int64_t or_intersect_brute(const or_scene* sc, const double o[3], const double d[3],
                           double* t_hit, double* cos_hit) {
    double best_t = INFINITY, best_c = 0.0;
    int64_t best = -1;
    for (int64_t id = 0; id < sc->n_tri; ++id) {
        double t, smin, c;
        if (!tri_eval(&sc->tv[9 * id], o, d, &t, &smin, &c)) continue;
        if (smin < 0.0) continue;
        if (t < best_t) { best_t = t; best = id; best_c = c; }
    }
    *t_hit = best_t;
    *cos_hit = best_c;
    return best;
}

/* ------------------------------------------------------------------------ */
/* 3b. voxel grid: a plain FP64 DDA (Amanatides & Woo, 1987).  Each crossing  */
/* time is computed per plane, (plane - o)/d, without accumulation.  This    */
/* replaces the epsilon re-cast of Sec. 5.1 by exact plane crossings.       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t vid;     /* voxel index within grid gi */
    double t_in, t_out;
    double sigma;
    int corner;      /* 1: another axis crossed within eps of the exit */
    int64_t alt_vid; /* the voxel an FP32 march could visit instead at that corner */
    int axis;        /* axis of the face the ray entered through, -1: started inside */
    int gi;          /* grid */
    int alt_axis;    /* corner: the axis whose plane is crossed within eps of the exit */
} vseg;

typedef struct { vseg* v; int64_t n, cap; } vlist;

static void vpush(vlist* L, vseg s) {
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 256;
        L->v = (vseg*)realloc(L->v, sizeof(vseg) * L->cap);
    }
    L->v[L->n++] = s;
}

/* sigma = G * density (Eq. extinction).  With a leaf-angle table (Table ladlut)
 * G depends on the subray direction: the table holds G at mu_i = i/(n-1) of
 * mu = |d_z| (d a unit vector) and is read by linear interpolation. */
static double proj_factor(const struct or_grid* g, const double d[3]) {
    if (g->lad_n < 2) return g->G;
    double t = fmin(fabs(d[2]), 1.0) * (double)(g->lad_n - 1);
    int64_t i = (int64_t)floor(t);
    if (i > g->lad_n - 2) i = g->lad_n - 2;
    double f = t - (double)i;
    double g0 = (double)g->lad[i], g1 = (double)g->lad[i + 1];
    return g0 + f * (g1 - g0);
}

/* voxel id in outputs and the index of its transmission draw */
static int64_t vox_id(const or_scene* sc, const vseg* v, int64_t vid) {
    return sc->n_tri + sc->grid[v->gi].vox_off + vid;
}
static int64_t vox_draw(const or_scene* sc, const vseg* v, int64_t vid) {
    return sc->grid[v->gi].vox_off + vid;
}

static double plane_t(const struct or_grid* g, int a, int64_t i, const double o[3], const double d[3]) {
    return (g->g0[a] + (double)i * g->gc - o[a]) / d[a];
}

/* entry and exit of the ray o + t d (t >= 0) with grid g's box; 0: no overlap */
static int grid_span(const struct or_grid* g, const double o[3], const double d[3],
                     double tlo[3], double thi[3], double* t_enter, double* t_exit) {
    *t_enter = 0.0;
    *t_exit = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = g->g0[a], hi = g->g0[a] + (double)g->gd[a] * g->gc;
        if (d[a] == 0.0) {
            if (o[a] < lo || o[a] >= hi) return 0;
            tlo[a] = -INFINITY; thi[a] = INFINITY;
        } else {
            double ta = (lo - o[a]) / d[a], tb = (hi - o[a]) / d[a];
            tlo[a] = ta < tb ? ta : tb;
            thi[a] = ta < tb ? tb : ta;
        }
        if (tlo[a] > *t_enter) *t_enter = tlo[a];
        if (thi[a] < *t_exit) *t_exit = thi[a];
    }
    return *t_enter < *t_exit;
}

/* all voxels of grid gi with positive segment length in [max(t_enter,0), min(t_exit,t_hi)) */
static void march_grid(const or_scene* sc, int gi, const double o[3], const double d[3], double t_hi,
                       vlist* L) {
    const struct or_grid* g = &sc->grid[gi];
    double tlo[3], thi[3];
    double t_enter, t_exit;
    if (!grid_span(g, o, d, tlo, thi, &t_enter, &t_exit)) return;
    double t_end = t_exit < t_hi ? t_exit : t_hi;
    if (!(t_enter < t_end)) return;
    const double G = proj_factor(g, d);
    int64_t idx[3];
    int step[3];
    double tn[3];
    for (int a = 0; a < 3; ++a) {
        step[a] = d[a] > 0.0 ? 1 : (d[a] < 0.0 ? -1 : 0);
        if (t_enter > 0.0 && tlo[a] == t_enter && d[a] != 0.0) {
            idx[a] = d[a] > 0.0 ? 0 : g->gd[a] - 1;
        } else {
            double p = o[a] + t_enter * d[a];
            double f = floor((p - g->g0[a]) / g->gc);
            if (f < 0) f = 0;
            if (f > g->gd[a] - 1) f = g->gd[a] - 1;
            idx[a] = (int64_t)f;
        }
        if (step[a] > 0) tn[a] = plane_t(g, a, idx[a] + 1, o, d);
        else if (step[a] < 0) tn[a] = plane_t(g, a, idx[a], o, d);
        else tn[a] = INFINITY;
    }
    double t_in = t_enter;
    int entry = -1;      /* the grid face crossed at t_enter (lowest axis on a tie) */
    if (t_enter > 0.0)
        for (int a = 2; a >= 0; --a)
            if (d[a] != 0.0 && tlo[a] == t_enter) entry = a;
    const int64_t nx = g->gd[0], ny = g->gd[1];
    for (int64_t guard = 0; guard < 4 * (int64_t)(g->gd[0] + g->gd[1] + g->gd[2]) + 8; ++guard) {
        int a = 0;
        if (tn[1] < tn[a]) a = 1;
        if (tn[2] < tn[a]) a = 2;
        double t_out = tn[a] < t_end ? tn[a] : t_end;
        int64_t vid = (idx[2] * ny + idx[1]) * nx + idx[0];
        if (t_out > t_in) {
            vseg s = {vid, t_in, t_out, G * (double)g->dens[vid], 0, -1, entry, gi, -1};
            /* second-smallest crossing near the exit: order ambiguous in FP32 */
            for (int b = 0; b < 3; ++b) {
                if (b == a || step[b] == 0) continue;
                if (tn[a] < t_end && tn[b] - tn[a] <= eps_rel(tn[a])) {
                    int64_t j[3] = {idx[0], idx[1], idx[2]};
                    j[b] += step[b];
                    if (j[b] >= 0 && j[b] < g->gd[b]) {
                        s.corner = 1;
                        s.alt_vid = (j[2] * ny + j[1]) * nx + j[0];
                        s.alt_axis = b;
                    }
                }
            }
            vpush(L, s);
        }
        if (tn[a] >= t_end) break;
        idx[a] += step[a];
        if (idx[a] < 0 || idx[a] >= g->gd[a]) break;
        entry = a;
        t_in = tn[a] > t_in ? tn[a] : t_in;
        tn[a] = step[a] > 0 ? plane_t(g, a, idx[a] + 1, o, d) : plane_t(g, a, idx[a], o, d);
    }
}

/* The voxels along the ray up to t_hi, over all grids: the grids' boxes have
 * disjoint interiors, so their segments follow one another in the order of
 * the boxes' entry points; each grid is marched in that order. */
static void march(const or_scene* sc, const double o[3], const double d[3], double t_hi, vlist* L) {
    L->n = 0;
    if (sc->n_grid == 0) return;
    double te_all[OR_MAX_GRIDS];
    int order[OR_MAX_GRIDS];
    int n = 0;
    for (int gi = 0; gi < sc->n_grid; ++gi) {
        double tlo[3], thi[3], te, tx;
        if (!grid_span(&sc->grid[gi], o, d, tlo, thi, &te, &tx) || !(te < t_hi)) continue;
        /* insertion by (entry, grid index) */
        int j = n++;
        while (j > 0 && te_all[order[j - 1]] > te) { order[j] = order[j - 1]; --j; }
        order[j] = gi;
        te_all[gi] = te;
    }
    for (int i = 0; i < n; ++i) march_grid(sc, order[i], o, d, t_hi, L);
}

int64_t or_march(const or_scene* sc, const double o[3], const double d[3], double t_hi,
                 int64_t cap, int64_t* vid, double* t_in, double* t_out) {
    vlist L = {0};
    march(sc, o, d, t_hi, &L);
    int64_t n = L.n;
    for (int64_t i = 0; i < n && i < cap; ++i) {
        vid[i] = vox_draw(sc, &L.v[i], L.v[i].vid);
        t_in[i] = L.v[i].t_in;
        t_out[i] = L.v[i].t_out;
    }
    free(L.v);
    return n;
}

/* ------------------------------------------------------------------------ */
/* per-pulse simulation                                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double R;      /* range of the return */
    double P;      /* returned power, weight included */
    int64_t id;    /* primitive: triangle, or n_tri + voxel */
    int s;         /* subray */
} ret_t;

typedef struct { ret_t* r; int64_t n, cap; } rlist;

static void rpush(rlist* L, ret_t x) {
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 256;
        L->r = (ret_t*)realloc(L->r, sizeof(ret_t) * L->cap);
    }
    L->r[L->n++] = x;
}

typedef struct {
    /* per-thread scratch */
    vlist vl;
    rlist rl;
    double* W;
    double* contrib;
    /* adjoint accumulation lists */
    int64_t* gid;
    double* gval;
    int64_t gn, gcap;
} scratch_t;

static void gpush(scratch_t* S, int64_t id, double v) {
    if (S->gn == S->gcap) {
        S->gcap = S->gcap ? 2 * S->gcap : 4096;
        S->gid = (int64_t*)realloc(S->gid, sizeof(int64_t) * S->gcap);
        S->gval = (double*)realloc(S->gval, sizeof(double) * S->gcap);
    }
    S->gid[S->gn] = id;
    S->gval[S->gn] = v;
    S->gn++;
}

static double voxel_power(const or_scanner* sn, const struct or_grid* g, double Is, double R) {
    /* Eq. ladlut_intensity for a voxel return; reading: leaf reflectance, cos := 1 */
    return or_triangle_power(sn, Is, R, g->leaf_refl, 1.0);
}

static double delay_ns(double R) { return 2.0 * R / OR_C * 1e9; }

static int n_pre_bins(const or_scanner* sn) {
    if (sn->pulse_shape != 0) return 0;
    double s = sn->pulse_fwhm_ns / (2.0 * sqrt(2.0 * log(2.0)));
    return (int)ceil(3.0 * s / sn->bin_ns);
}

typedef struct {
    const or_scene* sc;
    const or_scanner* sn;
    const or_leg* lg;
    const int64_t* pulses;
    int64_t n;
    int mode;
    uint64_t seed;
    const int32_t* fixed_window;
    const int64_t* force_hit; /* [n][S] or NULL: events given per subray (OR_FREE_HIT: none) */
    const or_out* out;
    const double* g;      /* adjoint only */
    int adjoint;
    int64_t begin, end;
    scratch_t S;
} job_t;

/* expected (differentiable) mode, over the voxels marched into J->S.vl: voxel
 * k returns w_k = T_k (1 - e^{-sigma_k l_k}) at its segment midpoint, the
 * triangle tri (if any) returns the transmitted T. */
static void expected_returns(job_t* J, int s, const double ds[3], double alpha, int64_t tri,
                             double t_tri, double cos_tri, int64_t* ev_id, double* ev_R) {
    const or_scene* sc = J->sc;
    const or_scanner* sn = J->sn;
    vlist* L = &J->S.vl;
    double T = 1.0;
    for (int64_t i = 0; i < L->n; ++i) {
        vseg* v = &L->v[i];
        const struct or_grid* g = &sc->grid[v->gi];
        if (v->sigma <= 0.0) continue;
        if (g->opaque) {
            /* an opaque voxel returns all that reaches it and passes nothing;
             * the subray record keeps the triangle hit, as in every expected-mode
             * scan (it is the adjoint's checkpoint) */
            double R = v->t_in, c = v->axis >= 0 ? fabs(ds[v->axis]) : 1.0;
            double Is = or_subray_intensity(sn, R, alpha);
            ret_t r = {R, T * or_triangle_power(sn, Is, R, g->leaf_refl, c), vox_id(sc, v, v->vid), s};
            rpush(&J->S.rl, r);
            if (tri >= 0) {
                *ev_id = tri;
                *ev_R = t_tri;
            }
            return;
        }
        double len = v->t_out - v->t_in;
        double a = exp(-v->sigma * len);
        double R = 0.5 * (v->t_in + v->t_out);
        double Is = or_subray_intensity(sn, R, alpha);
        ret_t r = {R, T * (1.0 - a) * voxel_power(sn, g, Is, R), vox_id(sc, v, v->vid), s};
        rpush(&J->S.rl, r);
        T *= a;
    }
    if (tri >= 0) {
        double Is = or_subray_intensity(sn, t_tri, alpha);
        ret_t r = {t_tri, T * or_triangle_power(sn, Is, t_tri, (double)sc->refl[tri], cos_tri), tri, s};
        rpush(&J->S.rl, r);
        *ev_id = tri;
        *ev_R = t_tri;
    }
}

/* one subray: fill the return list (stochastic: <= 1 return; expected: voxels
 * then triangle).  Returns the primitive of the event and its range. */
static void trace_subray(job_t* J, int64_t k, int s, const double o[3], const double ds[3],
                         double alpha, uint32_t* flags, int64_t* ev_id, double* ev_R) {
    const or_scene* sc = J->sc;
    const or_scanner* sn = J->sn;
    double t_tri, cos_tri;
    uint32_t f = 0;
    int64_t tri = or_intersect(sc, o, ds, &t_tri, &cos_tri, &f);
    *flags |= f;
    *ev_id = -1;
    *ev_R = 0.0;
    march(sc, o, ds, t_tri, &J->S.vl);
    vlist* L = &J->S.vl;
    if (J->mode == 0) {
        /* stochastic transmission (Eq. intersection_dist): s = -ln(u)/sigma; an
         * echo at entry + s if s < traversed length, else continue (Sec. 5.2).
         * Non-transmissive grids (Sec. 3.5.4): the first voxel of non-zero
         * density stops the subray where it enters it, Lambertian on the face
         * entered (cos = |d . n|; 1 when the ray starts inside). */
        for (int64_t i = 0; i < L->n; ++i) {
            vseg* v = &L->v[i];
            const struct or_grid* g = &sc->grid[v->gi];
            if (g->opaque) {
                if (v->corner && v->alt_vid >= 0 && (g->dens[v->alt_vid] > 0.0f) != (v->sigma > 0.0))
                    *flags |= OR_F_VOX;
                if (v->sigma <= 0.0) continue;
                double R = v->t_in, c = v->axis >= 0 ? fabs(ds[v->axis]) : 1.0;
                double Is = or_subray_intensity(sn, R, alpha);
                ret_t r = {R, or_triangle_power(sn, Is, R, g->leaf_refl, c), vox_id(sc, v, v->vid), s};
                rpush(&J->S.rl, r);
                *ev_id = r.id;
                *ev_R = R;
                return;
            }
            if (v->corner && v->alt_vid >= 0) {
                double sa = proj_factor(g, ds) * (double)g->dens[v->alt_vid];
                if (sa > 0.0) {
                    uint32_t w[4];
                    draw(J->seed, J->lg->leg_id, k, 0, (uint32_t)s, (uint64_t)vox_draw(sc, v, v->alt_vid), w);
                    double sal = -log(or_uniform24(w[0])) / sa;
                    if (sal <= 2.0 * eps_rel(v->t_out)) *flags |= OR_F_VOX;
                }
            }
            if (v->sigma <= 0.0) continue;
            uint32_t w[4];
            draw(J->seed, J->lg->leg_id, k, 0, (uint32_t)s, (uint64_t)vox_draw(sc, v, v->vid), w);
            double u = or_uniform24(w[0]);
            double sdist = -log(u) / v->sigma;
            double len = v->t_out - v->t_in;
            if (fabs(sdist - len) <= 1e-6 * sdist + 1e-12) *flags |= OR_F_VOX;
            if (len < eps_rel(v->t_in) && sdist <= len + eps_rel(v->t_in)) *flags |= OR_F_VOX;
            if (sdist < len) {
                double R = v->t_in + sdist;
                double Is = or_subray_intensity(sn, R, alpha);
                ret_t r = {R, voxel_power(sn, g, Is, R), vox_id(sc, v, v->vid), s};
                rpush(&J->S.rl, r);
                *ev_id = r.id;
                *ev_R = R;
                return;
            }
        }
        if (tri >= 0) {
            double Is = or_subray_intensity(sn, t_tri, alpha);
            ret_t r = {t_tri, or_triangle_power(sn, Is, t_tri, (double)sc->refl[tri], cos_tri), tri, s};
            rpush(&J->S.rl, r);
            *ev_id = tri;
            *ev_R = t_tri;
        }
        return;
    }
    expected_returns(J, s, ds, alpha, tri, t_tri, cos_tri, ev_id, ev_R);
}

/* 1 when the ray meets, at some 0 < t <= t_max, an edge shared by two
 * triangles (the same two vertex positions) within eps of that edge in both:
 * a watertight triangle test hits one of the two there, so no FP32 path may
 * pass between them. */
static int closed_edge_before(const or_scene* sc, const double o[3], const double d[3],
                              double t_max) {
    if (sc->n_tri == 0 || !(t_max > 0.0)) return 0;
    int64_t stack[256];
    int sp = 0;
    int64_t near_id[64];
    int near_k[64];
    int nn = 0;
    stack[sp++] = 0;
    while (sp > 0 && nn < 64) {
        const bnode* nd = &sc->nodes[stack[--sp]];
        double te;
        double bound = isinf(t_max) ? INFINITY : t_max + eps_rel(t_max) + sc->eps_box;
        if (!box_enter(nd->lo, nd->hi, sc->eps_box, o, d, bound, &te)) continue;
        if (nd->left < 0) {
            for (int64_t i = nd->start; i < nd->start + nd->count && nn < 64; ++i) {
                int64_t id = sc->order[i];
                const double* v = &sc->tv[9 * id];
                double t, smin, c;
                if (!tri_eval(v, o, d, &t, &smin, &c) || t > t_max) continue;
                if (fabs(smin) >= eps_rel(t)) continue;
                /* the edge the point is nearest to */
                double e1[3], e2[3], n[3], p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
                sub3(&v[3], &v[0], e1);
                sub3(&v[6], &v[0], e2);
                cross3(e1, e2, n);
                double nrm = norm3(n), best = DBL_MAX;
                int kb = 0;
                for (int k = 0; k < 3; ++k) {
                    const double* a = &v[3 * k];
                    const double* b = &v[3 * ((k + 1) % 3)];
                    double ab[3], ap[3], cr[3];
                    sub3(b, a, ab);
                    sub3(p, a, ap);
                    cross3(ab, ap, cr);
                    double sk = dot3(cr, n) / (nrm * norm3(ab));
                    if (sk < best) { best = sk; kb = k; }
                }
                near_id[nn] = id;
                near_k[nn] = kb;
                nn++;
            }
        } else if (sp + 2 <= 256) {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
    for (int i = 0; i < nn; ++i) {
        const double* a0 = &sc->tv[9 * near_id[i] + 3 * near_k[i]];
        const double* a1 = &sc->tv[9 * near_id[i] + 3 * ((near_k[i] + 1) % 3)];
        for (int j = i + 1; j < nn; ++j) {
            const double* b0 = &sc->tv[9 * near_id[j] + 3 * near_k[j]];
            const double* b1 = &sc->tv[9 * near_id[j] + 3 * ((near_k[j] + 1) % 3)];
            int same = (memcmp(a0, b0, 24) == 0 && memcmp(a1, b1, 24) == 0) ||
                       (memcmp(a0, b1, 24) == 0 && memcmp(a1, b0, 24) == 0);
            if (same) return 1;
        }
    }
    return 0;
}

/* Parity support: one subray re-run with its event given.  An FP32 path may
 * legitimately decide differently where the oracle raised a flag (a hit within
 * eps of an edge, near-equal hits, a transmission draw within rounding of the
 * segment length, a voxel corner).  `forced` is the event it reported: a
 * triangle id, n_tri + voxel (stochastic mode: the voxel it stopped in), or -1
 * (no event).  The subray's returns are formed from that event with the
 * oracle's arithmetic.  OR_F_FORCED_BAD is raised when no flagged decision
 * allows the event: a triangle the ray misses by more than eps, an event
 * behind a hit no FP32 evaluation could miss or behind an edge shared by two
 * triangles (a watertight test hits one of them), or a voxel passed although
 * its draw stops the subray clearly inside it. */
static void trace_subray_forced(job_t* J, int64_t k, int s, const double o[3], const double ds[3],
                                double alpha, int64_t forced, uint32_t* flags, int64_t* ev_id,
                                double* ev_R) {
    const or_scene* sc = J->sc;
    const or_scanner* sn = J->sn;
    double t_clear, cos_clear;
    intersect_impl(sc, o, ds, 1, &t_clear, &cos_clear, NULL);
    const double lim = isinf(t_clear) ? INFINITY : t_clear + eps_rel(t_clear);
    int64_t tri = -1, fvox = -1;
    double t_tri = INFINITY, cos_tri = 0.0;
    *ev_id = -1;
    *ev_R = 0.0;
    if (forced >= 0 && forced < sc->n_tri) {
        double smin;
        tri = forced;
        if (!tri_eval(&sc->tv[9 * forced], o, ds, &t_tri, &smin, &cos_tri) ||
            smin < -eps_rel(t_tri) || t_tri > lim ||
            closed_edge_before(sc, o, ds, t_tri - eps_rel(t_tri))) {
            *flags |= OR_F_FORCED_BAD;
            return;
        }
    } else if (forced >= sc->n_tri) {
        fvox = forced - sc->n_tri;
        if (J->mode != 0) { *flags |= OR_F_FORCED_BAD; return; }
    } else if (!isinf(t_clear) || closed_edge_before(sc, o, ds, INFINITY)) {
        *flags |= OR_F_FORCED_BAD;
        return;
    }
    march(sc, o, ds, tri >= 0 ? t_tri : t_clear, &J->S.vl);
    vlist* L = &J->S.vl;
    if (J->mode != 0) {
        expected_returns(J, s, ds, alpha, tri, t_tri, cos_tri, ev_id, ev_R);
        return;
    }
    for (int64_t i = 0; i < L->n; ++i) {
        vseg* v = &L->v[i];
        const struct or_grid* g = &sc->grid[v->gi];
        int alt = v->corner && v->alt_vid >= 0;
        int hit_main = fvox >= 0 && vox_draw(sc, v, v->vid) == fvox;
        int hit_alt = fvox >= 0 && alt && vox_draw(sc, v, v->alt_vid) == fvox;
        if (g->opaque) {
            if (hit_main || hit_alt) {
                double R = hit_main ? v->t_in : v->t_out;
                /* the corner voxel is entered through the face crossed within eps of this exit */
                double c = hit_main ? (v->axis >= 0 ? fabs(ds[v->axis]) : 1.0) : fabs(ds[v->alt_axis]);
                double Is = or_subray_intensity(sn, R, alpha);
                ret_t r = {R, or_triangle_power(sn, Is, R, g->leaf_refl, c), sc->n_tri + fvox, s};
                if (hit_main && v->sigma <= 0.0) *flags |= OR_F_FORCED_BAD;
                if (closed_edge_before(sc, o, ds, R - eps_rel(R))) *flags |= OR_F_FORCED_BAD;
                rpush(&J->S.rl, r);
                *ev_id = r.id;
                *ev_R = R;
                return;
            }
            if (v->sigma > 0.0 && !(alt && g->dens[v->alt_vid] <= 0.0f)) {
                *flags |= OR_F_FORCED_BAD;
                return;
            }
            continue;
        }
        if (hit_main || hit_alt) {
            int64_t vv = hit_main ? v->vid : v->alt_vid;
            double sg = proj_factor(g, ds) * (double)g->dens[vv];
            uint32_t w[4];
            draw(J->seed, J->lg->leg_id, k, 0, (uint32_t)s, (uint64_t)vox_draw(sc, v, vv), w);
            double sdist = sg > 0.0 ? -log(or_uniform24(w[0])) / sg : INFINITY;
            double len = v->t_out - v->t_in;
            double R;
            if (hit_main) {
                if (!(sdist <= len + 1e-6 * sdist + 1e-12 ||
                      (len < eps_rel(v->t_in) && sdist <= len + eps_rel(v->t_in))))
                    *flags |= OR_F_FORCED_BAD;
                R = v->t_in + (sdist < len ? sdist : len);
            } else {
                if (!(sdist <= 2.0 * eps_rel(v->t_out))) *flags |= OR_F_FORCED_BAD;
                R = v->t_out;
            }
            if (closed_edge_before(sc, o, ds, R - eps_rel(R))) *flags |= OR_F_FORCED_BAD;
            double Is = or_subray_intensity(sn, R, alpha);
            ret_t r = {R, voxel_power(sn, g, Is, R), sc->n_tri + fvox, s};
            rpush(&J->S.rl, r);
            *ev_id = r.id;
            *ev_R = R;
            return;
        }
        if (v->sigma <= 0.0) continue;
        uint32_t w[4];
        draw(J->seed, J->lg->leg_id, k, 0, (uint32_t)s, (uint64_t)vox_draw(sc, v, v->vid), w);
        double sdist = -log(or_uniform24(w[0])) / v->sigma;
        double len = v->t_out - v->t_in;
        int near = fabs(sdist - len) <= 1e-6 * sdist + 1e-12 ||
                   (len < eps_rel(v->t_in) && sdist <= len + eps_rel(v->t_in));
        if (sdist < len && !near) {
            *flags |= OR_F_FORCED_BAD;
            return;
        }
    }
    if (fvox >= 0) {
        *flags |= OR_F_FORCED_BAD;
        return;
    }
    if (tri >= 0) {
        double Is = or_subray_intensity(sn, t_tri, alpha);
        ret_t r = {t_tri, or_triangle_power(sn, Is, t_tri, (double)sc->refl[tri], cos_tri), tri, s};
        rpush(&J->S.rl, r);
        *ev_id = tri;
        *ev_R = t_tri;
    }
}

/* adjoint of one subray in expected mode (window fixed): A_k = sum_b g_b P_k p(t_b - tau_k) */
static void adjoint_subray(job_t* J, const double* g, int32_t m,
                           const double o[3], const double ds[3], double alpha) {
    const or_scene* sc = J->sc;
    const or_scanner* sn = J->sn;
    double t_tri, cos_tri;
    uint32_t f = 0;
    int64_t tri = or_intersect(sc, o, ds, &t_tri, &cos_tri, &f);
    march(sc, o, ds, t_tri, &J->S.vl);
    vlist* L = &J->S.vl;
    const int nb = sn->n_bins;
    const double dt = sn->bin_ns;
    /* forward quantities */
    int64_t nv = 0;
    for (int64_t i = 0; i < L->n; ++i)
        if (L->v[i].sigma > 0.0) L->v[nv++] = L->v[i];
    double* A = (double*)malloc(sizeof(double) * (nv + 1));
    double* T = (double*)malloc(sizeof(double) * (nv + 2));
    double* wk = (double*)malloc(sizeof(double) * (nv + 1));
    T[0] = 1.0;
    for (int64_t i = 0; i < nv; ++i) {
        vseg* v = &L->v[i];
        double len = v->t_out - v->t_in;
        double a = exp(-v->sigma * len);
        double R = 0.5 * (v->t_in + v->t_out);
        double Is = or_subray_intensity(sn, R, alpha);
        double P = voxel_power(sn, &sc->grid[v->gi], Is, R);
        double tau = delay_ns(R);
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc += g[b] * P * or_pulse_shape(sn, (double)(m + b) * dt - tau);
        A[i] = acc;
        wk[i] = T[i] * (1.0 - a);
        T[i + 1] = T[i] * a;
    }
    double suffix = 0.0;
    if (tri >= 0) {
        double Is = or_subray_intensity(sn, t_tri, alpha);
        double P1 = or_triangle_power(sn, Is, t_tri, 1.0, cos_tri);
        double tau = delay_ns(t_tri);
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc += g[b] * P1 * or_pulse_shape(sn, (double)(m + b) * dt - tau);
        double wtri = T[nv];
        /* dL/drho = A_tri(rho=1) * w_tri */
        gpush(&J->S, tri, acc * wtri);
        suffix = acc * (double)sc->refl[tri] * wtri;
    }
    /* dL/dsigma_j = A_j T_j l_j e^{-sigma_j l_j} - l_j (sum_{k>j} A_k w_k + A_tri w_tri);
     * dL/ddensity_j = G(d) dL/dsigma_j */
    for (int64_t i = nv - 1; i >= 0; --i) {
        vseg* v = &L->v[i];
        double len = v->t_out - v->t_in;
        double a = exp(-v->sigma * len);
        double dsig = A[i] * T[i] * len * a - len * suffix;
        gpush(&J->S, vox_id(sc, v, v->vid), proj_factor(&sc->grid[v->gi], ds) * dsig);
        suffix += A[i] * wk[i];
    }
    free(A); free(T); free(wk);
}

/* Echoes (Sec. 3.4: local maxima of the waveform above a threshold; the
 * threshold as a fraction of the pulse's own maximum bin).  A bin is an echo
 * when it rises strictly above its left neighbour, does not fall below its
 * right neighbour (so a plateau gives its leftmost bin), is positive and is at
 * or above thr_rel * max W; outside the window W counts as 0.  Bins are taken
 * in order and the first K kept. */
int or_echo_peaks(const double* W, int nb, double thr_rel, int K, int32_t* bins, int* overflow,
                  int* near) {
    double wmax = 0.0;
    for (int b = 0; b < nb; ++b)
        if (W[b] > wmax) wmax = W[b];
    double thr = thr_rel * wmax;
    double tol = 1e-4 * wmax;
    int ne = 0;
    *overflow = 0;
    *near = 0;
    for (int b = 0; b < nb; ++b) {
        double c = W[b];
        double l = b > 0 ? W[b - 1] : 0.0;
        double r = b + 1 < nb ? W[b + 1] : 0.0;
        if (c >= thr - tol && (fabs(c - l) <= tol || fabs(c - r) <= tol)) *near = 1;
        int is_max = c > l && c >= r && c >= thr && c > 0.0;
        if (is_max && fabs(c - thr) <= tol) *near = 1;
        if (!is_max) continue;
        if (ne >= K) { *overflow = 1; continue; }
        bins[ne++] = b;
    }
    return ne;
}

/* Echo object: the primitive whose return contributes most to the waveform at
 * time tb; on equal contributions the first in summation order (subray order,
 * then along the subray).  *near: the two largest within 1e-4 relative. */
static int64_t echo_object_list(const or_scanner* sn, const ret_t* r, int64_t n, double tb,
                                int* near, int64_t* second_id) {
    double best = -1.0, second = -1.0;
    int64_t bid = -1, sid = -1;
    for (int64_t i = 0; i < n; ++i) {
        double v = r[i].P * or_pulse_shape(sn, tb - delay_ns(r[i].R));
        if (v > best) { second = best; sid = bid; best = v; bid = r[i].id; }
        else if (v > second) { second = v; sid = r[i].id; }
    }
    *near = second >= 0.0 && best - second <= 1e-4 * best;
    if (second_id) *second_id = *near ? sid : -1;
    return bid;
}

int64_t or_echo_object(const or_scanner* sn, int64_t n, const double* P, const double* R,
                       const int64_t* id, double tb_ns, int* near) {
    ret_t* r = (ret_t*)malloc(sizeof(ret_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        r[i].R = R[i];
        r[i].P = P[i];
        r[i].id = id[i];
        r[i].s = 0;
    }
    int64_t b = echo_object_list(sn, r, n, tb_ns, near, NULL);
    free(r);
    return b;
}

static void simulate_pulse(job_t* J, int64_t row) {
    const or_scanner* sn = J->sn;
    const or_leg* lg = J->lg;
    const or_out* out = J->out;
    int64_t k = J->pulses[row];
    int q = lg->quality >= 0 ? lg->quality : sn->quality;
    int S = or_subray_count(q);
    int nb = sn->n_bins, K = sn->max_echoes;
    double o[3], d[3];
    or_pulse_ray(sn, lg, k, J->seed, o, d);
    uint32_t flags = 0;
    if (J->adjoint) {
        const double* g = &J->g[row * nb];
        int32_t m = J->fixed_window[row];
        if (m == OR_NO_WINDOW) return;
        for (int s = 0; s < S; ++s) {
            double alpha, phi, ds[3];
            or_subray_angles(q, 0.5 * sn->divergence_rad, s, &alpha, &phi);
            or_subray_dir(sn, q, s, d, ds);
            adjoint_subray(J, g, m, o, ds, alpha);
        }
        return;
    }
    J->S.rl.n = 0;
    for (int s = 0; s < S; ++s) {
        double alpha, phi, ds[3];
        or_subray_angles(q, 0.5 * sn->divergence_rad, s, &alpha, &phi);
        or_subray_dir(sn, q, s, d, ds);
        int64_t ev;
        double R;
        uint32_t sf = 0;
        int64_t fh = J->force_hit ? J->force_hit[row * S + s] : OR_FREE_HIT;
        if (fh != OR_FREE_HIT) trace_subray_forced(J, k, s, o, ds, alpha, fh, &sf, &ev, &R);
        else trace_subray(J, k, s, o, ds, alpha, &sf, &ev, &R);
        flags |= sf;
        if (out->subray_flags) out->subray_flags[row * S + s] = sf;
        if (out->subray_hit) out->subray_hit[row * S + s] = ev;
        if (out->subray_range) out->subray_range[row * S + s] = R;
    }
    rlist* RL = &J->S.rl;
    double* W = &out->waveform[row * nb];
    for (int b = 0; b < nb; ++b) W[b] = 0.0;
    out->echo_count[row] = 0;
    for (int e = 0; e < K; ++e) {
        out->echo_bin[row * K + e] = -1;
        out->echo_amp[row * K + e] = 0.0;
        out->echo_range[row * K + e] = 0.0;
        out->echo_range_clean[row * K + e] = 0.0;
        out->echo_object[row * K + e] = -1;
        if (out->echo_object_alt) out->echo_object_alt[row * K + e] = -1;
        if (out->echo_width) out->echo_width[row * K + e] = 0.0;
    }
    if (RL->n == 0) {
        out->window_bin[row] = OR_NO_WINDOW;
        out->flags[row] = flags | OR_F_NOHIT;
        return;
    }
    /* 5. window anchored on the nearest return (reading: integer start bin m on
     * the global grid t = j * bin, n_pre bins of lead for the Gaussian). */
    double Rmin = RL->r[0].R;
    for (int64_t i = 1; i < RL->n; ++i)
        if (RL->r[i].R < Rmin) Rmin = RL->r[i].R;
    const double dt = sn->bin_ns;
    int32_t m;
    if (J->fixed_window) {
        m = J->fixed_window[row];
    } else {
        double x = delay_ns(Rmin) / dt;
        double fr = x - floor(x);
        if (fr < 1e-6 || fr > 1.0 - 1e-6) flags |= OR_F_WIN;
        m = (int32_t)floor(x) - n_pre_bins(sn);
    }
    out->window_bin[row] = m;
    /* W[b] = sum over returns (subray order, then march order) of P p(t_b - tau) */
    for (int64_t i = 0; i < RL->n; ++i) {
        double tau = delay_ns(RL->r[i].R);
        for (int b = 0; b < nb; ++b)
            W[b] += RL->r[i].P * or_pulse_shape(sn, (double)(m + b) * dt - tau);
    }
    /* 6. echoes: 3-bin local maxima at or above threshold * max(W), first K by bin */
    int32_t eb[OR_MAX_ECHOES];
    int overflow = 0, near = 0;
    int ne = or_echo_peaks(W, nb, sn->echo_threshold_rel, K, eb, &overflow, &near);
    if (near) flags |= OR_F_ECHO;
    if (overflow) flags |= OR_F_OVERFLOW;
    for (int e = 0; e < ne; ++e) {
        int b = eb[e];
        double tb = (double)(m + b) * dt;
        double Rc = sn->pulse_shape == 0 ? 0.5 * OR_C * tb * 1e-9
                                         : 0.5 * OR_C * (tb - 2.0 * sn->pulse_length_ns / 1.75) * 1e-9;
        uint32_t w[4];
        draw(J->seed, lg->leg_id, k, 1, (uint32_t)e, 0, w);
        double u1 = or_uniform24(w[0]), u2 = or_uniform24(w[1]);
        double z = sqrt(-2.0 * log(u1)) * cos(2.0 * OR_PI * u2);
        int tie = 0;
        int64_t sid = -1;
        int64_t bid = echo_object_list(sn, RL->r, RL->n, tb, &tie, &sid);
        if (tie) flags |= OR_F_OBJ;
        if (out->echo_object_alt) out->echo_object_alt[row * K + e] = sid;
        out->echo_bin[row * K + e] = b;
        out->echo_amp[row * K + e] = W[b];
        out->echo_range_clean[row * K + e] = Rc;
        out->echo_range[row * K + e] = Rc + sn->range_noise_sigma_m * z;
        out->echo_object[row * K + e] = bid;
        if (out->echo_width && sn->pulse_shape == 0) {
            int ftie = 0;
            double sig_b = sn->pulse_fwhm_ns / (2.0 * sqrt(2.0 * log(2.0))) / dt;
            out->echo_width[row * K + e] = or_echo_width(W, nb, b, sig_b, &ftie) * dt;
            if (ftie) flags |= OR_F_FIT;
        }
    }
    out->echo_count[row] = ne;
    out->flags[row] = flags;
}

/* ------------------------------------------------------------------------ */
/* 7. echo width (Sec. 3.4: an optional non-linear least-squares estimate).  */
/* Reading: model f(b) = A exp(-(b - mu)^2 / (2 s^2)) in bin units over the  */
/* bins within ceil(2 sigma_b) of the echo; Levenberg-Marquardt with the     */
/* damping added to the diagonal (H + lambda diag(H)), lambda from 1e-3,     */
/* divided by 10 on an accepted step and multiplied by 10 on a rejected      */
/* one; exactly 10 iterations; the width is the fitted s.                   */
/* ------------------------------------------------------------------------ */
static double fit_sse(const double* W, int lo, int hi, double A, double mu, double s) {
    double e = 0.0;
    for (int b = lo; b <= hi; ++b) {
        double x = ((double)b - mu) / s;
        double r = W[b] - A * exp(-0.5 * x * x);
        e += r * r;
    }
    return e;
}

double or_echo_width(const double* W, int nb, int p, double sigma_b, int* near_tie) {
    int h = (int)ceil(2.0 * sigma_b);
    int lo = p - h < 0 ? 0 : p - h, hi = p + h > nb - 1 ? nb - 1 : p + h;
    double A = W[p], mu = (double)p, s = sigma_b, lam = 1e-3;
    double E = fit_sse(W, lo, hi, A, mu, s);
    double energy = 0.0;   /* scale of FP32 rounding in the errors */
    for (int b = lo; b <= hi; ++b) energy += W[b] * W[b];
    if (near_tie) *near_tie = 0;
    for (int it = 0; it < 10; ++it) {
        /* normal equations of the linearised model at (A, mu, s) */
        double H[3][3] = {{0}}, g[3] = {0};
        for (int b = lo; b <= hi; ++b) {
            double u = (double)b - mu;
            double e = exp(-0.5 * u * u / (s * s));
            double Jr[3] = {e, A * e * u / (s * s), A * e * u * u / (s * s * s)};
            double r = W[b] - A * e;
            for (int i = 0; i < 3; ++i) {
                g[i] += Jr[i] * r;
                for (int j = 0; j < 3; ++j) H[i][j] += Jr[i] * Jr[j];
            }
        }
        double M[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[i][j] = H[i][j] + (i == j ? lam * H[i][i] : 0.0);
        /* Cramer's rule for M delta = g */
        double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                     M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                     M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        if (!(fabs(det) > 0.0)) break;
        double dA = (g[0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                     M[0][1] * (g[1] * M[2][2] - M[1][2] * g[2]) +
                     M[0][2] * (g[1] * M[2][1] - M[1][1] * g[2])) / det;
        double dmu = (M[0][0] * (g[1] * M[2][2] - M[1][2] * g[2]) -
                      g[0] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                      M[0][2] * (M[1][0] * g[2] - g[1] * M[2][0])) / det;
        double ds = (M[0][0] * (M[1][1] * g[2] - g[1] * M[2][1]) -
                     M[0][1] * (M[1][0] * g[2] - g[1] * M[2][0]) +
                     g[0] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) / det;
        double s2 = s + ds;
        double E2 = s2 > 0.0 ? fit_sse(W, lo, hi, A + dA, mu + dmu, s2) : INFINITY;
        /* a decision FP32 may take the other way, on a step that matters */
        if (near_tie && s2 > 0.0 && fabs(E2 - E) <= 1e-6 * energy && fabs(ds) > 1e-5 * s) *near_tie = 1;
        if (E2 < E) {
            A += dA; mu += dmu; s = s2; E = E2;
            lam *= 0.1;
        } else {
            lam *= 10.0;
        }
    }
    return s;
}

int64_t or_trace_returns(const or_scene* sc, const or_scanner* sn, const double o[3],
                         const double ds[3], double alpha, int mode, uint64_t seed, uint32_t leg_id,
                         int64_t pulse, int s, int64_t cap, double* R, double* P, int64_t* id,
                         uint32_t* flags) {
    job_t J;
    memset(&J, 0, sizeof(J));
    J.sc = sc; J.sn = sn; J.mode = mode; J.seed = seed;
    or_leg lg;
    memset(&lg, 0, sizeof(lg));
    lg.leg_id = leg_id;
    J.lg = &lg;
    int64_t ev;
    double evR;
    uint32_t f = 0;
    trace_subray(&J, pulse, s, o, ds, alpha, &f, &ev, &evR);
    int64_t n = J.S.rl.n;
    for (int64_t i = 0; i < n && i < cap; ++i) {
        R[i] = J.S.rl.r[i].R;
        P[i] = J.S.rl.r[i].P;
        id[i] = J.S.rl.r[i].id;
    }
    if (flags) *flags = f;
    free(J.S.vl.v);
    free(J.S.rl.r);
    return n;
}

static void* worker(void* arg) {
    job_t* J = (job_t*)arg;
    for (int64_t r = J->begin; r < J->end; ++r) simulate_pulse(J, r);
    return NULL;
}

static int n_threads_default(int n_threads) {
    if (n_threads > 0) return n_threads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

static int run_jobs(job_t* proto, int64_t n, int n_threads, job_t** jobs_out, int* nt_out) {
    int nt = n_threads_default(n_threads);
    if (nt > n) nt = (int)(n > 0 ? n : 1);
    job_t* jobs = (job_t*)calloc(nt, sizeof(job_t));
    pthread_t* th = (pthread_t*)calloc(nt, sizeof(pthread_t));
    for (int i = 0; i < nt; ++i) {
        jobs[i] = *proto;
        memset(&jobs[i].S, 0, sizeof(scratch_t));
        jobs[i].begin = n * i / nt;
        jobs[i].end = n * (i + 1) / nt;
    }
    for (int i = 1; i < nt; ++i) pthread_create(&th[i], NULL, worker, &jobs[i]);
    worker(&jobs[0]);
    for (int i = 1; i < nt; ++i) pthread_join(th[i], NULL);
    free(th);
    *jobs_out = jobs;
    *nt_out = nt;
    return 0;
}

static void free_jobs(job_t* jobs, int nt) {
    for (int i = 0; i < nt; ++i) {
        free(jobs[i].S.vl.v);
        free(jobs[i].S.rl.r);
        free(jobs[i].S.gid);
        free(jobs[i].S.gval);
    }
    free(jobs);
}

int or_scan(const or_scene* sc, const or_scanner* sn, const or_leg* lg,
            const int64_t* pulses, int64_t n, int mode, uint64_t seed,
            const int32_t* fixed_window, const int64_t* force_hit, const or_out* out,
            int n_threads) {
    if (n <= 0) return 0;
    if (sn->max_echoes < 1 || sn->max_echoes > OR_MAX_ECHOES) return -1;
    job_t proto;
    memset(&proto, 0, sizeof(proto));
    proto.sc = sc; proto.sn = sn; proto.lg = lg; proto.pulses = pulses; proto.n = n;
    proto.mode = mode; proto.seed = seed; proto.fixed_window = fixed_window; proto.out = out;
    proto.force_hit = force_hit;
    job_t* jobs;
    int nt;
    run_jobs(&proto, n, n_threads, &jobs, &nt);
    free_jobs(jobs, nt);
    return 0;
}

int or_adjoint(const or_scene* sc, const or_scanner* sn, const or_leg* lg,
               const int64_t* pulses, int64_t n, const double* g, const int32_t* window,
               double* d_refl, double* d_density, int n_threads) {
    if (n <= 0) return 0;
    job_t proto;
    memset(&proto, 0, sizeof(proto));
    proto.sc = sc; proto.sn = sn; proto.lg = lg; proto.pulses = pulses; proto.n = n;
    proto.mode = 1; proto.fixed_window = window; proto.g = g; proto.adjoint = 1;
    job_t* jobs;
    int nt;
    run_jobs(&proto, n, n_threads, &jobs, &nt);
    /* deterministic merge in thread order */
    for (int i = 0; i < nt; ++i) {
        for (int64_t j = 0; j < jobs[i].S.gn; ++j) {
            int64_t id = jobs[i].S.gid[j];
            if (id < sc->n_tri) d_refl[id] += jobs[i].S.gval[j];
            else d_density[id - sc->n_tri] += jobs[i].S.gval[j];
        }
    }
    free_jobs(jobs, nt);
    return 0;
}
