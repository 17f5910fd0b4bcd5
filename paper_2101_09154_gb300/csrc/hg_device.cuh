// hg_device.cuh - device-side data layout and building blocks of the pulse kernels.
//
// Everything here runs on sm_103a.  FP32 is used for the BVH traversal, the
// voxel march and the waveform; FP64 only where the method's tolerances need
// it (pulse pose, subray direction, final hit range, voxel segment ends).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

namespace hg {

constexpr int kMaxMesh = 16;
constexpr int kMaxScenes = 16;
constexpr int kMaxScanners = 4;
constexpr int kMaxLegs = 128;
constexpr int kMaxGrids = 4096;        // voxel grids per scene
constexpr double kC = 299792458.0;        // speed of light (Sec. 3.4)
constexpr double kPi = 3.14159265358979323846;
constexpr double kDelayPerMetre = 2.0e9 / kC;  // round-trip delay in ns per metre of range
// the same constant as a float pair, and half the speed of light in m/ns
constexpr float kDelayHi = (float)kDelayPerMetre;
constexpr float kDelayLo = (float)(kDelayPerMetre - (double)kDelayHi);
constexpr float kHalfCns = (float)(0.5e-9 * kC);

// ---------------------------------------------------------------------------
// scene: BVH nodes, packed triangles, per-mesh reflectance, optional grid
// ---------------------------------------------------------------------------
// Internal node i occupies nodes[4i .. 4i+3] (64 bytes):
//   [0] = (c0.lo.x, c0.lo.y, c0.lo.z, c0.hi.x)
//   [1] = (c0.hi.y, c0.hi.z, c1.lo.x, c1.lo.y)
//   [2] = (c1.lo.z, c1.hi.x, c1.hi.y, c1.hi.z)
//   [3] = (child0, child1, parent, axis) as int bits
// child >= 0 is an internal node, child < 0 is the leaf ~tri (a triangle).
// child0 is the lower child along `axis`, so the near child of a ray with
// d[axis] >= 0 is child0.  Triangle t occupies tris[3t .. 3t+2]:
//   (v0, global id), (v1, mesh), (v2, face).
constexpr int64_t kMaxPulseIndex = (int64_t)1 << 44;   // pulse indices of the draws' counter
constexpr int64_t kMaxVoxelId = (int64_t)1 << 40;      // voxel ids of the draws' counter
constexpr int kReturnListCap = 256;   // expected-mode returns listed per lane and pulse
constexpr int kConeCap = 16;          // candidate triangles per pulse in shared memory
constexpr int kConeExt = 112;         // more in global scratch (non-static scans)
constexpr int kBrickLog2 = 2;   // 4^3-voxel bricks for empty-space skipping
constexpr int kBrick = 1 << kBrickLog2;

// One voxel grid (Sec. 3.5.4).  Voxel (x,y,z) spans g0 + [x, x+1) cell etc.;
// its id in outputs is n_tri + vox_off + (z ny + y) nx + x, and its
// transmission draw is keyed by vox_off + (z ny + y) nx + x.
struct DevGrid {
    const float* density;       // [nz][ny][nx]
    const uint32_t* occ;        // brick occupancy bits (x fastest), NULL: not used
    const float* lad;           // leaf-angle table G(mu_i), mu_i = i/(lad_n-1)
    float* ddens;               // adjoint: dL/ddensity of this grid, NULL: not wanted
    float g0[3];
    float cell;
    int32_t dims[3];
    int32_t opaque;             // non-transmissive voxels
    int32_t bdims[3];           // bricks of kBrick^3 voxels per axis
    int32_t lad_n;              // 0: constant G
    float G, leaf_refl;
    int64_t vox_off;            // voxels of the scene's earlier grids
    float icell_h, icell_l;     // 1 / cell as a float pair, formed on the host
};

struct DevScene {
    const float4* nodes;
    const float4* nodes4;       // 4-wide collapse of the same tree (8 float4 per node)
    const float4* tris;
    const int32_t* tri_index;   // global triangle id -> packed (sorted) position
    const float* refl[kMaxMesh];
    int32_t mesh_first[kMaxMesh + 1];
    int32_t n_tri, n_int, n_mesh, has_grid;
    int32_t n_node4;
    int32_t n_grid;
    DevGrid grid;               // the grid of a one-grid scene
    const DevGrid* grids;       // all grids of a scene with several (device)
    const float4* gnodes;       // BVH over their boxes: 4 float4 per node, leaf ~grid
};

// sigma = G density (Eq. extinction).  With a leaf-angle table (Table ladlut)
// G depends on the subray direction: linear interpolation at mu = |d_z| of the
// unit direction between entries at mu_i = i/(n-1); without one, the grid's
// constant G.  Evaluated once per subray and grid, before its march.
__device__ __forceinline__ float proj_factor(const DevGrid& g, float dz) {
    if (g.lad_n < 2) return g.G;
    const float t = fminf(fabsf(dz), 1.0f) * (float)(g.lad_n - 1);   // NaN -> the last entry
    const int i = min((int)t, g.lad_n - 2);
    const float f = t - (float)i;
    const float g0 = __ldg(g.lad + i), g1 = __ldg(g.lad + i + 1);
    return fmaf(f, g1 - g0, g0);
}

// Instrument constants derived once per call (host side, FP64).
struct DevScanner {
    double prf;
    double bin_ns;
    double echo_offset_ns;   // pulse peak delay removed from echo ranges (0: Gaussian)
    double theta_r;          // half divergence
    double scan_freq, amax, head_rate, el_min, el_max;
    float w0sq;              // beam waist squared
    float zk;                // lambda / (pi w0^2)
    float focus;
    float pconst;            // I0 Dr^2 eta_sys eta_atm / 4
    float gk2;               // Gaussian: log2(e) / (2 sigma^2)   [1/ns^2]
    float ctau_inv;          // Carlsson: 1/tau                   [1/ns]
    float cut_lo, cut_hi;    // support of the pulse shape around the delay [ns]
    float thr_rel, noise_sigma;
    double bins_per_metre;   // 2 / (c * bin) in bins per metre of range
    float inv_bin;           // 1 / bin_ns
    float bpm_hi, bpm_lo;    // bins_per_metre as a float pair
    float bin_hi, bin_lo;    // bin_ns as a float pair
    float echo_offset_f;     // echo_offset_ns in FP32
    float inv_s2;            // Gaussian: 1 / sigma^2 [1/ns^2]
    float sigma_bins;        // Gaussian: sigma / bin
    int32_t q_default, pulse_shape, n_bins, max_echoes;
    int32_t deflector, n_az, n_el, n_pre;
    int32_t n_fibres, pad0;
};

// One leg, with offsets into the concatenated outputs.
struct DevLeg {
    double start[3];
    double dir[3];           // unit vector start -> end (linear platform)
    double length, speed, t0;
    double rpy[3];           // roll, pitch, yaw (heading included)
    double platform_noise;   // sigma of the per-pulse platform position noise (m)
    int64_t n_pulses;        // pulses scanned: leg pulse indices k_first .. k_first + n_pulses - 1
    int64_t k_first;
    int64_t pulse_off, wave_off, sub_off, echo_off;   // output index of leg pulse k: off + k (x row size)
    int64_t item_begin;      // first work item of this leg
    int32_t scene, scanner, platform, q;
    int32_t S, pulses_per_item;    // pulses per work item
    uint32_t leg_id;
    int32_t pulses_per_sub;        // pulses per subray/waveform batch within an item
};

struct Outputs {
    float* waveform;
    int32_t* window_bin;
    int32_t* echo_count;
    float* echo_range;
    float* echo_amp;
    int32_t* echo_bin;
    int64_t* echo_object;
    uint8_t* pulse_flags;
    int64_t* subray_hit;
    float* subray_range;
    uint32_t* status;
    float* echo_width;           // optional: fitted echo sigma (ns), Gaussian pulses
};

// FP64 pulse pose (origin, unit direction, ONB axes), computed once per pulse.
struct PulseFrame {
    double o[3], d[3], u[3], v[3];
};
// The same pose as kept in shared memory: origin and direction as unevaluated
// float pairs hi + lo (about 48 significant bits), the ONB axes in FP32 (they
// only scale the sub-milliradian subray offsets).
struct PulseFF {
    float oh[3], ol[3];
    float dh[3], dl[3];
    float u[3], v[3];
};
// Per-subray constants: 1 - cos(alpha), sin(alpha)cos(phi), sin(alpha)sin(phi), tan(alpha).
struct SubrayConst {
    float eps, sacp, sasp, tan_a;
};

constexpr uint32_t kPfEchoOverflow = 0x01u;
constexpr uint32_t kPfTraversalCap = 0x02u;
constexpr uint32_t kPfMarchCap = 0x04u;
constexpr uint32_t kPfNoReturn = 0x08u;
constexpr uint32_t kStTraversalCap = 0x01u;
constexpr uint32_t kStMarchCap = 0x02u;
constexpr uint32_t kStEchoOverflow = 0x04u;
constexpr int32_t kNoWindow = INT32_MIN;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): its 32 x 32 -> 64-bit
// products are single multiplies here (a 64-bit Philox multiply is several).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           uint32_t k0, uint32_t k1, uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t h0 = __umulhi(M0, c0), l0 = M0 * c0;
        const uint32_t h1 = __umulhi(M1, c2), l1 = M1 * c2;
        const uint32_t y0 = h1 ^ c1 ^ k0, y2 = h0 ^ c3 ^ k1;
        c0 = y0; c1 = l1; c2 = y2; c3 = l0;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// One draw's four words.  The 128-bit counter: pulse bits 0-31; pulse bits
// 32-43 | stream << 12 | subray-or-echo index << 14 | voxel id bits 32-39 << 23;
// voxel id bits 0-31; leg id.  The key is the seed.  Streams: 0 voxel
// transmission (index = subray), 1 range noise (index = echo), 2 platform
// noise.  The API keeps pulses below 2^44 and voxel ids below 2^40.
__device__ __forceinline__ void draw4(uint64_t seed, uint32_t leg, int64_t pulse, uint32_t stream,
                                      uint32_t idx, int64_t vox, uint32_t out[4]) {
    const uint64_t p = (uint64_t)pulse, v = (uint64_t)vox;
    philox4x32((uint32_t)p,
               ((uint32_t)(p >> 32) & 0xFFFu) | (stream << 12) | ((idx & 0x1FFu) << 14) |
                   (((uint32_t)(v >> 32) & 0xFFu) << 23),
               (uint32_t)v, leg, (uint32_t)seed, (uint32_t)(seed >> 32), out);
}

// (top 23 bits + 1/2) * 2^-23: odd multiples of 2^-24, exact in FP32
__device__ __forceinline__ float uniform23(uint32_t w) {
    return ((float)(w >> 9) + 0.5f) * (1.0f / 8388608.0f);
}

// ---------------------------------------------------------------------------
// pulse pose (Sec. 3.2, 3.3) in FP64
// ---------------------------------------------------------------------------
// world = Rz(yaw) Ry(pitch) Rx(roll) platform; rot = (sr, cr, sp, cp, sy, cy)
__device__ __forceinline__ void rot_rpy(const double rot[6], double x, double y, double z,
                                        double out[3]) {
    const double sr = rot[0], cr = rot[1], sp = rot[2], cp = rot[3], sy = rot[4], cy = rot[5];
    double y1 = y * cr - z * sr, z1 = y * sr + z * cr;
    double x2 = x * cp + z1 * sp, z2 = -x * sp + z1 * cp;
    out[0] = x2 * cy - y1 * sy;
    out[1] = x2 * sy + y1 * cy;
    out[2] = z2;
}

__device__ __forceinline__ void pulse_frame(const DevScanner& sn, const DevLeg& lg,
                                            const double rot[6], int64_t k, uint64_t seed,
                                            PulseFrame& f) {
    double elapsed = (double)k / sn.prf;
    double t = lg.t0 + elapsed;
    for (int a = 0; a < 3; ++a) f.o[a] = lg.start[a];
    if (lg.platform == 1 && lg.length > 0.0) {
        double s = lg.speed * elapsed;
        if (s > lg.length) s = lg.length;
        for (int a = 0; a < 3; ++a) f.o[a] = lg.start[a] + s * lg.dir[a];
    }
    if (lg.platform_noise > 0.0) {
        // platform noise (Sec. 3.7): N(0, sigma) per axis, Box-Muller on the
        // Philox draw of stream 2 for this pulse
        uint32_t w[4];
        draw4(seed, lg.leg_id, k, 2u, 0u, 0, w);
        const double r1 = sqrt(-2.0 * log((double)uniform23(w[0])));
        const double r2 = sqrt(-2.0 * log((double)uniform23(w[2])));
        const double a1 = 2.0 * kPi * (double)uniform23(w[1]), a2 = 2.0 * kPi * (double)uniform23(w[3]);
        f.o[0] += lg.platform_noise * r1 * cos(a1);
        f.o[1] += lg.platform_noise * r1 * sin(a1);
        f.o[2] += lg.platform_noise * r2 * cos(a2);
    }
    double x, y, z;
    switch (sn.deflector) {
    case 0: {
        double ph = sn.scan_freq * t;
        ph -= floor(ph);
        double th = -sn.amax + 2.0 * sn.amax * ph;
        double st, ct;
        sincos(th, &st, &ct);
        x = 0.0; y = st; z = -ct;
        break;
    }
    case 1: {
        // sin(2 pi f t) from the phase's fractional part: no FP64 argument reduction
        double ph = sn.scan_freq * t;
        ph -= floor(ph);
        double th = sn.amax * sinpi(2.0 * ph);
        double st, ct;
        sincos(th, &st, &ct);
        x = 0.0; y = st; z = -ct;
        break;
    }
    case 4: {
        // fibre-optic line: pulse k leaves fibre k mod n, fanned over [-max, max]
        const int64_t n = sn.n_fibres > 0 ? sn.n_fibres : 1;
        const int64_t i = k % n;
        const double th = n > 1 ? -sn.amax + 2.0 * sn.amax * (double)i / (double)(n - 1) : 0.0;
        double st, ct;
        sincos(th, &st, &ct);
        x = 0.0; y = st; z = -ct;
        break;
    }
    case 5: {
        // Palmer (slanted rotating mirror): a cone at max off nadir, azimuth 2 pi frac(f t)
        double ph = sn.scan_freq * t;
        ph -= floor(ph);
        double sa, ca, sm, cm;
        sincos(2.0 * kPi * ph, &sa, &ca);
        sincos(sn.amax, &sm, &cm);
        x = sm * ca; y = sm * sa; z = -cm;
        break;
    }
    case 2: {
        int64_t i = k / sn.n_el, j = k % sn.n_el;
        double az = 2.0 * kPi * (double)i / (double)sn.n_az;
        double el = sn.el_min;
        if (sn.n_el > 1) el = sn.el_min + (sn.el_max - sn.el_min) * (double)j / (double)(sn.n_el - 1);
        double sa, ca, se, ce;
        sincos(az, &sa, &ca);
        sincos(el, &se, &ce);
        x = ce * ca; y = ce * sa; z = se;
        break;
    }
    default: {
        double az = sn.head_rate * t;
        double ph = sn.scan_freq * t;
        ph -= floor(ph);
        double el = -sn.amax + 2.0 * sn.amax * ph;
        double sa, ca, se, ce;
        sincos(az, &sa, &ca);
        sincos(el, &se, &ce);
        x = ce * ca; y = ce * sa; z = se;
        break;
    }
    }
    rot_rpy(rot, x, y, z, f.d);
    // orthonormal basis around d (Duff et al., JCGT 2017), in FP32: it only
    // scales the sub-milliradian subray offsets, and is kept as floats
    const float d0 = (float)f.d[0], d1 = (float)f.d[1], d2 = (float)f.d[2];
    const float sign = copysignf(1.0f, d2);
    const float a = -1.0f / (sign + d2);
    const float b = d0 * d1 * a;
    f.u[0] = 1.0f + sign * d0 * d0 * a;
    f.u[1] = sign * b;
    f.u[2] = -sign * d0;
    f.v[0] = b;
    f.v[1] = sign + d1 * d1 * a;
    f.v[2] = -d1;
}

// subray s of quality q (Sec. 3.4): ring i at angle (i/q) theta_r, floor(2 pi i) per ring
__device__ __forceinline__ void subray_const(int q, double theta_r, int s, SubrayConst& c) {
    double alpha = 0.0, phi = 0.0;
    if (s > 0) {
        int idx = s - 1;
        for (int i = 1; i <= q; ++i) {
            int n = (int)floor(2.0 * kPi * (double)i);
            if (idx < n) {
                alpha = ((double)i / (double)q) * theta_r;
                phi = 2.0 * kPi * (double)idx / (double)n;
                break;
            }
            idx -= n;
        }
    }
    double sa, ca, sp, cp;
    sincos(alpha, &sa, &ca);
    sincos(phi, &sp, &cp);
    // 1 - cos(alpha) without cancellation: 2 sin^2(alpha/2)
    double sh = sin(0.5 * alpha);
    c.eps = (float)(2.0 * sh * sh);
    c.sacp = (float)(sa * cp);
    c.sasp = (float)(sa * sp);
    c.tan_a = (float)tan(alpha);
}

// ---------------------------------------------------------------------------
// float-float helpers (error-free transformations: Knuth TwoSum, FMA TwoProd)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

__device__ __forceinline__ void split_store(const PulseFrame& f, PulseFF& g) {
    for (int a = 0; a < 3; ++a) {
        g.oh[a] = (float)f.o[a];
        g.ol[a] = (float)(f.o[a] - (double)g.oh[a]);
        g.dh[a] = (float)f.d[a];
        g.dl[a] = (float)(f.d[a] - (double)g.dh[a]);
        g.u[a] = (float)f.u[a];
        g.v[a] = (float)f.v[a];
    }
}

// unit subray direction as hi + lo: d_s = (1 - eps) d + sin(a)(cos(p) u + sin(p) v);
// the correction to d is below 2e-4 in size, so FP32 carries it to ~1e-11.
__device__ __forceinline__ void subray_dir_ff(const PulseFF& f, const SubrayConst& c,
                                              float dh[3], float dl[3]) {
    for (int a = 0; a < 3; ++a) {
        float corr = fmaf(-c.eps, f.dh[a], fmaf(c.sacp, f.u[a], c.sasp * f.v[a]));
        float s, e;
        two_sum(f.dh[a], corr, s, e);
        dh[a] = s;
        dl[a] = e + f.dl[a];
    }
}

__device__ __forceinline__ double ff2d(float hi, float lo) { return (double)hi + (double)lo; }

// normalised float pair (|lo| <= ulp(hi)/2) and its order
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_norm(float hi, float lo) {
    FF r;
    two_sum(hi, lo, r.hi, r.lo);
    return r;
}

// s += x with the rounding error of the addition kept in s.lo
__device__ __forceinline__ void ff_acc(FF& s, float x) {
    float h, e;
    two_sum(s.hi, x, h, e);
    s = ff_norm(h, e + s.lo);
}
__device__ __forceinline__ bool ff_less(const FF& a, const FF& b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ FF ff_split(double x) {
    FF r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}
// float-float arithmetic (error-free transformations; about 2^-44 relative)
__device__ __forceinline__ FF ff_add(const FF& a, const FF& b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return ff_norm(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ FF ff_sub(const FF& a, const FF& b) {
    return ff_add(a, FF{-b.hi, -b.lo});
}
__device__ __forceinline__ FF ff_mul(const FF& a, const FF& b) {
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    return ff_norm(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
// 1/b (b.hi != 0): the FP32 quotient r and one Newton step, r + r (1 - b r),
// with 1 - b r formed from the exact product b.hi r
__device__ __forceinline__ FF ff_rcp(const FF& b) {
    const float r = 1.0f / b.hi;
    float p, pe;
    two_prod(b.hi, r, p, pe);
    const float e = ((1.0f - p) - pe) - b.lo * r;
    return ff_norm(r, r * e);
}
__device__ __forceinline__ FF ff_min(const FF& a, const FF& b) { return ff_less(b, a) ? b : a; }
__device__ __forceinline__ FF ff_max(const FF& a, const FF& b) { return ff_less(a, b) ? b : a; }
__device__ __forceinline__ bool ff_eq(const FF& a, const FF& b) { return a.hi == b.hi && a.lo == b.lo; }
// the pair n * c exactly (|n| < 2^24)
__device__ __forceinline__ FF ff_int_mul(int n, float c) {
    float p, e;
    two_prod((float)n, c, p, e);
    return ff_norm(p, e);
}

// floor(a * b) for a normalised pair a and a constant pair (bh, bl)
__device__ __forceinline__ int ff_floor_mul(const FF& a, float bh, float bl) {
    float p, e;
    two_prod(a.hi, bh, p, e);
    e += fmaf(a.hi, bl, a.lo * bh);
    float s, t;
    two_sum(p, e, s, t);
    float f = floorf(s);
    if (f == s && t < 0.0f) f -= 1.0f;
    return (int)f;
}
// a * (bh + bl) - (ch + cl) to FP32, for a product close to c (Sterbenz)
__device__ __forceinline__ float ff_mul_sub(const FF& a, float bh, float bl, float ch, float cl) {
    float p, e;
    two_prod(a.hi, bh, p, e);
    e += fmaf(a.hi, bl, a.lo * bh);
    return (p - ch) + (e - cl);
}

// ---------------------------------------------------------------------------
// FP32 ray for traversal
// ---------------------------------------------------------------------------
struct RayF {
    float ox, oy, oz;        // origin: high words of the float-float pair
    float lx, ly, lz;        // origin: low words (the triangle test subtracts both)
    float idx, idy, idz;     // 1/d (tiny components replaced by +-1e-20)
    float oix, oiy, oiz;     // o * (1/d)
    float sx, sy, sz;        // watertight shear constants
    int kx, ky, kz;
};

__device__ __forceinline__ float safe_inv(float d) {
    return 1.0f / (fabsf(d) < 1e-20f ? copysignf(1e-20f, d) : d);
}

__device__ __forceinline__ float sel3(int k, float x, float y, float z) {
    return k == 0 ? x : (k == 1 ? y : z);
}

// origin and watertight-test setup (Woop, Benthin & Wald, JCGT 2013): all a
// ray needs for tri_hit
__device__ __forceinline__ void make_ray_tri(const float o[3], const float ol[3], const float d[3],
                                             RayF& r) {
    r.ox = o[0]; r.oy = o[1]; r.oz = o[2];
    r.lx = ol[0]; r.ly = ol[1]; r.lz = ol[2];
    const float dx = d[0], dy = d[1], dz = d[2];
    const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const float dkz = sel3(kz, dx, dy, dz);
    if (dkz < 0.0f) { int t = kx; kx = ky; ky = t; }
    r.kx = kx; r.ky = ky; r.kz = kz;
    const float inv = 1.0f / dkz;
    r.sx = sel3(kx, dx, dy, dz) * inv;
    r.sy = sel3(ky, dx, dy, dz) * inv;
    r.sz = inv;
}

// slab-test setup (box tests of the traversals)
__device__ __forceinline__ void make_ray_slab(const float d[3], RayF& r) {
    r.idx = safe_inv(d[0]); r.idy = safe_inv(d[1]); r.idz = safe_inv(d[2]);
    r.oix = r.ox * r.idx; r.oiy = r.oy * r.idy; r.oiz = r.oz * r.idz;
}

__device__ __forceinline__ void make_ray(const float o[3], const float ol[3], const float d[3], RayF& r) {
    make_ray_tri(o, ol, d, r);
    make_ray_slab(d, r);
}

// slab test of one box against [0, tmax]
__device__ __forceinline__ bool slab(const RayF& r, float lx, float ly, float lz, float hx,
                                     float hy, float hz, float tmax) {
    float tx0 = fmaf(lx, r.idx, -r.oix), tx1 = fmaf(hx, r.idx, -r.oix);
    float ty0 = fmaf(ly, r.idy, -r.oiy), ty1 = fmaf(hy, r.idy, -r.oiy);
    float tz0 = fmaf(lz, r.idz, -r.oiz), tz1 = fmaf(hz, r.idz, -r.oiz);
    float tmn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
    float tmx = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
    return tmn <= tmx;
}

// Watertight ray-triangle test; on a hit closer than t_best updates t_best.
__device__ __forceinline__ bool tri_hit(const RayF& r, float4 a, float4 b, float4 c,
                                        float& t_best) {
    // Vertices relative to the float-float origin.  The first difference is
    // exact for a vertex within a factor of two of the origin's coordinate,
    // so a far-from-zero origin (a street 2 km long) keeps its low word; an
    // origin rounded to FP32 alone moves edge crossings by its rounding error
    // (up to 6e-5 m at 1 km), more than the edge distance hits are resolved to.
    // Each vertex maps the same way in every triangle: still watertight.
    float Ax = (a.x - r.ox) - r.lx, Ay = (a.y - r.oy) - r.ly, Az = (a.z - r.oz) - r.lz;
    float Bx = (b.x - r.ox) - r.lx, By = (b.y - r.oy) - r.ly, Bz = (b.z - r.oz) - r.lz;
    float Cx = (c.x - r.ox) - r.lx, Cy = (c.y - r.oy) - r.ly, Cz = (c.z - r.oz) - r.lz;
    float akx = sel3(r.kx, Ax, Ay, Az), aky = sel3(r.ky, Ax, Ay, Az), akz = sel3(r.kz, Ax, Ay, Az);
    float bkx = sel3(r.kx, Bx, By, Bz), bky = sel3(r.ky, Bx, By, Bz), bkz = sel3(r.kz, Bx, By, Bz);
    float ckx = sel3(r.kx, Cx, Cy, Cz), cky = sel3(r.ky, Cx, Cy, Cz), ckz = sel3(r.kz, Cx, Cy, Cz);
    float ax_ = fmaf(-r.sx, akz, akx), ay_ = fmaf(-r.sy, akz, aky);
    float bx_ = fmaf(-r.sx, bkz, bkx), by_ = fmaf(-r.sy, bkz, bky);
    float cx_ = fmaf(-r.sx, ckz, ckx), cy_ = fmaf(-r.sy, ckz, cky);
    float U = cx_ * by_ - cy_ * bx_;
    float V = ax_ * cy_ - ay_ * cx_;
    float W = bx_ * ay_ - by_ * ax_;
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        // edge case: recompute the edge functions in double precision
        U = (float)((double)cx_ * (double)by_ - (double)cy_ * (double)bx_);
        V = (float)((double)ax_ * (double)cy_ - (double)ay_ * (double)cx_);
        W = (float)((double)bx_ * (double)ay_ - (double)by_ * (double)ax_);
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
    float det = U + V + W;
    if (det == 0.0f) return false;
    float T = U * (r.sz * akz) + V * (r.sz * bkz) + W * (r.sz * ckz);
    if (det < 0.0f) { det = -det; T = -T; }
    if (T <= 0.0f || T >= t_best * det) return false;
    t_best = T / det;
    return true;
}

// ---------------------------------------------------------------------------
// Warp-coherent stackless BVH traversal (closest hit).
//
// All 32 lanes call it together; every branch depends only on warp-uniform
// values (node index, depth, trail, votes), so the warp walks one node
// sequence while each lane keeps its own closest hit.  There is no stack:
// the walk goes up through parent links, and a 128-bit trail holds, per
// depth, whether the far child of the node on the current path was hit by
// some lane when the node was entered.  On the way up a node whose far child
// was already culled is passed with a 16-byte link load and no box test
// (t_best only shrinks, so a culled box stays culled).  A Karras tree over
// 63-bit codes with index tie-breaks is at most 95 levels deep, so the trail
// never overflows; the loop is also bounded by 3 x (internal nodes).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void child_box(const float4& n0, const float4& n1, const float4& n2,
                                          bool second, float b[6]) {
    if (!second) { b[0] = n0.x; b[1] = n0.y; b[2] = n0.z; b[3] = n0.w; b[4] = n1.x; b[5] = n1.y; }
    else { b[0] = n1.z; b[1] = n1.w; b[2] = n2.x; b[3] = n2.y; b[4] = n2.z; b[5] = n2.w; }
}

__device__ __forceinline__ void leaf_test(const DevScene& S, const RayF& r, int child, bool h,
                                          float& t_best, int& hit) {
    if (h) {
        int t = ~child;
        const float4* tp = S.tris + 3 * (size_t)t;
        float4 a = __ldg(tp), b = __ldg(tp + 1), c = __ldg(tp + 2);
        if (tri_hit(r, a, b, c, t_best)) hit = t;
    }
}

__device__ __forceinline__ void traverse(const DevScene& S, const RayF& r, bool active,
                                         float& t_best, int& hit, uint32_t& flags) {
    const unsigned full = 0xffffffffu;
    if (S.n_tri == 0) return;
    if (S.n_int == 0) {
        if (active) {
            float4 a = __ldg(&S.tris[0]), b = __ldg(&S.tris[1]), c = __ldg(&S.tris[2]);
            if (tri_hit(r, a, b, c, t_best)) hit = 0;
        }
        return;
    }
    unsigned am = __ballot_sync(full, active);
    if (am == 0u) return;
    int rep = __ffs(am) - 1;
    // near/far order from one representative ray of the packet
    const bool px = __shfl_sync(full, r.idx, rep) >= 0.0f;
    const bool py = __shfl_sync(full, r.idy, rep) >= 0.0f;
    const bool pz = __shfl_sync(full, r.idz, rep) >= 0.0f;
    const float tscale = 1.0f + 4.0f * 1.1920929e-7f;
    uint64_t trail0 = 0, trail1 = 0;   // bit d: far child at depth d still pending
    int cur = 0, depth = 0;
    bool down = true;
    const int max_steps = 3 * S.n_int + 8;
    for (int step = 0;; ++step) {
        if (step >= max_steps) { flags |= kPfTraversalCap; break; }
        const float4* nd = S.nodes + 4 * (size_t)cur;
        if (down) {
            float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
            int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
            int axis = __float_as_int(n3.w) & 3;
            bool pos = axis == 0 ? px : (axis == 1 ? py : pz);
            int cn = pos ? c0 : c1, cf = pos ? c1 : c0;
            float bn[6], bf[6];
            child_box(n0, n1, n2, !pos, bn);
            child_box(n0, n1, n2, pos, bf);
            float tmax = t_best * tscale;
            bool hn = active && slab(r, bn[0], bn[1], bn[2], bn[3], bn[4], bn[5], tmax);
            bool hf = active && slab(r, bf[0], bf[1], bf[2], bf[3], bf[4], bf[5], tmax);
            bool an = __any_sync(full, hn), af = __any_sync(full, hf);
            if (an && cn < 0) { leaf_test(S, r, cn, hn, t_best, hit); an = false; }
            if (af && cf < 0) {
                // re-check the far leaf against the (possibly) shorter t_best
                bool h2 = hf && slab(r, bf[0], bf[1], bf[2], bf[3], bf[4], bf[5], t_best * tscale);
                leaf_test(S, r, cf, h2, t_best, hit);
                af = false;
            }
            if (an) {
                if (af) { if (depth < 64) trail0 |= 1ull << depth; else trail1 |= 1ull << (depth - 64); }
                cur = cn; ++depth;
                continue;
            }
            if (af) { cur = cf; ++depth; continue; }
            down = false;   // nothing below: leave this node
            continue;
        }
        // going up: leave `cur` for its parent
        if (cur == 0) break;
        int parent = __float_as_int(__ldg(nd + 3).z);
        --depth;
        bool pending = depth < 64 ? ((trail0 >> depth) & 1ull) : ((trail1 >> (depth - 64)) & 1ull);
        cur = parent;
        if (!pending) continue;
        if (depth < 64) trail0 &= ~(1ull << depth); else trail1 &= ~(1ull << (depth - 64));
        // the far child of `parent` is still pending: re-test it now
        const float4* pd = S.nodes + 4 * (size_t)parent;
        float4 n0 = __ldg(pd), n1 = __ldg(pd + 1), n2 = __ldg(pd + 2), n3 = __ldg(pd + 3);
        int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
        int axis = __float_as_int(n3.w) & 3;
        bool pos = axis == 0 ? px : (axis == 1 ? py : pz);
        int cf = pos ? c1 : c0;
        float bf[6];
        child_box(n0, n1, n2, pos, bf);
        bool hf = active && slab(r, bf[0], bf[1], bf[2], bf[3], bf[4], bf[5], t_best * tscale);
        if (__any_sync(full, hf)) {
            // cf is internal: leaves were tested when `parent` was entered
            cur = cf; ++depth; down = true;
        }
    }
}

// ---------------------------------------------------------------------------
// Beam-cone candidate search.  The subrays of a pulse leave one origin inside
// a cone of half-angle atan(ta) around the pulse axis: a subray point at
// distance t lies within t * ta of the axis point at the same t.  A box all of
// whose points are within D of the origin (D: distance to its farthest
// corner) and that a subray meets is therefore met by the axis ray once it is
// grown by R = ta * D on every side: on axis a that widens the slab interval
// by R / |d_a| (ta carries a margin for FP32 rounding).  The warp walks the
// union of its lanes' cones (one pulse per lane), without range culling; the
// leaves met are the pulse's candidate triangles, in walk order.  The closest hit of every subray is among them,
// so testing a subray against the list gives its traversal result.
// n > cap + ecap: the list overflowed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool cone_slab(const RayF& r, float ta, const float ad[3], const float b[6]) {
    const float fx = fmaxf(fabsf(b[0] - r.ox), fabsf(b[3] - r.ox));
    const float fy = fmaxf(fabsf(b[1] - r.oy), fabsf(b[4] - r.oy));
    const float fz = fmaxf(fabsf(b[2] - r.oz), fabsf(b[5] - r.oz));
    // q rsqrt(q) is within 2^-22 of sqrt(q): far inside the cone's 0.1% angle
    // margin (ta), so the test stays conservative at a third of the cost
    const float q = fmaxf(fmaf(fx, fx, fmaf(fy, fy, fz * fz)), 1.0e-30f);
    const float R = ta * (q * rsqrtf(q));
    float tx0 = fmaf(b[0], r.idx, -r.oix), tx1 = fmaf(b[3], r.idx, -r.oix);
    float ty0 = fmaf(b[1], r.idy, -r.oiy), ty1 = fmaf(b[4], r.idy, -r.oiy);
    float tz0 = fmaf(b[2], r.idz, -r.oiz), tz1 = fmaf(b[5], r.idz, -r.oiz);
    float tmn = fmaxf(fmaxf(fminf(tx0, tx1) - R * ad[0], fminf(ty0, ty1) - R * ad[1]),
                      fmaxf(fminf(tz0, tz1) - R * ad[2], 0.0f));
    float tmx = fminf(fminf(fmaxf(tx0, tx1) + R * ad[0], fmaxf(ty0, ty1) + R * ad[1]),
                      fmaxf(tz0, tz1) + R * ad[2]);
    return tmn <= tmx;
}

// candidate i of a pulse: the first cap in shared memory, the next ecap in
// global scratch
__device__ __forceinline__ void cone_store(int32_t* cand, int cap, int32_t* ext, int ecap, int i,
                                           int32_t t) {
    if (i < cap) cand[i] = t;
    else if (i < cap + ecap) ext[i - cap] = t;
}

// The walk runs over the 4-wide collapse of the tree: a node's four slot
// boxes are tested per lane, leaves met go to the lane's list, and the slots
// of internal children met by any lane are visited in slot order; a 4-bit
// mask per level (192 bits for the 48 levels a 95-level binary tree collapses
// to) holds the slots still pending.
__device__ __forceinline__ float f4c(const float4& v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
__device__ __forceinline__ int i4c(const int4& v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

__device__ __forceinline__ void cone_candidates4(const DevScene& S, const RayF& r, float ta,
                                                 bool active, int32_t* cand, int cap,
                                                 int32_t* ext, int ecap, int& n) {
    const unsigned full = 0xffffffffu;
    n = 0;
    if (S.n_tri == 0) return;
    if (S.n_int == 0) {
        if (active) cand[n++] = 0;
        return;
    }
    if (__ballot_sync(full, active) == 0u) return;
    const float ad[3] = {fabsf(r.idx), fabsf(r.idy), fabsf(r.idz)};
    uint64_t tr0 = 0, tr1 = 0, tr2 = 0;   // 4 bits per level: slots still pending
    int cur = 0, depth = 0;
    bool down = true, live = active;
    const int max_steps = 4 * S.n_node4 + 8;
    for (int step = 0;; ++step) {
        if (step >= max_steps || depth >= 48) {
            if (live) n = cap + ecap + 1;
            break;
        }
        const float4* nd = S.nodes4 + 8 * (size_t)cur;
        if (down) {
            const float4 lx = __ldg(nd), ly = __ldg(nd + 1), lz = __ldg(nd + 2);
            const float4 hx = __ldg(nd + 3), hy = __ldg(nd + 4), hz = __ldg(nd + 5);
            const int4 rf = __ldg(reinterpret_cast<const int4*>(nd + 6));
            const int vm = __ldg(reinterpret_cast<const int4*>(nd + 7)).y;
            unsigned hm = 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float b[6] = {f4c(lx, k), f4c(ly, k), f4c(lz, k), f4c(hx, k), f4c(hy, k), f4c(hz, k)};
                if (live && ((vm >> k) & 1) && cone_slab(r, ta, ad, b)) {
                    const int ref = i4c(rf, k);
                    if (ref < 0) {
                        cone_store(cand, cap, ext, ecap, n, ~ref);
                        ++n;
                    } else {
                        hm |= 1u << k;
                    }
                }
            }
            live = live && n <= cap + ecap;
            const unsigned m = __reduce_or_sync(full, live ? hm : 0u);
            if (m) {
                const int first = __ffs(m) - 1;
                const uint64_t rest = (uint64_t)(m & (m - 1)) << (4 * (depth & 15));
                if (depth < 16) tr0 |= rest; else if (depth < 32) tr1 |= rest; else tr2 |= rest;
                cur = i4c(rf, first);
                ++depth;
                continue;
            }
            down = false;
            continue;
        }
        if (cur == 0) break;
        const int parent = __ldg(reinterpret_cast<const int4*>(nd + 7)).x;
        --depth;
        const int sh = 4 * (depth & 15);
        const uint64_t tw = depth < 16 ? tr0 : (depth < 32 ? tr1 : tr2);
        const unsigned rest = (unsigned)(tw >> sh) & 15u;
        cur = parent;
        if (!rest) continue;
        if (!__any_sync(full, live)) break;
        const int first = __ffs(rest) - 1;
        const uint64_t clr = ~((uint64_t)(1u << first) << sh);
        if (depth < 16) tr0 &= clr; else if (depth < 32) tr1 &= clr; else tr2 &= clr;
        cur = i4c(__ldg(reinterpret_cast<const int4*>(S.nodes4 + 8 * (size_t)parent + 6)), first);
        ++depth;
        down = true;
    }
}

// Range to the plane of triangle t (the closest hit found in FP32 at t32).
// The ray is re-anchored at o' = o + t32 d, formed exactly as a float pair;
// the vertices relative to o' are then metre-sized, so the FP32 plane
// intersection from o' is good to ~1e-7 m.  Returns R = t32 + dt as (t32, dt)
// and |cos| of the incidence angle.
__device__ __forceinline__ float refine_hit_ff(const DevScene& S, int t, const float oh[3],
                                               const float ol[3], const float dh[3],
                                               const float dl[3], float t32, float& cos_inc) {
    const float4* tp = S.tris + 3 * (size_t)t;
    float4 a = __ldg(tp), b = __ldg(tp + 1), c = __ldg(tp + 2);
    float oph[3], opl[3];
    for (int k = 0; k < 3; ++k) {
        float p, pe, s, se;
        two_prod(t32, dh[k], p, pe);
        two_sum(oh[k], p, s, se);
        oph[k] = s;
        opl[k] = ol[k] + (pe + se) + t32 * dl[k];
    }
    float w0x = (a.x - oph[0]) - opl[0], w0y = (a.y - oph[1]) - opl[1], w0z = (a.z - oph[2]) - opl[2];
    float e1x = b.x - a.x, e1y = b.y - a.y, e1z = b.z - a.z;
    float e2x = c.x - a.x, e2y = c.y - a.y, e2z = c.z - a.z;
    float nx = e1y * e2z - e1z * e2y;
    float ny = e1z * e2x - e1x * e2z;
    float nz = e1x * e2y - e1y * e2x;
    float num = nx * w0x + ny * w0y + nz * w0z;
    float den = nx * dh[0] + ny * dh[1] + nz * dh[2];
    float n2 = nx * nx + ny * ny + nz * nz;
    cos_inc = fminf(fabsf(den) * rsqrtf(n2), 1.0f);
    return __fdividef(num, den);
}

// FP32 plane distance along dh from oh to triangle t: an anchor for
// refine_hit_ff when only the triangle id is known.
__device__ __forceinline__ float plane_t32(const DevScene& S, int t, const float oh[3],
                                           const float dh[3]) {
    const float4* tp = S.tris + 3 * (size_t)t;
    float4 a = __ldg(tp), b = __ldg(tp + 1), c = __ldg(tp + 2);
    float e1x = b.x - a.x, e1y = b.y - a.y, e1z = b.z - a.z;
    float e2x = c.x - a.x, e2y = c.y - a.y, e2z = c.z - a.z;
    float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    return (nx * (a.x - oh[0]) + ny * (a.y - oh[1]) + nz * (a.z - oh[2])) /
           (nx * dh[0] + ny * dh[1] + nz * dh[2]);
}

// ---------------------------------------------------------------------------
// Voxel march (Amanatides & Woo 1987): FP32 index stepping, FP64 segment ends.
// ---------------------------------------------------------------------------
struct March {
    int ix, iy, iz;
    int sx, sy, sz;
    int px, py, pz;           // first plane crossed on each axis
    float tnx, tny, tnz;      // next crossing per axis, FP32 (ordering only)
    // Crossing of plane p on axis a: t = (f0_a + (p - p_a) c) / d_a, where
    // f0_a = (g0_a + p_a c) - o_a is formed in FP64 like the plain definition
    // (g0 + p c - o)/d, so nearly parallel axes never cancel large terms.
    // f0 and 1/d are kept as float pairs: segment ends are float-float
    // (~1e-13 relative), with no FP64 instruction per voxel.
    float f0hx, f0hy, f0hz, f0lx, f0ly, f0lz;
    float ivhx, ivhy, ivhz, ivlx, ivly, ivlz;
    float cell;
    FF t_enter, t_end;
    int entry_axis;           // axis crossed to enter the current voxel, -1: grid entry
    int face0;                // grid face crossed at t_enter (-1: the ray starts inside)
    int steps_left;
};

__device__ __forceinline__ float cross32(int p, int p0, int s, float f0, float iv, float c) {
    return s == 0 ? 3.0e38f : fmaf((float)(p - p0), c, f0) * iv;
}

// set up the march along o + t d for t in [t_enter, min(t_exit, t_hi)); false: no voxel
// The grid's box along o + t d (o, d as float pairs): each axis's slab
// [tlo, thi] (an axis the ray is parallel to: the whole line, or false when
// the origin is outside the slab), 1/d per axis, and the entry
// te = max(0, tlo) and exit min(thi, t_hi).  Float-float throughout.
__device__ __forceinline__ bool grid_span_ff(const DevGrid& S, const FF o[3], const FF d[3],
                                             const FF& t_hi, FF tlo[3], FF iv[3], FF& te, FF& tend) {
    te = FF{0.0f, 0.0f};
    FF tx = t_hi;
    for (int a = 0; a < 3; ++a) {
        const FF lo = {S.g0[a], 0.0f};
        const FF hi = ff_add(lo, ff_int_mul(S.dims[a], S.cell));
        if (d[a].hi == 0.0f) {
            if (ff_less(o[a], lo) || !ff_less(o[a], hi)) return false;
            tlo[a] = FF{-CUDART_INF_F, 0.0f};
            iv[a] = FF{0.0f, 0.0f};
            continue;
        }
        iv[a] = ff_rcp(d[a]);
        const FF ta = ff_mul(ff_sub(lo, o[a]), iv[a]), tb = ff_mul(ff_sub(hi, o[a]), iv[a]);
        tlo[a] = ff_min(ta, tb);
        te = ff_max(te, tlo[a]);
        tx = ff_min(tx, ff_max(ta, tb));
    }
    tend = tx;
    return ff_less(te, tend);
}

// set up the march along o + t d for t in [t_enter, min(t_exit, t_hi)); false:
// no voxel.  Float-float throughout (no FP64 instruction): the entry, the first
// voxel's indices and each axis's first crossing numerator f0.
__device__ __forceinline__ bool march_init(const DevGrid& S, const FF o[3], const FF d[3],
                                           const FF& t_hi, March& m) {
    FF tlo[3], ivd[3], te, tend;
    if (!grid_span_ff(S, o, d, t_hi, tlo, ivd, te, tend)) return false;
    const int dims[3] = {S.dims[0], S.dims[1], S.dims[2]};
    const FF icell = {S.icell_h, S.icell_l};
    const bool te_pos = te.hi > 0.0f;
    int idx[3], stp[3], p0[3];
    FF f0[3];
    for (int a = 0; a < 3; ++a) {
        stp[a] = d[a].hi > 0.0f ? 1 : (d[a].hi < 0.0f ? -1 : 0);
        if (te_pos && stp[a] != 0 && ff_eq(tlo[a], te)) {
            idx[a] = stp[a] > 0 ? 0 : dims[a] - 1;
        } else {
            // floor(x / cell) for x = p - g0: the estimate x * (1/cell), then
            // corrected against n cell and (n + 1) cell (exact pairs), so a point
            // on a voxel boundary (a ray inside a boundary plane) takes the
            // voxel above it, as the exact quotient does
            const FF p = ff_add(o[a], ff_mul(te, d[a]));
            const FF x = ff_sub(p, FF{S.g0[a], 0.0f});
            const FF v = ff_mul(x, icell);
            float f = floorf(v.hi);
            if (f == v.hi && v.lo < 0.0f) f -= 1.0f;
            f = fminf(fmaxf(f, -1.0f), (float)dims[a]);
            int n = (int)f;
            if (ff_less(x, ff_int_mul(n, S.cell))) --n;
            else if (!ff_less(x, ff_int_mul(n + 1, S.cell))) ++n;
            idx[a] = min(max(n, 0), dims[a] - 1);
        }
        p0[a] = stp[a] > 0 ? idx[a] + 1 : idx[a];
        f0[a] = stp[a] != 0 ? ff_sub(ff_add(FF{S.g0[a], 0.0f}, ff_int_mul(p0[a], S.cell)), o[a])
                            : FF{0.0f, 0.0f};
    }
    m.ix = idx[0]; m.iy = idx[1]; m.iz = idx[2];
    m.sx = stp[0]; m.sy = stp[1]; m.sz = stp[2];
    m.px = p0[0]; m.py = p0[1]; m.pz = p0[2];
    m.f0hx = f0[0].hi; m.f0hy = f0[1].hi; m.f0hz = f0[2].hi;
    m.f0lx = f0[0].lo; m.f0ly = f0[1].lo; m.f0lz = f0[2].lo;
    m.ivhx = ivd[0].hi; m.ivhy = ivd[1].hi; m.ivhz = ivd[2].hi;
    m.ivlx = ivd[0].lo; m.ivly = ivd[1].lo; m.ivlz = ivd[2].lo;
    m.cell = S.cell;
    m.tnx = cross32(m.px, m.px, m.sx, m.f0hx, m.ivhx, m.cell);
    m.tny = cross32(m.py, m.py, m.sy, m.f0hy, m.ivhy, m.cell);
    m.tnz = cross32(m.pz, m.pz, m.sz, m.f0hz, m.ivhz, m.cell);
    m.t_enter = te;
    m.t_end = tend;
    m.entry_axis = -1;
    m.face0 = -1;
    if (te_pos)
        for (int a = 2; a >= 0; --a)
            if (stp[a] != 0 && ff_eq(tlo[a], te)) m.face0 = a;
    m.steps_left = dims[0] + dims[1] + dims[2] + 4;
    return true;
}

// float-float crossing time of the entry (or exit) face of the current voxel on axis a
__device__ __forceinline__ FF plane_ff(const March& m, int a, bool entry) {
    int i = a == 0 ? m.ix : (a == 1 ? m.iy : m.iz);
    int s = a == 0 ? m.sx : (a == 1 ? m.sy : m.sz);
    int p0 = a == 0 ? m.px : (a == 1 ? m.py : m.pz);
    float f0h = a == 0 ? m.f0hx : (a == 1 ? m.f0hy : m.f0hz);
    float f0l = a == 0 ? m.f0lx : (a == 1 ? m.f0ly : m.f0lz);
    float ivh = a == 0 ? m.ivhx : (a == 1 ? m.ivhy : m.ivhz);
    float ivl = a == 0 ? m.ivlx : (a == 1 ? m.ivly : m.ivlz);
    int plane = entry ? (s > 0 ? i : i + 1) : (s > 0 ? i + 1 : i);
    float ph, pl;                       // (plane - p0) * cell, exactly
    two_prod((float)(plane - p0), m.cell, ph, pl);
    float sh, sl;                       // f0 + (ph + pl)
    two_sum(f0h, ph, sh, sl);
    sl += f0l + pl;
    FF n = ff_norm(sh, sl);
    float th, tl;                       // (f0 + ...) * (1/d)
    two_prod(n.hi, ivh, th, tl);
    tl = fmaf(n.hi, ivl, fmaf(n.lo, ivh, tl));
    return ff_norm(th, tl);
}

// Current voxel: linear id and exit axis.  Returns false once outside the grid.
struct VoxSeg {
    int64_t vid;
    int exit_axis;
    float t_out32;
};

__device__ __forceinline__ bool march_current(const DevGrid& S, const March& m, VoxSeg& v) {
    if (m.ix < 0 || m.iy < 0 || m.iz < 0 || m.ix >= S.dims[0] || m.iy >= S.dims[1] ||
        m.iz >= S.dims[2])
        return false;
    int a = 0;
    float tn = m.tnx;
    if (m.tny < tn) { a = 1; tn = m.tny; }
    if (m.tnz < tn) { a = 2; tn = m.tnz; }
    v.vid = ((int64_t)m.iz * S.dims[1] + m.iy) * S.dims[0] + m.ix;
    v.exit_axis = a;
    v.t_out32 = tn;
    return true;
}

// Density of the current voxel.  A voxel inside a brick whose occupancy bit is
// clear has density <= 0 (or NaN) by construction of the mask, so the grid is
// not read there; 0 is returned, or with MARK_EMPTY -1, which a march may
// answer with march_skip_brick.  Every caller treats either as empty.
template <bool MARK_EMPTY = false>
__device__ __forceinline__ float voxel_density(const DevGrid& S, const March& m, const VoxSeg& v) {
    if (S.occ != nullptr) {
        int b = ((m.iz >> kBrickLog2) * S.bdims[1] + (m.iy >> kBrickLog2)) * S.bdims[0] +
                (m.ix >> kBrickLog2);
        if (!((__ldg(&S.occ[b >> 5]) >> (b & 31)) & 1u)) return MARK_EMPTY ? -1.0f : 0.0f;
    }
    return __ldg(&S.density[v.vid]);
}

// float-float segment of the current voxel, clipped to [t_enter, t_end]
__device__ __forceinline__ void march_segment_ff(const March& m, const VoxSeg& v, FF& t_in,
                                                 FF& t_out) {
    t_in = m.t_enter;
    if (m.entry_axis >= 0) {
        FF p = plane_ff(m, m.entry_axis, true);
        if (ff_less(t_in, p)) t_in = p;
    }
    t_out = plane_ff(m, v.exit_axis, false);
    if (ff_less(m.t_end, t_out)) t_out = m.t_end;
}

// FP32 estimate of the current voxel's segment length, ending at t1 (its exit
// crossing clipped to t_end, in FP32): the entry crossing is formed in FP32
// like the exit ones.  Each end is within a few ulps of the float-float one
// (no cancellation: the crossings grow away from the origin), so the length
// is within 1e-6 of t1 of the exact one.
__device__ __forceinline__ float segment_len32(const March& m, float t1) {
    float t0 = m.t_enter.hi;
    const int a = m.entry_axis;
    if (a >= 0) {
        const int i = a == 0 ? m.ix : (a == 1 ? m.iy : m.iz);
        const int s = a == 0 ? m.sx : (a == 1 ? m.sy : m.sz);
        const int p0 = a == 0 ? m.px : (a == 1 ? m.py : m.pz);
        const float f0h = a == 0 ? m.f0hx : (a == 1 ? m.f0hy : m.f0hz);
        const float ivh = a == 0 ? m.ivhx : (a == 1 ? m.ivhy : m.ivhz);
        t0 = fmaxf(t0, cross32(s > 0 ? i : i + 1, p0, s, f0h, ivh, m.cell));
    }
    return t1 - t0;
}

// b - a for close float pairs (the hi difference is exact)
__device__ __forceinline__ float ff_diff(const FF& b, const FF& a) {
    return (b.hi - a.hi) + (b.lo - a.lo);
}
__device__ __forceinline__ FF ff_add_f(const FF& a, float x) {
    float s, e;
    two_sum(a.hi, x, s, e);
    return ff_norm(s, e + a.lo);
}

// advance to the next voxel; false when past t_end or out of steps
__device__ __forceinline__ bool march_step(March& m, const VoxSeg& v, uint32_t& flags) {
    if (--m.steps_left <= 0) { flags |= kPfMarchCap; return false; }
    if (v.t_out32 >= m.t_end.hi) {
        // FP32 ordering says the segment ends here; confirm in float-float
        if (!ff_less(plane_ff(m, v.exit_axis, false), m.t_end)) return false;
    }
    int a = v.exit_axis;
    if (a == 0) {
        m.ix += m.sx;
        m.tnx = cross32(m.sx > 0 ? m.ix + 1 : m.ix, m.px, m.sx, m.f0hx, m.ivhx, m.cell);
    } else if (a == 1) {
        m.iy += m.sy;
        m.tny = cross32(m.sy > 0 ? m.iy + 1 : m.iy, m.py, m.sy, m.f0hy, m.ivhy, m.cell);
    } else {
        m.iz += m.sz;
        m.tnz = cross32(m.sz > 0 ? m.iz + 1 : m.iz, m.pz, m.sz, m.f0hz, m.ivhz, m.cell);
    }
    m.entry_axis = a;
    return true;
}

// float-float crossing time of voxel-boundary plane `plane` on axis a
__device__ __forceinline__ FF plane_ff_at(const March& m, int a, int plane) {
    const int p0 = a == 0 ? m.px : (a == 1 ? m.py : m.pz);
    const float f0h = a == 0 ? m.f0hx : (a == 1 ? m.f0hy : m.f0hz);
    const float f0l = a == 0 ? m.f0lx : (a == 1 ? m.f0ly : m.f0lz);
    const float ivh = a == 0 ? m.ivhx : (a == 1 ? m.ivhy : m.ivhz);
    const float ivl = a == 0 ? m.ivlx : (a == 1 ? m.ivly : m.ivlz);
    float ph, pl;
    two_prod((float)(plane - p0), m.cell, ph, pl);
    float sh, sl;
    two_sum(f0h, ph, sh, sl);
    sl += f0l + pl;
    FF n = ff_norm(sh, sl);
    float th, tl;
    two_prod(n.hi, ivh, th, tl);
    tl = fmaf(n.hi, ivl, fmaf(n.lo, ivh, tl));
    return ff_norm(th, tl);
}

// From a voxel of an empty brick, jump to the first voxel past the brick.
// The one-voxel march takes crossings in (time, axis) order, each axis's
// crossing times being non-decreasing; so it leaves the brick at the least
// (time, axis) among the three exit planes, and before that it crosses, on
// every other axis, exactly the inner planes ordered before that event.
// Taking those crossings here gives the voxel, next-crossing times and entry
// axis the one-voxel march would reach.  false: the march ends in the brick.
__device__ __forceinline__ bool march_skip_brick(const DevGrid& S, March& m, uint32_t& flags) {
    const int bx0 = m.ix & ~(kBrick - 1), by0 = m.iy & ~(kBrick - 1), bz0 = m.iz & ~(kBrick - 1);
    const int bx1 = min(bx0 + kBrick - 1, S.dims[0] - 1);
    const int by1 = min(by0 + kBrick - 1, S.dims[1] - 1);
    const int bz1 = min(bz0 + kBrick - 1, S.dims[2] - 1);
    // exit planes (voxel-boundary indices) in the step directions
    const int ex = m.sx > 0 ? bx1 + 1 : bx0, ey = m.sy > 0 ? by1 + 1 : by0, ez = m.sz > 0 ? bz1 + 1 : bz0;
    const float Tx = cross32(ex, m.px, m.sx, m.f0hx, m.ivhx, m.cell);
    const float Ty = cross32(ey, m.py, m.sy, m.f0hy, m.ivhy, m.cell);
    const float Tz = cross32(ez, m.pz, m.sz, m.f0hz, m.ivhz, m.cell);
    int a = 0;
    float T = Tx;
    if (Ty < T) { a = 1; T = Ty; }
    if (Tz < T) { a = 2; T = Tz; }
    if (T >= m.t_end.hi) {
        // FP32 ordering says the march may end in the brick; confirm in float-float
        if (!ff_less(plane_ff_at(m, a, a == 0 ? ex : (a == 1 ? ey : ez)), m.t_end)) return false;
    }
    const int ox = m.ix, oy = m.iy, oz = m.iz;
    // the other axes: inner crossings ordered before (T, a)
    if (a != 0 && m.sx != 0) {
        for (int k = 0; k < kBrick; ++k) {
            const int pl = m.sx > 0 ? m.ix + 1 : m.ix;
            if (pl == ex) break;
            const float t = cross32(pl, m.px, m.sx, m.f0hx, m.ivhx, m.cell);
            if (!(t < T || t == T)) break;      // ties go to x, the lowest axis
            m.ix += m.sx;
        }
    }
    if (a != 1 && m.sy != 0) {
        for (int k = 0; k < kBrick; ++k) {
            const int pl = m.sy > 0 ? m.iy + 1 : m.iy;
            if (pl == ey) break;
            const float t = cross32(pl, m.py, m.sy, m.f0hy, m.ivhy, m.cell);
            if (!(t < T || (t == T && a == 2))) break;
            m.iy += m.sy;
        }
    }
    if (a != 2 && m.sz != 0) {
        for (int k = 0; k < kBrick; ++k) {
            const int pl = m.sz > 0 ? m.iz + 1 : m.iz;
            if (pl == ez) break;
            const float t = cross32(pl, m.pz, m.sz, m.f0hz, m.ivhz, m.cell);
            if (!(t < T)) break;                // z loses every tie
            m.iz += m.sz;
        }
    }
    // the exit axis: through the brick and out of it
    if (a == 0) m.ix = m.sx > 0 ? bx1 + 1 : bx0 - 1;
    else if (a == 1) m.iy = m.sy > 0 ? by1 + 1 : by0 - 1;
    else m.iz = m.sz > 0 ? bz1 + 1 : bz0 - 1;
    m.tnx = cross32(m.sx > 0 ? m.ix + 1 : m.ix, m.px, m.sx, m.f0hx, m.ivhx, m.cell);
    m.tny = cross32(m.sy > 0 ? m.iy + 1 : m.iy, m.py, m.sy, m.f0hy, m.ivhy, m.cell);
    m.tnz = cross32(m.sz > 0 ? m.iz + 1 : m.iz, m.pz, m.sz, m.f0hz, m.ivhz, m.cell);
    m.entry_axis = a;
    m.steps_left -= abs(m.ix - ox) + abs(m.iy - oy) + abs(m.iz - oz);
    if (m.steps_left <= 0) { flags |= kPfMarchCap; return false; }
    return true;
}

// ---------------------------------------------------------------------------
// scenes with several grids: their boxes have disjoint interiors, so the
// segments of a ray in them follow one another in the order of the boxes'
// entry points.  A grid's key is (t_enter, index), t_enter = max(0, entry)
// in FP64 exactly as march_init forms it.  The grid BVH holds the boxes
// widened at build time; its FP32 slab tests only cull (conservatively: a
// box the FP64 march enters is never dropped).  next_grid returns the grid of
// least key above the cursor that the ray enters before t_hi; each call is
// one bounded walk of the grid BVH.
// ---------------------------------------------------------------------------
constexpr int kGridStack = 32;

struct GridRay {
    float of[3], ivf[3];        // FP32 culling
    FF o[3], d[3];              // the ray as float pairs
};

struct GridCursor {
    FF te;          // key of the last grid returned
    int gi;         // -1: none yet
};

__device__ __forceinline__ void box_span(const float o[3], const float iv[3], const float lo[3],
                                         const float hi[3], float& tn, float& tf) {
    tn = 0.0f;
    tf = 3.0e38f;
    for (int a = 0; a < 3; ++a) {
        const float t0 = (lo[a] - o[a]) * iv[a], t1 = (hi[a] - o[a]) * iv[a];
        tn = fmaxf(tn, fminf(t0, t1));
        tf = fminf(tf, fmaxf(t0, t1));
    }
}

// entry of o + t d (t >= 0) into grid g's box, formed exactly as march_init
// forms it; false: the ray does not enter it before t_hi
__device__ __forceinline__ bool grid_entry_ff(const DevGrid& g, const GridRay& r, const FF& t_hi, FF& te) {
    FF tlo[3], iv[3], tend;
    return grid_span_ff(g, r.o, r.d, t_hi, tlo, iv, te, tend);
}

__device__ __forceinline__ int next_grid(const DevScene& sc, const GridRay& r, const FF& t_hi, GridCursor& c) {
    if (sc.n_grid == 1) {
        if (c.gi >= 0) return -1;
        c.gi = 0;
        return 0;
    }
    const float th = t_hi.hi * 1.0001f + 1.0e-3f;
    const float cte = c.gi >= 0 ? c.te.hi * 0.9999f - 1.0e-3f : -1.0e30f;   // below the cursor, for culling
    FF best_t = t_hi;
    int best = -1;
    int stack[kGridStack];
    int sp = 0, node = 0;
    for (int guard = 0; guard < 2 * sc.n_grid + 4; ++guard) {
        const float4* n = sc.gnodes + 4 * (size_t)node;
        const float4 a = __ldg(n), b = __ldg(n + 1), e = __ldg(n + 2);
        const int4 ch = __ldg(reinterpret_cast<const int4*>(n + 3));
        const float lo0[3] = {a.x, a.y, a.z}, hi0[3] = {a.w, b.x, b.y};
        const float lo1[3] = {b.z, b.w, e.x}, hi1[3] = {e.y, e.z, e.w};
        const float bt = best_t.hi * 1.0001f + 1.0e-3f;
        for (int k = 0; k < 2; ++k) {
            float tn, tf;
            box_span(r.of, r.ivf, k ? lo1 : lo0, k ? hi1 : hi0, tn, tf);
            if (!(tn <= tf) || tf < cte || tn > bt || !(tn < th)) continue;
            const int child = k ? ch.y : ch.x;
            if (child < 0) {
                const int gi = ~child;
                FF te;
                if (!grid_entry_ff(sc.grids[gi], r, t_hi, te)) continue;
                const bool after = c.gi < 0 || ff_less(c.te, te) || (ff_eq(te, c.te) && gi > c.gi);
                const bool before = best < 0 || ff_less(te, best_t) || (ff_eq(te, best_t) && gi < best);
                if (after && before) {
                    best_t = te;
                    best = gi;
                }
            } else if (sp < kGridStack) {
                stack[sp++] = child;
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
    if (best >= 0) {
        c.te = best_t;
        c.gi = best;
    }
    return best;
}

__device__ __forceinline__ void grid_ray(const FF o[3], const FF d[3], GridRay& r) {
    for (int a = 0; a < 3; ++a) {
        r.o[a] = o[a];
        r.d[a] = d[a];
        r.of[a] = o[a].hi;
        r.ivf[a] = d[a].hi != 0.0f ? 1.0f / d[a].hi : 1.0e30f;
    }
}

// the march set up on the next grid (in entry order) that the march enters
// before t_hi; NULL when none is left
__device__ __forceinline__ const DevGrid* next_march(const DevScene& sc, const GridRay& r, const FF& t_hi,
                                                     GridCursor& c, March& m) {
    for (int guard = 0; guard < sc.n_grid; ++guard) {
        const int gi = next_grid(sc, r, t_hi, c);
        if (gi < 0) return nullptr;
        const DevGrid* G = sc.n_grid == 1 ? &sc.grid : sc.grids + gi;
        if (march_init(*G, r.o, r.d, t_hi, m)) return G;
    }
    return nullptr;
}

// body(G, m) on each grid the ray crosses before t_hi, in entry order, with
// m set up on it; body returns false to end the walk.  GK 1: the scene has
// at most one grid (sc.grid); GK 2: any number.  o and d as float pairs.
template <int GK, class F>
__device__ __forceinline__ void walk_grids(const DevScene& sc, const FF o[3], const FF d[3], const FF& t_hi,
                                           F&& body) {
    if (GK == 1) {
        March m;
        if (march_init(sc.grid, o, d, t_hi, m)) body(sc.grid, m);
        return;
    }
    GridRay r;
    grid_ray(o, d, r);
    GridCursor c = {{0.0f, 0.0f}, -1};
    March m;
    for (int guard = 0; guard < sc.n_grid; ++guard) {
        const DevGrid* G = next_march(sc, r, t_hi, c, m);
        if (!G || !body(*G, m)) return;
    }
}

// ---------------------------------------------------------------------------
// power (Eq. beamdiv, Eq. beamdiv_w, Eq. ladlut_intensity with a Lambertian
// cross-section): P = I0 exp(-2 r^2/w^2) Dr^2 eta rho cos / (4 R^2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float return_power(const DevScanner& sn, float R, float tan_a,
                                              float rho, float cos_inc) {
    float z = sn.zk * (R - sn.focus);
    float w2 = sn.w0sq * (1.0f + z * z);
    float r = R * tan_a;
    float Is = __expf(__fdividef(-2.0f * r * r, w2));
    return __fdividef(sn.pconst * Is * rho * cos_inc, R * R);
}

// pulse shape at time x (ns) relative to the return's delay
__device__ __forceinline__ float pulse_shape(const DevScanner& sn, float x) {
    if (sn.pulse_shape == 0) return exp2f(-x * x * sn.gk2);
    if (x < 0.0f) return 0.0f;
    float y = x * sn.ctau_inv;
    return y * y * expf(-y);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace hg
