/* helios.h - C ABI of the GB300 per-pulse beam-scene interaction library
 * (libhelios_gb300.so).
 *
 * The library simulates full-waveform laser scanning as in HELIOS++
 * (Winiwarter et al., "Virtual laser scanning with HELIOS++"): every emitted
 * pulse is split into divergence subrays (Sec. 3.4), each subray is traced
 * through triangle meshes and transmissive voxels (Sec. 3.5, Sec. 5.1, 5.2),
 * the hits become return power through the laser radar equation with a
 * Lambertian target (Eq. beamdiv, Eq. beamdiv_w, Eq. ladlut_intensity), the
 * returns are summed into a per-pulse waveform and echoes are detected as
 * local maxima above a threshold (Sec. 3.4) with Gaussian range noise
 * (Sec. 3.7).  The argument structs follow the paper's survey / scene /
 * scanner / platform / leg split (Sec. 3.1, Fig. file_overview).
 *
 * Conventions shared by every call:
 *  - Array pointers inside the *_desc and helios_outputs structs are DEVICE
 *    pointers owned by the caller; the library never frees them.  The structs
 *    themselves (and arrays of structs passed as arguments) are HOST memory,
 *    read during the call only.
 *  - Every call returns a helios_status: 0 on success, a negative code on
 *    failure.  helios_last_error() returns a message for the calling thread's
 *    most recent failure.  No C++ exception crosses this boundary.
 *  - Argument errors are detected on the host and returned before anything
 *    is launched.  Kernels are enqueued on `cuda_stream` (a cudaStream_t; NULL
 *    is the legacy default stream) and run asynchronously; a call returns
 *    once its work is enqueued.  Conditions found on the device are reported
 *    through per-pulse flags and the optional device status word.
 *  - Scene geometry is FP32.  Instrument, platform and leg parameters are
 *    FP64 so that host-side and device-side geometry agree to FP64.
 *  - Each call is one NVTX range named after it (visible under a profiler).
 *  - Host-side fault injection for tests, read from the environment at every
 *    call: HELIOS_FAULT=badarg makes every call except helios_last_error and
 *    helios_version return HELIOS_ERR_INVALID_ARG at entry; HELIOS_FAULT=oom
 *    makes a call that would allocate device memory return HELIOS_ERR_OOM
 *    where it first would (nothing is launched before, everything it
 *    allocated is released).  No fault is injected on the device.
 */
#ifndef HELIOS_GB300_H
#define HELIOS_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define HELIOS_API __attribute__((visibility("default")))
#else
#define HELIOS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t helios_status;
#define HELIOS_OK               0
#define HELIOS_ERR_INVALID_ARG (-1)  /* a pointer, size or parameter is invalid */
#define HELIOS_ERR_OOM         (-2)  /* a device allocation failed */
#define HELIOS_ERR_CUDA        (-3)  /* a CUDA runtime call failed */
#define HELIOS_ERR_TIMEOUT     (-4)  /* a bounded device loop reached its cap */
#define HELIOS_ERR_OVERFLOW    (-5)  /* an output capacity was exceeded */
#define HELIOS_ERR_UNSUPPORTED (-6)  /* valid request this build does not handle */

/* window_bin value of a pulse none of whose subrays returned */
#define HELIOS_NO_WINDOW INT32_MIN

/* per-pulse device flags (helios_outputs.pulse_flags) */
#define HELIOS_PF_ECHO_OVERFLOW 0x01u  /* more local maxima than max_echoes */
#define HELIOS_PF_TRAVERSAL_CAP 0x02u  /* BVH traversal hit its step cap */
#define HELIOS_PF_MARCH_CAP     0x04u  /* voxel march hit its step cap */
#define HELIOS_PF_NO_RETURN     0x08u  /* no subray returned */

/* device status word bits (helios_outputs.status, OR-ed by the kernels) */
#define HELIOS_ST_TRAVERSAL_CAP 0x01u
#define HELIOS_ST_MARCH_CAP     0x02u
#define HELIOS_ST_ECHO_OVERFLOW 0x04u

/* deflectors (Sec. 3.3) and platforms (Sec. 3.2) */
#define HELIOS_DEFL_POLYGON       0  /* rotating polygon mirror: sawtooth across track */
#define HELIOS_DEFL_OSCILLATING   1  /* swinging mirror: sinusoidal across track */
#define HELIOS_DEFL_TLS_GRID      2  /* static scanner: azimuth x elevation grid */
#define HELIOS_DEFL_ROTATING_HEAD 3  /* head turning at head_rate, polygon in elevation */
#define HELIOS_DEFL_FIBRE         4  /* fibre-optic line: n_fibres fixed angles in turn */
#define HELIOS_DEFL_PALMER        5  /* slanted rotating mirror: cone at scan_angle_max off nadir */
#define HELIOS_PLATFORM_STATIC 0
#define HELIOS_PLATFORM_LINEAR 1
#define HELIOS_PULSE_GAUSSIAN  0
#define HELIOS_PULSE_CARLSSON  1     /* Eq. beam_time: (t/tau)^2 exp(-t/tau) */
#define HELIOS_MODE_STOCHASTIC 0     /* Eq. intersection_dist with Philox4x32-10 draws */
#define HELIOS_MODE_EXPECTED   1     /* expected transmittance, differentiable */

typedef struct helios_scene helios_scene; /* opaque; owns its BVH buffers */

/* One triangle mesh part (Sec. 3.5.1 / 3.5.2).  verts: device float[n_verts][3],
 * faces: device int32[n_faces][3] (indices into verts), reflectance: device
 * float[n_faces], Lambertian reflectance per face.  reflectance is REFERENCED,
 * not copied: it must stay valid while the scene is used, and updates to it
 * are seen by later scans without a rebuild.  verts/faces are read during
 * helios_build_scene only. */
typedef struct {
    const float* verts;
    int64_t n_verts;
    const int32_t* faces;
    int64_t n_faces;
    const float* reflectance;
    int32_t object_id;
    int32_t reserved;
} helios_mesh_desc;

/* One transmissive voxel part (Sec. 3.5.4, Eq. extinction: sigma = G * density).
 * density: device float[dims[2]][dims[1]][dims[0]] plant area density in
 * m^2/m^3, REFERENCED (not copied) like mesh reflectance.  Voxel (x,y,z) spans
 * [origin + (x,y,z)*cell, origin + (x+1,y+1,z+1)*cell).
 * G is the constant projection factor, unless lad_table is given: then G
 * depends on the subray's unit direction d through the leaf-angle table
 * (Table ladlut), G(d) = linear interpolation of lad_table at mu = |d_z|
 * between entries at mu_i = i/(lad_n - 1).  lad_table: device or host
 * float[lad_n], 2 <= lad_n <= 65536, entries finite and >= 0 (INVALID_ARG
 * otherwise); COPIED by helios_build_scene (the caller may free it after).
 * helios_lad_table fills one for the distributions the paper names. */
typedef struct {
    float origin[3];
    float cell;
    int32_t dims[3];
    float G;
    float leaf_reflectance;
    int32_t object_id;
    int32_t opaque;               /* 1: non-transmissive (Sec. 3.5.4): a voxel of density > 0
                                     stops the subray where it enters, Lambertian on that face */
    const float* density;
    const float* lad_table;       /* NULL: constant G */
    int32_t lad_n;
    int32_t reserved;
} helios_voxel_desc;

/* A scene: meshes are concatenated in order; triangle id = offset of its mesh
 * + face index.  At most 16 meshes, 4096 voxel grids and 2^40 - 1 voxels in
 * all per scene (HELIOS_ERR_UNSUPPORTED otherwise).  The grids' boxes must have disjoint
 * interiors (touching faces are allowed, and so are overlaps thinner than
 * 1e-6 of the largest box edge; INVALID_ARG otherwise): a ray's
 * segments in them then follow the order of its entry points, which is the
 * order its transmission is applied in.  Voxel primitive ids are n_triangles +
 * (voxels of the earlier grids) + (z*ny + y)*nx + x; the stochastic
 * transmission draw of a voxel is keyed by that id minus n_triangles. */
typedef struct {
    const helios_mesh_desc* meshes;
    int32_t n_meshes;
    int32_t n_grids;
    const helios_voxel_desc* grids;
} helios_scene_desc;

typedef struct {
    int64_t n_triangles;
    int64_t n_bvh_nodes;       /* internal nodes of the binary BVH */
    int64_t device_bytes;      /* bytes owned by the scene */
    int32_t n_meshes;
    int32_t n_grids;
    int64_t n_bvh4_nodes;      /* nodes of its 4-wide collapse (the beam-cone walk's tree) */
} helios_scene_info;

/* Build the acceleration structure on the device (Sec. 5.1's role, here an
 * LBVH: Morton codes, radix sort, Karras 2012 hierarchy, bottom-up refit).
 * The kernels run on cuda_stream; face indices are checked on the device and
 * the call synchronises cuda_stream once to read that check, so *out is
 * complete on return.  Temporary buffers are stream-ordered allocations
 * (cudaMallocAsync) freed before return; the scene's own buffers come from
 * cudaMalloc.  Errors: INVALID_ARG (NULL or negative sizes, a face index
 * outside its mesh, overlapping grid boxes, a bad leaf-angle table),
 * UNSUPPORTED (more than 16 meshes or 4096 grids, ids beyond 32 bits), OOM,
 * CUDA.  With several grids the build also forms a BVH over their boxes (host,
 * median split) and a device array of their descriptors. */
HELIOS_API helios_status helios_build_scene(const helios_scene_desc* desc, void* cuda_stream,
                                 helios_scene** out);
/* Leaf-angle distributions (de Wit) for helios_lad_table, Sec. 3.5.4. */
#define HELIOS_LAD_PLANOPHILE   1    /* f(t) = (2/pi)(1 + cos 2t), t = leaf-normal zenith */
#define HELIOS_LAD_ERECTOPHILE  2    /* (2/pi)(1 - cos 2t) */
#define HELIOS_LAD_PLAGIOPHILE  3    /* (2/pi)(1 - cos 4t) */
#define HELIOS_LAD_EXTREMOPHILE 4    /* (2/pi)(1 + cos 4t) */
#define HELIOS_LAD_UNIFORM      5    /* 2/pi */
#define HELIOS_LAD_SPHERICAL    6    /* sin t (G = 1/2 at every angle) */

/* Fill a leaf-angle table for helios_voxel_desc.lad_table (Eq. extinction,
 * Table ladlut): table[i] = G at a beam with |cos zenith| = mu_i = i/(n-1),
 *   G(theta) = (1/2pi) int over leaf normals of g_L |Omega'.Omega_L| dOmega_L
 *            = int_0^{pi/2} f(t) psi(theta, t) dt,
 * psi Ross's azimuthal kernel, for azimuthally uniform leaves with inclination
 * density f = `distribution` (HELIOS_LAD_*).  Computed on the device in FP64
 * (composite Simpson on the two pieces split at t = pi/2 - theta), rounded to
 * float.  table: DEVICE float[n], written asynchronously on cuda_stream.
 * Errors: INVALID_ARG (unknown distribution, n outside 2..65536, NULL table),
 * CUDA. */
HELIOS_API helios_status helios_lad_table(int32_t distribution, int32_t n, float* table,
                                          void* cuda_stream);

/* Frees the scene's device buffers (synchronises the device first). */
HELIOS_API helios_status helios_free_scene(helios_scene* scene);
HELIOS_API helios_status helios_scene_get_info(const helios_scene* scene, helios_scene_info* info);

/* Instrument (Sec. 3.3 deflector + Sec. 3.4 beam and waveform settings). */
typedef struct {
    double prf_hz;
    double divergence_rad;        /* full beam divergence at the 1/e^2 points */
    int32_t beam_sample_quality;  /* q: subray rings; S = 1 + sum_i floor(2 pi i) */
    int32_t pulse_shape;          /* HELIOS_PULSE_* */
    double wavelength_m;
    double beam_waist_m;          /* <= 0: lambda / (pi * divergence/2) */
    double focus_m;
    double peak_power_w;
    double receiver_diam_m;
    double eta_sys, eta_atm;
    double pulse_fwhm_ns;         /* Gaussian pulse */
    double pulse_length_ns;       /* Carlsson pulse: tau = length / 1.75 */
    double bin_ns;                /* waveform bin width */
    int32_t n_bins;               /* bins per pulse waveform, 4..4096 */
    int32_t max_echoes;           /* echoes kept per pulse, 1..32 */
    double echo_threshold_rel;    /* echo threshold as a fraction of the pulse's maximum bin */
    double range_noise_sigma_m;   /* sigma of the Gaussian ranging error */
    int32_t deflector;            /* HELIOS_DEFL_* */
    int32_t grid_n_az, grid_n_el; /* HELIOS_DEFL_TLS_GRID */
    int32_t n_fibres;             /* HELIOS_DEFL_FIBRE: pulse k leaves fibre k mod n_fibres, at
                                     -max + 2 max i/(n_fibres - 1) across track (>= 1) */
    double scan_freq_hz;          /* mirror lines (polygon) or swings (oscillating) per second */
    double scan_angle_max_rad;
    double head_rate_rad_s;
    double el_min_rad, el_max_rad;
} helios_scanner_desc;

/* One leg (Sec. 3.1): the platform moves from start towards end at speed_mps
 * (LINEAR) heading at the next waypoint, or stays at start (STATIC).  Pulse k
 * is emitted at t0 + k/prf.  leg_id keys the random draws of this leg.  A leg
 * interrupted after its first K pulses is resumed with first_pulse = K. */
typedef struct {
    int32_t scene_index;
    int32_t scanner_index;
    int32_t platform;
    int32_t beam_sample_quality;  /* < 0: the scanner's */
    double start[3];
    double end[3];
    double speed_mps;
    double attitude_rpy[3];       /* roll, pitch, yaw offset (radians) */
    double t0;
    int64_t n_pulses;
    uint32_t leg_id;
    float platform_noise_m;       /* sigma of an N(0, s) offset of the platform position on each
                                     axis, drawn per pulse (Sec. 3.7 platform noise); 0: none */
    int64_t first_pulse;          /* resume: the leg's pulses first_pulse .. first_pulse +
                                     n_pulses - 1 are scanned into n_pulses output rows.  Every
                                     draw is keyed by the absolute pulse index, so the rows equal
                                     those of the whole leg (first_pulse >= 0 and
                                     first_pulse + n_pulses <= 2^44; INVALID_ARG otherwise) */
} helios_leg_desc;

typedef struct {
    int32_t mode;                 /* HELIOS_MODE_* */
    int32_t persistent;           /* 1: all legs in one launch over a work queue */
    uint64_t seed;                /* Philox4x32-10 key (counter: pulse, stream, subray or echo,
                                     voxel id, leg id) */
    int32_t block_threads;        /* 0: default (256) */
    int32_t rays_per_block;       /* 0: default (768); target subrays per work item (scan and
                                     adjoint), <= 4096 */
    int32_t blocks_per_sm;        /* 0: occupancy-derived */
    int32_t reserved;
} helios_scan_opts;

/* Outputs: per-pulse arrays are concatenated over legs in leg order (leg l
 * starts at pulse_offset[l] of helios_output_layout); the waveform holds leg
 * l's rows of scanner(l).n_bins floats starting at wave_offset[l]; subray
 * arrays hold leg l's [n_pulses][S_l] block at subray_offset[l].  Every
 * pointer is a device pointer; optional ones may be NULL.  echo_* arrays are
 * [total_pulses][max_echoes of the leg's scanner] at pulse_offset*K.
 * For mode EXPECTED subray_hit/subray_range hold the triangle hit, which is
 * the checkpoint helios_scan_adjoint reuses. */
typedef struct {
    float* waveform;              /* required */
    int32_t* window_bin;          /* required: absolute index m of the first bin (bin b is t=(m+b)*bin_ns) */
    int32_t* echo_count;          /* required */
    float* echo_range;            /* required: metres, range noise included */
    float* echo_amp;              /* optional */
    int32_t* echo_bin;            /* optional: b within the window */
    int64_t* echo_object;         /* optional: primitive id of the strongest contributor
                                     (triangle id, or n_triangles + voxel id: voxels are
                                     numbered over the scene's grids in order, so ids can
                                     exceed 2^31), -1 in unused slots */
    uint8_t* pulse_flags;         /* optional: HELIOS_PF_* */
    int64_t* subray_hit;          /* optional: event primitive (as echo_object) or -1 */
    float* subray_range;          /* optional */
    uint32_t* status;             /* optional: one word, OR-ed HELIOS_ST_* */
    float* echo_width;            /* optional [total_pulses][K]: echo width (Sec. 3.4), the sigma
                                     in ns of a Gaussian fitted to the waveform over the bins
                                     within 2 pulse sigmas of the echo by 10 Levenberg-Marquardt
                                     steps; Gaussian pulses only (0 otherwise and in unused
                                     slots); NULL: not fitted (no cost) */
} helios_outputs;

typedef struct {
    int64_t total_pulses;
    int64_t waveform_floats;
    int64_t subray_elems;
    int64_t echo_elems;
} helios_layout;

/* Host-only: offsets of each leg inside the output arrays (any pointer may be
 * NULL).  Errors: INVALID_ARG. */
HELIOS_API helios_status helios_output_layout(const helios_scanner_desc* scanners, int32_t n_scanners,
                                   const helios_leg_desc* legs, int32_t n_legs,
                                   int64_t* pulse_offset, int64_t* wave_offset,
                                   int64_t* subray_offset, int64_t* echo_offset,
                                   helios_layout* totals);

/* Simulate the legs: pulse generation (Sec. 3.2-3.3), subrays (Sec. 3.4),
 * intersection (Sec. 5.1-5.2), power (Eq. beamdiv, beamdiv_w,
 * ladlut_intensity), waveform (Sec. 3.4), echoes and range noise (Sec. 3.4,
 * 3.7), echo widths when out->echo_width is set.  With opts->persistent the
 * legs share one launch fed by a work queue; otherwise one launch per leg.
 * Scratch (the queue counter, candidate lists, voxel brick masks, moment bins
 * and return lists in expected mode, echo bins for the width fit) is
 * stream-ordered memory allocated and freed on cuda_stream.  The call returns
 * once the work is queued.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
HELIOS_API helios_status helios_scan_legs(helios_scene* const* scenes, int32_t n_scenes,
                               const helios_scanner_desc* scanners, int32_t n_scanners,
                               const helios_leg_desc* legs, int32_t n_legs,
                               const helios_scan_opts* opts, const helios_outputs* out,
                               void* cuda_stream);

/* helios_scan_legs_static: helios_scan_legs in persistent mode that allocates
 * nothing.  The paper has no counterpart; this is a deployment variant.
 * Some callers cannot allocate device memory during a scan: processes whose
 * device memory is owned by another allocator (a framework's caching
 * allocator holding the budget), code running while a CUDA graph is captured
 * into a memory pool it does not control, and real-time loops that cannot let
 * an allocation fail or stall mid-run.  helios_scan_legs allocates its
 * scratch (work-queue counter, candidate lists, occupancy masks, moment bins)
 * with cudaMallocAsync; this variant keeps the queue counters in a
 * static device array of 16 int32 (64 bytes, held by every GPU that loads the
 * library until exit), so it takes at most 16 x 128 = 2048 legs per call and
 * returns HELIOS_ERR_INVALID_ARG beyond that.  Host-side staging is static too
 * (no heap use).  Each call made outside a stream capture looks the array's
 * address up with cudaGetSymbolAddress (so a device reset between calls is
 * harmless); a call inside a capture reuses the address of the last call
 * outside one, so make the first call on each device before any stream
 * capture (HELIOS_ERR_UNSUPPORTED otherwise).  Stochastic mode keeps the
 * Hermite table of merged returns (it lives in shared memory), so its
 * results are those of helios_scan_legs; expected mode sums each waveform
 * directly instead of through moment bins (device scratch) and finds echo
 * objects from its own return list, which agrees with helios_scan_legs within
 * the waveform tolerance.
 * All calls share the array: each call zeroes the counters it uses on its
 * stream, and calls whose work overlaps on the GPU (e.g. on two streams) race
 * on them.  opts->persistent is ignored (always one launch per 128 legs).
 * out->echo_width needs out->echo_bin here (the fit reads the bins back).
 * Arguments, outputs and results are those of helios_scan_legs. */
HELIOS_API helios_status helios_scan_legs_static(helios_scene* const* scenes, int32_t n_scenes,
                                                 const helios_scanner_desc* scanners,
                                                 int32_t n_scanners, const helios_leg_desc* legs,
                                                 int32_t n_legs, const helios_scan_opts* opts,
                                                 const helios_outputs* out, void* cuda_stream);

/* helios_scan_legs with the outputs in HOST memory.  The paper has no
 * counterpart; this is the end-to-end form for callers that consume the
 * results on the host.  host_out holds host pointers with the layout of
 * helios_outputs (status alone stays a device pointer, or NULL).  The pulses
 * are cut into chunks of whole work items of about chunk_pulses pulses
 * (> 0); each chunk is scanned on cuda_stream into one of two device staging
 * slots (stream-ordered allocations, freed on cuda_stream) and copied to the
 * host on a second stream while the next chunk is scanned.  Each pulse is
 * computed exactly as by helios_scan_legs, so the results are identical.  The
 * call returns once the work is queued: the host buffers are complete when
 * cuda_stream reaches the point after this call (synchronise it before
 * reading them).  Copies overlap the scan only for page-locked host buffers;
 * pageable ones are still filled correctly.  Errors: those of
 * helios_scan_legs. */
HELIOS_API helios_status helios_scan_legs_host(helios_scene* const* scenes, int32_t n_scenes,
                                               const helios_scanner_desc* scanners,
                                               int32_t n_scanners, const helios_leg_desc* legs,
                                               int32_t n_legs, const helios_scan_opts* opts,
                                               const helios_outputs* host_out,
                                               int64_t chunk_pulses, void* cuda_stream);

/* Gradient buffers of one scene: d_reflectance[i] (device float[n_faces of
 * mesh i], or NULL to skip) and d_density[j] (device float[n voxels of grid
 * j], or NULL).  Gradients are ADDED to these buffers. */
typedef struct {
    float* const* d_reflectance;
    float* const* d_density;
} helios_scene_grads;

/* Adjoint of the EXPECTED-mode waveform (opts->mode must be EXPECTED):
 * given dL/dW (same layout as helios_outputs.waveform) and the forward's
 * window_bin (held fixed), accumulate dL/d(reflectance) and dL/d(density)
 * with the hit sets held fixed.  subray_hit (optional, the forward's
 * checkpoint) skips the BVH traversal.  Voxels of zero density receive no
 * gradient (the density support is part of the fixed hit set).  Gradients
 * are accumulated with device atomics (summation order not fixed).
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
HELIOS_API helios_status helios_scan_adjoint(helios_scene* const* scenes, int32_t n_scenes,
                                  const helios_scanner_desc* scanners, int32_t n_scanners,
                                  const helios_leg_desc* legs, int32_t n_legs,
                                  const helios_scan_opts* opts, const float* d_waveform,
                                  const int32_t* window_bin, const int64_t* subray_hit,
                                  const helios_scene_grads* grads, void* cuda_stream);

/* Fetch counts of one pulse: what it needs from memory, as a union over its
 * subrays.  A measurement aid for the roofline's algorithmic bytes (the
 * paper has no counterpart): a pulse's bytes are its output row plus
 * 128 nodes + 48 triangles + 4 voxels. */
typedef struct {
    int64_t nodes;         /* 4-wide BVH nodes (128 B) the beam cone enters: the root and
                              each internal slot whose box the cone overlaps */
    int64_t triangles;     /* triangles (48 B) whose widened box the cone overlaps: the
                              candidates every subray of the pulse tests */
    int64_t voxels;        /* distinct voxels (4 B density) the subrays march through, each
                              up to where the scan's march stops in the given mode */
    int64_t voxel_visits;  /* voxel visits summed over the subrays */
    int32_t flags;         /* HELIOS_FC_* */
    int32_t reserved;
} helios_fetch_counts;

#define HELIOS_FC_STACK         0x01  /* cone walk stack full: nodes, triangles undercounted */
#define HELIOS_FC_LIST_OVERFLOW 0x02  /* more candidates than the scan's per-pulse list holds
                                         (128): the scan traverses per subray for this pulse */
#define HELIOS_FC_SET_FULL      0x04  /* over 3072 distinct voxels: later visits counted as
                                         distinct (an upper bound) */
#define HELIOS_FC_MARCH_CAP     0x08  /* a march hit its step cap */

/* Fetch counts of `count` pulses of one leg: pulse first + i * stride of the
 * leg (0-based within the leg's n_pulses; first >= 0, stride >= 1, the last
 * one < n_pulses), poses and draws as helios_scan_legs with the same seed
 * and mode (Sec. 3.2-3.5).  The cone is the one the scan walks: half-angle
 * atan of the half divergence (Sec. 3.4), from the pulse origin, unbounded
 * in range, tested against boxes conservatively (each box grown by the
 * cone's radius at its farthest corner); with one subray per pulse the scan
 * traverses per ray instead, and the count is still the cone's.  Voxel marches stop at the stochastic event (Eq.
 * intersection_dist) in mode STOCHASTIC, at the subray's triangle hit in
 * mode EXPECTED, at the first dense voxel of an opaque grid in both.  out:
 * device array of `count` entries, written on cuda_stream (not on the scan
 * path; not timed with it).  Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
HELIOS_API helios_status helios_fetch_counts_sample(helios_scene* scene,
                                                    const helios_scanner_desc* scanner,
                                                    const helios_leg_desc* leg, int32_t mode,
                                                    uint64_t seed, int64_t first, int64_t stride,
                                                    int64_t count, helios_fetch_counts* out,
                                                    void* cuda_stream);

/* Number of subrays for beam sample quality q (Sec. 3.4), or -1 if q < 0. */
HELIOS_API int32_t helios_subray_count(int32_t q);

/* Message of the calling thread's last failure ("" if none). */
HELIOS_API const char* helios_last_error(void);

/* Library version string. */
HELIOS_API const char* helios_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HELIOS_GB300_H */
