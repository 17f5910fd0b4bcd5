// helios_api.cu - the extern "C" boundary of libhelios_gb300.so: argument
// validation, derived instrument constants, scene lifetime and launches.
#include "hg_host.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>

namespace hg {

static thread_local std::string g_err;

helios_status set_error(helios_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

helios_status set_cuda_error(const char* what, cudaError_t e) {
    (void)cudaGetLastError();  // clear a non-sticky error
    return set_error(e == cudaErrorMemoryAllocation ? HELIOS_ERR_OOM : HELIOS_ERR_CUDA, "%s: %s",
                     what, cudaGetErrorString(e));
}

// one NVTX range per API call
struct CallRange {
    explicit CallRange(const char* name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange&) = delete;
    CallRange& operator=(const CallRange&) = delete;
};

// host-side fault injection for tests (HELIOS_FAULT=badarg|oom, read per call)
enum { kFaultNone = 0, kFaultBadArg = 1, kFaultOom = 2 };
static int injected_fault() {
    const char* f = std::getenv("HELIOS_FAULT");
    if (!f) return kFaultNone;
    if (!strcmp(f, "badarg")) return kFaultBadArg;
    if (!strcmp(f, "oom")) return kFaultOom;
    return kFaultNone;
}

// device allocations of the API layer: an injected oom fails the first one
static cudaError_t dev_malloc(void** p, size_t n) {
    if (injected_fault() == kFaultOom) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, n);
}
static cudaError_t dev_malloc_async(void** p, size_t n, cudaStream_t st) {
    if (injected_fault() == kFaultOom) return cudaErrorMemoryAllocation;
    return cudaMallocAsync(p, n, st);
}
// a scan's first device allocation is its scratch (masks, lists, queues)
static helios_status scratch_fault() {
    if (injected_fault() == kFaultOom)
        return set_error(HELIOS_ERR_OOM, "scan scratch: injected fault (HELIOS_FAULT=oom)");
    return HELIOS_OK;
}

static int32_t subray_count(int32_t q) {
    if (q < 0) return -1;
    int32_t s = 1;
    for (int i = 1; i <= q; ++i) s += (int32_t)std::floor(2.0 * kPi * (double)i);
    return s;
}

static helios_status check_scanner(const helios_scanner_desc& s, int idx) {
    auto bad = [&](const char* what) {
        return set_error(HELIOS_ERR_INVALID_ARG, "scanner %d: %s", idx, what);
    };
    if (!(s.prf_hz > 0.0) || !std::isfinite(s.prf_hz)) return bad("prf_hz must be > 0");
    if (!(s.divergence_rad > 0.0) || !(s.divergence_rad < 0.5)) return bad("divergence_rad must be in (0, 0.5)");
    if (s.beam_sample_quality < 0 || s.beam_sample_quality > 9) return bad("beam_sample_quality must be in 0..9");
    if (!(s.wavelength_m > 0.0)) return bad("wavelength_m must be > 0");
    if (!(s.bin_ns > 0.0)) return bad("bin_ns must be > 0");
    if (s.n_bins < 4 || s.n_bins > 4096) return bad("n_bins must be in 4..4096");
    if (s.max_echoes < 1 || s.max_echoes > 32) return bad("max_echoes must be in 1..32");
    if (!(s.echo_threshold_rel >= 0.0 && s.echo_threshold_rel <= 1.0)) return bad("echo_threshold_rel must be in [0,1]");
    if (!(s.range_noise_sigma_m >= 0.0)) return bad("range_noise_sigma_m must be >= 0");
    if (!(s.peak_power_w >= 0.0) || !(s.receiver_diam_m >= 0.0)) return bad("power parameters must be >= 0");
    if (s.pulse_shape == HELIOS_PULSE_GAUSSIAN) {
        if (!(s.pulse_fwhm_ns > 0.0)) return bad("pulse_fwhm_ns must be > 0");
    } else if (s.pulse_shape == HELIOS_PULSE_CARLSSON) {
        if (!(s.pulse_length_ns > 0.0)) return bad("pulse_length_ns must be > 0");
    } else {
        return bad("unknown pulse_shape");
    }
    if (s.deflector < 0 || s.deflector > 5) return bad("unknown deflector");
    if (s.deflector == HELIOS_DEFL_FIBRE && s.n_fibres < 1) return bad("n_fibres must be >= 1");
    if (s.deflector == HELIOS_DEFL_TLS_GRID && (s.grid_n_az < 1 || s.grid_n_el < 1))
        return bad("TLS grid needs grid_n_az, grid_n_el >= 1");
    return HELIOS_OK;
}

static DevScanner derive_scanner(const helios_scanner_desc& s) {
    DevScanner d;
    memset(&d, 0, sizeof(d));
    d.prf = s.prf_hz;
    d.bin_ns = s.bin_ns;
    d.theta_r = 0.5 * s.divergence_rad;
    d.scan_freq = s.scan_freq_hz;
    d.amax = s.scan_angle_max_rad;
    d.head_rate = s.head_rate_rad_s;
    d.el_min = s.el_min_rad;
    d.el_max = s.el_max_rad;
    double w0 = s.beam_waist_m > 0.0 ? s.beam_waist_m : s.wavelength_m / (kPi * d.theta_r);
    d.w0sq = (float)(w0 * w0);
    d.zk = (float)(s.wavelength_m / (kPi * w0 * w0));
    d.focus = (float)s.focus_m;
    d.pconst = (float)(s.peak_power_w * s.receiver_diam_m * s.receiver_diam_m * s.eta_sys * s.eta_atm / 4.0);
    // pulse support: where the shape falls below 2^-30 of its peak
    if (s.pulse_shape == HELIOS_PULSE_GAUSSIAN) {
        double sig = s.pulse_fwhm_ns / (2.0 * std::sqrt(2.0 * std::log(2.0)));
        double gk2 = 1.4426950408889634 / (2.0 * sig * sig);
        d.gk2 = (float)gk2;
        d.inv_s2 = (float)(1.0 / (sig * sig));
        d.sigma_bins = (float)(sig / s.bin_ns);
        d.cut_lo = d.cut_hi = (float)std::sqrt(30.0 / gk2);
        d.n_pre = (int32_t)std::ceil(3.0 * sig / s.bin_ns);
        d.echo_offset_ns = 0.0;
    } else {
        double tau = s.pulse_length_ns / 1.75;
        d.ctau_inv = (float)(1.0 / tau);
        double peak = 4.0 * std::exp(-2.0), y = 2.0;
        while (y * y * std::exp(-y) >= std::ldexp(peak, -30)) y += 0.25;
        d.cut_lo = 0.0f;
        d.cut_hi = (float)(y * tau);
        d.n_pre = 0;
        d.echo_offset_ns = 2.0 * tau;
    }
    d.bins_per_metre = kDelayPerMetre / s.bin_ns;
    d.inv_bin = (float)(1.0 / s.bin_ns);
    d.bpm_hi = (float)d.bins_per_metre;
    d.bpm_lo = (float)(d.bins_per_metre - (double)d.bpm_hi);
    d.bin_hi = (float)s.bin_ns;
    d.bin_lo = (float)(s.bin_ns - (double)d.bin_hi);
    d.echo_offset_f = (float)d.echo_offset_ns;
    d.thr_rel = (float)s.echo_threshold_rel;
    d.noise_sigma = (float)s.range_noise_sigma_m;
    d.q_default = s.beam_sample_quality;
    d.pulse_shape = s.pulse_shape;
    d.n_bins = s.n_bins;
    d.max_echoes = s.max_echoes;
    d.deflector = s.deflector;
    d.n_az = s.grid_n_az;
    d.n_el = s.grid_n_el;
    d.n_fibres = s.n_fibres;
    return d;
}

static DevScene dev_scene(const helios_scene* s) {
    DevScene d;
    memset(&d, 0, sizeof(d));
    d.nodes = s->nodes;
    d.nodes4 = s->nodes4;
    d.n_node4 = (int32_t)s->n_node4;
    d.tris = s->tris;
    d.tri_index = s->tri_index;
    for (int m = 0; m < s->n_mesh; ++m) d.refl[m] = s->refl[m];
    for (int m = 0; m <= s->n_mesh; ++m) d.mesh_first[m] = s->mesh_first[m];
    d.n_tri = (int32_t)s->n_tri;
    d.n_int = (int32_t)s->n_int;
    d.n_mesh = s->n_mesh;
    d.n_grid = s->n_grid;
    d.has_grid = s->n_grid > 0;
    if (s->n_grid == 1) d.grid = s->grids[0];
    if (s->n_grid > 1) {
        d.grids = s->grids_d;
        d.gnodes = s->gnodes;
    }
    return d;
}

static void free_scene_buffers(helios_scene* s) {
    cudaFree(s->nodes);
    cudaFree(s->nodes4);
    cudaFree(s->tris);
    cudaFree(s->tri_index);
    for (float* p : s->lads) cudaFree(p);
    s->lads.clear();
    cudaFree(s->grids_d);
    cudaFree(s->gnodes);
    s->nodes = s->tris = s->nodes4 = s->gnodes = nullptr;
    s->tri_index = nullptr;
    s->grids_d = nullptr;
}

// Boxes of a scene's grids must have disjoint interiors (touching faces are
// fine): then a ray's segments in them follow the order of the entry points.
// Sweep along x over the boxes sorted by their low x.
static helios_status check_grid_boxes(const helios_voxel_desc* g, int n) {
    if (n < 2) return HELIOS_OK;
    std::vector<std::array<double, 6>> b((size_t)n);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            b[i][a] = (double)g[i].origin[a];
            b[i][3 + a] = (double)g[i].origin[a] + (double)g[i].dims[a] * (double)g[i].cell;
        }
    std::vector<int> order((size_t)n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return b[x][0] < b[y][0]; });
    // overlaps thinner than 1e-6 of the boxes' size are rounding of the
    // corners (e.g. FP32 origins i * width): taken as touching
    double ext = 0.0;
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) ext = std::max(ext, b[i][3 + a] - b[i][a]);
    const double eps = 1e-6 * ext;
    for (int i = 0; i < n; ++i) {
        const auto& p = b[order[i]];
        for (int j = i + 1; j < n && b[order[j]][0] < p[3] - eps; ++j) {
            const auto& q = b[order[j]];
            if (p[1] < q[4] - eps && q[1] < p[4] - eps && p[2] < q[5] - eps && q[2] < p[5] - eps)
                return set_error(HELIOS_ERR_INVALID_ARG, "grids %d and %d overlap", order[i], order[j]);
        }
    }
    return HELIOS_OK;
}

// BVH over the grids' boxes (median split on the longest axis of the box
// centres), nodes in the layout of the triangle BVH: child boxes and
// (child0, child1) with leaf children ~grid.  Boxes are widened so that a
// ray the FP64 march takes into a grid is never culled by the FP32 test.
static int grid_bvh_rec(const std::vector<std::array<float, 6>>& box, std::vector<int>& idx, int lo, int hi,
                        std::vector<float4>& nodes, std::array<float, 6>& out_box) {
    auto merge = [](std::array<float, 6>& a, const std::array<float, 6>& c) {
        for (int k = 0; k < 3; ++k) {
            a[k] = std::min(a[k], c[k]);
            a[3 + k] = std::max(a[3 + k], c[3 + k]);
        }
    };
    if (hi - lo == 1) {
        out_box = box[idx[lo]];
        return ~idx[lo];
    }
    float cmin[3] = {3e38f, 3e38f, 3e38f}, cmax[3] = {-3e38f, -3e38f, -3e38f};
    for (int i = lo; i < hi; ++i)
        for (int k = 0; k < 3; ++k) {
            const float c = 0.5f * (box[idx[i]][k] + box[idx[i]][3 + k]);
            cmin[k] = std::min(cmin[k], c);
            cmax[k] = std::max(cmax[k], c);
        }
    int ax = 0;
    for (int k = 1; k < 3; ++k)
        if (cmax[k] - cmin[k] > cmax[ax] - cmin[ax]) ax = k;
    const int mid = (lo + hi) / 2;
    std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, [&](int x, int y) {
        return box[x][ax] + box[x][3 + ax] < box[y][ax] + box[y][3 + ax];
    });
    const int node = (int)(nodes.size() / 4);
    nodes.resize(nodes.size() + 4);
    std::array<float, 6> b0, b1;
    const int c0 = grid_bvh_rec(box, idx, lo, mid, nodes, b0);
    const int c1 = grid_bvh_rec(box, idx, mid, hi, nodes, b1);
    float4* n = &nodes[(size_t)node * 4];
    n[0] = make_float4(b0[0], b0[1], b0[2], b0[3]);
    n[1] = make_float4(b0[4], b0[5], b1[0], b1[1]);
    n[2] = make_float4(b1[2], b1[3], b1[4], b1[5]);
    int4 ch = make_int4(c0, c1, -1, ax);
    memcpy(&n[3], &ch, sizeof(ch));
    out_box = b0;
    merge(out_box, b1);
    return node;
}

// The grids' device descriptors, leaf-angle table copies and, with several
// grids, their BVH.
static helios_status build_grids(helios_scene* s, const helios_scene_desc* desc, cudaStream_t st) {
    const int n = desc->n_grids;
    s->grids.assign((size_t)n, DevGrid{});
    int64_t vox = 0;
    for (int i = 0; i < n; ++i) {
        const helios_voxel_desc& g = desc->grids[i];
        DevGrid& d = s->grids[i];
        d.density = g.density;
        for (int a = 0; a < 3; ++a) {
            d.g0[a] = g.origin[a];
            d.dims[a] = g.dims[a];
            d.bdims[a] = (g.dims[a] + kBrick - 1) >> kBrickLog2;
        }
        d.cell = g.cell;
        {
            const double ic = 1.0 / (double)g.cell;
            d.icell_h = (float)ic;
            d.icell_l = (float)(ic - (double)d.icell_h);
        }
        d.opaque = g.opaque != 0;
        d.G = g.G;
        d.leaf_refl = g.leaf_reflectance;
        d.vox_off = vox;
        vox += (int64_t)g.dims[0] * g.dims[1] * g.dims[2];
        if (g.lad_table) {
            // leaf-angle table: read (host or device memory), checked, copied
            const int32_t m = g.lad_n;
            std::vector<float> h((size_t)m);
            cudaError_t e = cudaMemcpyAsync(h.data(), g.lad_table, sizeof(float) * (size_t)m, cudaMemcpyDefault, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return set_cuda_error("reading a leaf-angle table", e);
            for (int32_t k = 0; k < m; ++k)
                if (!(h[k] >= 0.0f && h[k] <= 3.0e38f))
                    return set_error(HELIOS_ERR_INVALID_ARG, "grid %d: lad_table[%d] is negative or not finite", i, k);
            float* dl = nullptr;
            e = dev_malloc(reinterpret_cast<void**>(&dl), sizeof(float) * (size_t)m);
            if (e != cudaSuccess) return set_cuda_error("leaf-angle table allocation", e);
            s->lads.push_back(dl);
            e = cudaMemcpy(dl, h.data(), sizeof(float) * (size_t)m, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return set_cuda_error("leaf-angle table copy", e);
            d.lad = dl;
            d.lad_n = m;
            s->bytes += (int64_t)sizeof(float) * m;
        }
    }
    if (n < 2) return HELIOS_OK;
    std::vector<std::array<float, 6>> box((size_t)n);
    for (int i = 0; i < n; ++i) {
        const DevGrid& d = s->grids[i];
        double m = 0.0;
        for (int a = 0; a < 3; ++a)
            m = std::max(m, std::max(std::fabs((double)d.g0[a]),
                                     std::fabs((double)d.g0[a] + (double)d.dims[a] * d.cell)));
        const double w = 1e-5 * m + 1e-3 * (double)d.cell;
        for (int a = 0; a < 3; ++a) {
            box[i][a] = (float)((double)d.g0[a] - w);
            box[i][3 + a] = (float)((double)d.g0[a] + (double)d.dims[a] * d.cell + w);
        }
    }
    std::vector<int> idx((size_t)n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::vector<float4> nodes;
    nodes.reserve((size_t)4 * (n - 1));
    std::array<float, 6> root;
    grid_bvh_rec(box, idx, 0, n, nodes, root);
    cudaError_t e = dev_malloc(reinterpret_cast<void**>(&s->gnodes), sizeof(float4) * nodes.size());
    if (e == cudaSuccess) e = cudaMemcpy(s->gnodes, nodes.data(), sizeof(float4) * nodes.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void**>(&s->grids_d), sizeof(DevGrid) * (size_t)n);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->grids_d, s->grids.data(), sizeof(DevGrid) * (size_t)n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_cuda_error("grid BVH", e);
    s->bytes += (int64_t)(sizeof(float4) * nodes.size() + sizeof(DevGrid) * (size_t)n);
    return HELIOS_OK;
}

struct LegPlan {
    std::vector<DevLeg> legs;
    int64_t total_pulses = 0, wave = 0, sub = 0, echo = 0;
};

// Pulses per work item: whole batches of `sub` pulses.  Stochastic scans take
// up to 256 (the cone walk groups ~32 pulses per warp); expected-mode scans
// keep one batch, since their larger per-warp scratch leaves no shared memory
// for a longer item at two blocks per SM.
static int32_t item_pulses(int32_t sub, int mode) {
    return mode == HELIOS_MODE_EXPECTED ? sub : sub * (256 / sub);
}

static helios_status plan_legs(const helios_scanner_desc* scanners, int32_t n_scanners,
                               const helios_leg_desc* legs, int32_t n_legs, int32_t n_scenes,
                               int rays_per_item, int mode, LegPlan& P) {
    if (n_legs < 0 || (n_legs > 0 && !legs)) return set_error(HELIOS_ERR_INVALID_ARG, "legs is NULL");
    if (n_scanners < 1 || n_scanners > kMaxScanners || !scanners)
        return set_error(HELIOS_ERR_INVALID_ARG, "n_scanners must be in 1..%d", kMaxScanners);
    for (int i = 0; i < n_scanners; ++i) {
        helios_status st = check_scanner(scanners[i], i);
        if (st != HELIOS_OK) return st;
    }
    P.legs.clear();
    for (int l = 0; l < n_legs; ++l) {
        const helios_leg_desc& L = legs[l];
        if (n_scenes >= 0 && (L.scene_index < 0 || L.scene_index >= n_scenes))
            return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: scene_index out of range", l);
        if (L.scanner_index < 0 || L.scanner_index >= n_scanners)
            return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: scanner_index out of range", l);
        if (L.platform != HELIOS_PLATFORM_STATIC && L.platform != HELIOS_PLATFORM_LINEAR)
            return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: unknown platform", l);
        if (L.n_pulses < 0) return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: n_pulses < 0", l);
        // draws are keyed by the absolute pulse index in 44 bits
        if (L.first_pulse < 0 || L.first_pulse > kMaxPulseIndex - L.n_pulses)
            return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: first_pulse + n_pulses must be in 0..2^44", l);
        if (!(L.platform_noise_m >= 0.0f))
            return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: platform_noise_m must be >= 0", l);
        if (L.platform == HELIOS_PLATFORM_LINEAR && !(L.speed_mps >= 0.0))
            return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: speed_mps must be >= 0", l);
        const helios_scanner_desc& sc = scanners[L.scanner_index];
        int q = L.beam_sample_quality >= 0 ? L.beam_sample_quality : sc.beam_sample_quality;
        if (q > 9) return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: beam_sample_quality must be <= 9", l);
        DevLeg d;
        memset(&d, 0, sizeof(d));
        double D[3];
        double len2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            d.start[a] = L.start[a];
            D[a] = L.end[a] - L.start[a];
            len2 += D[a] * D[a];
            d.rpy[a] = L.attitude_rpy[a];
        }
        d.length = std::sqrt(len2);
        if (L.platform == HELIOS_PLATFORM_LINEAR && d.length > 0.0) {
            for (int a = 0; a < 3; ++a) d.dir[a] = D[a] / d.length;
            d.rpy[2] += std::atan2(D[1], D[0]);  // heading towards the next waypoint
        }
        d.speed = L.speed_mps;
        d.t0 = L.t0;
        d.n_pulses = L.n_pulses;
        d.scene = L.scene_index;
        d.scanner = L.scanner_index;
        d.platform = L.platform;
        d.q = q;
        d.S = subray_count(q);
        int ppi = rays_per_item / d.S;
        d.pulses_per_sub = ppi < 1 ? 1 : (ppi > 256 ? 256 : ppi);
        d.pulses_per_item = item_pulses(d.pulses_per_sub, mode);
        d.leg_id = L.leg_id;
        d.platform_noise = L.platform_noise_m;
        d.k_first = L.first_pulse;
        d.pulse_off = P.total_pulses;
        d.wave_off = P.wave;
        d.sub_off = P.sub;
        d.echo_off = P.echo;
        P.total_pulses += L.n_pulses;
        P.wave += L.n_pulses * sc.n_bins;
        P.sub += L.n_pulses * d.S;
        P.echo += L.n_pulses * sc.max_echoes;
        P.legs.push_back(d);
    }
    return HELIOS_OK;
}

// The kernels index the outputs of absolute pulse k at offset + k: the plan's
// offsets (where a leg's rows start) less first_pulse rows.
static DevLeg kernel_leg(DevLeg d, const helios_scanner_desc* scanners) {
    const helios_scanner_desc& sc = scanners[d.scanner];
    d.pulse_off -= d.k_first;
    d.wave_off -= d.k_first * sc.n_bins;
    d.sub_off -= d.k_first * d.S;
    d.echo_off -= d.k_first * sc.max_echoes;
    return d;
}

static helios_status check_scenes(helios_scene* const* scenes, int32_t n_scenes) {
    if (n_scenes < 1 || n_scenes > kMaxScenes || !scenes)
        return set_error(HELIOS_ERR_INVALID_ARG, "n_scenes must be in 1..%d", kMaxScenes);
    for (int i = 0; i < n_scenes; ++i)
        if (!scenes[i]) return set_error(HELIOS_ERR_INVALID_ARG, "scene %d is NULL", i);
    return HELIOS_OK;
}

}  // namespace hg

using namespace hg;

extern "C" {

const char* helios_last_error(void) { return g_err.c_str(); }

const char* helios_version(void) { return "helios_gb300 0.1 sm_103a"; }

int32_t helios_subray_count(int32_t q) { return subray_count(q); }

helios_status helios_build_scene(const helios_scene_desc* desc, void* cuda_stream,
                                 helios_scene** out) {
    g_err.clear();
    CallRange range_("helios_build_scene");
    if (injected_fault() == kFaultBadArg)
        return set_error(HELIOS_ERR_INVALID_ARG, "helios_build_scene: injected fault (HELIOS_FAULT=badarg)");
    if (!desc || !out) return set_error(HELIOS_ERR_INVALID_ARG, "desc and out must not be NULL");
    *out = nullptr;
    if (desc->n_meshes < 0 || desc->n_meshes > kMaxMesh)
        return set_error(HELIOS_ERR_UNSUPPORTED, "n_meshes must be in 0..%d", kMaxMesh);
    if (desc->n_meshes > 0 && !desc->meshes) return set_error(HELIOS_ERR_INVALID_ARG, "meshes is NULL");
    if (desc->n_grids < 0) return set_error(HELIOS_ERR_INVALID_ARG, "n_grids < 0");
    if (desc->n_grids > kMaxGrids)
        return set_error(HELIOS_ERR_UNSUPPORTED, "at most %d voxel grids per scene", kMaxGrids);
    if (desc->n_grids > 0 && !desc->grids) return set_error(HELIOS_ERR_INVALID_ARG, "grids is NULL");
    int64_t n_tri = 0;
    for (int m = 0; m < desc->n_meshes; ++m) {
        const helios_mesh_desc& M = desc->meshes[m];
        if (M.n_faces < 0 || M.n_verts < 0) return set_error(HELIOS_ERR_INVALID_ARG, "mesh %d: negative size", m);
        if (M.n_faces > 0 && (!M.verts || !M.faces || !M.reflectance || M.n_verts == 0))
            return set_error(HELIOS_ERR_INVALID_ARG, "mesh %d: NULL array", m);
        n_tri += M.n_faces;
    }
    int64_t n_vox = 0;
    for (int i = 0; i < desc->n_grids; ++i) {
        const helios_voxel_desc& g = desc->grids[i];
        if (g.dims[0] < 1 || g.dims[1] < 1 || g.dims[2] < 1)
            return set_error(HELIOS_ERR_INVALID_ARG, "grid %d: dims must be >= 1", i);
        if (!(g.cell > 0.0f)) return set_error(HELIOS_ERR_INVALID_ARG, "grid %d: cell must be > 0", i);
        if (!(g.G >= 0.0f)) return set_error(HELIOS_ERR_INVALID_ARG, "grid %d: G must be >= 0", i);
        if (!g.density) return set_error(HELIOS_ERR_INVALID_ARG, "grid %d: density is NULL", i);
        if (g.lad_table && (g.lad_n < 2 || g.lad_n > 65536))
            return set_error(HELIOS_ERR_INVALID_ARG, "grid %d: lad_n must be in 2..65536", i);
        const int64_t nv = (int64_t)g.dims[0] * g.dims[1] * g.dims[2];
        // within a grid the kernels index voxels (after the triangles) in 32 bits
        if (n_tri + nv >= (int64_t)INT32_MAX)
            return set_error(HELIOS_ERR_UNSUPPORTED, "grid %d: triangles + its voxels exceed 2^31 - 1", i);
        n_vox += nv;
    }
    // draws are keyed by the voxel id in 40 bits
    if (n_vox >= kMaxVoxelId)
        return set_error(HELIOS_ERR_UNSUPPORTED, "the grids hold %lld voxels; at most 2^40 - 1 per scene",
                         (long long)n_vox);
    helios_status r = check_grid_boxes(desc->grids, desc->n_grids);
    if (r != HELIOS_OK) return r;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    helios_scene* s = new helios_scene();
    cudaGetDevice(&s->device);
    s->n_tri = n_tri;
    s->n_int = n_tri > 1 ? n_tri - 1 : 0;
    s->n_mesh = desc->n_meshes;
    s->n_grid = desc->n_grids;
    int64_t off = 0;
    for (int m = 0; m < desc->n_meshes; ++m) {
        s->mesh_first[m] = (int32_t)off;
        s->mesh_faces[m] = desc->meshes[m].n_faces;
        s->refl[m] = desc->meshes[m].reflectance;
        off += desc->meshes[m].n_faces;
    }
    s->mesh_first[desc->n_meshes] = (int32_t)off;
    r = build_grids(s, desc, st);
    if (r != HELIOS_OK) {
        free_scene_buffers(s);
        delete s;
        return r;
    }
    cudaError_t e = cudaSuccess;
    if (s->n_int > 0) e = dev_malloc(reinterpret_cast<void**>(&s->nodes), sizeof(float4) * 4 * (size_t)s->n_int);
    if (e == cudaSuccess && n_tri > 0)
        e = dev_malloc(reinterpret_cast<void**>(&s->tris), sizeof(float4) * 3 * (size_t)n_tri);
    if (e == cudaSuccess && n_tri > 0)
        e = dev_malloc(reinterpret_cast<void**>(&s->tri_index), sizeof(int32_t) * (size_t)n_tri);
    if (e != cudaSuccess) {
        r = set_cuda_error("scene allocation", e);
        free_scene_buffers(s);
        delete s;
        return r;
    }
    s->bytes += (int64_t)sizeof(float4) * (4 * s->n_int + 3 * n_tri) + (int64_t)sizeof(int32_t) * n_tri;
    r = build_bvh(s, desc, st);
    if (r != HELIOS_OK) {
        cudaStreamSynchronize(st);
        free_scene_buffers(s);
        delete s;
        return r;
    }
    *out = s;
    return HELIOS_OK;
}

helios_status helios_free_scene(helios_scene* scene) {
    g_err.clear();
    CallRange range_("helios_free_scene");
    if (injected_fault() == kFaultBadArg)
        return set_error(HELIOS_ERR_INVALID_ARG, "helios_free_scene: injected fault (HELIOS_FAULT=badarg)");
    if (!scene) return HELIOS_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != scene->device) cudaSetDevice(scene->device);
    free_scene_buffers(scene);
    if (cur != scene->device) cudaSetDevice(cur);
    delete scene;
    return HELIOS_OK;
}

helios_status helios_lad_table(int32_t distribution, int32_t n, float* table, void* cuda_stream) {
    g_err.clear();
    CallRange range_("helios_lad_table");
    if (injected_fault() == kFaultBadArg)
        return set_error(HELIOS_ERR_INVALID_ARG, "helios_lad_table: injected fault (HELIOS_FAULT=badarg)");
    if (distribution < HELIOS_LAD_PLANOPHILE || distribution > HELIOS_LAD_SPHERICAL)
        return set_error(HELIOS_ERR_INVALID_ARG, "unknown leaf angle distribution %d", distribution);
    if (n < 2 || n > 65536) return set_error(HELIOS_ERR_INVALID_ARG, "n must be in 2..65536");
    if (!table) return set_error(HELIOS_ERR_INVALID_ARG, "table is NULL");
    return launch_lad_table(distribution, n, table, (cudaStream_t)cuda_stream);
}

helios_status helios_scene_get_info(const helios_scene* scene, helios_scene_info* info) {
    g_err.clear();
    CallRange range_("helios_scene_get_info");
    if (injected_fault() == kFaultBadArg)
        return set_error(HELIOS_ERR_INVALID_ARG, "helios_scene_get_info: injected fault (HELIOS_FAULT=badarg)");
    if (!scene || !info) return set_error(HELIOS_ERR_INVALID_ARG, "scene and info must not be NULL");
    info->n_triangles = scene->n_tri;
    info->n_bvh_nodes = scene->n_int;
    info->device_bytes = scene->bytes;
    info->n_meshes = scene->n_mesh;
    info->n_grids = scene->n_grid;
    info->n_bvh4_nodes = scene->n_node4;
    return HELIOS_OK;
}

helios_status helios_output_layout(const helios_scanner_desc* scanners, int32_t n_scanners,
                                   const helios_leg_desc* legs, int32_t n_legs,
                                   int64_t* pulse_offset, int64_t* wave_offset,
                                   int64_t* subray_offset, int64_t* echo_offset,
                                   helios_layout* totals) {
    g_err.clear();
    CallRange range_("helios_output_layout");
    if (injected_fault() == kFaultBadArg)
        return set_error(HELIOS_ERR_INVALID_ARG, "helios_output_layout: injected fault (HELIOS_FAULT=badarg)");
    LegPlan P;
    helios_status st = plan_legs(scanners, n_scanners, legs, n_legs, -1, 768, HELIOS_MODE_STOCHASTIC, P);
    if (st != HELIOS_OK) return st;
    for (int l = 0; l < n_legs; ++l) {
        if (pulse_offset) pulse_offset[l] = P.legs[l].pulse_off;
        if (wave_offset) wave_offset[l] = P.legs[l].wave_off;
        if (subray_offset) subray_offset[l] = P.legs[l].sub_off;
        if (echo_offset) echo_offset[l] = P.legs[l].echo_off;
    }
    if (totals) {
        totals->total_pulses = P.total_pulses;
        totals->waveform_floats = P.wave;
        totals->subray_elems = P.sub;
        totals->echo_elems = P.echo;
    }
    return HELIOS_OK;
}

helios_status helios_scan_legs(helios_scene* const* scenes, int32_t n_scenes,
                               const helios_scanner_desc* scanners, int32_t n_scanners,
                               const helios_leg_desc* legs, int32_t n_legs,
                               const helios_scan_opts* opts, const helios_outputs* out,
                               void* cuda_stream) {
    g_err.clear();
    CallRange range_("helios_scan_legs");
    if (injected_fault() == kFaultBadArg)
        return set_error(HELIOS_ERR_INVALID_ARG, "helios_scan_legs: injected fault (HELIOS_FAULT=badarg)");
    helios_status st = check_scenes(scenes, n_scenes);
    if (st != HELIOS_OK) return st;
    if (!opts || !out) return set_error(HELIOS_ERR_INVALID_ARG, "opts and out must not be NULL");
    if (opts->mode != HELIOS_MODE_STOCHASTIC && opts->mode != HELIOS_MODE_EXPECTED)
        return set_error(HELIOS_ERR_INVALID_ARG, "unknown mode");
    if (!out->waveform || !out->window_bin || !out->echo_count || !out->echo_range)
        return set_error(HELIOS_ERR_INVALID_ARG, "waveform, window_bin, echo_count, echo_range are required");
    if (out->subray_range && !out->subray_hit)
        return set_error(HELIOS_ERR_INVALID_ARG, "subray_range needs subray_hit");
    int threads = opts->block_threads > 0 ? opts->block_threads : 256;
    if (threads % 32 != 0 || threads < 64 || threads > 256)
        return set_error(HELIOS_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in 64..256");
    int rays = opts->rays_per_block > 0 ? opts->rays_per_block : 768;
    if (rays > 4096) return set_error(HELIOS_ERR_INVALID_ARG, "rays_per_block must be <= 4096");
    LegPlan P;
    st = plan_legs(scanners, n_scanners, legs, n_legs, n_scenes, rays, opts->mode, P);
    if (st != HELIOS_OK) return st;
    ScanLaunch L;
    for (int i = 0; i < n_scenes; ++i) L.scenes.push_back(dev_scene(scenes[i]));
    for (int i = 0; i < n_scanners; ++i) L.scanners.push_back(derive_scanner(scanners[i]));
    for (const DevLeg& d : P.legs) L.legs.push_back(kernel_leg(d, scanners));
    L.out.waveform = out->waveform;
    L.out.window_bin = out->window_bin;
    L.out.echo_count = out->echo_count;
    L.out.echo_range = out->echo_range;
    L.out.echo_amp = out->echo_amp;
    L.out.echo_bin = out->echo_bin;
    L.out.echo_object = out->echo_object;
    L.out.pulse_flags = out->pulse_flags;
    L.out.subray_hit = out->subray_hit;
    L.out.subray_range = out->subray_range;
    L.out.status = out->status;
    L.out.echo_width = out->echo_width;
    L.seed = opts->seed;
    L.mode = opts->mode;
    L.persistent = opts->persistent;
    L.threads = threads;
    L.blocks_per_sm = opts->blocks_per_sm;
    if (P.total_pulses == 0) return HELIOS_OK;
    st = scratch_fault();
    if (st != HELIOS_OK) return st;
    OccupancyMasks masks;
    st = build_occupancy(L.scenes, scenes, (cudaStream_t)cuda_stream, masks);
    if (st != HELIOS_OK) return st;
    return launch_scan(L, (cudaStream_t)cuda_stream);
}

helios_status helios_scan_adjoint(helios_scene* const* scenes, int32_t n_scenes,
                                  const helios_scanner_desc* scanners, int32_t n_scanners,
                                  const helios_leg_desc* legs, int32_t n_legs,
                                  const helios_scan_opts* opts, const float* d_waveform,
                                  const int32_t* window_bin, const int64_t* subray_hit,
                                  const helios_scene_grads* grads, void* cuda_stream) {
    g_err.clear();
    CallRange range_("helios_scan_adjoint");
    if (injected_fault() == kFaultBadArg)
        return set_error(HELIOS_ERR_INVALID_ARG, "helios_scan_adjoint: injected fault (HELIOS_FAULT=badarg)");
    helios_status st = check_scenes(scenes, n_scenes);
    if (st != HELIOS_OK) return st;
    if (!opts || !d_waveform || !window_bin || !grads)
        return set_error(HELIOS_ERR_INVALID_ARG, "opts, d_waveform, window_bin, grads must not be NULL");
    if (opts->mode != HELIOS_MODE_EXPECTED)
        return set_error(HELIOS_ERR_INVALID_ARG, "the adjoint is defined for mode EXPECTED only");
    for (int i = 0; i < n_scenes; ++i)
        for (const DevGrid& g : scenes[i]->grids)
            if (g.opaque)
                return set_error(HELIOS_ERR_UNSUPPORTED, "opaque voxels have no density gradient; the adjoint needs transmissive grids");
    int threads = opts->block_threads > 0 ? opts->block_threads : 256;
    if (threads % 32 != 0 || threads < 64 || threads > 256)
        return set_error(HELIOS_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in 64..256");
    // items of ~768 subrays (40 pulses at 19 subrays): with 8 warps per block a
    // smaller item leaves warps idle at the per-item barrier
    const int rays = opts->rays_per_block > 0 ? opts->rays_per_block : 768;
    if (rays > 4096) return set_error(HELIOS_ERR_INVALID_ARG, "rays_per_block must be <= 4096");
    LegPlan P;
    st = plan_legs(scanners, n_scanners, legs, n_legs, n_scenes, rays, HELIOS_MODE_EXPECTED, P);
    if (st != HELIOS_OK) return st;
    AdjointLaunch L;
    for (int i = 0; i < n_scenes; ++i) {
        L.scenes.push_back(dev_scene(scenes[i]));
        std::vector<float*> dr(kMaxMesh, nullptr);
        for (int m = 0; m < scenes[i]->n_mesh; ++m)
            dr[m] = grads[i].d_reflectance ? grads[i].d_reflectance[m] : nullptr;
        L.d_refl.push_back(dr);
        int32_t want = 0;
        if (grads[i].d_density)
            for (int g = 0; g < scenes[i]->n_grid; ++g) want |= grads[i].d_density[g] != nullptr;
        L.want_dens.push_back(want);
    }
    for (int i = 0; i < n_scanners; ++i) L.scanners.push_back(derive_scanner(scanners[i]));
    for (const DevLeg& d : P.legs) L.legs.push_back(kernel_leg(d, scanners));
    L.g = d_waveform;
    L.window = window_bin;
    L.subray_hit = subray_hit;
    L.seed = opts->seed;
    L.threads = threads;
    if (P.total_pulses == 0) return HELIOS_OK;
    st = scratch_fault();
    if (st != HELIOS_OK) return st;
    OccupancyMasks masks;
    st = build_occupancy(L.scenes, scenes, (cudaStream_t)cuda_stream, masks, grads);
    if (st != HELIOS_OK) return st;
    return launch_adjoint(L, (cudaStream_t)cuda_stream);
}

helios_status helios_fetch_counts_sample(helios_scene* scene, const helios_scanner_desc* scanner,
                                         const helios_leg_desc* leg, int32_t mode, uint64_t seed,
                                         int64_t first, int64_t stride, int64_t count,
                                         helios_fetch_counts* out, void* cuda_stream) {
    g_err.clear();
    if (!scene || !scanner || !leg) return set_error(HELIOS_ERR_INVALID_ARG, "scene, scanner, leg must not be NULL");
    if (mode != HELIOS_MODE_STOCHASTIC && mode != HELIOS_MODE_EXPECTED)
        return set_error(HELIOS_ERR_INVALID_ARG, "unknown mode %d", mode);
    if (count < 0 || first < 0 || stride < 1)
        return set_error(HELIOS_ERR_INVALID_ARG, "need count >= 0, first >= 0, stride >= 1");
    if (count > 0 && !out) return set_error(HELIOS_ERR_INVALID_ARG, "out must not be NULL");
    helios_leg_desc L = *leg;
    L.scene_index = 0;
    L.scanner_index = 0;
    LegPlan P;
    helios_status st = plan_legs(scanner, 1, &L, 1, 1, 256, mode, P);
    if (st != HELIOS_OK) return st;
    if (count > 0 && (first >= L.n_pulses || (count - 1) > (L.n_pulses - 1 - first) / stride))
        return set_error(HELIOS_ERR_INVALID_ARG, "sampled pulses must lie inside the leg's %lld pulses",
                         (long long)L.n_pulses);
    return launch_fetch_counts(dev_scene(scene), derive_scanner(*scanner), kernel_leg(P.legs[0], scanner),
                               mode, seed, first, stride, count, out, (cudaStream_t)cuda_stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// helios_scan_legs_static: the persistent scan without any allocation.
// Validation and leg planning mirror helios_scan_legs but write into
// fixed-size static arrays (no std::vector, no new, no device allocation).
// ---------------------------------------------------------------------------
namespace hg {
namespace {
std::mutex g_plan_mu;
DevScene g_plan_scenes[kMaxScenes];
DevScanner g_plan_scanners[kMaxScanners];
DevLeg g_plan_legs[16 * kMaxLegs];
}  // namespace
}  // namespace hg

extern "C" helios_status helios_scan_legs_static(helios_scene* const* scenes, int32_t n_scenes,
                                                 const helios_scanner_desc* scanners,
                                                 int32_t n_scanners, const helios_leg_desc* legs,
                                                 int32_t n_legs, const helios_scan_opts* opts,
                                                 const helios_outputs* out, void* cuda_stream) {
    g_err.clear();
    CallRange range_("helios_scan_legs_static");
    if (injected_fault() == kFaultBadArg)
        return set_error(HELIOS_ERR_INVALID_ARG, "helios_scan_legs_static: injected fault (HELIOS_FAULT=badarg)");
    helios_status st = check_scenes(scenes, n_scenes);
    if (st != HELIOS_OK) return st;
    if (!opts || !out) return set_error(HELIOS_ERR_INVALID_ARG, "opts and out must not be NULL");
    if (opts->mode != HELIOS_MODE_STOCHASTIC && opts->mode != HELIOS_MODE_EXPECTED)
        return set_error(HELIOS_ERR_INVALID_ARG, "unknown mode");
    if (!out->waveform || !out->window_bin || !out->echo_count || !out->echo_range)
        return set_error(HELIOS_ERR_INVALID_ARG, "waveform, window_bin, echo_count, echo_range are required");
    if (out->subray_range && !out->subray_hit)
        return set_error(HELIOS_ERR_INVALID_ARG, "subray_range needs subray_hit");
    if (out->echo_width && !out->echo_bin)
        return set_error(HELIOS_ERR_INVALID_ARG, "echo_width needs echo_bin in the allocation-free scan");
    const int max_legs = static_scan_max_legs();
    if (n_legs < 0 || (n_legs > 0 && !legs)) return set_error(HELIOS_ERR_INVALID_ARG, "legs is NULL");
    if (n_legs > max_legs)
        return set_error(HELIOS_ERR_INVALID_ARG, "helios_scan_legs_static takes at most %d legs, got %d",
                         max_legs, n_legs);
    int threads = opts->block_threads > 0 ? opts->block_threads : 256;
    if (threads % 32 != 0 || threads < 64 || threads > 256)
        return set_error(HELIOS_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in 64..256");
    int rays = opts->rays_per_block > 0 ? opts->rays_per_block : 768;
    if (rays > 4096) return set_error(HELIOS_ERR_INVALID_ARG, "rays_per_block must be <= 4096");
    if (n_scanners < 1 || n_scanners > kMaxScanners || !scanners)
        return set_error(HELIOS_ERR_INVALID_ARG, "n_scanners must be in 1..%d", kMaxScanners);
    for (int i = 0; i < n_scanners; ++i) {
        st = check_scanner(scanners[i], i);
        if (st != HELIOS_OK) return st;
    }
    std::lock_guard<std::mutex> lock(g_plan_mu);
    int64_t pulses = 0, wave = 0, sub = 0, echo = 0;
    for (int l = 0; l < n_legs; ++l) {
        const helios_leg_desc& L = legs[l];
        if (L.scene_index < 0 || L.scene_index >= n_scenes)
            return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: scene_index out of range", l);
        if (L.scanner_index < 0 || L.scanner_index >= n_scanners)
            return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: scanner_index out of range", l);
        if (L.platform != HELIOS_PLATFORM_STATIC && L.platform != HELIOS_PLATFORM_LINEAR)
            return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: unknown platform", l);
        if (L.n_pulses < 0) return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: n_pulses < 0", l);
        // draws are keyed by the absolute pulse index in 44 bits
        if (L.first_pulse < 0 || L.first_pulse > kMaxPulseIndex - L.n_pulses)
            return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: first_pulse + n_pulses must be in 0..2^44", l);
        if (!(L.platform_noise_m >= 0.0f))
            return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: platform_noise_m must be >= 0", l);
        if (L.platform == HELIOS_PLATFORM_LINEAR && !(L.speed_mps >= 0.0))
            return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: speed_mps must be >= 0", l);
        const helios_scanner_desc& sc = scanners[L.scanner_index];
        int q = L.beam_sample_quality >= 0 ? L.beam_sample_quality : sc.beam_sample_quality;
        if (q > 9) return set_error(HELIOS_ERR_INVALID_ARG, "leg %d: beam_sample_quality must be <= 9", l);
        DevLeg& d = g_plan_legs[l];
        memset(&d, 0, sizeof(d));
        double D[3], len2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            d.start[a] = L.start[a];
            D[a] = L.end[a] - L.start[a];
            len2 += D[a] * D[a];
            d.rpy[a] = L.attitude_rpy[a];
        }
        d.length = std::sqrt(len2);
        if (L.platform == HELIOS_PLATFORM_LINEAR && d.length > 0.0) {
            for (int a = 0; a < 3; ++a) d.dir[a] = D[a] / d.length;
            d.rpy[2] += std::atan2(D[1], D[0]);
        }
        d.speed = L.speed_mps;
        d.t0 = L.t0;
        d.n_pulses = L.n_pulses;
        d.scene = L.scene_index;
        d.scanner = L.scanner_index;
        d.platform = L.platform;
        d.q = q;
        d.S = subray_count(q);
        int ppi = rays / d.S;
        d.pulses_per_sub = ppi < 1 ? 1 : (ppi > 256 ? 256 : ppi);
        d.pulses_per_item = item_pulses(d.pulses_per_sub, opts->mode);
        d.leg_id = L.leg_id;
        d.platform_noise = L.platform_noise_m;
        // outputs of absolute pulse k at offset + k (rows start at first_pulse)
        d.k_first = L.first_pulse;
        d.pulse_off = pulses - L.first_pulse;
        d.wave_off = wave - L.first_pulse * sc.n_bins;
        d.sub_off = sub - L.first_pulse * d.S;
        d.echo_off = echo - L.first_pulse * sc.max_echoes;
        pulses += L.n_pulses;
        wave += L.n_pulses * sc.n_bins;
        sub += L.n_pulses * d.S;
        echo += L.n_pulses * sc.max_echoes;
    }
    for (int i = 0; i < n_scenes; ++i) g_plan_scenes[i] = dev_scene(scenes[i]);
    for (int i = 0; i < n_scanners; ++i) g_plan_scanners[i] = derive_scanner(scanners[i]);
    Outputs o;
    o.waveform = out->waveform;
    o.window_bin = out->window_bin;
    o.echo_count = out->echo_count;
    o.echo_range = out->echo_range;
    o.echo_amp = out->echo_amp;
    o.echo_bin = out->echo_bin;
    o.echo_object = out->echo_object;
    o.pulse_flags = out->pulse_flags;
    o.subray_hit = out->subray_hit;
    o.subray_range = out->subray_range;
    o.status = out->status;
    o.echo_width = out->echo_width;
    if (pulses == 0) return HELIOS_OK;
    return launch_scan_static(g_plan_scenes, n_scenes, g_plan_scanners, n_scanners, g_plan_legs,
                              n_legs, o, opts->seed, opts->mode, threads, opts->blocks_per_sm,
                              (cudaStream_t)cuda_stream);
}

// ---------------------------------------------------------------------------
// helios_scan_legs_host: the scan with outputs in host memory.  The pulses
// are cut into chunks of whole work items (so every pulse is computed exactly
// as by helios_scan_legs); chunk c is scanned on the caller's stream into
// staging slot c % 2 while a second stream copies chunk c - 1 to the host.
// ---------------------------------------------------------------------------
namespace hg {
namespace {

// one contiguous run of a leg's pulses inside a chunk
struct Piece {
    int leg;
    int64_t k0, n;
};

// output positions (pulse, waveform float, echo slot, subray slot) of global pulse g
struct Pos {
    int64_t p, w, e, s;
};

Pos out_pos(const LegPlan& P, const helios_scanner_desc* sc, int64_t g) {
    for (const DevLeg& d : P.legs) {
        if (d.n_pulses > 0 && g >= d.pulse_off && g < d.pulse_off + d.n_pulses) {
            const int64_t k = g - d.pulse_off;
            return {g, d.wave_off + k * sc[d.scanner].n_bins, d.echo_off + k * sc[d.scanner].max_echoes,
                    d.sub_off + k * d.S};
        }
    }
    return {P.total_pulses, P.wave, P.echo, P.sub};
}

struct HostStaging {
    void* buf[2] = {nullptr, nullptr};
    cudaStream_t s0 = nullptr, s1 = nullptr;
    cudaEvent_t scanned[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
    ~HostStaging() {
        // the caller's stream waits for the last copies before the slots are freed
        for (int i = 0; i < 2; ++i)
            if (copied[i]) cudaStreamWaitEvent(s0, copied[i], 0);
        for (int i = 0; i < 2; ++i) {
            if (buf[i]) cudaFreeAsync(buf[i], s0);
            if (scanned[i]) cudaEventDestroy(scanned[i]);
            if (copied[i]) cudaEventDestroy(copied[i]);
        }
        if (s1) cudaStreamDestroy(s1);
    }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace hg

extern "C" helios_status helios_scan_legs_host(helios_scene* const* scenes, int32_t n_scenes,
                                               const helios_scanner_desc* scanners,
                                               int32_t n_scanners, const helios_leg_desc* legs,
                                               int32_t n_legs, const helios_scan_opts* opts,
                                               const helios_outputs* host_out,
                                               int64_t chunk_pulses, void* cuda_stream) {
    using namespace hg;
    g_err.clear();
    CallRange range_("helios_scan_legs_host");
    if (injected_fault() == kFaultBadArg)
        return set_error(HELIOS_ERR_INVALID_ARG, "helios_scan_legs_host: injected fault (HELIOS_FAULT=badarg)");
    helios_status st = check_scenes(scenes, n_scenes);
    if (st != HELIOS_OK) return st;
    if (!opts || !host_out) return set_error(HELIOS_ERR_INVALID_ARG, "opts and host_out must not be NULL");
    if (opts->mode != HELIOS_MODE_STOCHASTIC && opts->mode != HELIOS_MODE_EXPECTED)
        return set_error(HELIOS_ERR_INVALID_ARG, "unknown mode");
    if (!host_out->waveform || !host_out->window_bin || !host_out->echo_count || !host_out->echo_range)
        return set_error(HELIOS_ERR_INVALID_ARG, "waveform, window_bin, echo_count, echo_range are required");
    if (host_out->subray_range && !host_out->subray_hit)
        return set_error(HELIOS_ERR_INVALID_ARG, "subray_range needs subray_hit");
    if (chunk_pulses <= 0) return set_error(HELIOS_ERR_INVALID_ARG, "chunk_pulses must be positive");
    int threads = opts->block_threads > 0 ? opts->block_threads : 256;
    if (threads % 32 != 0 || threads < 64 || threads > 256)
        return set_error(HELIOS_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in 64..256");
    int rays = opts->rays_per_block > 0 ? opts->rays_per_block : 768;
    if (rays > 4096) return set_error(HELIOS_ERR_INVALID_ARG, "rays_per_block must be <= 4096");
    LegPlan P;
    st = plan_legs(scanners, n_scanners, legs, n_legs, n_scenes, rays, opts->mode, P);
    if (st != HELIOS_OK) return st;
    if (P.total_pulses == 0) return HELIOS_OK;

    // chunks of whole work items, about chunk_pulses pulses each
    std::vector<std::vector<Piece>> chunks(1);
    int64_t in_chunk = 0;
    for (int l = 0; l < (int)P.legs.size(); ++l) {
        const DevLeg& d = P.legs[l];
        int64_t k = 0;
        while (k < d.n_pulses) {
            if (in_chunk >= chunk_pulses) { chunks.emplace_back(); in_chunk = 0; }
            const int64_t want = chunk_pulses - in_chunk;
            const int64_t items = (want + d.pulses_per_item - 1) / d.pulses_per_item;
            const int64_t n = std::min(d.n_pulses - k, items * d.pulses_per_item);
            chunks.back().push_back({l, k, n});
            k += n;
            in_chunk += n;
        }
    }
    // staging slot size: the largest chunk's outputs
    int64_t mx_p = 0, mx_w = 0, mx_e = 0, mx_s = 0;
    std::vector<std::pair<Pos, Pos>> span;
    for (const auto& c : chunks) {
        const DevLeg& a = P.legs[c.front().leg];
        const DevLeg& b = P.legs[c.back().leg];
        const Pos lo = out_pos(P, scanners, a.pulse_off + c.front().k0);
        const Pos hi = out_pos(P, scanners, b.pulse_off + c.back().k0 + c.back().n);
        span.push_back({lo, hi});
        mx_p = std::max(mx_p, hi.p - lo.p);
        mx_w = std::max(mx_w, hi.w - lo.w);
        mx_e = std::max(mx_e, hi.e - lo.e);
        mx_s = std::max(mx_s, hi.s - lo.s);
    }
    const helios_outputs& H = *host_out;
    const bool sub = H.subray_hit != nullptr;
    size_t off[11], bytes = 0;
    const size_t sz[11] = {sizeof(float) * mx_w, sizeof(int32_t) * mx_p, sizeof(int32_t) * mx_p,
                           sizeof(float) * mx_e, H.echo_amp ? sizeof(float) * mx_e : 0,
                           H.echo_bin ? sizeof(int32_t) * mx_e : 0, H.echo_object ? sizeof(int64_t) * mx_e : 0,
                           H.pulse_flags ? sizeof(uint8_t) * mx_p : 0, sub ? sizeof(int64_t) * mx_s : 0,
                           H.subray_range ? sizeof(float) * mx_s : 0,
                           H.echo_width ? sizeof(float) * mx_e : 0};
    for (int i = 0; i < 11; ++i) { off[i] = bytes; bytes += align256(sz[i]); }

    HostStaging hs;
    hs.s0 = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaStreamCreateWithFlags(&hs.s1, cudaStreamNonBlocking);
    if (e != cudaSuccess) { hs.s1 = nullptr; return set_cuda_error("cudaStreamCreate", e); }
    for (int i = 0; i < 2; ++i) {
        e = cudaEventCreateWithFlags(&hs.scanned[i], cudaEventDisableTiming);
        if (e != cudaSuccess) { hs.scanned[i] = nullptr; return set_cuda_error("cudaEventCreate", e); }
        e = cudaEventCreateWithFlags(&hs.copied[i], cudaEventDisableTiming);
        if (e != cudaSuccess) { hs.copied[i] = nullptr; return set_cuda_error("cudaEventCreate", e); }
        e = dev_malloc_async(&hs.buf[i], bytes, hs.s0);
        if (e != cudaSuccess) { hs.buf[i] = nullptr; return set_cuda_error("cudaMallocAsync(staging)", e); }
    }
    ScanLaunch L;
    for (int i = 0; i < n_scenes; ++i) L.scenes.push_back(dev_scene(scenes[i]));
    for (int i = 0; i < n_scanners; ++i) L.scanners.push_back(derive_scanner(scanners[i]));
    OccupancyMasks masks;
    st = build_occupancy(L.scenes, scenes, hs.s0, masks);
    if (st != HELIOS_OK) return st;
    L.seed = opts->seed;
    L.mode = opts->mode;
    L.persistent = opts->persistent;
    L.threads = threads;
    L.blocks_per_sm = opts->blocks_per_sm;
    for (size_t c = 0; c < chunks.size(); ++c) {
        const int slot = (int)(c & 1);
        const Pos lo = span[c].first, hi = span[c].second;
        if (c >= 2) cudaStreamWaitEvent(hs.s0, hs.copied[slot], 0);
        char* base = static_cast<char*>(hs.buf[slot]);
        L.out.waveform = reinterpret_cast<float*>(base + off[0]);
        L.out.window_bin = reinterpret_cast<int32_t*>(base + off[1]);
        L.out.echo_count = reinterpret_cast<int32_t*>(base + off[2]);
        L.out.echo_range = reinterpret_cast<float*>(base + off[3]);
        L.out.echo_amp = H.echo_amp ? reinterpret_cast<float*>(base + off[4]) : nullptr;
        L.out.echo_bin = H.echo_bin ? reinterpret_cast<int32_t*>(base + off[5]) : nullptr;
        L.out.echo_object = H.echo_object ? reinterpret_cast<int64_t*>(base + off[6]) : nullptr;
        L.out.pulse_flags = H.pulse_flags ? reinterpret_cast<uint8_t*>(base + off[7]) : nullptr;
        L.out.subray_hit = sub ? reinterpret_cast<int64_t*>(base + off[8]) : nullptr;
        L.out.subray_range = H.subray_range ? reinterpret_cast<float*>(base + off[9]) : nullptr;
        L.out.status = H.status;
        L.out.echo_width = H.echo_width ? reinterpret_cast<float*>(base + off[10]) : nullptr;
        // the chunk's legs, their outputs indexed from the slot's start
        L.legs.clear();
        for (const Piece& pc : chunks[c]) {
            // rows pc.k0 .. of the leg: absolute pulses first_pulse + pc.k0 ..
            DevLeg d = kernel_leg(P.legs[pc.leg], scanners);
            d.k_first += pc.k0;
            d.n_pulses = pc.n;
            d.pulse_off -= lo.p;
            d.wave_off -= lo.w;
            d.echo_off -= lo.e;
            d.sub_off -= lo.s;
            L.legs.push_back(d);
        }
        st = launch_scan(L, hs.s0);
        if (st != HELIOS_OK) return st;
        e = cudaEventRecord(hs.scanned[slot], hs.s0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hs.s1, hs.scanned[slot], 0);
        if (e != cudaSuccess) return set_cuda_error("chunk event", e);
        struct Copy { void* dst; const void* src; size_t n; };
        const Copy cp[11] = {
            {H.waveform + lo.w, L.out.waveform, sizeof(float) * (hi.w - lo.w)},
            {H.window_bin + lo.p, L.out.window_bin, sizeof(int32_t) * (hi.p - lo.p)},
            {H.echo_count + lo.p, L.out.echo_count, sizeof(int32_t) * (hi.p - lo.p)},
            {H.echo_range + lo.e, L.out.echo_range, sizeof(float) * (hi.e - lo.e)},
            {H.echo_amp ? H.echo_amp + lo.e : nullptr, L.out.echo_amp, sizeof(float) * (hi.e - lo.e)},
            {H.echo_bin ? H.echo_bin + lo.e : nullptr, L.out.echo_bin, sizeof(int32_t) * (hi.e - lo.e)},
            {H.echo_object ? H.echo_object + lo.e : nullptr, L.out.echo_object, sizeof(int64_t) * (hi.e - lo.e)},
            {H.pulse_flags ? H.pulse_flags + lo.p : nullptr, L.out.pulse_flags, sizeof(uint8_t) * (hi.p - lo.p)},
            {sub ? H.subray_hit + lo.s : nullptr, L.out.subray_hit, sizeof(int64_t) * (hi.s - lo.s)},
            {H.subray_range ? H.subray_range + lo.s : nullptr, L.out.subray_range, sizeof(float) * (hi.s - lo.s)},
            {H.echo_width ? H.echo_width + lo.e : nullptr, L.out.echo_width, sizeof(float) * (hi.e - lo.e)}};
        for (const Copy& x : cp) {
            if (!x.dst || x.n == 0) continue;
            e = cudaMemcpyAsync(x.dst, x.src, x.n, cudaMemcpyDeviceToHost, hs.s1);
            if (e != cudaSuccess) return set_cuda_error("cudaMemcpyAsync(D2H)", e);
        }
        e = cudaEventRecord(hs.copied[slot], hs.s1);
        if (e != cudaSuccess) return set_cuda_error("chunk event", e);
    }
    return HELIOS_OK;
}
