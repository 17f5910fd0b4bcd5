// stats.cu - per-pulse fetch counts for the algorithmic-bytes model of the
// roofline.  Not on the scan path: a separate kernel, run on a sample of a
// leg's pulses, counts what one pulse needs from memory as a union over its
// subrays (the subrays of a pulse are a fraction of a milliradian apart and
// share most fetches):
//   nodes      4-wide BVH nodes (8 float4, 128 B) the pulse's beam cone
//              enters: the root plus every internal slot whose box the cone
//              overlaps (the scan's per-pulse cone walk, Sec. 3.4 beam)
//   triangles  triangles (3 float4, 48 B) whose widened box the cone
//              overlaps: the pulse's candidate set, tested by every subray
//   voxels     distinct voxels (4 B of density) the subrays march through
//              (Sec. 3.5.4), each stopping where the scan's march stops in
//              the given mode: at its stochastic event (Eq. intersection_dist)
//              or, in expected mode, at its triangle hit
//   visits     voxel visits summed over the subrays (visits / voxels is the
//              subrays' coherence)
// One warp takes 32 sampled pulses: lanes are pulses for the cone walk (each
// lane walks its own cone with an explicit stack, so it counts exactly the
// nodes its pulse needs), then lanes are subrays for the marches, whose voxel
// ids go into a per-warp hash set in shared memory.
#include "hg_device.cuh"
#include "hg_host.h"

namespace hg {

namespace {

constexpr int kStatsThreads = 128;
constexpr int kHashSlots = 4096;                 // per warp: 32 KB of 64-bit keys
constexpr int kHashFill = kHashSlots * 3 / 4;    // beyond this, visits count as new
constexpr int kStackCap = 160;                   // 48 levels x 3 pending slots + 1

struct StatsParams {
    DevScene sc;
    DevScanner sn;
    DevLeg lg;
    int64_t first, stride, count;
    int32_t mode;
    uint64_t seed;
    helios_fetch_counts* out;
};

// The cone walk of one pulse on its own: every node popped is one node load.
__device__ void cone_count(const DevScene& S, const RayF& r, float ta, int64_t& nodes,
                           int64_t& tris, int32_t& flags) {
    nodes = 0;
    tris = 0;
    if (S.n_tri == 0) return;
    if (S.n_int == 0) {          // a single triangle, no tree
        tris = 1;
        return;
    }
    const float ad[3] = {fabsf(r.idx), fabsf(r.idy), fabsf(r.idz)};
    int stack[kStackCap];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const int cur = stack[--sp];
        ++nodes;
        const float4* nd = S.nodes4 + 8 * (size_t)cur;
        const float4 lx = __ldg(nd), ly = __ldg(nd + 1), lz = __ldg(nd + 2);
        const float4 hx = __ldg(nd + 3), hy = __ldg(nd + 4), hz = __ldg(nd + 5);
        const int4 rf = __ldg(reinterpret_cast<const int4*>(nd + 6));
        const int vm = __ldg(reinterpret_cast<const int4*>(nd + 7)).y;
        for (int k = 0; k < 4; ++k) {
            const float b[6] = {f4c(lx, k), f4c(ly, k), f4c(lz, k), f4c(hx, k), f4c(hy, k), f4c(hz, k)};
            if (!((vm >> k) & 1) || !cone_slab(r, ta, ad, b)) continue;
            const int ref = i4c(rf, k);
            if (ref < 0) {
                ++tris;
            } else if (sp < kStackCap) {
                stack[sp++] = ref;
            } else {
                flags |= HELIOS_FC_STACK;
            }
        }
    }
    if (tris > kConeCap + kConeExt) flags |= HELIOS_FC_LIST_OVERFLOW;
}

// Insert a key (> 0) into the warp's open-addressing set; true if it was new.
// Past kHashFill entries nothing is inserted and every key counts as new (an
// upper bound, flagged).
__device__ bool set_insert(unsigned long long* T, int* fill, unsigned long long key, bool& full) {
    if (*fill >= kHashFill) {
        full = true;
        return true;
    }
    uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 52) & (kHashSlots - 1);
    for (int i = 0; i < kHashSlots; ++i) {
        const unsigned long long prev = atomicCAS(&T[h], 0ull, key);
        if (prev == 0ull) {
            atomicAdd(fill, 1);
            return true;
        }
        if (prev == key) return false;
        h = (h + 1) & (kHashSlots - 1);
    }
    full = true;
    return true;
}

template <int GK>
__global__ void __launch_bounds__(kStatsThreads) stats_kernel(const __grid_constant__ StatsParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int nwarps = kStatsThreads / 32;
    unsigned long long* s_set = reinterpret_cast<unsigned long long*>(smem);      // [nwarps][slots]
    PulseFF* s_pf = reinterpret_cast<PulseFF*>(s_set + (size_t)nwarps * kHashSlots);   // [nwarps][32]
    SubrayConst* s_sc = reinterpret_cast<SubrayConst*>(s_pf + nwarps * 32);     // [S]
    __shared__ int s_fill[kStatsThreads / 32];
    __shared__ double s_rot[6];
    const unsigned full = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevScene& sc = P.sc;
    const DevScanner& sn = P.sn;
    const DevLeg& lg = P.lg;
    const int S = lg.S;
    for (int s = tid; s < S; s += blockDim.x) subray_const(lg.q, sn.theta_r, s, s_sc[s]);
    for (int i = tid; i < nwarps * kHashSlots; i += blockDim.x) s_set[i] = 0ull;
    if (tid < nwarps) s_fill[tid] = 0;
    if (tid == 0) {
        sincos(lg.rpy[0], &s_rot[0], &s_rot[1]);
        sincos(lg.rpy[1], &s_rot[2], &s_rot[3]);
        sincos(lg.rpy[2], &s_rot[4], &s_rot[5]);
    }
    __syncthreads();
    unsigned long long* T = s_set + (size_t)warp * kHashSlots;
    PulseFF* pf = s_pf + warp * 32;
    const float ta = fmaf(tanf((float)sn.theta_r), 1.001f, 1.0e-6f);
    const int64_t n_groups = (P.count + 31) / 32;
    for (int64_t grp = (int64_t)blockIdx.x * nwarps + warp; grp < n_groups; grp += (int64_t)gridDim.x * nwarps) {
        // lanes = pulses: pose and cone walk
        const int64_t i = grp * 32 + lane;
        const bool act = i < P.count;
        const int64_t k = lg.k_first + P.first + (act ? i : 0) * P.stride;
        {
            PulseFrame fr;
            pulse_frame(sn, lg, s_rot, k, P.seed, fr);
            split_store(fr, pf[lane]);
        }
        int64_t nodes = 0, tris = 0;
        int32_t flags = 0;
        if (act && sc.n_tri > 0) {
            float dh[3], dl[3];
            subray_dir_ff(pf[lane], s_sc[0], dh, dl);   // subray 0: the pulse axis
            RayF ray;
            make_ray(pf[lane].oh, pf[lane].ol, dh, ray);
            cone_count(sc, ray, ta, nodes, tris, flags);
        }
        __syncwarp();
        // lanes = subrays: the marches of each pulse in turn
        int64_t my_vox = 0, my_visits = 0;
        int32_t my_vflags = 0;
        const int n_here = (int)min((int64_t)32, P.count - grp * 32);
        for (int j = 0; j < n_here; ++j) {
            const int64_t kj = lg.k_first + P.first + (grp * 32 + j) * P.stride;
            const PulseFF& f = pf[j];
            int64_t vox = 0, visits = 0;
            bool set_full = false;
            uint32_t mfl = 0;
            for (int s0 = 0; s0 < S && GK > 0 && sc.has_grid; s0 += 32) {
                const int s = s0 + lane;
                const bool on = s < S;
                float dh[3], dl[3];
                subray_dir_ff(f, s_sc[on ? s : 0], dh, dl);
                RayF ray;
                make_ray(f.oh, f.ol, dh, ray);
                float tb = 3.0e38f;
                int hit = -1;
                traverse(sc, ray, on, tb, hit, mfl);    // all lanes: warp-coherent walk
                if (!on) continue;
                FF o[3], d[3];
                for (int a = 0; a < 3; ++a) {
                    o[a] = ff_norm(f.oh[a], f.ol[a]);
                    d[a] = ff_norm(dh[a], dl[a]);
                }
                const FF t_tri = hit >= 0 ? FF{tb, 0.0f} : FF{CUDART_INF_F, 0.0f};
                walk_grids<GK>(sc, o, d, t_tri, [&](const DevGrid& G, March& m) -> bool {
                    const float Gs = proj_factor(G, dh[2]);
                    for (;;) {
                        VoxSeg v;
                        if (!march_current(G, m, v)) return true;
                        ++visits;
                        if (set_insert(T, &s_fill[warp], (unsigned long long)(G.vox_off + v.vid) + 1ull, set_full))
                            ++vox;
                        const float dens = voxel_density<false>(G, m, v);
                        if (dens > 0.0f) {
                            FF t_in, t_out;
                            march_segment_ff(m, v, t_in, t_out);
                            const float len = ff_diff(t_out, t_in);
                            if (len > 0.0f && G.opaque) return false;
                            if (len > 0.0f && P.mode == HELIOS_MODE_STOCHASTIC) {
                                uint32_t w[4];
                                draw4(P.seed, lg.leg_id, kj, 0u, (uint32_t)s, G.vox_off + v.vid, w);
                                const float sdist = -logf(uniform23(w[0])) / (Gs * dens);
                                if (sdist < len) return false;
                            }
                        }
                        if (!march_step(m, v, mfl)) return true;
                    }
                });
            }
            // the pulse's totals to its lane; empty the set for the next pulse
            vox = __reduce_add_sync(full, (unsigned)vox);
            visits = __reduce_add_sync(full, (unsigned)visits);
            const bool any_full = __any_sync(full, set_full);
            const unsigned any_cap = __reduce_or_sync(full, mfl & kPfMarchCap);
            if (lane == j) {
                my_vox = vox;
                my_visits = visits;
                my_vflags = (any_full ? HELIOS_FC_SET_FULL : 0) | (any_cap ? HELIOS_FC_MARCH_CAP : 0);
            }
            __syncwarp();
            for (int t = lane; t < kHashSlots; t += 32) T[t] = 0ull;
            if (lane == 0) s_fill[warp] = 0;
            __syncwarp();
        }
        if (act) {
            helios_fetch_counts c;
            c.nodes = nodes;
            c.triangles = tris;
            c.voxels = my_vox;
            c.voxel_visits = my_visits;
            c.flags = flags | my_vflags;
            c.reserved = 0;
            P.out[i] = c;
        }
        __syncwarp();
    }
}

}  // namespace

helios_status launch_fetch_counts(const DevScene& sc, const DevScanner& sn, const DevLeg& lg,
                                  int mode, uint64_t seed, int64_t first, int64_t stride,
                                  int64_t count, helios_fetch_counts* out, cudaStream_t st) {
    if (count == 0) return HELIOS_OK;
    StatsParams p;
    memset(&p, 0, sizeof(p));
    p.sc = sc;
    p.sn = sn;
    p.lg = lg;
    p.first = first;
    p.stride = stride;
    p.count = count;
    p.mode = mode;
    p.seed = seed;
    p.out = out;
    const int nwarps = kStatsThreads / 32;
    const size_t smem = sizeof(unsigned long long) * (size_t)nwarps * kHashSlots +
                        sizeof(PulseFF) * nwarps * 32 + sizeof(SubrayConst) * (size_t)lg.S;
    if (smem > 227 * 1024) return set_error(HELIOS_ERR_UNSUPPORTED, "fetch counts need %zu bytes of shared memory", smem);
    auto kern = sc.n_grid > 1 ? stats_kernel<2> : (sc.has_grid ? stats_kernel<1> : stats_kernel<0>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_cuda_error("cudaFuncSetAttribute(fetch counts)", e);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t groups = (count + 31) / 32;
    const int64_t want = (groups + nwarps - 1) / nwarps;
    const int grid = (int)(want < 4LL * sms ? want : 4LL * sms);
    kern<<<grid, kStatsThreads, smem, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error("fetch-count kernel launch", e);
    return HELIOS_OK;
}

}  // namespace hg
